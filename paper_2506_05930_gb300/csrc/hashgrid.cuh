// Device helpers of the multi-resolution hash-grid encoding (Sections 3.1
// and 3.3 of the paper): the 8 corner rows of a cell and their trilinear
// weights, and vector loads of one table row.
#pragma once

#include "nvc_internal.cuh"

namespace nvc {

template <int F>
struct FeatVec {
  float v[F];
};

template <int F>
__device__ __forceinline__ FeatVec<F> load_feat(const float* p) {
  FeatVec<F> r;
  if constexpr (F == 1) {
    r.v[0] = __ldg(p);
  } else if constexpr (F == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(p));
    r.v[0] = a.x;
    r.v[1] = a.y;
  } else {
#pragma unroll
    for (int k = 0; k < F; k += 4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p + k));
      r.v[k] = a.x;
      r.v[k + 1] = a.y;
      r.v[k + 2] = a.z;
      r.v[k + 3] = a.w;
    }
  }
  return r;
}

// Corner rows and trilinear weights of one (position, level).
struct Corners {
  uint32_t row[8];
  float w[8];
};

__device__ __forceinline__ void level_corners(const EncodeParams& ep, int l, float x, float y,
                                              float z, Corners& cr) {
  const int n = ep.res[l];
  int cx, cy, cz;
  float fx, fy, fz;
  grid_cell(x, n, cx, fx);
  grid_cell(y, n, cy, fy);
  grid_cell(z, n, cz, fz);
  const uint32_t mask = (1u << ep.log2_table) - 1u;
  const float gx[2] = {1.0f - fx, fx}, gy[2] = {1.0f - fy, fy}, gz[2] = {1.0f - fz, fz};
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
    cr.row[d] = grid_hash((uint32_t)(cx + dx), (uint32_t)(cy + dy), (uint32_t)(cz + dz)) & mask;
    cr.w[d] = gx[dx] * gy[dy] * gz[dz];
  }
}

}  // namespace nvc
