// Multi-resolution hash-grid encoding (Sections 3.1 and 3.3 of the paper,
// after Mueller et al. 2022) and its adjoint.
//
// One thread per (position, level), level fastest, so a warp covers two
// positions x 16 levels and its feature stores are contiguous.  Each
// thread hashes the 8 corners of its cell and gathers F float32 features
// per corner (one 8-byte load for F = 2) from the level's table; at the
// table sizes used here the tables stay resident in L2.
#include "nvc_internal.cuh"
#include "hashgrid.cuh"

namespace nvc {

EncodeParams encode_params(const nvc_handle* h) {
  EncodeParams ep{};
  ep.n_levels = h->cfg.n_levels;
  ep.log2_table = h->cfg.log2_table_size;
  for (int d = 0; d < 3; ++d) {
    ep.lo[d] = h->cfg.bounds_min[d];
    ep.ext[d] = h->cfg.bounds_max[d] - h->cfg.bounds_min[d];  // host float32 subtraction
  }
  for (int l = 0; l < h->cfg.n_levels; ++l) {
    ep.res[l] = h->res[l];
    ep.resf[l] = (float)h->res[l];
  }
  return ep;
}

template <int F>
__global__ void __launch_bounds__(256) encode_fwd_kernel(const float* __restrict__ pos,
                                                         int64_t n, const float* __restrict__ table,
                                                         EncodeParams ep,
                                                         float* __restrict__ feat) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int L = ep.n_levels;
  if (t >= n * L) return;
  const int64_t i = t / L;
  const int l = (int)(t - i * L);
  const float x = normalise(__ldg(pos + 3 * i + 0), ep.lo[0], ep.ext[0]);
  const float y = normalise(__ldg(pos + 3 * i + 1), ep.lo[1], ep.ext[1]);
  const float z = normalise(__ldg(pos + 3 * i + 2), ep.lo[2], ep.ext[2]);
  Corners cr;
  level_corners(ep, l, x, y, z, cr);
  const float* tab = table + ((int64_t)l << ep.log2_table) * F;
  float acc[F];
#pragma unroll
  for (int f = 0; f < F; ++f) acc[f] = 0.0f;
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const FeatVec<F> v = load_feat<F>(tab + (int64_t)cr.row[d] * F);
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = fmaf(cr.w[d], v.v[f], acc[f]);
  }
  float* out = feat + i * (int64_t)L * F + l * F;
#pragma unroll
  for (int f = 0; f < F; ++f) out[f] = acc[f];
}

template <int F>
__global__ void __launch_bounds__(256) encode_bwd_kernel(const float* __restrict__ pos, int64_t n,
                                                         const float* __restrict__ dfeat,
                                                         EncodeParams ep, float* grad,
                                                         int32_t* status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int L = ep.n_levels;
  if (t >= n * L) return;
  const int64_t i = t / L;
  const int l = (int)(t - i * L);
  float g[F];
  bool finite = true;
#pragma unroll
  for (int f = 0; f < F; ++f) {
    g[f] = __ldg(dfeat + i * (int64_t)L * F + l * F + f);
    finite = finite && isfinite(g[f]);
  }
  if (!finite) {
    atomicOr(status + kStNonFinite, 1);
    return;
  }
  const float x = normalise(__ldg(pos + 3 * i + 0), ep.lo[0], ep.ext[0]);
  const float y = normalise(__ldg(pos + 3 * i + 1), ep.lo[1], ep.ext[1]);
  const float z = normalise(__ldg(pos + 3 * i + 2), ep.lo[2], ep.ext[2]);
  Corners cr;
  level_corners(ep, l, x, y, z, cr);
  float* tab = grad + ((int64_t)l << ep.log2_table) * F;
  if constexpr (F == 2) {
    // The x-corners d, d + 1 of each (y, z) pair: when their rows are the two
    // rows of one aligned 16-byte pair -- always for an even cell x, as the
    // x prime is 1 and so hash(x + 1) = hash(x) ^ 1 -- one 16-byte atomic
    // adds both; otherwise two 8-byte atomics.
#pragma unroll
    for (int d = 0; d < 8; d += 2) {
      const uint32_t r0 = cr.row[d], r1 = cr.row[d + 1];
      const float2 g0 = make_float2(cr.w[d] * g[0], cr.w[d] * g[1]);
      const float2 g1 = make_float2(cr.w[d + 1] * g[0], cr.w[d + 1] * g[1]);
      if ((r0 ^ r1) == 1u) {
        const float4 v = (r0 & 1u) ? make_float4(g1.x, g1.y, g0.x, g0.y)
                                   : make_float4(g0.x, g0.y, g1.x, g1.y);
        atomicAdd(reinterpret_cast<float4*>(tab + (int64_t)(r0 & ~1u) * 2), v);
      } else {
        atomicAdd(reinterpret_cast<float2*>(tab + (int64_t)r0 * 2), g0);
        atomicAdd(reinterpret_cast<float2*>(tab + (int64_t)r1 * 2), g1);
      }
    }
    return;
  }
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    float* dst = tab + (int64_t)cr.row[d] * F;
    if constexpr (F % 4 == 0) {
#pragma unroll
      for (int k = 0; k < F; k += 4)
        atomicAdd(reinterpret_cast<float4*>(dst + k),
                  make_float4(cr.w[d] * g[k], cr.w[d] * g[k + 1], cr.w[d] * g[k + 2],
                              cr.w[d] * g[k + 3]));
    } else {
#pragma unroll
      for (int f = 0; f < F; ++f) atomicAdd(dst + f, cr.w[d] * g[f]);
    }
  }
}

template <int F>
static cudaError_t enc_fwd(const nvc_handle* h, const float* pos, int64_t n, float* feat,
                           cudaStream_t s) {
  const int64_t total = n * h->cfg.n_levels;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  encode_fwd_kernel<F><<<(unsigned)blocks, threads, 0, s>>>(pos, n, h->params, encode_params(h),
                                                              feat);
  return cudaGetLastError();
}

template <int F>
static cudaError_t enc_bwd(const nvc_handle* h, const float* pos, int64_t n, const float* dfeat,
                           float* grad, int32_t* status, cudaStream_t s) {
  const int64_t total = n * h->cfg.n_levels;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  encode_bwd_kernel<F><<<(unsigned)blocks, threads, 0, s>>>(pos, n, dfeat, encode_params(h), grad,
                                                              status);
  return cudaGetLastError();
}

cudaError_t launch_encode_fwd(const nvc_handle* h, const float* pos, int64_t n, float* feat,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  switch (h->F) {
    case 1: return enc_fwd<1>(h, pos, n, feat, s);
    case 2: return enc_fwd<2>(h, pos, n, feat, s);
    case 4: return enc_fwd<4>(h, pos, n, feat, s);
    case 8: return enc_fwd<8>(h, pos, n, feat, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_encode_bwd(const nvc_handle* h, const float* pos, int64_t n,
                              const float* dfeat, float* grad_table, int32_t* status,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  switch (h->F) {
    case 1: return enc_bwd<1>(h, pos, n, dfeat, grad_table, status, s);
    case 2: return enc_bwd<2>(h, pos, n, dfeat, grad_table, status, s);
    case 4: return enc_bwd<4>(h, pos, n, dfeat, grad_table, status, s);
    case 8: return enc_bwd<8>(h, pos, n, dfeat, grad_table, status, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nvc
