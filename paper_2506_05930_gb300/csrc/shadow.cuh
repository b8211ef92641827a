// Binary shadow rays against the analytic occluders (Section 3.4 targets,
// the shading pass of Section 3.1 and the all-lights reference of Section
// 4.4 share them).  The segment x + t d, t in [1e-4, 1 - 1e-4], d = l - x,
// is blocked by a sphere whose centre is strictly closer than its radius to
// the segment, or by a box the segment meets (closed slab test).  The
// arithmetic is correctly rounded float32 in a fixed order, so the binary
// decision is reproducible operation by operation.
#pragma once
#include "nvc_internal.cuh"

namespace nvc {

// The divisions are taken once per (position, light): 1/|d|^2 for the
// spheres' closest-point parameter and 1/d per axis for the boxes' slabs;
// each occluder then costs multiplications only.
__device__ __forceinline__ bool sphere_blocks(float px, float py, float pz, float dx, float dy,
                                              float dz, float inv_dd, float4 s) {
  const float t0 = bits_f(kSegT0Bits), t1 = bits_f(kSegT1Bits);
  const float ox = __fsub_rn(s.x, px), oy = __fsub_rn(s.y, py), oz = __fsub_rn(s.z, pz);
  float tc = __fmul_rn(dot3_rn(ox, oy, oz, dx, dy, dz), inv_dd);
  tc = fminf(fmaxf(tc, t0), t1);
  const float ex = __fsub_rn(s.x, __fadd_rn(px, __fmul_rn(tc, dx)));
  const float ey = __fsub_rn(s.y, __fadd_rn(py, __fmul_rn(tc, dy)));
  const float ez = __fsub_rn(s.z, __fadd_rn(pz, __fmul_rn(tc, dz)));
  return dot3_rn(ex, ey, ez, ex, ey, ez) < __fmul_rn(s.w, s.w);
}

__device__ __forceinline__ void slab(float xa, float da, float inv_da, float lo, float hi,
                                     float& tmin, float& tmax, bool& miss) {
  if (da == 0.0f) {
    miss = miss || xa < lo || xa > hi;
    return;
  }
  const float ta = __fmul_rn(__fsub_rn(lo, xa), inv_da);
  const float tb = __fmul_rn(__fsub_rn(hi, xa), inv_da);
  tmin = fmaxf(tmin, fminf(ta, tb));
  tmax = fminf(tmax, fmaxf(ta, tb));
}

__device__ __forceinline__ bool box_blocks(float px, float py, float pz, float dx, float dy,
                                           float dz, float ix, float iy, float iz,
                                           const float* b) {
  float tmin = bits_f(kSegT0Bits), tmax = bits_f(kSegT1Bits);
  bool miss = false;
  slab(px, dx, ix, b[0], b[3], tmin, tmax, miss);
  slab(py, dy, iy, b[1], b[4], tmin, tmax, miss);
  slab(pz, dz, iz, b[2], b[5], tmin, tmax, miss);
  return !miss && tmin <= tmax;
}

// Whether the segment from (px, py, pz) to the light at (lx, ly, lz) is
// blocked by one of the staged occluders (spheres as float4 centre + radius,
// boxes as 6 floats lo, hi).
__device__ __forceinline__ bool segment_blocked(float px, float py, float pz, float lx, float ly,
                                                float lz, const float4* sph, int n_sph,
                                                const float* box, int n_box) {
  const float dx = __fsub_rn(lx, px), dy = __fsub_rn(ly, py), dz = __fsub_rn(lz, pz);
  const float dd = dot3_rn(dx, dy, dz, dx, dy, dz);
  const float inv_dd = dd > 0.0f ? __fdiv_rn(1.0f, dd) : 0.0f;
  const float ix = dx != 0.0f ? __fdiv_rn(1.0f, dx) : 0.0f;
  const float iy = dy != 0.0f ? __fdiv_rn(1.0f, dy) : 0.0f;
  const float iz = dz != 0.0f ? __fdiv_rn(1.0f, dz) : 0.0f;
  bool occ = false;
  for (int k = 0; k < n_sph && !occ; ++k)
    occ = sphere_blocks(px, py, pz, dx, dy, dz, inv_dd, sph[k]);
  for (int k = 0; k < n_box && !occ; ++k)
    occ = box_blocks(px, py, pz, dx, dy, dz, ix, iy, iz, box + 6 * k);
  return occ;
}

// ---- training positions (Section 3.4) ------------------------------------------
// Samples [0, n_world) are uniform in the world box (stream tag 1); the rest
// copy G-buffer pixel floor(r * n_screen / 2^32) (stream tag 2).
struct PosGen {
  float3 lo, ext;
  const float* screen;
  int64_t n_screen, n_world;
  uint32_t k0, k1, frame;
};

__device__ __forceinline__ float3 training_position(int64_t j, const PosGen& g) {
  if (j < g.n_world) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)j, g.frame, 0u, kTagWorld), g.k0, g.k1);
    return make_float3(__fadd_rn(g.lo.x, __fmul_rn(uniform24(r.x), g.ext.x)),
                       __fadd_rn(g.lo.y, __fmul_rn(uniform24(r.y), g.ext.y)),
                       __fadd_rn(g.lo.z, __fmul_rn(uniform24(r.z), g.ext.z)));
  }
  const uint32_t s = (uint32_t)(j - g.n_world);
  const uint4 r = philox4x32_10(make_uint4(s, g.frame, 0u, kTagScreen), g.k0, g.k1);
  const int64_t pix = (int64_t)(((uint64_t)r.x * (uint64_t)g.n_screen) >> 32);
  return make_float3(g.screen[3 * pix], g.screen[3 * pix + 1], g.screen[3 * pix + 2]);
}

// The generator of a training batch (train.cu): n_world = -1 for the
// default split ceil(batch / 2); every position is world space without
// screen positions.
PosGen pos_gen(const nvc_scene* sc, const float* screen_pos, int64_t n_screen, int64_t batch,
               uint64_t seed, uint32_t frame, int64_t n_world);

}  // namespace nvc
