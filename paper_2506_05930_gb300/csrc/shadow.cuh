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

// ---- the occluders as the tests read them -----------------------------------
// Kernels stage the scene's occluders in shared memory in this layout:
//   sphere pairs, 32 bytes each: float4 {cx_a, cx_b, cy_a, cy_b}, float4
//   {cz_a, cz_b, r_a^2, r_b^2} (r^2 = fl(r r)); an odd count's last slot is
//   a sphere with r^2 = -1, which blocks nothing;
//   boxes, 24 bytes each: (lo_x, hi_x), (lo_y, hi_y), (lo_z, hi_z).
// A slab's two planes go through each packed float32x2 subtraction and
// multiplication (Blackwell's sub/mul.rn.f32x2), each lane the correctly
// rounded operation of the scalar test; the sphere pairs are read with two
// 16-byte loads and tested lane by lane in scalar operations.
struct Occluders {
  const float4* sph;   // 2 float4 per sphere pair
  int n_pairs;
  const float2* box;   // 3 float2 per box
  int n_box;
};

__host__ __device__ __forceinline__ size_t occluder_bytes(int n_sph, int n_box) {
  return 32 * (size_t)((n_sph + 1) / 2) + 24 * (size_t)n_box;
}

// Stages the occluders at dst (16-byte aligned; occluder_bytes(...) long),
// threads tid of nthreads sharing the work; the caller synchronises.
__device__ __forceinline__ Occluders stage_occluders(const float* __restrict__ spheres, int n_sph,
                                                     const float* __restrict__ boxes, int n_box,
                                                     void* dst, int tid, int nthreads) {
  Occluders o;
  float* f = static_cast<float*>(dst);
  o.sph = reinterpret_cast<const float4*>(dst);
  o.n_pairs = (n_sph + 1) / 2;
  for (int e = tid; e < 2 * o.n_pairs; e += nthreads) {
    const int pair = e >> 1, lane = e & 1;
    float4 sp = make_float4(0.0f, 0.0f, 0.0f, -1.0f);   // r^2 = -1: blocks nothing
    if (e < n_sph) {
      sp = reinterpret_cast<const float4*>(spheres)[e];
      sp.w = __fmul_rn(sp.w, sp.w);
    }
    float* q = f + 8 * pair + lane;
    q[0] = sp.x;
    q[2] = sp.y;
    q[4] = sp.z;
    q[6] = sp.w;
  }
  float* b = f + 8 * o.n_pairs;
  for (int e = tid; e < n_box; e += nthreads) {
    const float* src = boxes + 6 * e;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      b[6 * e + 2 * a] = src[a];
      b[6 * e + 2 * a + 1] = src[3 + a];
    }
  }
  o.box = reinterpret_cast<const float2*>(b);
  o.n_box = n_box;
  return o;
}

// The view of occluders already staged at src (as stage_occluders left them).
__device__ __forceinline__ Occluders staged_occluders(const void* src, int n_sph, int n_box) {
  Occluders o;
  o.sph = reinterpret_cast<const float4*>(src);
  o.n_pairs = (n_sph + 1) / 2;
  o.box = reinterpret_cast<const float2*>(static_cast<const float*>(src) + 8 * o.n_pairs);
  o.n_box = n_box;
  return o;
}

// ---- the tests ----------------------------------------------------------------
// The divisions are taken once per (position, light): 1/|d|^2 for the
// spheres' closest-point parameter and 1/d per axis for the boxes' slabs;
// each occluder then costs multiplications only.  Sphere (c, r): the
// segment's closest point q = x + t_c d, t_c = clamp(((c - x).d) / |d|^2,
// t0, t1), blocks when |c - q|^2 < r^2.

// One sphere of a staged pair (lane 0 or 1), in scalar correctly rounded
// operations: the compiler fuses a packed multiply into a following packed
// add (one rounding instead of two) even when both carry .rn, so products
// that feed sums stay scalar here.
__device__ __forceinline__ bool sphere_lane_blocks(float px, float py, float pz, float dx,
                                                   float dy, float dz, float inv_dd, float cx,
                                                   float cy, float cz, float r2) {
  const float t0 = bits_f(kSegT0Bits), t1 = bits_f(kSegT1Bits);
  const float ox = __fsub_rn(cx, px), oy = __fsub_rn(cy, py), oz = __fsub_rn(cz, pz);
  float tc = __fmul_rn(dot3_rn(ox, oy, oz, dx, dy, dz), inv_dd);
  tc = fminf(fmaxf(tc, t0), t1);
  const float ex = __fsub_rn(cx, __fadd_rn(px, __fmul_rn(tc, dx)));
  const float ey = __fsub_rn(cy, __fadd_rn(py, __fmul_rn(tc, dy)));
  const float ez = __fsub_rn(cz, __fadd_rn(pz, __fmul_rn(tc, dz)));
  return dot3_rn(ex, ey, ez, ex, ey, ez) < r2;
}

// Two spheres: A = {cx_a, cx_b, cy_a, cy_b}, B = {cz_a, cz_b, r_a^2, r_b^2}.
__device__ __forceinline__ bool sphere_pair_blocks(float px, float py, float pz, float dx,
                                                   float dy, float dz, float inv_dd, float4 A,
                                                   float4 B) {
  return sphere_lane_blocks(px, py, pz, dx, dy, dz, inv_dd, A.x, A.z, B.x, B.z) ||
         sphere_lane_blocks(px, py, pz, dx, dy, dz, inv_dd, A.y, A.w, B.y, B.w);
}

// Closed slab test of one box when no component of d is zero: the entry and
// exit parameters (lo - x) / d and (hi - x) / d of every axis, two per
// packed operation; blocked when max(t0, nearer planes) <= min(t1, farther).
__device__ __forceinline__ bool box_blocks_oblique(float2 px, float2 py, float2 pz, float2 ix,
                                                   float2 iy, float2 iz, const float2* b) {
  const float2 tx = fmul2_rn(fsub2(b[0], px), ix);
  const float2 ty = fmul2_rn(fsub2(b[1], py), iy);
  const float2 tz = fmul2_rn(fsub2(b[2], pz), iz);
  const float tmin = fmaxf(fmaxf(fmaxf(bits_f(kSegT0Bits), fminf(tx.x, tx.y)), fminf(ty.x, ty.y)),
                           fminf(tz.x, tz.y));
  const float tmax = fminf(fminf(fminf(bits_f(kSegT1Bits), fmaxf(tx.x, tx.y)), fmaxf(ty.x, ty.y)),
                           fmaxf(tz.x, tz.y));
  return tmin <= tmax;
}

// The same test with any component of d zero: that axis only checks that x
// lies between its planes.
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

__device__ __forceinline__ bool box_blocks_general(float px, float py, float pz, float dx, float dy,
                                                   float dz, float ix, float iy, float iz,
                                                   const float2* b) {
  float tmin = bits_f(kSegT0Bits), tmax = bits_f(kSegT1Bits);
  bool miss = false;
  slab(px, dx, ix, b[0].x, b[0].y, tmin, tmax, miss);
  slab(py, dy, iy, b[1].x, b[1].y, tmin, tmax, miss);
  slab(pz, dz, iz, b[2].x, b[2].y, tmin, tmax, miss);
  return !miss && tmin <= tmax;
}

// Whether the segment from (px, py, pz) to the light at (lx, ly, lz) is
// blocked by one of the staged occluders.
__device__ __forceinline__ bool segment_blocked(float px, float py, float pz, float lx, float ly,
                                                float lz, const Occluders& occ) {
  const float dx = __fsub_rn(lx, px), dy = __fsub_rn(ly, py), dz = __fsub_rn(lz, pz);
  const float dd = dot3_rn(dx, dy, dz, dx, dy, dz);
  // a zero-length segment (light on the point): t stays at t0
  const float inv_dd = dd > 0.0f ? __fdiv_rn(1.0f, dd) : 0.0f;
  const float ix = dx != 0.0f ? __fdiv_rn(1.0f, dx) : 0.0f;
  const float iy = dy != 0.0f ? __fdiv_rn(1.0f, dy) : 0.0f;
  const float iz = dz != 0.0f ? __fdiv_rn(1.0f, dz) : 0.0f;
  const float2 px2 = make_float2(px, px), py2 = make_float2(py, py), pz2 = make_float2(pz, pz);
  bool blocked = false;
  for (int k = 0; k < occ.n_pairs && !blocked; ++k)
    blocked = sphere_pair_blocks(px, py, pz, dx, dy, dz, inv_dd, occ.sph[2 * k], occ.sph[2 * k + 1]);
  if (blocked) return true;
  if (dx != 0.0f && dy != 0.0f && dz != 0.0f) {
    const float2 ix2 = make_float2(ix, ix), iy2 = make_float2(iy, iy), iz2 = make_float2(iz, iz);
    for (int k = 0; k < occ.n_box && !blocked; ++k)
      blocked = box_blocks_oblique(px2, py2, pz2, ix2, iy2, iz2, occ.box + 3 * k);
  } else {
    for (int k = 0; k < occ.n_box && !blocked; ++k)
      blocked = box_blocks_general(px, py, pz, dx, dy, dz, ix, iy, iz, occ.box + 3 * k);
  }
  return blocked;
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
