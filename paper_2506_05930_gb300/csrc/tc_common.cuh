// tcgen05 / TMEM / mbarrier wrappers (inline PTX for sm_103a), the
// no-swizzle core-matrix operand layout, and the per-(pixel, level) hash-grid
// encode shared by the tensor-core kernels.
#pragma once

#include <cuda_fp8.h>

#include "nvc_internal.cuh"
#include "hashgrid.cuh"

namespace nvc {
namespace tc {

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of the barrier, for at most ~1 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > 1000000000ull) return false;
  }
  return true;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(holder),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start, leading (K-direction)
// and stride (M/N-direction) byte offsets, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  return d;
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// E4M3 x E4M3 -> fp32 (kind::f8f6f4): K = 32 per instruction.
__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Two floats -> two saturating round-to-nearest E4M3 bytes (low = a).
__device__ __forceinline__ uint32_t pack_e4m3x2(float a, float b) {
  return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane; the registers are
// tied to the wait so no use can be scheduled before the load completes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                 "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                 "+r"(r[30]), "+r"(r[31])::"memory");
}

// 16 consecutive fp32 columns of this thread's TMEM lane (same contract as
// tmem_ld32).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])::"memory");
}

// Stores N (16 or 32) 32-bit words of this thread into TMEM columns [taddr,
// taddr + N) of its lane (the 32x32b shape tmem_ld16/32 read) and waits
// until the stores have completed, so a later load of the columns sees them.
// Warp-collective, like the loads.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
        "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]),
        "r"(r[14]), "r"(r[15])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
        "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]),
        "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]),
        "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---- operand packing ------------------------------------------------------
// Byte offset of element (row, k) of a K-major operand with K columns in the
// no-swizzle core-matrix layout.
__host__ __device__ __forceinline__ uint32_t cm_offset(int row, int k, int K, int esize) {
  // a core-matrix row is 16 bytes: 16 / esize elements of K
  const int cpr = 16 / esize;
  return (uint32_t)((row >> 3) * (K * 8 * esize) + (k / cpr) * 128 + (row & 7) * 16 +
                    (k % cpr) * esize);
}

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (PREC == NVC_PREC_BF16) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

// ---- encode of one (pixel, level) ------------------------------------------
// One table row of F half-precision features, widened to float32 (one 2-,
// 4-, 8- or 16-byte load).
__device__ __forceinline__ float2 h2f2(uint32_t u) {
  return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

template <int F>
__device__ __forceinline__ FeatVec<F> load_row(const __half* p) {
  FeatVec<F> r;
  if constexpr (F == 1) {
    r.v[0] = __half2float(__ldg(p));
  } else if constexpr (F == 2) {
    const float2 a = h2f2(__ldg(reinterpret_cast<const unsigned int*>(p)));
    r.v[0] = a.x;
    r.v[1] = a.y;
  } else if constexpr (F == 4) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = h2f2(u.x), b = h2f2(u.y);
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = b.x; r.v[3] = b.y;
  } else {
    static_assert(F == 8, "F is 1, 2, 4 or 8");
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 a = h2f2(w[q]);
      r.v[2 * q] = a.x;
      r.v[2 * q + 1] = a.y;
    }
  }
  return r;
}

template <int F>
__device__ __forceinline__ FeatVec<F> load_row(const float* p) {
  return load_feat<F>(p);
}

// The separate encode kernel's float32 cell and hashed corners, with the
// hash's per-axis terms shared between the corners that use them; rows are
// read from a float32 or a half-precision table (TT).
//   LERP = false: the trilinear blend sum_d w_d v_d with the weights
//     w_d = prod_a (d_a ? f_a : 1 - f_a), corners in order, as the separate
//     encode kernel and the hash-grid backward form it (the training
//     forward uses this, so its features are the ones the backward's
//     corner weights differentiate).
//   LERP = true (inference): for an even number of features, three rounds
//     of linear interpolation, v0 + f (v1 - v0) along x, then y, then z,
//     two features per packed float32x2 operation -- 14 instructions for 8
//     corners instead of 12 weight products and 16 fused multiply-adds;
//     equal to the weighted sum up to rounding.
// The cell of x_hat at level l: the 8 corner rows (within the level's table)
// and the fractions.  (a ^ b ^ c) & m = (a & m) ^ (b & m) ^ (c & m): masking
// the six axis terms leaves one three-input XOR per corner.  XSMALL: the
// caller knows every level's N_l + 1 < T, so the x terms need no mask.
struct LevelCell {
  uint32_t row[8];
  float fx, fy, fz;
};

template <bool XSMALL>
__device__ __forceinline__ LevelCell level_cell(const EncodeParams& ep, int l, float x, float y,
                                                float z) {
  LevelCell c;
  const int n = ep.res[l];
  const float nf = ep.resf[l];
  int cx = __float2int_rd(__fmul_rn(x, nf)), cy = __float2int_rd(__fmul_rn(y, nf)),
      cz = __float2int_rd(__fmul_rn(z, nf));
  cx = min(cx, n - 1);
  cy = min(cy, n - 1);
  cz = min(cz, n - 1);
  c.fx = __fsub_rn(__fmul_rn(x, nf), (float)cx);
  c.fy = __fsub_rn(__fmul_rn(y, nf), (float)cy);
  c.fz = __fsub_rn(__fmul_rn(z, nf), (float)cz);
  const uint32_t mask = (1u << ep.log2_table) - 1u;
  const uint32_t hx[2] = {XSMALL ? (uint32_t)cx : (uint32_t)cx & mask,
                          XSMALL ? (uint32_t)cx + 1u : ((uint32_t)cx + 1u) & mask};
  const uint32_t hy0 = (uint32_t)cy * kPrime1, hz0 = (uint32_t)cz * kPrime2;
  const uint32_t hy[2] = {hy0 & mask, (hy0 + kPrime1) & mask};
  const uint32_t hz[2] = {hz0 & mask, (hz0 + kPrime2) & mask};
#pragma unroll
  for (int d = 0; d < 8; ++d) c.row[d] = hx[d & 1] ^ hy[(d >> 1) & 1] ^ hz[d >> 2];
  return c;
}

// Packed linear interpolation of 8 corners' feature pairs (f, f + 1):
// v0 + f (v1 - v0) along x, then y, then z.
__device__ __forceinline__ float2 lerp_corners(const float2 (&v)[8], float fx, float fy, float fz) {
  const float2 fx2 = make_float2(fx, fx), fy2 = make_float2(fy, fy), fz2 = make_float2(fz, fz);
  float2 e[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) e[k] = __ffma2_rn(fx2, fsub2(v[2 * k + 1], v[2 * k]), v[2 * k]);
  const float2 e0 = __ffma2_rn(fy2, fsub2(e[1], e[0]), e[0]);
  const float2 e1 = __ffma2_rn(fy2, fsub2(e[3], e[2]), e[2]);
  return __ffma2_rn(fz2, fsub2(e1, e0), e0);
}

template <int F, bool XSMALL = false, bool LERP = true, typename TT = float>
__device__ __forceinline__ void encode_level(const EncodeParams& ep, const TT* __restrict__ table,
                                             int l, float x, float y, float z, float (&acc)[F]) {
  const LevelCell c = level_cell<XSMALL>(ep, l, x, y, z);
  const TT* tab = table + ((size_t)l << ep.log2_table) * F;
  FeatVec<F> v[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) v[d] = load_row<F>(tab + (size_t)c.row[d] * F);
  if constexpr (LERP && F % 2 == 0) {
#pragma unroll
    for (int f = 0; f < F; f += 2) {
      float2 vv[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) vv[d] = make_float2(v[d].v[f], v[d].v[f + 1]);
      const float2 r = lerp_corners(vv, c.fx, c.fy, c.fz);
      acc[f] = r.x;
      acc[f + 1] = r.y;
    }
  } else {
    const float gx[2] = {1.0f - c.fx, c.fx}, gy[2] = {1.0f - c.fy, c.fy},
                gz[2] = {1.0f - c.fz, c.fz};
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = 0.0f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const float w = gx[d & 1] * gy[(d >> 1) & 1] * gz[d >> 2];
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f] = fmaf(w, v[d].v[f], acc[f]);
    }
  }
}

// Two levels of a half-precision, two-feature table at once: both cells'
// 16 rows are requested before either is blended, so twice as many row
// loads are in flight.  The rows stay packed half2 words (one register a
// corner) until the blend widens them.  Same results as two encode_level
// calls.
template <bool XSMALL>
__device__ __forceinline__ void encode_two_levels_h2(const EncodeParams& ep,
                                                     const __half* __restrict__ table, int la,
                                                     float x, float y, float z, float (&acc)[4]) {
  const LevelCell ca = level_cell<XSMALL>(ep, la, x, y, z);
  const LevelCell cb = level_cell<XSMALL>(ep, la + 1, x, y, z);
  const unsigned int* ta = reinterpret_cast<const unsigned int*>(table) + ((size_t)la << ep.log2_table);
  const unsigned int* tb = ta + ((size_t)1 << ep.log2_table);
  uint32_t ua[8], ub[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) ua[d] = __ldg(ta + ca.row[d]);
#pragma unroll
  for (int d = 0; d < 8; ++d) ub[d] = __ldg(tb + cb.row[d]);
  float2 va[8], vb[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) va[d] = h2f2(ua[d]);
  const float2 ra = lerp_corners(va, ca.fx, ca.fy, ca.fz);
#pragma unroll
  for (int d = 0; d < 8; ++d) vb[d] = h2f2(ub[d]);
  const float2 rb = lerp_corners(vb, cb.fx, cb.fy, cb.fz);
  acc[0] = ra.x;
  acc[1] = ra.y;
  acc[2] = rb.x;
  acc[3] = rb.y;
}

}  // namespace tc
}  // namespace nvc
