// Declarations shared by the fused shading kernels' translation units: the
// kernel argument block, the weight-image geometry and the sampler's device
// arithmetic.
#pragma once
#include <type_traits>
#include "nvc_internal.cuh"
#include "hashgrid.cuh"
#include "tc_common.cuh"

namespace nvc {
namespace fz {

using namespace tc;

constexpr int kTileM = 128;
constexpr int kMaxLayers = NVC_MAX_HIDDEN_LAYERS + 1;

struct LayerDesc {
  int K;           // reduction size (multiple of 16)
  int N;           // MMA width (multiple of 16)
  int N_real;      // real output neurons of the layer
  int K_real;      // real inputs of the layer
  int w_byte_off;  // offset of the packed matrix in the weight image
  uint32_t idesc;  // tcgen05 instruction descriptor
};

constexpr int kMaxViews = 16;

// One view of a launch: its pixels, outputs and first tile.
struct ViewDesc {
  const float* pos;
  const float* nrm;
  int64_t n;
  int64_t tile_start;   // tiles of earlier views
  int64_t pixel_offset;
  uint32_t view;
  int32_t* idx;
  float* pdf;
  float* wsum;
  float* radiance;
  float* vis_out;
  float* w_out;
};

struct FusedArgs {
  int n_views;
  int64_t n_tiles;
  ViewDesc v[kMaxViews];
  const float* table;
  const __half* table16;     // half-precision copy read instead of `table` (may be NULL)
  EncodeParams ep;
  int F;
  const uint4* wimg;
  int wimg_bytes;
  int n_layers;
  LayerDesc layer[kMaxLayers];
  int kmax;
  float slope;
  int L;
  uint32_t tmem_cols;
  const float* lights;
  uint32_t k0, k1, frame;
  uint2 rkey[10];    // Philox round keys for (k0, k1)
  int32_t* status;
  const float* fp8_scales;   // [0, kMaxLayers): activation scales, [kMaxLayers, 2 kMaxLayers): weight scales
  // warp-specialised layout (byte offsets into shared memory)
  int ws_a0[2], ws_h, ws_c[2], ws_l, ws_bar, ws_cs;
  // monolithic layout: activation tile, light table, mbarrier + TMEM word
  int mono_a, mono_l, mono_bar;
  int pair_x;   // two-threads-per-pixel kernel: the halves' exchange area
  // several-tiles-per-CTA kernel: first activation tile, tile stride, light
  // table, mbarriers; TMEM columns per group
  int multi_a, multi_stride, multi_l, multi_bar, multi_cols;
  // phase profile of the several-tiles-per-CTA kernel (nvc_shade_phases):
  // summed SM cycles of [0] encode, [1] MLP, [2] sampler, [3] whole tile
  // loop, over every group; NULL in ordinary launches
  unsigned long long* phase_cycles;
  // resident CTAs per SM the launch may use (the autotuner's occupancy
  // knob); 0 = as many as fit
  int max_ctas_per_sm;
  // MLP-only launches (nvc_mlp_infer_features): the layer-0 operands,
  // [n][layer[0].K] 16-bit values, read instead of encoding; NULL otherwise
  const uint16_t* feat16;
};

// ---- the encode's chunks of CH features -------------------------------------
// Chunk c of a pixel's layer-0 input (one 16-byte core-matrix row: 8
// 16-bit or 16 E4M3 operands): levels c LPC .. c LPC + LPC - 1 (F divides
// CH), zero beyond the real inputs or for a dead pixel.  TT is the table's
// element type (float32 master or half-precision copy); the fused kernels
// branch on it once per tile, not per level.
template <int F, bool XSMALL, int CH, typename TT>
__device__ __forceinline__ void encode_chunk(const EncodeParams& ep, const TT* table, int c,
                                             int din, float x, float y, float z, bool live,
                                             float (&fv)[CH]) {
  constexpr int LPC = F >= CH ? 1 : CH / F;
#pragma unroll
  for (int s = 0; s < CH; ++s) fv[s] = 0.0f;
  if constexpr (F == 2 && LPC % 2 == 0 && std::is_same<TT, __half>::value) {
    // half-precision rows: two levels' loads in flight at once
    if (live) {
#pragma unroll
      for (int q = 0; q < LPC; q += 2) {
        const int l = c * LPC + q;
        if ((l + 1) * F < din) {
          float acc[4];
          encode_two_levels_h2<XSMALL>(ep, table, l, x, y, z, acc);
#pragma unroll
          for (int f = 0; f < 4; ++f) fv[q * F + f] = acc[f];
        } else if (l * F < din) {
          float acc[F];
          encode_level<F, XSMALL, true, TT>(ep, table, l, x, y, z, acc);
#pragma unroll
          for (int f = 0; f < F; ++f) fv[q * F + f] = acc[f];
        }
      }
    }
    return;
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < LPC; ++q) {
      const int l = c * LPC + q;
      if (l * F < din) {
        float acc[F];
        encode_level<F, XSMALL, true, TT>(ep, table, l, x, y, z, acc);
#pragma unroll
        for (int f = 0; f < F; ++f) fv[q * F + f] = acc[f];
      }
    }
  }
}

// ---- the tile scheduler -------------------------------------------------------
// The persistent shading kernels hand out 128-pixel tiles at run time: a
// tile stream takes its next tile from a ticket counter in the handle's
// status words when it finishes one, so a stream that met cheaper tiles
// takes more of them and the launch ends within about one tile of the mean
// (a fixed round-robin deal left the slowest stream 19% behind the mean at
// 1080p).  The last stream to finish puts the counter back to zero for the
// next launch; the calls on one handle are ordered, so launches never share
// the counter.
__device__ __forceinline__ uint32_t take_tile(int32_t* status) {
  return atomicAdd(reinterpret_cast<uint32_t*>(status + kStTileNext), 1u);
}

__device__ __forceinline__ void finish_tiles(int32_t* status, uint32_t n_streams) {
  __threadfence();
  uint32_t* next = reinterpret_cast<uint32_t*>(status + kStTileNext);
  uint32_t* done = reinterpret_cast<uint32_t*>(status + kStTileDone);
  if (atomicAdd(done, 1u) == n_streams - 1u) {
    atomicExch(next, 0u);
    atomicExch(done, 0u);
  }
}

// ---- the sampler's arithmetic ----------------------------------------------
// The two-threads-per-pixel kernel gives lights [0, H) to one thread and
// [H, L) to the other, H = ceil(L / 2) rounded up to a multiple of 16.
__host__ __device__ __forceinline__ int split_h(int L) { return ((((L + 1) >> 1) + 15) >> 4) << 4; }

// sigma(z) = 1 / (1 + 2^(-z log2(e))) with the hardware's approximate base-2
// exponential and reciprocal (ex2.approx, rcp.approx; subnormals flushed):
// z -> -inf gives 2^inf = inf and 1/inf = 0, z -> +inf gives 1.
__device__ __forceinline__ float sigmoid_fast(float z) {
  const float t = __fmul_rn(z, -1.4426950408889634f);
  float e, v;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(t));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(__fadd_rn(e, 1.0f)));
  return v;
}

// sigmoid_fast of two values, the multiply and the add as packed float32x2
// operations: each lane equals sigmoid_fast of that lane.
__device__ __forceinline__ float2 sigmoid2_fast(float2 z) {
  const float2 t = __fmul2_rn(z, make_float2(-1.4426950408889634f, -1.4426950408889634f));
  float2 e, v;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(t.x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(t.y));
  const float2 d = __fadd2_rn(e, make_float2(1.0f, 1.0f));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(v.x) : "f"(d.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(v.y) : "f"(d.y));
  return v;
}

// Exported visibilities: the sigmoid of N accumulator words (times mul)
// into dst[0 .. min(n, N)).  A full, 16-byte aligned run goes out as N/4
// 16-byte stores; otherwise one checked store per value.
template <int N>
__device__ __forceinline__ void store_sigmoid_row(float* dst, const uint32_t (&r)[N], int n,
                                                  float mul) {
  if (n >= N && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q)
      reinterpret_cast<float4*>(dst)[q] =
          make_float4(sigmoid_fast(__uint_as_float(r[4 * q]) * mul),
                      sigmoid_fast(__uint_as_float(r[4 * q + 1]) * mul),
                      sigmoid_fast(__uint_as_float(r[4 * q + 2]) * mul),
                      sigmoid_fast(__uint_as_float(r[4 * q + 3]) * mul));
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (j < n) dst[j] = sigmoid_fast(__uint_as_float(r[j]) * mul);
  }
}

// Unshadowed contribution of a point light (Lambertian, albedo 1):
// (I/pi) * (n.d) / (|d| * max(|d|^2, 1e-6)) for n.d > 0, with a hardware
// reciprocal square root r of |d|^2 + 1e-30 (the 1e-30 rides in the last
// fused multiply-add; it changes |d|^2 only below about 1e-22, where it
// keeps r finite) and 1 / max(|d|^2, 1e-6) taken as min(r^2, 1e6).
__device__ __forceinline__ float contribution_fast(float px, float py, float pz, float nx,
                                                   float ny, float nz, float4 l) {
  const float dx = l.x - px, dy = l.y - py, dz = l.z - pz;
  const float d2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-30f)));
  const float ndl = fmaf(nx, dx, fmaf(ny, dy, nz * dz));
  const float r = rsqrtf(d2);
  const float inv = fminf(r * r, 1e6f);
  return fmaxf(l.w * ndl * r * inv, 0.0f);   // n.d <= 0 gives c <= 0 -> 0
}

// contribution_fast of two lights at once, lane by lane the same operations
// (x - p as x + (-p)), from a light table staged in pairs, coordinate-major:
// A = {x, x', y, y'}, B = {z, z', I/pi, I'/pi} (stage_light_pairs).
__device__ __forceinline__ float2 contribution2_fast(float2 npx, float2 npy, float2 npz,
                                                     float2 nx2, float2 ny2, float2 nz2,
                                                     float4 A, float4 B) {
  const float2 dx = __fadd2_rn(make_float2(A.x, A.y), npx);
  const float2 dy = __fadd2_rn(make_float2(A.z, A.w), npy);
  const float2 dz = __fadd2_rn(make_float2(B.x, B.y), npz);
  const float2 d2 =
      __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, make_float2(1e-30f, 1e-30f))));
  const float2 ndl = __ffma2_rn(nx2, dx, __ffma2_rn(ny2, dy, __fmul2_rn(nz2, dz)));
  const float2 rq = make_float2(rsqrtf(d2.x), rsqrtf(d2.y));
  const float2 rr = __fmul2_rn(rq, rq);
  const float2 inv = make_float2(fminf(rr.x, 1e6f), fminf(rr.y, 1e6f));
  float2 c = __fmul2_rn(__fmul2_rn(__fmul2_rn(make_float2(B.z, B.w), ndl), rq), inv);
  c.x = fmaxf(c.x, 0.0f);   // n.d <= 0 gives c <= 0 -> 0
  c.y = fmaxf(c.y, 0.0f);
  return c;
}

// Stages the L lights (float4 x, y, z, I) as pairs for contribution2_fast,
// I scaled by 1/pi; an odd count's last slot is zero.  Threads t of
// nthreads share the work; the caller synchronises.
__device__ __forceinline__ void stage_light_pairs(float4* s_pairs, const float* lights, int L,
                                                  int t, int nthreads) {
  const int Lp = (L + 1) & ~1;
  for (int e = t; e < Lp; e += nthreads) {
    float4 l = e < L ? reinterpret_cast<const float4*>(lights)[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    l.w = __fmul_rn(l.w, bits_f(kInvPiBits));
    float* q = reinterpret_cast<float*>(s_pairs) + (e >> 1) * 8 + (e & 1);
    q[0] = l.x;
    q[2] = l.y;
    q[4] = l.z;
    q[6] = l.w;
  }
}

// Per-pixel scales for q = max(1, floor(w 2^(23 - e))), e = ilogb(wmax), by
// exact multiplications only: when wmax < 2^-104 the weights are first
// multiplied by 2^64 (a power of two, so exact, and every w <= wmax stays
// far from overflow); then e' = ilogb(wmax 2^64) = e + 64 and
// w 2^64 2^(23 - e') = w 2^(23 - e), with 2^(23 - e') a normal float.
struct QuantScale {
  float pre, scale;
};
__device__ __forceinline__ QuantScale quant_scale(float wmax) {
  const bool tiny = (__float_as_uint(wmax) >> 23) < 23u;
  const float pre = tiny ? 0x1p64f : 1.0f;
  const uint32_t E = max(__float_as_uint(__fmul_rn(wmax, pre)) >> 23, 23u);
  return {pre, __uint_as_float((277u - E) << 23)};   // 2^(150 - E) = 2^(23 - e')
}

// q = max(1, floor(w * scale)) for w > 0, else 0, with scale = 2^(23 - e)
// from quant_scale (w already multiplied by its `pre`): the product is exact
// whenever it is a normal float, and truncating a subnormal or zero product
// gives 0, which the max(1, .) rule then lifts to 1.
__device__ __forceinline__ uint32_t quantize_scaled(float w, float scale) {
  const uint32_t q = __float2uint_rz(w * scale);
  return (w > 0.0f && q == 0u) ? 1u : q;
}

// One 16-byte core-matrix row of an operand: 8 fp16/bf16 or 16 E4M3 values
// (the latter multiplied by the tensor's scale first).
template <int PREC, int CH>
__device__ __forceinline__ uint4 pack_chunk(const float (&v)[CH], float scale) {
  uint4 pk;
  if constexpr (PREC == NVC_PREC_FP8) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      w[q] = pack_e4m3x2(v[4 * q] * scale, v[4 * q + 1] * scale) |
             (pack_e4m3x2(v[4 * q + 2] * scale, v[4 * q + 3] * scale) << 16);
    pk = make_uint4(w[0], w[1], w[2], w[3]);
  } else {
    pk.x = pack2<PREC>(v[0], v[1]);
    pk.y = pack2<PREC>(v[2], v[3]);
    pk.z = pack2<PREC>(v[4], v[5]);
    pk.w = pack2<PREC>(v[6], v[7]);
  }
  return pk;
}

// Two fp32 pre-activations -> packed 16-bit leaky ReLU (0 <= slope < 1).
template <int PREC>
__device__ __forceinline__ uint32_t leaky2(uint32_t za, uint32_t zb, float slope) {
  if constexpr (PREC == NVC_PREC_FP8) {
    return 0u;   // the E4M3 path converts in fp32 (see the hidden-layer store)
  } else if constexpr (PREC == NVC_PREC_BF16) {
    const __nv_bfloat162 z = __floats2bfloat162_rn(__uint_as_float(za), __uint_as_float(zb));
    const __nv_bfloat162 h = __hmax2(z, __hmul2(z, __float2bfloat162_rn(slope)));
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __half2 z = __floats2half2_rn(__uint_as_float(za), __uint_as_float(zb));
    const __half2 h = __hmax2(z, __hmul2(z, __float2half2_rn(slope)));
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}

// Philox-4x32-10 with the ten round keys (k0 + r W0, k1 + r W1) given: the
// same function as philox4x32_10, the key schedule done once on the host.
__device__ __forceinline__ uint4 philox_keyed(uint4 c, const uint2 (&rk)[10]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk[r].x, lo1, hi0 ^ c.w ^ rk[r].y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint32_t pick_word(uint4 r, int lane) {
  return lane == 0 ? r.x : lane == 1 ? r.y : lane == 2 ? r.z : r.w;
}

// View that tile `tile` belongs to (views are few and tiles sorted by view).
__device__ __forceinline__ int view_of(const FusedArgs& a, int64_t tile) {
  int v = 0;
  while (v + 1 < a.n_views && tile >= a.v[v + 1].tile_start) ++v;
  return v;
}

// Geometry of the tensor-core weight image.
struct PackArgs {
  int n_layers;
  int K[kMaxLayers], N[kMaxLayers], K_real[kMaxLayers], N_real[kMaxLayers];
  int64_t w_off[kMaxLayers];     // float offset of W_k in the parameter vector
  int byte_off[kMaxLayers + 1];  // byte offset of layer k in the image
  int esize;
};

}  // namespace fz

// Shading with several tile streams per CTA (fused_multi.cu); `a` holds the
// other launches' fields, tpc is 2 or 4, L <= 32.
cudaError_t launch_shade_multi(fz::FusedArgs a, const nvc_handle* h, const fz::PackArgs& p, int tpc,
                               bool bf16, cudaStream_t s);

}  // namespace nvc
