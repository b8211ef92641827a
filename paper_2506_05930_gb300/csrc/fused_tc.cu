// The per-pixel hot path in one kernel: hash-grid encode -> MLP on the
// 5th-generation tensor cores (tcgen05, accumulators in TMEM) -> sigmoid ->
// light weights -> weighted reservoir sampling + Neural DI (Sections 3.1 to
// 3.3 of the paper).
//
// Layout.  One CTA = 128 threads = one 128-pixel tile at a time (persistent
// over tiles); thread t owns pixel row t, which is also TMEM lane t of the
// M = 128 accumulator, so every thread encodes its own pixel, reads its own
// row of every layer's output and runs its own pixel's sampler.  Operands
// live in shared memory in the no-swizzle K-major core-matrix layout (8 rows
// x 16 bytes per core matrix; the K-adjacent core matrix 128 bytes on, the
// next 8-row group K*2*8 bytes on).  All layers' weights are loaded once
// per CTA; the activation tile is rewritten in place between layers.  One
// elected thread issues the layer's tcgen05.mma (M=128, N=layer width, fp32
// accumulate; K/16 of kind::f16 for fp16 / bf16 operands, K/32 of
// kind::f8f6f4 for scaled E4M3) and commits to an mbarrier.
// Several CTAs per SM overlap one CTA's gathers with another's MMAs and
// sampler arithmetic; the TMEM columns per CTA are a power of two and the
// CTAs per SM are capped so that their columns fit the 512 available.
//
// Every wait on the mbarrier is bounded (about one second); a timeout sets
// an error flag in the handle's status and every thread of the CTA leaves
// the tile loop together, freeing TMEM on the way out.
//
// Two other kernels compute the same function for the autotuner: a
// warp-specialised one (producer warps encode the next tile while consumer
// warps run the MLP and the sampler) and one with two threads per pixel
// (256-thread CTAs splitting levels, columns and lights).
#include "nvc_internal.cuh"
#include "hashgrid.cuh"
#include "tc_common.cuh"
#include "fused_common.cuh"

namespace nvc {

namespace {

using namespace tc;
using namespace fz;

// ---- the kernel ----------------------------------------------------------------
template <int F, int PREC, bool LSMALL>
__global__ void __launch_bounds__(kTileM, 5) fused_shade_kernel(const __grid_constant__ FusedArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // offsets computed by the host (fused_smem), which sized the allocation
  uint8_t* s_w = smem;
  uint8_t* s_a = smem + a.mono_a;
  float4* s_l = reinterpret_cast<float4*>(smem + a.mono_l);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.mono_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + 1);
  uint32_t* s_next = s_tmem + 1;   // the CTA's next tile
  const int t = threadIdx.x;
  const int warp = t >> 5;

  for (int e = t; e < a.wimg_bytes / 16; e += kTileM)
    reinterpret_cast<uint4*>(s_w)[e] = a.wimg[e];
  if (a.lights) stage_light_pairs(s_l, a.lights, a.L, t, kTileM);
  const uint32_t bar = smem_u32(s_bar);
  if (t == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(s_tmem), a.tmem_cols);
  if (t == 0) *s_next = take_tile(a.status);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t a_base = smem_u32(s_a);
  const uint32_t w_base = smem_u32(s_w);
  uint32_t phase = 0;
  bool failed = false;

  constexpr bool kF8 = PREC == NVC_PREC_FP8;
  constexpr int CH = kF8 ? 16 : 8;     // operand elements per 16-byte core-matrix row
  constexpr int ES = kF8 ? 1 : 2;      // bytes per operand element
  constexpr int KS = kF8 ? 32 : 16;    // K per MMA instruction
  // E4M3: layer k's accumulator times s_mult[k] is the next layer's scaled
  // input (or, for the last layer, the logit)
  __shared__ float s_mult[kMaxLayers];
  float s_in0 = 1.0f;
  if constexpr (kF8) {
    const float* sa = a.fp8_scales;
    const float* sw = a.fp8_scales + kMaxLayers;
    s_in0 = sa[0];
    if (t < a.n_layers)
      s_mult[t] = (t + 1 < a.n_layers ? sa[t + 1] : 1.0f) / (sa[t] * sw[t]);
    __syncthreads();
  }

  const int din = a.ep.n_levels * F;
  const int K0 = a.layer[0].K;
  const int64_t n_tiles = a.n_tiles;

  for (int64_t tile = *s_next; tile < n_tiles && !failed; tile = *s_next) {
    const ViewDesc& V = a.v[view_of(a, tile)];
    const int64_t row = (tile - V.tile_start) * kTileM + t;
    const bool live = row < V.n;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (live) {
      px = __ldg(V.pos + 3 * row);
      py = __ldg(V.pos + 3 * row + 1);
      pz = __ldg(V.pos + 3 * row + 2);
    }
    // ---- encode this pixel into the layer-0 A tile ------------------------
    {
      const float x = normalise(px, a.ep.lo[0], a.ep.ext[0]);
      const float y = normalise(py, a.ep.lo[1], a.ep.ext[1]);
      const float z = normalise(pz, a.ep.lo[2], a.ep.ext[2]);
      auto encode_all = [&](const auto* tab) {
        for (int c = 0; c < K0 / CH; ++c) {
          float fv[CH];
          encode_chunk<F, false, CH>(a.ep, tab, c, din, x, y, z, live, fv);
          *reinterpret_cast<uint4*>(s_a + cm_offset(t, c * CH, K0, ES)) =
              pack_chunk<PREC, CH>(fv, s_in0);
        }
      };
      if (a.table16)
        encode_all(a.table16);
      else
        encode_all(a.table);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();

    // ---- the MLP, layer by layer --------------------------------------------
    for (int k = 0; k < a.n_layers && !failed; ++k) {
      const LayerDesc ld = a.layer[k];
      if (t == 0) {
        tc_fence_after();
        const uint32_t sbo = (uint32_t)ld.K * 8u * ES;
        const uint32_t wb = w_base + (uint32_t)ld.w_byte_off;
        for (int kk = 0; kk < ld.K / KS; ++kk) {
          if constexpr (kF8)
            mma_f8(tmem, smem_desc(a_base + kk * 256, 128, sbo),
                   smem_desc(wb + kk * 256, 128, sbo), ld.idesc, kk > 0 ? 1u : 0u);
          else
            mma_f16(tmem, smem_desc(a_base + kk * 256, 128, sbo),
                    smem_desc(wb + kk * 256, 128, sbo), ld.idesc, kk > 0 ? 1u : 0u);
        }
        mma_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      tc_fence_after();
      if (k + 1 < a.n_layers) {
        // hidden activation -> operand A of the next layer (K = this N)
        const int Kn = ld.N;
        for (int c0 = 0; c0 < ld.N; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(t_lane + (uint32_t)c0, r);
          if constexpr (kF8) {
            // leaky ReLU is positively homogeneous: leaky(m z) = m leaky(z)
            const float m = s_mult[k];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              float v[16];
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const float zz = __uint_as_float(r[g * 16 + q]) * m;
                v[q] = fmaxf(zz, a.slope * zz);
              }
              if (c0 + g * 16 < Kn)
                *reinterpret_cast<uint4*>(s_a + cm_offset(t, c0 + g * 16, Kn, 1)) =
                    pack_chunk<PREC, 16>(v, 1.0f);
            }
          } else {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              // convert pairs, then leaky ReLU max(z, slope z) in packed 16-bit math
              uint4 pk;
              pk.x = leaky2<PREC>(r[g * 8 + 0], r[g * 8 + 1], a.slope);
              pk.y = leaky2<PREC>(r[g * 8 + 2], r[g * 8 + 3], a.slope);
              pk.z = leaky2<PREC>(r[g * 8 + 4], r[g * 8 + 5], a.slope);
              pk.w = leaky2<PREC>(r[g * 8 + 6], r[g * 8 + 7], a.slope);
              if (c0 + g * 8 < Kn)
                *reinterpret_cast<uint4*>(s_a + cm_offset(t, c0 + g * 8, Kn, 2)) = pk;
            }
          }
        }
        fence_async_smem();
        tc_fence_before();
        failed = __syncthreads_or(!ok) != 0;
        continue;
      }

      // ---- output layer: sigmoid, light weights, WRS, Neural DI -------------
      const int L = LSMALL ? (a.L < 32 ? a.L : 32) : a.L;
      const float outmul = kF8 ? s_mult[a.n_layers - 1] : 1.0f;
      if (V.vis_out) {
        for (int c0 = 0; c0 < L; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(t_lane + (uint32_t)c0, r);
          if (live) store_sigmoid_row<32>(V.vis_out + row * L + c0, r, L - c0, outmul);
        }
      } else {
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (live) {
          nx = __ldg(V.nrm + 3 * row);
          ny = __ldg(V.nrm + 3 * row + 1);
          nz = __ldg(V.nrm + 3 * row + 2);
        }
        float wreg[32];
        float wmax = 0.0f, sum = 0.0f, di = 0.0f;
        const float2 npx = make_float2(-px, -px), npy = make_float2(-py, -py),
                     npz = make_float2(-pz, -pz);
        const float2 nx2 = make_float2(nx, nx), ny2 = make_float2(ny, ny), nz2 = make_float2(nz, nz);
        for (int c0 = 0; c0 < L; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(t_lane + (uint32_t)c0, r);
          // two lights per packed operation (pair (c0 + j) / 2 of the table)
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            const int i = c0 + j;
            wreg[j] = 0.0f;
            wreg[j + 1] = 0.0f;
            if (i < L) {
              const float2 c = contribution2_fast(npx, npy, npz, nx2, ny2, nz2, s_l[i], s_l[i + 1]);
              const float v0 = sigmoid_fast(__uint_as_float(r[j]) * outmul);
              const float w0 = __fmul_rn(fmaxf(v0, bits_f(kVisClampBits)), c.x);
              wmax = fmaxf(wmax, w0);
              sum += w0;
              di = fmaf(v0, c.x, di);
              wreg[j] = w0;
              if (i + 1 < L) {
                const float v1 = sigmoid_fast(__uint_as_float(r[j + 1]) * outmul);
                const float w1 = __fmul_rn(fmaxf(v1, bits_f(kVisClampBits)), c.y);
                wmax = fmaxf(wmax, w1);
                sum += w1;
                di = fmaf(v1, c.y, di);
                wreg[j + 1] = w1;
              }
            }
          }
          if (V.w_out != nullptr && live) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (c0 + j < L) V.w_out[row * L + c0 + j] = wreg[j];
          }
          if (!LSMALL) {
            // the weights replace their logits in the (now read) output
            // accumulator, so the pick pass reads them instead of computing
            // them again
            uint32_t wb[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) wb[j] = __float_as_uint(wreg[j]);
            tmem_st32(t_lane + (uint32_t)c0, wb);
          }
        }
        int sel = -1;
        float wsel = 0.0f;
        // tcgen05.ld is warp-collective: the chunk loop runs in every thread,
        // the per-pixel work only where there is something to pick
        const bool active = live && wmax > 0.0f;
        const QuantScale qs = quant_scale(wmax);
        // the pick runs on pre-scaled weights; pdf = (pre w_sel) / (pre sum)
        // is the same correctly rounded quotient (pre is a power of two)
        const float sum_q = __fmul_rn(sum, qs.pre);
        if (LSMALL && active && qs.pre != 1.0f) {
#pragma unroll
          for (int j = 0; j < 32; ++j) wreg[j] = __fmul_rn(wreg[j], qs.pre);
        }
        const uint32_t pixel = (uint32_t)(V.pixel_offset + row);
        uint32_t Q = 0;
        uint4 rr = make_uint4(0, 0, 0, 0);
        for (int c0 = 0; c0 < L; c0 += 32) {
          uint32_t r[32];
          if (!LSMALL) tmem_ld32(t_lane + (uint32_t)c0, r);
          if (active) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int i = c0 + j;
              if (i < L) {
                float w = wreg[j];
                if (!LSMALL) w = __fmul_rn(__uint_as_float(r[j]), qs.pre);
                if ((i & 3) == 0)
                  rr = philox_keyed(make_uint4(pixel, a.frame, V.view,
                                               ((uint32_t)(i >> 2) << 4) | kTagWrs),
                                    a.rkey);
                const uint32_t q = quantize_scaled(w, qs.scale);
                Q += q;
                // r*Q < q*2^32  <=>  hi32(r*Q) < q  (Q < 2^32); false for q = 0
                if (__umulhi(pick_word(rr, i & 3), Q) < q) {
                  sel = i;
                  wsel = w;
                }
              }
            }
          }
        }
        if (live) {
          if (V.idx) V.idx[row] = sel;
          if (V.pdf) V.pdf[row] = sel >= 0 ? wsel / sum_q : 0.0f;
          if (V.wsum) V.wsum[row] = sum;
          if (V.radiance) V.radiance[row] = di;
        }
      }
      if (t == 0) *s_next = take_tile(a.status);
      tc_fence_before();
      failed = __syncthreads_or(!ok) != 0;   // also publishes *s_next
    }
  }
  if (failed && t == 0) atomicOr(a.status + kStFlags, kFlagTimeout);
  if (t == 0) finish_tiles(a.status, gridDim.x);
  __syncthreads();
  if (failed) mbar_wait_bounded(bar, phase ^ 1u);   // let an MMA in flight land
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

// ---- two threads per pixel (256 threads, 128-pixel tiles) -------------------
// Thread t serves pixel row t % 128 (TMEM lane; warps w and w + 4 read the
// same 32 lanes) and half h = t / 128 of that pixel's work: every other
// 8-feature chunk of the encode, every other 32-column chunk of each hidden
// epilogue, and lights [0, H) or [H, L) of the sampler (H = the half of L
// rounded up to 16).  The halves meet in shared memory three times per
// tile, each time behind a 64-thread named barrier of the warp pair:
//   1. max w, sum w and Neural DI of each half -> both halves;
//   2. Q_A, the first half's integer weight total -> the second half, whose
//      prefix sums start there (so every Q_i is the one-thread value);
//   3. the second half's pick, which wins when there is one (it is the
//      later light) -> the first half, which writes the pixel's outputs.
// Sum w and Neural DI are the first half's sum plus the second half's, so
// they can differ from the other variants' one-pass sums in the last bits;
// the picks are the same integers from the same float32 weights.
// (constant barrier ids, so the CTA holds five hardware barriers, not 16)
__device__ __forceinline__ void pair_sync(int warp) {
  switch (warp & 3) {
    case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
  }
}

template <int F, int PREC, bool HSMALL>
__global__ void __launch_bounds__(2 * kTileM, 3) fused_shade_pair_kernel(const __grid_constant__ FusedArgs a) {
  constexpr int kThreads = 2 * kTileM;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* s_w = smem;
  uint8_t* s_a = smem + a.mono_a;
  float4* s_l = reinterpret_cast<float4*>(smem + a.mono_l);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.mono_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + 1);
  uint32_t* s_next = s_tmem + 1;                                     // the CTA's next tile
  float4* s_x = reinterpret_cast<float4*>(smem + a.pair_x);          // [2][128] partials
  uint32_t* s_q = reinterpret_cast<uint32_t*>(s_x + 2 * kTileM);     // [2][128] parts of Q_A
  int2* s_s = reinterpret_cast<int2*>(s_q + 2 * kTileM);             // [128] (sel, w_sel bits) of half 1
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int rw = t & (kTileM - 1);
  const int half = t >> 7;

  for (int e = t; e < a.wimg_bytes / 16; e += kThreads)
    reinterpret_cast<uint4*>(s_w)[e] = a.wimg[e];
  if (a.lights) stage_light_pairs(s_l, a.lights, a.L, t, kThreads);
  const uint32_t bar = smem_u32(s_bar);
  if (t == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(s_tmem), a.tmem_cols);
  if (t == 0) *s_next = take_tile(a.status);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t t_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t a_base = smem_u32(s_a);
  const uint32_t w_base = smem_u32(s_w);
  uint32_t phase = 0;
  bool failed = false;

  constexpr bool kF8 = PREC == NVC_PREC_FP8;
  constexpr int CH = kF8 ? 16 : 8;     // operand elements per 16-byte core-matrix row
  constexpr int ES = kF8 ? 1 : 2;      // bytes per operand element
  constexpr int KS = kF8 ? 32 : 16;    // K per MMA instruction
  // E4M3: layer k's accumulator times s_mult[k] is the next layer's scaled
  // input (or, for the last layer, the logit), as in the monolithic kernel
  __shared__ float s_mult[kMaxLayers];
  float s_in0 = 1.0f;
  if constexpr (kF8) {
    const float* sa = a.fp8_scales;
    const float* sw = a.fp8_scales + kMaxLayers;
    s_in0 = sa[0];
    if (t < a.n_layers)
      s_mult[t] = (t + 1 < a.n_layers ? sa[t + 1] : 1.0f) / (sa[t] * sw[t]);
    __syncthreads();
  }
  const int din = a.ep.n_levels * F;
  const int K0 = a.layer[0].K;
  const int64_t n_tiles = a.n_tiles;
  const int L = a.L;
  const int H = split_h(L);   // first half: lights [0, H)
  const int lo = half ? H : 0;
  const int hi = half ? L : (H < L ? H : L);

  for (int64_t tile = *s_next; tile < n_tiles && !failed; tile = *s_next) {
    const ViewDesc& V = a.v[view_of(a, tile)];
    const int64_t row = (tile - V.tile_start) * kTileM + rw;
    const bool live = row < V.n;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (live) {
      px = __ldg(V.pos + 3 * row);
      py = __ldg(V.pos + 3 * row + 1);
      pz = __ldg(V.pos + 3 * row + 2);
    }
    // ---- encode: this half's 8-feature chunks of the layer-0 A tile -------
    {
      const float x = normalise(px, a.ep.lo[0], a.ep.ext[0]);
      const float y = normalise(py, a.ep.lo[1], a.ep.ext[1]);
      const float z = normalise(pz, a.ep.lo[2], a.ep.ext[2]);
      auto encode_half = [&](const auto* tab) {
        for (int c = half; c < K0 / CH; c += 2) {
          float fv[CH];
          encode_chunk<F, false, CH>(a.ep, tab, c, din, x, y, z, live, fv);
          *reinterpret_cast<uint4*>(s_a + cm_offset(rw, c * CH, K0, ES)) =
              pack_chunk<PREC, CH>(fv, s_in0);
        }
      };
      if (a.table16)
        encode_half(a.table16);
      else
        encode_half(a.table);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();

    // ---- the MLP -------------------------------------------------------------
    for (int k = 0; k < a.n_layers && !failed; ++k) {
      const LayerDesc ld = a.layer[k];
      if (t == 0) {
        tc_fence_after();
        const uint32_t sbo = (uint32_t)ld.K * 8u * ES;
        const uint32_t wb = w_base + (uint32_t)ld.w_byte_off;
        for (int kk = 0; kk < ld.K / KS; ++kk) {
          if constexpr (kF8)
            mma_f8(tmem, smem_desc(a_base + kk * 256, 128, sbo), smem_desc(wb + kk * 256, 128, sbo),
                   ld.idesc, kk > 0 ? 1u : 0u);
          else
            mma_f16(tmem, smem_desc(a_base + kk * 256, 128, sbo),
                    smem_desc(wb + kk * 256, 128, sbo), ld.idesc, kk > 0 ? 1u : 0u);
        }
        mma_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      tc_fence_after();
      if (k + 1 < a.n_layers) {
        const int Kn = ld.N;
        for (int c0 = half * 32; c0 < ld.N; c0 += 64) {
          uint32_t r[32];
          tmem_ld32(t_lane + (uint32_t)c0, r);
          if constexpr (kF8) {
            // leaky ReLU is positively homogeneous: leaky(m z) = m leaky(z)
            const float m = s_mult[k];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              float v[16];
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const float zz = __uint_as_float(r[g * 16 + q]) * m;
                v[q] = fmaxf(zz, a.slope * zz);
              }
              if (c0 + g * 16 < Kn)
                *reinterpret_cast<uint4*>(s_a + cm_offset(rw, c0 + g * 16, Kn, 1)) =
                    pack_chunk<PREC, 16>(v, 1.0f);
            }
          } else {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              uint4 pk;
              pk.x = leaky2<PREC>(r[g * 8 + 0], r[g * 8 + 1], a.slope);
              pk.y = leaky2<PREC>(r[g * 8 + 2], r[g * 8 + 3], a.slope);
              pk.z = leaky2<PREC>(r[g * 8 + 4], r[g * 8 + 5], a.slope);
              pk.w = leaky2<PREC>(r[g * 8 + 6], r[g * 8 + 7], a.slope);
              if (c0 + g * 8 < Kn)
                *reinterpret_cast<uint4*>(s_a + cm_offset(rw, c0 + g * 8, Kn, 2)) = pk;
            }
          }
        }
        fence_async_smem();
        tc_fence_before();
        failed = __syncthreads_or(!ok) != 0;
        continue;
      }

      // ---- output layer: this half's lights -----------------------------------
      const float outmul = kF8 ? s_mult[a.n_layers - 1] : 1.0f;
      if (V.vis_out) {
        for (int c0 = lo; c0 < hi; c0 += 16) {
          uint32_t r[16];
          tmem_ld16(t_lane + (uint32_t)c0, r);
          if (live) store_sigmoid_row<16>(V.vis_out + row * L + c0, r, hi - c0, outmul);
        }
      } else {
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (live) {
          nx = __ldg(V.nrm + 3 * row);
          ny = __ldg(V.nrm + 3 * row + 1);
          nz = __ldg(V.nrm + 3 * row + 2);
        }
        float wreg[16];
        float wmax = 0.0f, sum = 0.0f, di = 0.0f;
        const float2 npx = make_float2(-px, -px), npy = make_float2(-py, -py),
                     npz = make_float2(-pz, -pz);
        const float2 nx2 = make_float2(nx, nx), ny2 = make_float2(ny, ny), nz2 = make_float2(nz, nz);
        for (int c0 = lo; c0 < hi; c0 += 16) {
          uint32_t r[16];
          tmem_ld16(t_lane + (uint32_t)c0, r);
          // two lights per packed operation (pair (c0 + j) / 2 of the table)
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int i = c0 + j;
            wreg[j] = 0.0f;
            wreg[j + 1] = 0.0f;
            if (i < hi) {
              const float2 c = contribution2_fast(npx, npy, npz, nx2, ny2, nz2, s_l[i], s_l[i + 1]);
              float2 z01 = make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1]));
              if constexpr (kF8) z01 = __fmul2_rn(z01, make_float2(outmul, outmul));
              const float2 v01 = sigmoid2_fast(z01);
              const float w0 = __fmul_rn(fmaxf(v01.x, bits_f(kVisClampBits)), c.x);
              wmax = fmaxf(wmax, w0);
              sum += w0;
              di = fmaf(v01.x, c.x, di);
              wreg[j] = w0;
              if (i + 1 < hi) {
                const float w1 = __fmul_rn(fmaxf(v01.y, bits_f(kVisClampBits)), c.y);
                wmax = fmaxf(wmax, w1);
                sum += w1;
                di = fmaf(v01.y, c.y, di);
                wreg[j + 1] = w1;
              }
            }
          }
          if (V.w_out != nullptr && live) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < hi) V.w_out[row * L + c0 + j] = wreg[j];
          }
          if (!HSMALL) {
            // the weights replace their logits in this half's (now read)
            // accumulator columns, so the later passes read them instead of
            // computing them again
            uint32_t wb[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) wb[j] = __float_as_uint(wreg[j]);
            tmem_st16(t_lane + (uint32_t)c0, wb);
          }
        }
        // exchange 1: the other half's max, sum and DI (and, with the
        // weights in TMEM, the other half's columns for exchange 2)
        s_x[half * kTileM + rw] = make_float4(wmax, sum, di, 0.0f);
        if (!HSMALL) tc_fence_before();
        pair_sync(warp);
        if (!HSMALL) tc_fence_after();
        const float4 o = s_x[(half ^ 1) * kTileM + rw];
        wmax = fmaxf(wmax, o.x);
        const float sumA = half ? o.y : sum, sumB = half ? sum : o.y;
        const float diA = half ? o.z : di, diB = half ? di : o.z;
        sum = sumA + sumB;
        di = diA + diB;
        const bool active = live && wmax > 0.0f;
        const QuantScale qs = quant_scale(wmax);
        const float sum_q = __fmul_rn(sum, qs.pre);
        if (HSMALL && active && qs.pre != 1.0f) {
#pragma unroll
          for (int j = 0; j < 16; ++j) wreg[j] = __fmul_rn(wreg[j], qs.pre);
        }
        // the first half's integer weight total Q_A (exchange 2 hands it to
        // half 1).  With the weights in TMEM both halves share the sum:
        // half h quantizes the first half's chunks h, h + 2, ...
        uint32_t Q = 0;
        if (!HSMALL) {
          const int hiA = H < L ? H : L;
          uint32_t part = 0;
          for (int c0 = half * 16; c0 < hiA; c0 += 32) {
            uint32_t r[16];
            tmem_ld16(t_lane + (uint32_t)c0, r);
            if (active) {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (c0 + j < hiA)
                  part += quantize_scaled(__fmul_rn(__uint_as_float(r[j]), qs.pre), qs.scale);
            }
          }
          s_q[half * kTileM + rw] = part;
        } else if (half == 0) {
          uint32_t QA = 0;
          for (int c0 = lo; c0 < hi; c0 += 16) {
            uint32_t r[16];
            if (!HSMALL) tmem_ld16(t_lane + (uint32_t)c0, r);
            if (active) {
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int i = c0 + j;
                if (i < hi) {
                  float w = wreg[j];
                  if (!HSMALL) w = __fmul_rn(__uint_as_float(r[j]), qs.pre);
                  QA += quantize_scaled(w, qs.scale);
                }
              }
            }
          }
          s_q[rw] = QA;
        }
        pair_sync(warp);
        if (half == 1) Q = HSMALL ? s_q[rw] : s_q[rw] + s_q[kTileM + rw];
        // the pick over this half's lights, prefix sums continuing from Q
        int sel = -1;
        float wsel = 0.0f;
        const uint32_t pixel = (uint32_t)(V.pixel_offset + row);
        uint4 rr = make_uint4(0, 0, 0, 0);
        for (int c0 = lo; c0 < hi; c0 += 16) {
          uint32_t r[16];
          if (!HSMALL) tmem_ld16(t_lane + (uint32_t)c0, r);
          if (active) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int i = c0 + j;
              if (i < hi) {
                float w = wreg[j];
                if (!HSMALL) w = __fmul_rn(__uint_as_float(r[j]), qs.pre);
                if ((i & 3) == 0)
                  rr = philox_keyed(make_uint4(pixel, a.frame, V.view,
                                               ((uint32_t)(i >> 2) << 4) | kTagWrs),
                                    a.rkey);
                const uint32_t q = quantize_scaled(w, qs.scale);
                Q += q;
                if (__umulhi(pick_word(rr, i & 3), Q) < q) {
                  sel = i;
                  wsel = w;
                }
              }
            }
          }
        }
        // exchange 3: the second half's pick is the later light
        if (half == 1) s_s[rw] = make_int2(sel, __float_as_int(wsel));
        pair_sync(warp);
        if (half == 0 && live) {
          const int2 b = s_s[rw];
          if (b.x >= 0) {
            sel = b.x;
            wsel = __int_as_float(b.y);
          }
          if (V.idx) V.idx[row] = sel;
          if (V.pdf) V.pdf[row] = sel >= 0 ? wsel / sum_q : 0.0f;
          if (V.wsum) V.wsum[row] = sum;
          if (V.radiance) V.radiance[row] = di;
        }
      }
      if (t == 0) *s_next = take_tile(a.status);
      tc_fence_before();
      failed = __syncthreads_or(!ok) != 0;   // also publishes *s_next
    }
  }
  if (failed && t == 0) atomicOr(a.status + kStFlags, kFlagTimeout);
  if (t == 0) finish_tiles(a.status, gridDim.x);
  __syncthreads();
  if (failed) mbar_wait_bounded(bar, phase ^ 1u);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

// ---- warp-specialised variant (L <= 32) -----------------------------------
// 256 threads.  Warps 4-7 produce: for tile i they encode their pixel into
// the layer-0 operand A0[i % 2] and precompute its 32 light contributions
// into C[i % 2], then arrive on full[i % 2].  Warps 0-3 consume: wait on
// full[i % 2], run the MLP (tcgen05, activations through one hidden tile H),
// the sigmoid and the sampler with the precomputed contributions, write the
// pixel's outputs and arrive on empty[i % 2] so the producer may refill the
// buffer.  The producers' gathers thus overlap the consumers' tensor-core
// and ALU work.  Same arithmetic as fused_shade_kernel.
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// bar.sync over the 128 consumer threads (barrier 1) with an OR of `v`.
__device__ __forceinline__ bool consumers_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

template <int F, int PREC, int PW, bool PRE_C>
__global__ void __launch_bounds__(kTileM + PW * 32, PW == 4 ? 2 : 1) fused_shade_ws_kernel(const __grid_constant__ FusedArgs a) {
  constexpr int kThreads = kTileM + PW * 32;
  constexpr int kParts = PW / 4;   // producer threads per pixel
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* s_w = smem;
  uint8_t* s_h = smem + a.ws_h;
  float4* s_l = reinterpret_cast<float4*>(smem + a.ws_l);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.ws_bar);   // mma, full0, full1, empty0, empty1
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + 5);
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int CS = a.ws_cs;

  for (int e = t; e < a.wimg_bytes / 16; e += kThreads)
    reinterpret_cast<uint4*>(s_w)[e] = a.wimg[e];
  if (a.lights) {
    for (int e = t; e < a.L; e += kThreads) {
      float4 l = reinterpret_cast<const float4*>(a.lights)[e];
      l.w = __fmul_rn(l.w, bits_f(kInvPiBits));
      s_l[e] = l;
    }
  }
  const uint32_t bar_mma = smem_u32(s_bar);
  // full[b] at s_bar + 1 + b, empty[b] at s_bar + 3 + b (8 bytes each)
  const uint32_t bar_full0 = bar_mma + 8u, bar_empty0 = bar_mma + 24u;
  if (t == 0) {
    mbar_init(bar_mma, 1);
    mbar_init(bar_full0, PW * 32);
    mbar_init(bar_full0 + 8u, PW * 32);
    mbar_init(bar_empty0, kTileM);
    mbar_init(bar_empty0 + 8u, kTileM);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(s_tmem), a.tmem_cols);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const int din = a.ep.n_levels * F;
  const int K0 = a.layer[0].K;
  const int L = a.L;
  const int64_t n_tiles = a.n_tiles;
  bool failed = false;

  if (warp >= 4) {
    // ================================ producers ================================
    const int p = (t - kTileM) & (kTileM - 1);
    const int part = (t - kTileM) >> 7;
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
      const int b = i & 1;
      if (i >= 2 && !mbar_wait_bounded(bar_empty0 + 8u * b, ((i >> 1) - 1) & 1)) {
        failed = true;
        break;
      }
      const ViewDesc& V = a.v[view_of(a, tile)];
      const int64_t row = (tile - V.tile_start) * kTileM + p;
      const bool live = row < V.n;
      float px = 0.f, py = 0.f, pz = 0.f;
      if (live) {
        px = __ldg(V.pos + 3 * row);
        py = __ldg(V.pos + 3 * row + 1);
        pz = __ldg(V.pos + 3 * row + 2);
      }
      uint8_t* a0 = smem + (b ? a.ws_a0[1] : a.ws_a0[0]);
      {
        const float x = normalise(px, a.ep.lo[0], a.ep.ext[0]);
        const float y = normalise(py, a.ep.lo[1], a.ep.ext[1]);
        const float z = normalise(pz, a.ep.lo[2], a.ep.ext[2]);
        auto encode_part = [&](const auto* tab) {
          for (int c = part; c < K0 / 8; c += kParts) {
            float f8[8];
            encode_chunk<F, false, 8>(a.ep, tab, c, din, x, y, z, live, f8);
            uint4 pk;
            pk.x = pack2<PREC>(f8[0], f8[1]);
            pk.y = pack2<PREC>(f8[2], f8[3]);
            pk.z = pack2<PREC>(f8[4], f8[5]);
            pk.w = pack2<PREC>(f8[6], f8[7]);
            *reinterpret_cast<uint4*>(a0 + cm_offset(p, c * 8, K0, 2)) = pk;
          }
        };
        if (a.table16)
          encode_part(a.table16);
        else
          encode_part(a.table);
      }
      if (PRE_C && a.lights) {
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (live) {
          nx = __ldg(V.nrm + 3 * row);
          ny = __ldg(V.nrm + 3 * row + 1);
          nz = __ldg(V.nrm + 3 * row + 2);
        }
        float* cr = reinterpret_cast<float*>(smem + (b ? a.ws_c[1] : a.ws_c[0])) + p * CS;
#pragma unroll 4
        for (int j = part; j < L; j += kParts)
          cr[j] = contribution_fast(px, py, pz, nx, ny, nz, s_l[j]);
      }
      fence_async_smem();
      mbar_arrive(bar_full0 + 8u * b);
    }
  } else {
    // ================================ consumers ================================
    const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t w_base = smem_u32(s_w);
    const uint32_t h_base = smem_u32(s_h);
    uint32_t mphase = 0;
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
      const int b = i & 1;
      const bool got = mbar_wait_bounded(bar_full0 + 8u * b, (i >> 1) & 1);
      if (consumers_sync_or(!got)) {
        failed = true;
        break;
      }
      tc_fence_after();
      const ViewDesc& V = a.v[view_of(a, tile)];
      const int64_t row = (tile - V.tile_start) * kTileM + t;
      const bool live = row < V.n;
      const uint32_t a0_base = smem_u32(smem + (b ? a.ws_a0[1] : a.ws_a0[0]));
      bool ok = true;
      for (int k = 0; k < a.n_layers; ++k) {
        const LayerDesc ld = a.layer[k];
        if (t == 0) {
          tc_fence_after();
          const uint32_t sbo = (uint32_t)ld.K * 16u;
          const uint32_t ab = k == 0 ? a0_base : h_base;
          const uint32_t wb = w_base + (uint32_t)ld.w_byte_off;
          for (int kk = 0; kk < ld.K / 16; ++kk)
            mma_f16(tmem, smem_desc(ab + kk * 256, 128, sbo), smem_desc(wb + kk * 256, 128, sbo),
                    ld.idesc, kk > 0 ? 1u : 0u);
          mma_commit(bar_mma);
        }
        ok = mbar_wait_bounded(bar_mma, mphase) && ok;
        mphase ^= 1u;
        tc_fence_after();
        if (k + 1 < a.n_layers) {
          const int Kn = ld.N;
          for (int c0 = 0; c0 < ld.N; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(t_lane + (uint32_t)c0, r);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              uint4 pk;
              pk.x = leaky2<PREC>(r[g * 8 + 0], r[g * 8 + 1], a.slope);
              pk.y = leaky2<PREC>(r[g * 8 + 2], r[g * 8 + 3], a.slope);
              pk.z = leaky2<PREC>(r[g * 8 + 4], r[g * 8 + 5], a.slope);
              pk.w = leaky2<PREC>(r[g * 8 + 6], r[g * 8 + 7], a.slope);
              if (c0 + g * 8 < Kn)
                *reinterpret_cast<uint4*>(s_h + cm_offset(t, c0 + g * 8, Kn, 2)) = pk;
            }
          }
          fence_async_smem();
          tc_fence_before();
          if (consumers_sync_or(!ok)) {
            failed = true;
            break;
          }
          continue;
        }
        // ---- output layer: sigmoid, weights, WRS, Neural DI --------------------
        uint32_t r[32];
        tmem_ld32(t_lane, r);
        if (V.vis_out) {
          if (live) store_sigmoid_row<32>(V.vis_out + row * L, r, L, 1.0f);
        } else {
          const float* cr =
              reinterpret_cast<const float*>(smem + (b ? a.ws_c[1] : a.ws_c[0])) + t * CS;
          float px = 0.f, py = 0.f, pz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
          if (!PRE_C && live) {
            px = __ldg(V.pos + 3 * row);
            py = __ldg(V.pos + 3 * row + 1);
            pz = __ldg(V.pos + 3 * row + 2);
            nx = __ldg(V.nrm + 3 * row);
            ny = __ldg(V.nrm + 3 * row + 1);
            nz = __ldg(V.nrm + 3 * row + 2);
          }
          float wreg[32];
          float wmax = 0.0f, sum = 0.0f, di = 0.0f;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float w = 0.0f;
            if (j < L) {
              const float v = sigmoid_fast(__uint_as_float(r[j]));
              const float c =
                  PRE_C ? cr[j] : contribution_fast(px, py, pz, nx, ny, nz, s_l[j]);
              w = __fmul_rn(fmaxf(v, bits_f(kVisClampBits)), c);
              wmax = fmaxf(wmax, w);
              sum += w;
              di = fmaf(v, c, di);
            }
            wreg[j] = w;
          }
          if (V.w_out != nullptr && live) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < L) V.w_out[row * L + j] = wreg[j];
          }
          int sel = -1;
          float wsel = 0.0f;
          const QuantScale qs = quant_scale(wmax);
          const float sum_q = __fmul_rn(sum, qs.pre);
          if (live && wmax > 0.0f) {
            if (qs.pre != 1.0f) {
#pragma unroll
              for (int j = 0; j < 32; ++j) wreg[j] = __fmul_rn(wreg[j], qs.pre);
            }
            const uint32_t pixel = (uint32_t)(V.pixel_offset + row);
            uint32_t Q = 0;
            uint4 rr = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (j < L) {
                if ((j & 3) == 0)
                  rr = philox_keyed(make_uint4(pixel, a.frame, V.view,
                                               ((uint32_t)(j >> 2) << 4) | kTagWrs),
                                    a.rkey);
                const float w = wreg[j];
                const uint32_t q = quantize_scaled(w, qs.scale);
                Q += q;
                if (__umulhi(pick_word(rr, j & 3), Q) < q) {
                  sel = j;
                  wsel = w;
                }
              }
            }
          }
          if (live) {
            if (V.idx) V.idx[row] = sel;
            if (V.pdf) V.pdf[row] = sel >= 0 ? wsel / sum_q : 0.0f;
            if (V.wsum) V.wsum[row] = sum;
            if (V.radiance) V.radiance[row] = di;
          }
        }
      }
      if (failed) break;
      mbar_arrive(bar_empty0 + 8u * b);
      tc_fence_before();
      if (consumers_sync_or(!ok)) {
        failed = true;
        break;
      }
    }
    if (failed && t == 0) atomicOr(a.status + kStFlags, kFlagTimeout);
    if (failed) mbar_wait_bounded(bar_mma, mphase ^ 1u);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

// ---- weight packing (fp32 master -> tensor-core operand image) -------------

template <int PREC>
__global__ void pack_mlp_kernel(const float* __restrict__ params, PackArgs p, uint8_t* out) {
  const int total = p.byte_off[p.n_layers] / p.esize;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < p.n_layers && e * p.esize >= p.byte_off[k + 1]) ++k;
    const int local = e - p.byte_off[k] / p.esize;
    // invert cm_offset: 64 elements per core matrix, K/8 core matrices per row group
    const int grp = local >> 6, within = local & 63;
    const int kg = grp % (p.K[k] / 8), ng = grp / (p.K[k] / 8);
    const int n = ng * 8 + (within >> 3), kk = kg * 8 + (within & 7);
    const float v = (n < p.N_real[k] && kk < p.K_real[k])
                        ? params[p.w_off[k] + (int64_t)n * p.K_real[k] + kk]
                        : 0.0f;
    if constexpr (PREC == NVC_PREC_BF16)
      reinterpret_cast<__nv_bfloat16*>(out + p.byte_off[k])[local] = __float2bfloat16_rn(v);
    else
      reinterpret_cast<__half*>(out + p.byte_off[k])[local] = __float2half_rn(v);
  }
}

// E4M3 weight image: one block per layer finds max |W_k|, sets the layer's
// scale 448 / max (1 when the layer is zero), then writes round(W_k * scale).
__global__ void pack_mlp_fp8_kernel(const float* __restrict__ params, PackArgs p, uint8_t* out,
                                    float* w_scales) {
  const int k = blockIdx.x;
  __shared__ float s_max[32];
  const int nr = p.N_real[k], kr = p.K_real[k];
  const float* W = params + p.w_off[k];
  float m = 0.0f;
  for (int e = threadIdx.x; e < nr * kr; e += blockDim.x) m = fmaxf(m, fabsf(W[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (int)(blockDim.x >> 5) ? s_max[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) s_max[0] = m;
  }
  __syncthreads();
  const float scale = s_max[0] > 0.0f ? 448.0f / s_max[0] : 1.0f;
  if (threadIdx.x == 0) w_scales[k] = scale;
  const int K = p.K[k], total = p.N[k] * K;
  uint8_t* dst = out + p.byte_off[k];
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    // invert cm_offset for 1-byte elements: 128 elements per core matrix
    const int grp = e >> 7, within = e & 127;
    const int kg = grp % (K / 16), ng = grp / (K / 16);
    const int n = ng * 8 + (within >> 4), kk = kg * 16 + (within & 15);
    const float v = (n < nr && kk < kr) ? W[(int64_t)n * kr + kk] * scale : 0.0f;
    dst[e] = (uint8_t)(pack_e4m3x2(v, 0.0f) & 0xFFu);
  }
}

int round16(int x) { return (x + 15) & ~15; }
int round32(int x) { return (x + 31) & ~31; }

uint32_t make_idesc(int M, int N, int prec) {
  // kind::f16: 0 = f16, 1 = bf16; kind::f8f6f4: 0 = E4M3
  const uint32_t ab = prec == NVC_PREC_BF16 ? 1u : 0u;
  return (1u << 4)                                       // D = f32
         | (ab << 7) | (ab << 10)                        // A, B formats; both K-major
         | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

bool tc_precision(int prec) {
  return prec == NVC_PREC_FP16 || prec == NVC_PREC_BF16 || prec == NVC_PREC_FP8;
}

void layer_geometry(const nvc_handle* h, PackArgs& p) {
  p.n_layers = h->n_layers;
  const bool f8 = h->cfg.precision == NVC_PREC_FP8;
  p.esize = f8 ? 1 : 2;
  int off = 0;
  for (int k = 0; k < h->n_layers; ++k) {
    p.K_real[k] = h->w_in[k];
    p.N_real[k] = h->w_out[k];
    p.K[k] = f8 ? round32(h->w_in[k]) : round16(h->w_in[k]);
    p.N[k] = round16(h->w_out[k]);
    p.w_off[k] = h->w_off[k];
    p.byte_off[k] = off;
    off += p.K[k] * p.N[k] * p.esize;
  }
  p.byte_off[h->n_layers] = off;
}

uint32_t tmem_cols_for(const PackArgs& p) {
  int mx = 32;
  for (int k = 0; k < p.n_layers; ++k) mx = p.N[k] > mx ? p.N[k] : mx;
  uint32_t c = 32;
  while ((int)c < mx) c <<= 1;
  return c;
}

// Shared-memory plan of the monolithic kernel: weight image, one activation
// tile (128 rows x the widest K, p.esize bytes each), light table, then the
// mbarrier and TMEM address word.  Fills the offsets when `a` is given.
size_t fused_smem(const nvc_handle* h, const PackArgs& p, FusedArgs* a = nullptr) {
  int kmax = 16;
  for (int k = 0; k < p.n_layers; ++k) kmax = p.K[k] > kmax ? p.K[k] : kmax;
  size_t off = (size_t)p.byte_off[p.n_layers];
  const size_t a_off = off;
  off += (size_t)kTileM * kmax * p.esize;
  off = (off + 15) & ~(size_t)15;
  const size_t l_off = off;
  off += 16 * (size_t)(h->L > 0 ? ((h->L + 1) & ~1) : 2);   // lights in pairs
  const size_t bar_off = off;
  off += 64;
  if (a) {
    a->mono_a = (int)a_off;
    a->mono_l = (int)l_off;
    a->mono_bar = (int)bar_off;
  }
  return off;
}

// The monolithic plan followed by the exchange area of the two-threads-per-
// pixel kernel: partials [2][128] float4, Q_A parts [2][128] uint32, pick [128] int2.
size_t pair_smem(const nvc_handle* h, const PackArgs& p, FusedArgs* a = nullptr) {
  size_t off = fused_smem(h, p, a);
  off = (off + 15) & ~(size_t)15;
  if (a) a->pair_x = (int)off;
  return off + 2 * kTileM * 16 + 2 * kTileM * 4 + kTileM * 8;
}

template <int F, int PREC>
cudaError_t launch_pair_typed(const FusedArgs& a, size_t smem_needed, int num_sms, cudaStream_t s) {
  const int H = split_h(a.L);
  auto kern = H <= 16 ? fused_shade_pair_kernel<F, PREC, true> : fused_shade_pair_kernel<F, PREC, false>;
  const int max_ctas = (int)(512u / a.tmem_cols);
  size_t smem = smem_needed;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)kern);
  if (e != cudaSuccess) return e;
  const size_t dyn_max = 227 * 1024 - fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
  if (e != cudaSuccess) return e;
  int occ = blocks_per_sm((const void*)kern, 2 * kTileM, smem);
  while (occ > max_ctas && smem + 4096 <= dyn_max) {
    smem += 4096;
    occ = blocks_per_sm((const void*)kern, 2 * kTileM, smem);
  }
  if (occ > max_ctas) return cudaErrorInvalidConfiguration;
  const int64_t n_tiles = a.n_tiles;
  const int per_sm = a.max_ctas_per_sm > 0 && a.max_ctas_per_sm < occ ? a.max_ctas_per_sm : occ;
  const int64_t cap = (int64_t)per_sm * num_sms;
  const int grid = (int)(n_tiles < cap ? n_tiles : cap);
  kern<<<grid, 2 * kTileM, smem, s>>>(a);
  return cudaGetLastError();
}

template <int F, int PREC>
cudaError_t launch_typed(const FusedArgs& a, size_t smem_needed, int num_sms, cudaStream_t s) {
  auto kern = a.L <= 32 ? fused_shade_kernel<F, PREC, true> : fused_shade_kernel<F, PREC, false>;
  // cap CTAs per SM so their TMEM columns fit in 512
  const int max_ctas = (int)(512u / a.tmem_cols);
  size_t smem = smem_needed;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)kern);
  if (e != cudaSuccess) return e;
  const size_t dyn_max = 227 * 1024 - fa.sharedSizeBytes;   // static + dynamic <= 227 KB
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
  if (e != cudaSuccess) return e;
  int occ = blocks_per_sm((const void*)kern, kTileM, smem);
  while (occ > max_ctas && smem + 4096 <= dyn_max) {
    smem += 4096;
    occ = blocks_per_sm((const void*)kern, kTileM, smem);
  }
  if (occ > max_ctas) return cudaErrorInvalidConfiguration;
  const int64_t n_tiles = a.n_tiles;
  const int per_sm = a.max_ctas_per_sm > 0 && a.max_ctas_per_sm < occ ? a.max_ctas_per_sm : occ;
  const int64_t cap = (int64_t)per_sm * num_sms;
  const int grid = (int)(n_tiles < cap ? n_tiles : cap);
  kern<<<grid, kTileM, smem, s>>>(a);
  return cudaGetLastError();
}

// Shared-memory plan of the warp-specialised kernel; returns its size.
size_t plan_ws(const PackArgs& p, int L, bool pre_c, FusedArgs& a) {
  int off = p.byte_off[p.n_layers];
  const int K0 = p.K[0];
  int Kh = 16;
  for (int k = 1; k < p.n_layers; ++k) Kh = p.K[k] > Kh ? p.K[k] : Kh;
  a.ws_a0[0] = off;
  off += kTileM * K0 * 2;
  a.ws_a0[1] = off;
  off += kTileM * K0 * 2;
  a.ws_h = off;
  off += kTileM * Kh * 2;
  a.ws_cs = L | 1;   // odd row stride: conflict-free per-thread rows
  a.ws_c[0] = off;
  if (pre_c) off += kTileM * a.ws_cs * 4;
  a.ws_c[1] = off;
  if (pre_c) off += kTileM * a.ws_cs * 4;
  off = (off + 15) & ~15;
  a.ws_l = off;
  off += 16 * L;
  a.ws_bar = off;
  off += 64;
  return (size_t)off;
}

template <int F, int PREC, int PW, bool PRE_C>
cudaError_t launch_ws_typed(const FusedArgs& a, size_t smem_needed, int num_sms, cudaStream_t s) {
  auto kern = fused_shade_ws_kernel<F, PREC, PW, PRE_C>;
  constexpr int kThreads = kTileM + PW * 32;
  const int max_ctas = (int)(512u / a.tmem_cols);
  size_t smem = smem_needed;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)kern);
  if (e != cudaSuccess) return e;
  const size_t dyn_max = 227 * 1024 - fa.sharedSizeBytes;   // static + dynamic <= 227 KB
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
  if (e != cudaSuccess) return e;
  int occ = blocks_per_sm((const void*)kern, kThreads, smem);
  while (occ > max_ctas && smem + 4096 <= dyn_max) {
    smem += 4096;
    occ = blocks_per_sm((const void*)kern, kThreads, smem);
  }
  if (occ > max_ctas) return cudaErrorInvalidConfiguration;
  const int64_t n_tiles = a.n_tiles;
  const int per_sm = a.max_ctas_per_sm > 0 && a.max_ctas_per_sm < occ ? a.max_ctas_per_sm : occ;
  const int64_t cap = (int64_t)per_sm * num_sms;
  const int grid = (int)(n_tiles < cap ? n_tiles : cap);
  kern<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t mlp_packed_bytes(const nvc_handle* h) {
  if (!tc_precision(h->cfg.precision) && h->cfg.train_precision != NVC_PREC_FP16) return 0;
  PackArgs p{};
  layer_geometry(h, p);
  return (size_t)p.byte_off[p.n_layers];
}

bool mlp_image_map(const nvc_handle* h, MlpImageMap* m) {
  if (!h->mlp_packed || h->cfg.precision == NVC_PREC_FP8 || h->cfg.precision == NVC_PREC_FP32)
    return false;
  PackArgs p{};
  layer_geometry(h, p);
  m->n_layers = p.n_layers;
  for (int k = 0; k < p.n_layers; ++k) {
    m->w_off[k] = p.w_off[k];
    m->K_real[k] = p.K_real[k];
    m->K[k] = p.K[k];
    m->byte_off[k] = p.byte_off[k];
  }
  m->w_off[p.n_layers] = p.w_off[p.n_layers - 1] + (int64_t)p.N_real[p.n_layers - 1] *
                                                       p.K_real[p.n_layers - 1];
  m->bf16 = h->cfg.precision == NVC_PREC_BF16;
  return true;
}

cudaError_t launch_pack_mlp(nvc_handle* h, cudaStream_t s) {
  if (!h->mlp_packed) return cudaSuccess;
  PackArgs p{};
  layer_geometry(h, p);
  const int total = p.byte_off[p.n_layers] / p.esize;
  const int blocks = (total + 255) / 256;
  if (h->cfg.precision == NVC_PREC_FP8)
    pack_mlp_fp8_kernel<<<p.n_layers, 256, 0, s>>>(h->params, p, (uint8_t*)h->mlp_packed,
                                                    h->fp8_scales + kMaxLayers);
  else if (h->cfg.precision == NVC_PREC_BF16)
    pack_mlp_kernel<NVC_PREC_BF16><<<blocks, 256, 0, s>>>(h->params, p, (uint8_t*)h->mlp_packed);
  else
    pack_mlp_kernel<NVC_PREC_FP16><<<blocks, 256, 0, s>>>(h->params, p, (uint8_t*)h->mlp_packed);
  return cudaGetLastError();
}

// The half-precision copy of the hash table (nvc_set_table_precision):
// table16[i] = fp16(params[i]) for i < n_table, round to nearest even.
__global__ void pack_table_kernel(const float4* __restrict__ params, uint2* __restrict__ table16,
                                  int64_t n4) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = params[e];
    const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    table16[e] = make_uint2(*reinterpret_cast<const uint32_t*>(&a),
                            *reinterpret_cast<const uint32_t*>(&b));
  }
}

cudaError_t launch_pack_table(nvc_handle* h, cudaStream_t s) {
  if (!h->table16) return cudaSuccess;
  pack_table_kernel<<<h->num_sms * 8, 256, 0, s>>>(reinterpret_cast<const float4*>(h->params),
                                                    reinterpret_cast<uint2*>(h->table16),
                                                    h->n_table / 4);
  return cudaGetLastError();
}

bool fused_supported(const nvc_handle* h, std::string* why) {
  if (!tc_precision(h->cfg.precision)) {
    *why = "the fused tensor-core kernel runs in FP16, BF16 or FP8 precision";
    return false;
  }
  if (h->cfg.precision == NVC_PREC_FP8 && !h->fp8_calibrated) {
    *why = "FP8 needs activation scales: call nvc_calibrate first";
    return false;
  }
  PackArgs p{};
  layer_geometry(h, p);
  for (int k = 0; k < p.n_layers; ++k)
    if (p.N[k] > 256) {
      *why = "layer wider than 256";
      return false;
    }
  if (fused_smem(h, p) > 227 * 1024) {
    *why = "weights and tile exceed shared memory";
    return false;
  }
  return true;
}

cudaError_t launch_shade_fused_views(const nvc_handle* h, const nvc_scene* sc,
                                     const FusedView* views, int n_views, uint64_t seed,
                                     uint32_t frame, cudaStream_t s,
                                     unsigned long long* phase_cycles, const uint16_t* feat16) {
  // views beyond one launch's table go to further launches
  if (n_views > kMaxViews) {
    if (feat16) return cudaErrorInvalidValue;   // one view of features per launch
    cudaError_t e = launch_shade_fused_views(h, sc, views, kMaxViews, seed, frame, s, phase_cycles);
    if (e != cudaSuccess) return e;
    return launch_shade_fused_views(h, sc, views + kMaxViews, n_views - kMaxViews, seed, frame, s,
                                    phase_cycles);
  }
  PackArgs p{};
  layer_geometry(h, p);
  FusedArgs a{};
  int64_t tiles = 0;
  for (int i = 0; i < n_views; ++i) {
    const FusedView& fv = views[i];
    if (fv.n <= 0) continue;
    ViewDesc& V = a.v[a.n_views++];
    V.pos = fv.pos;
    V.nrm = fv.nrm;
    V.n = fv.n;
    V.tile_start = tiles;
    V.pixel_offset = fv.pixel_offset;
    V.view = fv.view;
    V.idx = fv.idx;
    V.pdf = fv.pdf;
    V.wsum = fv.wsum;
    V.radiance = fv.radiance;
    V.vis_out = fv.vis_out;
    V.w_out = fv.w_out;
    tiles += (fv.n + kTileM - 1) / kTileM;
  }
  if (tiles == 0) return cudaSuccess;
  a.n_tiles = tiles;
  a.table = h->params;
  a.table16 = h->table16;
  a.ep = encode_params(h);
  a.F = h->F;
  a.wimg = reinterpret_cast<const uint4*>(h->mlp_packed);
  a.wimg_bytes = p.byte_off[p.n_layers];
  a.n_layers = h->n_layers;
  a.kmax = 16;
  for (int k = 0; k < h->n_layers; ++k) {
    a.layer[k].K = p.K[k];
    a.layer[k].N = p.N[k];
    a.layer[k].N_real = p.N_real[k];
    a.layer[k].K_real = p.K_real[k];
    a.layer[k].w_byte_off = p.byte_off[k];
    a.layer[k].idesc = make_idesc(kTileM, p.N[k], h->cfg.precision);
    a.kmax = p.K[k] > a.kmax ? p.K[k] : a.kmax;
  }
  a.slope = h->cfg.leaky_slope;
  a.L = h->L;
  a.tmem_cols = tmem_cols_for(p);
  a.lights = sc ? sc->lights : nullptr;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r)
    a.rkey[r] = make_uint2(a.k0 + (uint32_t)r * kPhiloxW0, a.k1 + (uint32_t)r * kPhiloxW1);
  a.frame = frame;
  a.status = h->status;
  a.fp8_scales = h->fp8_scales;
  a.phase_cycles = phase_cycles;
  a.max_ctas_per_sm = h->shade_ctas_per_sm;
  a.feat16 = feat16;
  if (feat16) {
    // the MLP-only launch runs the tile-stream kernel (two streams per CTA
    // when the handle's shading point is variant 6, else four)
    if (h->cfg.precision == NVC_PREC_FP8 || h->L > 32) return cudaErrorInvalidValue;
    return launch_shade_multi(a, h, p, h->shade_variant == kShadeMulti2 ? 2 : 4,
                              h->cfg.precision == NVC_PREC_BF16, s);
  }
  if (h->cfg.precision == NVC_PREC_FP8 && h->shade_variant == kShadePair) {
    const size_t smem_p8 = pair_smem(h, p, &a);
    switch (h->F) {
      case 1: return launch_pair_typed<1, NVC_PREC_FP8>(a, smem_p8, h->num_sms, s);
      case 2: return launch_pair_typed<2, NVC_PREC_FP8>(a, smem_p8, h->num_sms, s);
      case 4: return launch_pair_typed<4, NVC_PREC_FP8>(a, smem_p8, h->num_sms, s);
      case 8: return launch_pair_typed<8, NVC_PREC_FP8>(a, smem_p8, h->num_sms, s);
    }
    return cudaErrorInvalidValue;
  }
  if (h->cfg.precision == NVC_PREC_FP8) {
    const size_t smem8 = fused_smem(h, p, &a);
    switch (h->F) {
      case 1: return launch_typed<1, NVC_PREC_FP8>(a, smem8, h->num_sms, s);
      case 2: return launch_typed<2, NVC_PREC_FP8>(a, smem8, h->num_sms, s);
      case 4: return launch_typed<4, NVC_PREC_FP8>(a, smem8, h->num_sms, s);
      case 8: return launch_typed<8, NVC_PREC_FP8>(a, smem8, h->num_sms, s);
    }
    return cudaErrorInvalidValue;
  }
  const bool bf16 = h->cfg.precision == NVC_PREC_BF16;
  const int variant = h->shade_variant;
  if ((variant == kShadeMulti2 || variant == kShadeMulti4) && h->L <= 32)
    return launch_shade_multi(a, h, p, variant == kShadeMulti2 ? 2 : 4, bf16, s);
  if (variant == kShadePair) {
    const size_t smem_p = pair_smem(h, p, &a);
    switch (h->F) {
      case 1: return bf16 ? launch_pair_typed<1, NVC_PREC_BF16>(a, smem_p, h->num_sms, s)
                          : launch_pair_typed<1, NVC_PREC_FP16>(a, smem_p, h->num_sms, s);
      case 2: return bf16 ? launch_pair_typed<2, NVC_PREC_BF16>(a, smem_p, h->num_sms, s)
                          : launch_pair_typed<2, NVC_PREC_FP16>(a, smem_p, h->num_sms, s);
      case 4: return bf16 ? launch_pair_typed<4, NVC_PREC_BF16>(a, smem_p, h->num_sms, s)
                          : launch_pair_typed<4, NVC_PREC_FP16>(a, smem_p, h->num_sms, s);
      case 8: return bf16 ? launch_pair_typed<8, NVC_PREC_BF16>(a, smem_p, h->num_sms, s)
                          : launch_pair_typed<8, NVC_PREC_FP16>(a, smem_p, h->num_sms, s);
    }
    return cudaErrorInvalidValue;
  }
  if (h->L <= 32 && variant != kShadeMono) {
    const bool pre_c = variant == kShadeWs4C || variant == kShadeWs8C;
    const bool p8 = variant == kShadeWs8 || variant == kShadeWs8C;
    const size_t smem_ws = plan_ws(p, h->L, pre_c, a);
    if (smem_ws <= 227 * 1024) {
#define NVC_WS(FF, PP)                                                                        \
  if (p8) return pre_c ? launch_ws_typed<FF, PP, 8, true>(a, smem_ws, h->num_sms, s)           \
                       : launch_ws_typed<FF, PP, 8, false>(a, smem_ws, h->num_sms, s);         \
  return pre_c ? launch_ws_typed<FF, PP, 4, true>(a, smem_ws, h->num_sms, s)                   \
               : launch_ws_typed<FF, PP, 4, false>(a, smem_ws, h->num_sms, s);
      switch (h->F) {
        case 1: if (bf16) { NVC_WS(1, NVC_PREC_BF16) } else { NVC_WS(1, NVC_PREC_FP16) }
        case 2: if (bf16) { NVC_WS(2, NVC_PREC_BF16) } else { NVC_WS(2, NVC_PREC_FP16) }
        case 4: if (bf16) { NVC_WS(4, NVC_PREC_BF16) } else { NVC_WS(4, NVC_PREC_FP16) }
        case 8: if (bf16) { NVC_WS(8, NVC_PREC_BF16) } else { NVC_WS(8, NVC_PREC_FP16) }
      }
#undef NVC_WS
    }
  }
  const size_t smem = fused_smem(h, p, &a);
  switch (h->F) {
    case 1: return bf16 ? launch_typed<1, NVC_PREC_BF16>(a, smem, h->num_sms, s)
                        : launch_typed<1, NVC_PREC_FP16>(a, smem, h->num_sms, s);
    case 2: return bf16 ? launch_typed<2, NVC_PREC_BF16>(a, smem, h->num_sms, s)
                        : launch_typed<2, NVC_PREC_FP16>(a, smem, h->num_sms, s);
    case 4: return bf16 ? launch_typed<4, NVC_PREC_BF16>(a, smem, h->num_sms, s)
                        : launch_typed<4, NVC_PREC_FP16>(a, smem, h->num_sms, s);
    case 8: return bf16 ? launch_typed<8, NVC_PREC_BF16>(a, smem, h->num_sms, s)
                        : launch_typed<8, NVC_PREC_FP16>(a, smem, h->num_sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_shade_fused(const nvc_handle* h, const nvc_scene* sc, const float* pos,
                               const float* nrm, int64_t n, uint64_t seed, uint32_t frame,
                               uint32_t view, int64_t pixel_offset, int32_t* idx, float* pdf,
                               float* wsum, float* radiance, float* vis_out, cudaStream_t s,
                               float* w_out) {
  if (n == 0) return cudaSuccess;
  FusedView v{pos, nrm, n, view, pixel_offset, idx, pdf, wsum, radiance, vis_out, w_out};
  return launch_shade_fused_views(h, sc, &v, 1, seed, frame, s);
}

}  // namespace nvc
