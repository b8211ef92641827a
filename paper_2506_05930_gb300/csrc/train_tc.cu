// Training forward + loss + hand-written backward on the tensor cores
// (Sections 3.3 and 3.4 of the paper; FP16 operands, FP32 accumulation in
// TMEM, static loss scaling).
//
// One CTA takes 128 training positions at a time (persistent over tiles);
// its four warpgroups share each sample row (= TMEM lane) by levels and by
// 16-column chunks.
//   forward:  encode -> act_0; z_k = act_k W_k^T (tcgen05, M=128) ->
//             act_{k+1} = leaky_relu(z_k) kept in shared memory (fp16);
//   loss:     logits from TMEM, targets from memory; delta_out =
//             scale * dl/dz per (sample, light) in fp16, where the mean's
//             1/(B*L) is applied later in fp32 so small deltas do not
//             underflow fp16;
//   backward: per layer k from the top, two MMAs on the same operands:
//             dW_k += delta_k^T act_k   (M = out rows, N = in, K = the 128
//                                       samples; accumulated in TMEM over
//                                       the CTA's tiles)
//             g    = delta_k W_k       (M = 128 samples, N = in, K = out)
//             then delta_{k-1} = g * act'(act_k), or for k = 0 the feature
//             gradient, scattered straight into the hash-table gradient
//             (the encoding's adjoint: 8 corner rows x trilinear weight).
// The transposed products read the sample-major buffers as MN-major
// operands: a K-major [rows][K] tile in the no-swizzle core-matrix layout
// is, read the other way, an MN-major tile with the same 128-byte core
// matrices (stride-byte offset 128, leading-byte offset 16 * row length).
// At the end each CTA adds its dW (times 1/(B*L)) into the gradient with
// fp32 atomics and writes its loss partial.
//
// GEN (the fused training data of Section 4.4): the kernel also makes the
// tile's training positions (training_position, as the separate data
// kernel) and traces their shadow rays to every light against the
// occluders staged in shared memory.  The rays of a tile are split into one
// slice per hidden layer, each traced by all threads between the layer's
// MMA issue and its wait, so the ray tests run while the tensor core works;
// the targets stay in shared memory for the loss (and are also written out
// with the positions, the batch nvc_training_batch reads back).
#include "nvc_internal.cuh"
#include "hashgrid.cuh"
#include "shadow.cuh"
#include "tc_common.cuh"

namespace nvc {

namespace {

using namespace tc;

constexpr int kTileM = 128;
constexpr int kMaxLayers = NVC_MAX_HIDDEN_LAYERS + 1;
constexpr int kGuardBytes = 4096;   // room for the M=128 reads past a delta tile

struct TrainTcArgs {
  const float* pos;
  const float* target;
  int64_t n;
  const float* table;
  EncodeParams ep;
  const uint4* wimg;
  int wimg_bytes;
  int n_layers;
  int K[kMaxLayers];          // padded inputs of layer k
  int N[kMaxLayers];          // padded outputs of layer k
  int K_real[kMaxLayers];
  int N_real[kMaxLayers];
  int w_byte_off[kMaxLayers];
  int64_t w_off[kMaxLayers];  // float offset of W_k in the parameter/gradient vector
  int act_off[kMaxLayers];    // smem byte offset of act_k (128 x K[k] fp16)
  int d_off[2];               // smem byte offsets of the two delta tiles
  int guard_off;
  int bar_off;
  uint32_t dw_col[kMaxLayers];
  uint32_t tmem_cols;
  uint32_t idesc_fwd[kMaxLayers], idesc_dw[kMaxLayers], idesc_bwd[kMaxLayers];
  float slope;
  int L;
  int loss;
  float loss_scale;
  float inv_count;            // 1 / (B * L)
  float* grad;
  double* partials;
  int32_t* status;
  // GEN only: the batch generator, the scene and where the batch goes
  PosGen pg;
  const float* lights;
  const float* spheres;
  const float* boxes;
  int n_sph, n_box;
  float* pos_out;             // [n][3]
  float* target_out;          // [n][L]
  int occ_off;                // smem: lights (float4), then the occluders (shadow.cuh layout)
  int tgt_off;                // smem: the tile's targets, 128 x L bytes
};

// Rays [r0, r1) of a tile's 128 x L (row-major by sample): the segment from
// the row's position to light i against every staged occluder; the binary
// target goes to shared memory and, for live rows, to target_out.
__device__ __forceinline__ void trace_slice(const TrainTcArgs& a, const float* s_pos,
                                            const Occluders& occ, const float4* s_lt,
                                            uint8_t* s_tgt, int64_t tile,
                                            int r0, int r1, int t, int n_threads) {
  for (int r = r0 + t; r < r1; r += n_threads) {
    const int row = r / a.L, i = r - row * a.L;
    const int64_t sample = tile * 128 + row;
    if (sample >= a.n) continue;
    const float4 lt = s_lt[i];
    const bool blocked = segment_blocked(s_pos[3 * row], s_pos[3 * row + 1], s_pos[3 * row + 2],
                                         lt.x, lt.y, lt.z, occ);
    s_tgt[r] = blocked ? 0 : 1;
    a.target_out[sample * a.L + i] = blocked ? 0.0f : 1.0f;
  }
}

template <int PREC>
__device__ __forceinline__ void unpack2(uint32_t u, float& a, float& b) {
  if constexpr (PREC == NVC_PREC_BF16) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
    a = __bfloat162float(h.x);
    b = __bfloat162float(h.y);
  } else {
    __half2 h = *reinterpret_cast<__half2*>(&u);
    a = __half2float(h.x);
    b = __half2float(h.y);
  }
}

// Store 16 fp32 values (columns c0..c0+15 of row `row`) as 16-bit values
// into a K-major tile with row length K, zero where the column is >= valid.
template <int PREC>
__device__ __forceinline__ void store_row16(uint8_t* tile, int row, int c0, int K, int valid,
                                            const float (&v)[16]) {
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int c = c0 + g * 8;
    if (c < K) {
      float h[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) h[s] = c + s < valid ? v[g * 8 + s] : 0.0f;
      uint4 pk;
      pk.x = pack2<PREC>(h[0], h[1]);
      pk.y = pack2<PREC>(h[2], h[3]);
      pk.z = pack2<PREC>(h[4], h[5]);
      pk.w = pack2<PREC>(h[6], h[7]);
      *reinterpret_cast<uint4*>(tile + cm_offset(row, c, K, 2)) = pk;
    }
  }
}

// kGroups warpgroups per CTA.  Thread t serves sample row t % 128 (its TMEM
// lane: warp w reads lanes 32 (w % 4) .. +31) and warpgroup t / 128 takes
// every kGroups-th share of the row's work -- the encode's 8-feature chunks,
// the hash-table scatter's levels and the epilogues' 16-column TMEM chunks --
// so a sample's gathers, atomics and conversions run kGroups ways in
// parallel instead of one after another in a single thread.
constexpr int kGroups = 4;

template <int F, int PREC, int NG, bool GEN>
__global__ void __launch_bounds__(kTileM * NG, 1) train_tc_kernel(const __grid_constant__ TrainTcArgs a) {
  constexpr int kThreads = kTileM * NG;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ double s_red[kThreads / 32];
  __shared__ float s_pos[GEN ? 3 * kTileM : 1];
  float4* s_lt = reinterpret_cast<float4*>(smem + a.occ_off);
  uint8_t* s_tgt = smem + a.tgt_off;
  Occluders occ = staged_occluders(s_lt + a.L, 0, 0);
  if constexpr (GEN) {
    occ = stage_occluders(a.spheres, a.n_sph, a.boxes, a.n_box, s_lt + a.L, threadIdx.x, kThreads);
    for (int e = threadIdx.x; e < a.L; e += kThreads)
      s_lt[e] = reinterpret_cast<const float4*>(a.lights)[e];
  }
  uint8_t* s_w = smem;
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.bar_off);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + 1);
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int rw = t & (kTileM - 1);   // sample row within the tile = TMEM lane
  const int wg = t / kTileM;         // this thread's share of the row's work

  for (int e = t; e < a.wimg_bytes / 16; e += kThreads)
    reinterpret_cast<uint4*>(s_w)[e] = a.wimg[e];
  for (int e = t; e < kGuardBytes / 16; e += kThreads)
    reinterpret_cast<uint4*>(smem + a.guard_off)[e] = make_uint4(0, 0, 0, 0);
  const uint32_t bar = smem_u32(s_bar);
  if (t == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(s_tmem), a.tmem_cols);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t t_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t s_base = smem_u32(smem);
  uint32_t phase = 0;
  bool failed = false;
  bool bad = false;
  double loss_acc = 0.0;
  int tiles_done = 0;
  const int last = a.n_layers - 1;
  const int din = a.ep.n_levels * F;
  const int64_t n_tiles = (a.n + kTileM - 1) / kTileM;

  for (int64_t tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
    const int64_t row = tile * kTileM + rw;
    const bool live = row < a.n;
    float x = 0.f, y = 0.f, z = 0.f;
    if (live) {
      float px, py, pz;
      if constexpr (GEN) {
        // every warpgroup makes its row's position (a cheaper way to share
        // it than a barrier); the first also stages and stores it
        const float3 q = training_position(row, a.pg);
        px = q.x;
        py = q.y;
        pz = q.z;
        if (wg == 0) {
          s_pos[3 * rw] = px;
          s_pos[3 * rw + 1] = py;
          s_pos[3 * rw + 2] = pz;
          a.pos_out[3 * row] = px;
          a.pos_out[3 * row + 1] = py;
          a.pos_out[3 * row + 2] = pz;
        }
      } else {
        px = __ldg(a.pos + 3 * row);
        py = __ldg(a.pos + 3 * row + 1);
        pz = __ldg(a.pos + 3 * row + 2);
      }
      x = normalise(px, a.ep.lo[0], a.ep.ext[0]);
      y = normalise(py, a.ep.lo[1], a.ep.ext[1]);
      z = normalise(pz, a.ep.lo[2], a.ep.ext[2]);
    }
    // ---- encode into act_0 (this warpgroup's 8-feature chunks) ------------
    {
      uint8_t* act0 = smem + a.act_off[0];
      const int K0 = a.K[0];
      constexpr int LPC = F >= 8 ? 1 : 8 / F;
      for (int c = wg; c < K0 / 8; c += NG) {
        float f8[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) f8[s] = 0.0f;
        if (live) {
#pragma unroll
          for (int q = 0; q < LPC; ++q) {
            const int l = c * LPC + q;   // F divides 8: chunk c holds levels c LPC ..
            if (l * F < din) {
              float acc[F];
              encode_level<F, false, false>(a.ep, a.table, l, x, y, z, acc);
#pragma unroll
              for (int f = 0; f < F; ++f) f8[q * F + f] = acc[f];
            }
          }
        }
        uint4 pk;
        pk.x = pack2<PREC>(f8[0], f8[1]);
        pk.y = pack2<PREC>(f8[2], f8[3]);
        pk.z = pack2<PREC>(f8[4], f8[5]);
        pk.w = pack2<PREC>(f8[6], f8[7]);
        *reinterpret_cast<uint4*>(act0 + cm_offset(rw, c * 8, K0, 2)) = pk;
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();

    // ---- forward ----------------------------------------------------------
    int cur = 0;
    for (int k = 0; k <= last && !failed; ++k) {
      const int K = a.K[k], N = a.N[k];
      if (t == 0) {
        tc_fence_after();
        const uint32_t ab = s_base + a.act_off[k], wb = s_base + a.w_byte_off[k];
        for (int kk = 0; kk < K / 16; ++kk)
          mma_f16(tmem, smem_desc(ab + kk * 256, 128, K * 16), smem_desc(wb + kk * 256, 128, K * 16),
                  a.idesc_fwd[k], kk > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      if constexpr (GEN) {
        // slice k of the tile's shadow rays while layer k's MMAs run; the
        // loss (layer `last`) reads them after this layer's barrier
        if (k < last) {
          const int R = kTileM * a.L;
          trace_slice(a, s_pos, occ, s_lt, s_tgt, tile, R * k / last, R * (k + 1) / last, t,
                      kThreads);
        }
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      tc_fence_after();
      if (k < last) {
        uint8_t* nxt = smem + a.act_off[k + 1];
        for (int c0 = wg * 16; c0 < N; c0 += 16 * NG) {
          uint32_t r[16];
          tmem_ld16(t_lane + (uint32_t)c0, r);
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float zz = __uint_as_float(r[j]);
            v[j] = live ? fmaxf(zz, a.slope * zz) : 0.0f;
          }
          store_row16<PREC>(nxt, rw, c0, N, a.N_real[k], v);
        }
      } else {
        // loss and the scaled gradient at the logits
        uint8_t* dt = smem + a.d_off[cur];
        const float* yrow = a.target + (live ? row : 0) * a.L;
        for (int c0 = wg * 16; c0 < N; c0 += 16 * NG) {
          uint32_t r[16];
          tmem_ld16(t_lane + (uint32_t)c0, r);
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int i = c0 + j;
            float g = 0.0f;
            if (live && i < a.L) {
              const float zz = __uint_as_float(r[j]);
              const float yy = GEN ? (float)s_tgt[rw * a.L + i] : __ldg(yrow + i);
              const float s = 1.0f / (1.0f + expf(-zz));
              if (a.loss == NVC_LOSS_BCE) {
                loss_acc += (double)(fmaxf(zz, 0.0f) + log1pf(expf(-fabsf(zz))) - yy * zz);
                g = s - yy;
              } else {
                const float d = s - yy;
                loss_acc += (double)d * (double)d;
                g = 2.0f * d * s * (1.0f - s);
              }
              g *= a.loss_scale;
              bad = bad || !isfinite(zz) || !isfinite(g);
            }
            v[j] = g;
          }
          store_row16<PREC>(dt, rw, c0, N, a.L, v);
        }
      }
      fence_async_smem();
      tc_fence_before();
      failed = __syncthreads_or(!ok) != 0;
    }

    // ---- backward ---------------------------------------------------------
    for (int k = last; k >= 0 && !failed; --k) {
      const int K = a.K[k], N = a.N[k];
      const uint32_t db = s_base + a.d_off[cur];
      const uint32_t ab = s_base + a.act_off[k], wb = s_base + a.w_byte_off[k];
      if (t == 0) {
        tc_fence_after();
        // dW_k (+)= delta_k^T act_k: both operands MN-major views of
        // sample-major tiles; K runs over the 128 samples
        for (int kk = 0; kk < kTileM / 16; ++kk)
          mma_f16(tmem + a.dw_col[k], smem_desc(db + kk * 2 * N * 16, N * 16, 128),
                  smem_desc(ab + kk * 2 * K * 16, K * 16, 128), a.idesc_dw[k],
                  (tiles_done > 0 || kk > 0) ? 1u : 0u);
        // g = delta_k W_k: delta K-major over the outputs, W_k read MN-major
        for (int kk = 0; kk < N / 16; ++kk)
          mma_f16(tmem, smem_desc(db + kk * 256, 128, N * 16),
                  smem_desc(wb + kk * 2 * K * 16, K * 16, 128), a.idesc_bwd[k],
                  kk > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      tc_fence_after();
      if (k > 0) {
        // delta_{k-1} = g * act'(z_{k-1}); act_k holds leaky_relu(z_{k-1})
        uint8_t* dn = smem + a.d_off[cur ^ 1];
        const uint8_t* act = smem + a.act_off[k];
        for (int c0 = wg * 16; c0 < K; c0 += 16 * NG) {
          uint32_t r[16];
          tmem_ld16(t_lane + (uint32_t)c0, r);
          float v[16];
#pragma unroll
          for (int g8 = 0; g8 < 2; ++g8) {
            const int c = c0 + g8 * 8;
            uint4 av = make_uint4(0, 0, 0, 0);
            if (c < K) av = *reinterpret_cast<const uint4*>(act + cm_offset(rw, c, K, 2));
            float h[8];
            unpack2<PREC>(av.x, h[0], h[1]);
            unpack2<PREC>(av.y, h[2], h[3]);
            unpack2<PREC>(av.z, h[4], h[5]);
            unpack2<PREC>(av.w, h[6], h[7]);
#pragma unroll
            for (int s = 0; s < 8; ++s) {
              const float g = __uint_as_float(r[g8 * 8 + s]);
              v[g8 * 8 + s] = live ? (h[s] > 0.0f ? g : a.slope * g) : 0.0f;
            }
          }
          store_row16<PREC>(dn, rw, c0, K, a.K_real[k], v);
        }
      } else {
        // feature gradient -> hash-table gradient (adjoint of the encoding);
        // level l is scattered by warpgroup l % NG.  F divides 16, so no
        // level straddles two 16-column chunks.
        float dfeat[NVC_MAX_FEATURES];
        for (int c0 = 0; c0 < K; c0 += 16) {
          uint32_t r[16];
          tmem_ld16(t_lane + (uint32_t)c0, r);
          if (live) {
#pragma unroll
            for (int q = 0; q < 16 / F; ++q) {
              const int l = c0 / F + q;
              if (l >= din / F || l % NG != wg) continue;
              bool any = false;
#pragma unroll
              for (int f = 0; f < F; ++f) {
                dfeat[f] = __uint_as_float(r[q * F + f]) * a.inv_count;
                any = any || dfeat[f] != 0.0f;
                bad = bad || !isfinite(dfeat[f]);
              }
              if (!any) continue;
              Corners cr;
              level_corners(a.ep, l, x, y, z, cr);
              float* gt = a.grad + ((int64_t)l << a.ep.log2_table) * F;
              if constexpr (F == 2) {
                // x-corners d, d + 1 whose rows form one aligned 16-byte pair
                // (always for an even cell x: hash(x + 1) = hash(x) ^ 1) go out
                // as one 16-byte atomic
#pragma unroll
                for (int d = 0; d < 8; d += 2) {
                  const uint32_t r0 = cr.row[d], r1 = cr.row[d + 1];
                  const float2 g0 = make_float2(cr.w[d] * dfeat[0], cr.w[d] * dfeat[1]);
                  const float2 g1 = make_float2(cr.w[d + 1] * dfeat[0], cr.w[d + 1] * dfeat[1]);
                  if ((r0 ^ r1) == 1u) {
                    const float4 v = (r0 & 1u) ? make_float4(g1.x, g1.y, g0.x, g0.y)
                                               : make_float4(g0.x, g0.y, g1.x, g1.y);
                    atomicAdd(reinterpret_cast<float4*>(gt + (int64_t)(r0 & ~1u) * 2), v);
                  } else {
                    atomicAdd(reinterpret_cast<float2*>(gt + (int64_t)r0 * 2), g0);
                    atomicAdd(reinterpret_cast<float2*>(gt + (int64_t)r1 * 2), g1);
                  }
                }
              } else {
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                  float* dst = gt + (int64_t)cr.row[d] * F;
#pragma unroll
                  for (int f = 0; f < F; ++f) atomicAdd(dst + f, cr.w[d] * dfeat[f]);
                }
              }
            }
          }
        }
      }
      fence_async_smem();
      tc_fence_before();
      failed = __syncthreads_or(!ok) != 0;
      cur ^= 1;
    }
    ++tiles_done;
  }

  // ---- flush this CTA's weight gradients ---------------------------------------
  if (!failed && tiles_done > 0) {
    tc_fence_after();
    for (int k = 0; k <= last; ++k) {
      const int out = a.N_real[k], in = a.K_real[k];
      const int j = rw;   // TMEM lane = output row j of dW_k
      for (int c0 = wg * 16; c0 < a.K[k]; c0 += 16 * NG) {
        uint32_t r[16];
        tmem_ld16(t_lane + a.dw_col[k] + (uint32_t)c0, r);
        if (j < out) {
          float* dst = a.grad + a.w_off[k] + (int64_t)j * in;
          float v[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            v[q] = __uint_as_float(r[q]) * a.inv_count;
            bad = bad || (c0 + q < in && !isfinite(v[q]));
          }
          if ((in & 3) == 0 && ((a.w_off[k] & 3) == 0)) {
            // 16-byte aligned rows: four 16-byte atomics instead of 16 scalar
#pragma unroll
            for (int q = 0; q < 16; q += 4)
              if (c0 + q < in)
                atomicAdd(reinterpret_cast<float4*>(dst + c0 + q),
                          make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]));
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (c0 + q < in) atomicAdd(dst + c0 + q, v[q]);
          }
        }
      }
    }
  }
  // ---- loss partial and the non-finite flag ------------------------------------
  double lsum = loss_acc;
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
  if ((t & 31) == 0) s_red[warp] = lsum;
  const bool any_bad = __syncthreads_or(bad) != 0;
  if (t == 0) {
    double p = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) p += s_red[w];
    a.partials[blockIdx.x] = p;
    if (any_bad) atomicOr(a.status + kStNonFinite, 1);
    if (failed) atomicOr(a.status + kStFlags, kFlagTimeout);
  }
  __syncthreads();
  if (failed) mbar_wait_bounded(bar, phase ^ 1u);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

int round16(int x) { return (x + 15) & ~15; }

uint32_t idesc(int M, int N, int prec, bool a_mn, bool b_mn) {
  const uint32_t ab = prec == NVC_PREC_BF16 ? 1u : 0u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory and TMEM plan; returns false with a reason when the network
// does not fit.
// gen (may be NULL): the scene of the fused-data variant, whose occluders,
// lights and targets then take shared memory too.
bool plan(const nvc_handle* h, TrainTcArgs& a, size_t* smem, std::string* why,
          const nvc_scene* gen = nullptr) {
  const int nl = h->n_layers;
  a.n_layers = nl;
  int wbytes = 0, work = 32;
  for (int k = 0; k < nl; ++k) {
    a.K_real[k] = h->w_in[k];
    a.N_real[k] = h->w_out[k];
    a.K[k] = round16(h->w_in[k]);
    a.N[k] = round16(h->w_out[k]);
    a.w_byte_off[k] = wbytes;
    a.w_off[k] = h->w_off[k];
    wbytes += a.K[k] * a.N[k] * 2;
    work = a.N[k] > work ? a.N[k] : work;
    work = a.K[k] > work ? a.K[k] : work;
  }
  a.wimg_bytes = wbytes;
  int off = wbytes;
  for (int k = 0; k < nl; ++k) {
    a.act_off[k] = off;
    off += kTileM * a.K[k] * 2;
  }
  // delta_k lives in tile (last - k) % 2; each tile is sized for its layers
  int dmax[2] = {16, 16};
  for (int k = 0; k < nl; ++k) {
    const int b = (nl - 1 - k) & 1;
    dmax[b] = a.N[k] > dmax[b] ? a.N[k] : dmax[b];
  }
  a.d_off[0] = off;
  off += kTileM * dmax[0] * 2;
  a.d_off[1] = off;
  off += kTileM * dmax[1] * 2;
  a.guard_off = off;
  off += kGuardBytes;
  a.bar_off = off;
  off += 64;
  if (gen) {
    a.occ_off = off;
    off += 16 * h->L + (int)((occluder_bytes(gen->n_spheres, gen->n_boxes) + 15) & ~(size_t)15);
    a.tgt_off = off;
    off += (kTileM * h->L + 15) & ~15;
  }
  uint32_t col = (uint32_t)((work + 31) & ~31);
  for (int k = 0; k < nl; ++k) {
    a.dw_col[k] = col;
    col += (uint32_t)a.K[k];
  }
  if (col > 512) {
    *why = "training network needs more than 512 TMEM columns";
    return false;
  }
  a.tmem_cols = 512;
  for (int k = 0; k < nl; ++k) {
    if (a.N[k] > 256 || a.K[k] > 256) {
      *why = "training layer wider than 256";
      return false;
    }
  }
  // one CTA per SM: it holds all 512 TMEM columns
  *smem = (size_t)off < 120 * 1024 ? 120 * 1024 : (size_t)off;
  if (*smem > 227 * 1024) {
    *why = "training tiles exceed shared memory";
    return false;
  }
  return true;
}

}  // namespace

bool train_tc_supported(const nvc_handle* h, std::string* why) {
  TrainTcArgs a{};
  size_t smem = 0;
  if (!h->mlp_packed) {
    *why = "no tensor-core weight image";
    return false;
  }
  return plan(h, a, &smem, why);
}

template <int F, int PREC, bool GEN>
cudaError_t launch_train_kernel(const TrainTcArgs& a, int grid, size_t smem, cudaStream_t s) {
  auto kern = train_tc_kernel<F, PREC, kGroups, GEN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kTileM * kGroups, smem, s>>>(a);
  return cudaGetLastError();
}

bool train_tc_gen_supported(const nvc_handle* h, const nvc_scene* sc) {
  TrainTcArgs a{};
  size_t smem = 0;
  std::string why;
  return h->mlp_packed && sc && sc->n_lights == h->L && plan(h, a, &smem, &why, sc);
}

cudaError_t launch_train_tc(nvc_handle* h, int64_t n, int* blocks_used, cudaStream_t s,
                            const nvc_scene* gen_scene, const PosGen* gen) {
  TrainTcArgs a{};
  size_t smem = 0;
  std::string why;
  if (!plan(h, a, &smem, &why, gen ? gen_scene : nullptr)) return cudaErrorNotSupported;
  if (gen) {
    a.pg = *gen;
    a.lights = gen_scene->lights;
    a.spheres = gen_scene->spheres;
    a.boxes = gen_scene->boxes;
    a.n_sph = gen_scene->n_spheres;
    a.n_box = gen_scene->n_boxes;
    a.pos_out = h->t_pos;
    a.target_out = h->t_target;
  }
  const int prec = h->cfg.precision == NVC_PREC_BF16 ? NVC_PREC_BF16 : NVC_PREC_FP16;
  a.pos = h->t_pos;
  a.target = h->t_target;
  a.n = n;
  a.table = h->params;
  a.ep = encode_params(h);
  a.wimg = reinterpret_cast<const uint4*>(h->mlp_packed);
  for (int k = 0; k < a.n_layers; ++k) {
    a.idesc_fwd[k] = idesc(kTileM, a.N[k], prec, false, false);
    a.idesc_dw[k] = idesc(kTileM, a.K[k], prec, true, true);
    a.idesc_bwd[k] = idesc(kTileM, a.K[k], prec, false, true);
  }
  a.slope = h->cfg.leaky_slope;
  a.L = h->L;
  a.loss = h->cfg.loss;
  a.loss_scale = h->cfg.loss_scale;
  a.inv_count = 1.0f / ((float)n * (float)h->L);
  a.grad = h->grad;
  a.partials = h->loss_partials;
  a.status = h->status;
  const int64_t n_tiles = (n + kTileM - 1) / kTileM;
  int grid = (int)(n_tiles < h->num_sms ? n_tiles : h->num_sms);
  if (grid > h->n_loss_partials) grid = h->n_loss_partials;
  *blocks_used = grid;
  if (prec == NVC_PREC_BF16) {
    switch (h->F) {
#define NVC_TRAIN_CASE(FF)                                                                      \
  case FF:                                                                                      \
    return gen ? launch_train_kernel<FF, NVC_PREC_BF16, true>(a, grid, smem, s)                   \
               : launch_train_kernel<FF, NVC_PREC_BF16, false>(a, grid, smem, s);
      NVC_TRAIN_CASE(1) NVC_TRAIN_CASE(2) NVC_TRAIN_CASE(4) NVC_TRAIN_CASE(8)
#undef NVC_TRAIN_CASE
    }
  } else {
    switch (h->F) {
#define NVC_TRAIN_CASE(FF)                                                                      \
  case FF:                                                                                      \
    return gen ? launch_train_kernel<FF, NVC_PREC_FP16, true>(a, grid, smem, s)                   \
               : launch_train_kernel<FF, NVC_PREC_FP16, false>(a, grid, smem, s);
      NVC_TRAIN_CASE(1) NVC_TRAIN_CASE(2) NVC_TRAIN_CASE(4) NVC_TRAIN_CASE(8)
#undef NVC_TRAIN_CASE
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace nvc
