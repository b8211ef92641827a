// Fused shading with several tile streams per CTA (variants 6 and 7 of
// nvc_shade): the same per-pixel path as fused_tc.cu's kernels -- hash-grid
// encode, tcgen05 MLP, sigmoid, light weights, weighted reservoir sampling
// and Neural DI (Sections 3.1 to 3.3 of the paper) -- with the CTA's weight
// image shared by its groups.  In its own translation unit so that the
// library builds in parallel.
#include "fused_common.cuh"

namespace nvc {

namespace {

using namespace tc;
using namespace fz;

// ---- several tiles per CTA sharing one weight copy ---------------------------
// TPC groups of four warps.  Group g runs its own stream of 128-pixel tiles
// (taken one at a time from the launch's ticket counter) the way the monolithic kernel
// does -- its own activation tile, mbarrier, TMEM columns [g C, (g + 1) C)
// and 128-thread named barrier -- while the weight image is held once per
// CTA for all groups.  Between the sampler's two passes the group's
// activation tile is idle, so it holds the pixels' light weights
// (a row of 36 floats per pixel) in place of 32 registers a thread.  Both savings
// buy warps per SM.  L <= 32, 16-bit operands; outputs bit-identical to the
// monolithic kernel's.  Instantiated separately for exactly 32 lights.
__device__ __forceinline__ void group_sync(int g) {
  switch (g) {
    case 0: asm volatile("bar.sync 1, 128;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 2, 128;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 3, 128;" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 128;" ::: "memory"); break;
  }
}

__device__ __forceinline__ bool group_sync_or(int g, bool v) {
  uint32_t r = 0;
#define NVC_GROUP_OR(ID)                                                      \
  asm volatile(                                                               \
      "{\n\t.reg .pred p, q;\n\t"                                             \
      "setp.ne.u32 q, %1, 0;\n\t"                                             \
      "bar.red.or.pred p, " #ID ", 128, q;\n\t"                               \
      "selp.u32 %0, 1, 0, p;\n\t}\n"                                          \
      : "=r"(r)                                                               \
      : "r"((uint32_t)v)                                                      \
      : "memory")
  switch (g) {
    case 0: NVC_GROUP_OR(1); break;
    case 1: NVC_GROUP_OR(2); break;
    case 2: NVC_GROUP_OR(3); break;
    default: NVC_GROUP_OR(4); break;
  }
#undef NVC_GROUP_OR
  return r != 0;
}

// FEAT: the MLP-only instantiation (nvc_mlp_infer_features): the tile's
// layer-0 operands are read from a.feat16 instead of encoded.
// STAMP: the phase-profile instantiation (nvc_shade_phases).  Thread 0 of
// each group reads the SM clock at four points of every tile -- tile start,
// the encoded A tile complete, the output layer's accumulator read, the end
// of the tile's sampler -- and adds the phases' cycles to a.phase_cycles
// once at exit; outputs are the same as the plain instantiation's.
template <int F, int PREC, int TPC, bool FULL, bool STAMP, bool FEAT = false>
__global__ void __launch_bounds__(kTileM * TPC, TPC == 2 ? 3 : 2)
    fused_shade_multi_kernel(const __grid_constant__ FusedArgs a) {
  constexpr int kThreads = kTileM * TPC;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* s_w = smem;
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int g = t >> 7;                  // this thread's group
  const int rw = t & (kTileM - 1);       // pixel row within the group's tile = TMEM lane
  uint8_t* s_a = smem + a.multi_a + g * a.multi_stride;
  // this pixel's 32 light weights between the passes: rows of 36 floats (16-byte
  // accesses, four wavefronts a warp, the fewest for 16 bytes a thread)
  float4* s_wst4 = reinterpret_cast<float4*>(s_a) + rw * 9;
  float4* s_l = reinterpret_cast<float4*>(smem + a.multi_l);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.multi_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + TPC);
  uint32_t* s_next = s_tmem + 1;         // each group's next tile

  for (int e = t; e < a.wimg_bytes / 16; e += kThreads)
    reinterpret_cast<uint4*>(s_w)[e] = a.wimg[e];
  if (a.lights) stage_light_pairs(s_l, a.lights, a.L, t, kThreads);
  if (t == 0) {
    for (int gg = 0; gg < TPC; ++gg) mbar_init(smem_u32(s_bar + gg), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(s_tmem), a.tmem_cols);
  if (rw == 0) s_next[g] = take_tile(a.status);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_all = *s_tmem;
  const uint32_t tmem = tmem_all + (uint32_t)(g * a.multi_cols);
  const uint32_t t_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t bar = smem_u32(s_bar + g);
  const uint32_t a_base = smem_u32(s_a);
  const uint32_t w_base = smem_u32(s_w);
  uint32_t phase = 0;
  bool failed = false;

  constexpr int CH = 8;
  constexpr int KS = 16;
  const int din = a.ep.n_levels * F;
  const int K0 = a.layer[0].K;
  const int64_t n_tiles = a.n_tiles;
  // FULL: exactly 32 lights, so the light tests fold away, and every level's
  // N_l + 1 < T (checked by the launcher), so the hash's x terms need no mask
  const int L = FULL ? 32 : a.L;
  unsigned long long cyc[3] = {0ull, 0ull, 0ull};
  long long c_tile = 0, c_mark = 0;
  const long long c_loop = STAMP ? clock64() : 0;

  for (int64_t tile = s_next[g]; tile < n_tiles && !failed; tile = s_next[g]) {
    if constexpr (STAMP) c_tile = clock64();
    const ViewDesc& V = a.v[view_of(a, tile)];
    const int64_t row = (tile - V.tile_start) * kTileM + rw;
    const bool live = row < V.n;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (live && !FEAT) {
      px = __ldg(V.pos + 3 * row);
      py = __ldg(V.pos + 3 * row + 1);
      pz = __ldg(V.pos + 3 * row + 2);
    }
    // ---- encode ------------------------------------------------------------
    if constexpr (FEAT) {
      const uint4* src = reinterpret_cast<const uint4*>(a.feat16 + row * K0);
      for (int c = 0; c < K0 / CH; ++c)
        *reinterpret_cast<uint4*>(s_a + cm_offset(rw, c * CH, K0, 2)) =
            live ? __ldg(src + c) : make_uint4(0u, 0u, 0u, 0u);
    } else {
      const float x = normalise(px, a.ep.lo[0], a.ep.ext[0]);
      const float y = normalise(py, a.ep.lo[1], a.ep.ext[1]);
      const float z = normalise(pz, a.ep.lo[2], a.ep.ext[2]);
      auto encode_all = [&](const auto* tab) {
        for (int c = 0; c < K0 / CH; ++c) {
          float fv[CH];
          encode_chunk<F, FULL, CH>(a.ep, tab, c, din, x, y, z, live, fv);
          *reinterpret_cast<uint4*>(s_a + cm_offset(rw, c * CH, K0, 2)) = pack_chunk<PREC, CH>(fv, 1.0f);
        }
      };
      if (a.table16)
        encode_all(a.table16);
      else
        encode_all(a.table);
    }
    fence_async_smem();
    tc_fence_before();
    group_sync(g);
    if constexpr (STAMP) {
      c_mark = clock64();
      cyc[0] += (unsigned long long)(c_mark - c_tile);
    }

    // ---- the MLP -------------------------------------------------------------
    for (int k = 0; k < a.n_layers && !failed; ++k) {
      const LayerDesc ld = a.layer[k];
      if (rw == 0) {
        tc_fence_after();
        const uint32_t sbo = (uint32_t)ld.K * 16u;
        const uint32_t wb = w_base + (uint32_t)ld.w_byte_off;
        for (int kk = 0; kk < ld.K / KS; ++kk)
          mma_f16(tmem, smem_desc(a_base + kk * 256, 128, sbo), smem_desc(wb + kk * 256, 128, sbo),
                  ld.idesc, kk > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      tc_fence_after();
      if (k + 1 < a.n_layers) {
        const int Kn = ld.N;
        for (int c0 = 0; c0 < ld.N; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(t_lane + (uint32_t)c0, r);
#pragma unroll
          for (int gq = 0; gq < 4; ++gq) {
            uint4 pk;
            pk.x = leaky2<PREC>(r[gq * 8 + 0], r[gq * 8 + 1], a.slope);
            pk.y = leaky2<PREC>(r[gq * 8 + 2], r[gq * 8 + 3], a.slope);
            pk.z = leaky2<PREC>(r[gq * 8 + 4], r[gq * 8 + 5], a.slope);
            pk.w = leaky2<PREC>(r[gq * 8 + 6], r[gq * 8 + 7], a.slope);
            if (c0 + gq * 8 < Kn) *reinterpret_cast<uint4*>(s_a + cm_offset(rw, c0 + gq * 8, Kn, 2)) = pk;
          }
        }
        fence_async_smem();
        tc_fence_before();
        failed = group_sync_or(g, !ok);
        continue;
      }

      // ---- output layer (the MMA that read this tile's A has completed) ------
      uint32_t r[32];
      tmem_ld32(t_lane, r);
      if constexpr (STAMP) {
        const long long c = clock64();
        cyc[1] += (unsigned long long)(c - c_mark);
        c_mark = c;
      }
      if (V.vis_out && L == 32 && (reinterpret_cast<uintptr_t>(V.vis_out) & 15) == 0) {
        // the tile's 128 x 32 visibilities are one contiguous block: staged
        // in the idle activation tile (row rw's float4 q at slot q ^ (rw & 7),
        // so a warp's writes spread over the banks), then stored by the
        // group in consecutive 16-byte pieces
        float4* s_v = reinterpret_cast<float4*>(s_a);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          s_v[rw * 8 + (q ^ (rw & 7))] =
              make_float4(sigmoid_fast(__uint_as_float(r[4 * q])),
                          sigmoid_fast(__uint_as_float(r[4 * q + 1])),
                          sigmoid_fast(__uint_as_float(r[4 * q + 2])),
                          sigmoid_fast(__uint_as_float(r[4 * q + 3])));
        group_sync(g);
        const int64_t row0 = (tile - V.tile_start) * kTileM;
        float4* dst = reinterpret_cast<float4*>(V.vis_out + row0 * 32);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
          const int e = rw + k2 * kTileM, rr = e >> 3, q = e & 7;
          if (row0 + rr < V.n) dst[e] = s_v[rr * 8 + (q ^ (rr & 7))];
        }
      } else if (V.vis_out) {
        if (live) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < L) V.vis_out[row * L + j] = sigmoid_fast(__uint_as_float(r[j]));
        }
      } else {
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (live) {
          nx = __ldg(V.nrm + 3 * row);
          ny = __ldg(V.nrm + 3 * row + 1);
          nz = __ldg(V.nrm + 3 * row + 2);
        }
        float wmax = 0.0f, sum = 0.0f, di = 0.0f;
        const float2 npx = make_float2(-px, -px), npy = make_float2(-py, -py),
                     npz = make_float2(-pz, -pz);
        const float2 nx2 = make_float2(nx, nx), ny2 = make_float2(ny, ny), nz2 = make_float2(nz, nz);
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4) {
          float w4[4];
#pragma unroll
          for (int up = 0; up < 2; ++up) {
            const int j = q4 * 4 + up * 2;
            w4[up * 2] = 0.0f;
            w4[up * 2 + 1] = 0.0f;
            if (j < L) {
              // pair j/2 of the staged table
              const float2 c = contribution2_fast(npx, npy, npz, nx2, ny2, nz2, s_l[j], s_l[j + 1]);
              const float2 v01 =
                  sigmoid2_fast(make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])));
              const float v0 = v01.x, v1 = v01.y;
              const float2 w2 = __fmul2_rn(make_float2(fmaxf(v0, bits_f(kVisClampBits)),
                                                       fmaxf(v1, bits_f(kVisClampBits))), c);
              wmax = fmaxf(wmax, w2.x);
              sum += w2.x;
              di = fmaf(v0, c.x, di);
              w4[up * 2] = w2.x;
              if (j + 1 < L) {
                wmax = fmaxf(wmax, w2.y);
                sum += w2.y;
                di = fmaf(v1, c.y, di);
                w4[up * 2 + 1] = w2.y;
              }
            }
          }
          if (q4 * 4 < L) s_wst4[q4] = make_float4(w4[0], w4[1], w4[2], w4[3]);
        }
        if (V.w_out != nullptr && live) {
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            const float4 w4 = s_wst4[q4];
            const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (q4 * 4 + u < L) V.w_out[row * L + q4 * 4 + u] = wv[u];
          }
        }
        int sel = -1;
        float wsel = 0.0f;
        const bool active = live && wmax > 0.0f;
        const QuantScale qs = quant_scale(wmax);
        const float sum_q = __fmul_rn(sum, qs.pre);
        const uint32_t pixel = (uint32_t)(V.pixel_offset + row);
        uint32_t Q = 0;
        uint4 rr = make_uint4(0, 0, 0, 0);
        if (active) {
          float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < L) {
              if ((j & 3) == 0) {
                w4 = s_wst4[j >> 2];
                if (qs.pre != 1.0f)
                  w4 = make_float4(__fmul_rn(w4.x, qs.pre), __fmul_rn(w4.y, qs.pre),
                                   __fmul_rn(w4.z, qs.pre), __fmul_rn(w4.w, qs.pre));
              }
              const float w = (j & 3) == 0 ? w4.x : (j & 3) == 1 ? w4.y : (j & 3) == 2 ? w4.z : w4.w;
              if ((j & 3) == 0)
                rr = philox_keyed(make_uint4(pixel, a.frame, V.view,
                                             ((uint32_t)(j >> 2) << 4) | kTagWrs),
                                  a.rkey);
              const uint32_t q = quantize_scaled(w, qs.scale);
              Q += q;
              if (__umulhi(pick_word(rr, j & 3), Q) < q) sel = j;
            }
          }
          // the picked weight, as the loop saw it
          if (sel >= 0) wsel = __fmul_rn(reinterpret_cast<const float*>(s_wst4)[sel], qs.pre);
        }
        if (live) {
          if (V.idx) V.idx[row] = sel;
          if (V.pdf) V.pdf[row] = sel >= 0 ? wsel / sum_q : 0.0f;
          if (V.wsum) V.wsum[row] = sum;
          if (V.radiance) V.radiance[row] = di;
        }
      }
      if (rw == 0) s_next[g] = take_tile(a.status);
      tc_fence_before();
      // also keeps the next tile's encode from overwriting weights that a
      // slower thread of the group still reads, and publishes s_next[g]
      failed = group_sync_or(g, !ok);
      if constexpr (STAMP) cyc[2] += (unsigned long long)(clock64() - c_mark);
    }
  }
  if constexpr (STAMP) {
    if (rw == 0 && a.phase_cycles) {
      atomicAdd(a.phase_cycles + 0, cyc[0]);
      atomicAdd(a.phase_cycles + 1, cyc[1]);
      atomicAdd(a.phase_cycles + 2, cyc[2]);
      atomicAdd(a.phase_cycles + 3, (unsigned long long)(clock64() - c_loop));
    }
  }
  if (failed && rw == 0) atomicOr(a.status + kStFlags, kFlagTimeout);
  if (rw == 0) finish_tiles(a.status, gridDim.x * TPC);
  if (failed) mbar_wait_bounded(bar, phase ^ 1u);   // let an MMA in flight land
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_all, a.tmem_cols);
  }
}

// Shared-memory plan of the several-tiles-per-CTA kernel: weight image, tpc
// activation tiles (each also holding the 128 pixels' light weights in rows
// of 36 floats), light table, tpc mbarriers, the TMEM address word and the
// groups' next-tile words.
size_t multi_smem(const nvc_handle* h, const PackArgs& p, int tpc, FusedArgs* a = nullptr) {
  int kmax = 16;
  for (int k = 0; k < p.n_layers; ++k) kmax = p.K[k] > kmax ? p.K[k] : kmax;
  size_t off = ((size_t)p.byte_off[p.n_layers] + 127) & ~(size_t)127;
  const size_t a_off = off;
  size_t stride = (size_t)kTileM * kmax * p.esize;
  if (stride < (size_t)kTileM * 36 * 4) stride = (size_t)kTileM * 36 * 4;
  stride = (stride + 127) & ~(size_t)127;
  off += (size_t)tpc * stride;
  const size_t l_off = off;
  off += 16 * (size_t)(h->L > 0 ? ((h->L + 1) & ~1) : 2);
  off = (off + 7) & ~(size_t)7;
  const size_t bar_off = off;
  off += 8 * (size_t)tpc + 8 + 4 * (size_t)tpc;
  if (a) {
    a->multi_a = (int)a_off;
    a->multi_stride = (int)stride;
    a->multi_l = (int)l_off;
    a->multi_bar = (int)bar_off;
  }
  return off;
}

template <int F, int PREC, int TPC>
cudaError_t launch_multi_typed(FusedArgs a, size_t smem_needed, int num_sms, cudaStream_t s) {
  int rmax = 0;
  for (int l = 0; l < a.ep.n_levels; ++l) rmax = a.ep.res[l] > rmax ? a.ep.res[l] : rmax;
  const bool full = a.L == 32 && (int64_t)rmax + 1 < ((int64_t)1 << a.ep.log2_table);
  auto kern = full ? fused_shade_multi_kernel<F, PREC, TPC, true, false>
                   : fused_shade_multi_kernel<F, PREC, TPC, false, false>;
  if (a.phase_cycles)
    kern = full ? fused_shade_multi_kernel<F, PREC, TPC, true, true>
                : fused_shade_multi_kernel<F, PREC, TPC, false, true>;
  if (a.feat16)
    kern = full ? fused_shade_multi_kernel<F, PREC, TPC, true, false, true>
                : fused_shade_multi_kernel<F, PREC, TPC, false, false, true>;
  a.multi_cols = (int)a.tmem_cols;              // per group
  a.tmem_cols = a.tmem_cols * (uint32_t)TPC;    // per CTA (a power of two)
  if (a.tmem_cols > 512u) return cudaErrorInvalidConfiguration;
  const int max_ctas = (int)(512u / a.tmem_cols);
  size_t smem = smem_needed;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)kern);
  if (e != cudaSuccess) return e;
  const size_t dyn_max = 227 * 1024 - fa.sharedSizeBytes;
  if (smem > dyn_max) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
  if (e != cudaSuccess) return e;
  int occ = blocks_per_sm((const void*)kern, TPC * kTileM, smem);
  while (occ > max_ctas && smem + 4096 <= dyn_max) {
    smem += 4096;
    occ = blocks_per_sm((const void*)kern, TPC * kTileM, smem);
  }
  if (occ < 1 || occ > max_ctas) return cudaErrorInvalidConfiguration;
  const int64_t groups = (a.n_tiles + TPC - 1) / TPC;
  const int per_sm = a.max_ctas_per_sm > 0 && a.max_ctas_per_sm < occ ? a.max_ctas_per_sm : occ;
  const int64_t cap = (int64_t)per_sm * num_sms;
  const int grid = (int)(groups < cap ? groups : cap);
  kern<<<grid, TPC * kTileM, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_shade_multi(FusedArgs a, const nvc_handle* h, const PackArgs& p, int tpc,
                               bool bf16, cudaStream_t s) {
  const size_t smem = multi_smem(h, p, tpc, &a);
#define NVC_MULTI(FF)                                                                          \
  if (tpc == 2) return bf16 ? launch_multi_typed<FF, NVC_PREC_BF16, 2>(a, smem, h->num_sms, s) \
                            : launch_multi_typed<FF, NVC_PREC_FP16, 2>(a, smem, h->num_sms, s); \
  return bf16 ? launch_multi_typed<FF, NVC_PREC_BF16, 4>(a, smem, h->num_sms, s)               \
              : launch_multi_typed<FF, NVC_PREC_FP16, 4>(a, smem, h->num_sms, s);
  switch (h->F) {
    case 1: NVC_MULTI(1)
    case 2: NVC_MULTI(2)
    case 4: NVC_MULTI(4)
    case 8: NVC_MULTI(8)
  }
#undef NVC_MULTI
  return cudaErrorInvalidValue;
}

}  // namespace nvc
