// Clustered neural visibility cache (Section 3.6 of the paper): the lights
// are grouped by k-means, the network's outputs are the clusters' average
// visibilities, and a light is sampled in two steps -- a weighted reservoir
// over the clusters, then streaming resampled importance sampling (RIS)
// among a few members of the chosen cluster.
//
// k-means runs on the host in float64 (Lloyd's iterations from given seed
// lights).  On the device:
//   cluster_targets_kernel   training targets: for each (position, cluster)
//                            the binary visibility of one member drawn
//                            uniformly, so the network learns the average;
//   sample_clustered_kernel  per pixel: c_hat_y = sum of the members'
//                            contributions, w_y = max(v_y, 0.001) c_hat_y,
//                            the integer reservoir over the clusters, then
//                            kRis uniform members of cluster y, one kept by
//                            the integer reservoir on their contributions,
//                            and its unbiased contribution weight
//                            W = (sum_j c_j / M) / (p(x) c(x)),
//                            p(x) = (w(y) / w_sum) / m_y.
// Every float32 result is rounded in a fixed order and every random choice
// is a fixed Philox word, so both kernels are reproducible bit for bit.
#include <vector>

#include "nvc_internal.cuh"
#include "shadow.cuh"

namespace nvc {

namespace {

constexpr uint32_t kTagRis = 4;       // candidates in the chosen cluster and their pick
constexpr uint32_t kTagCluster = 5;   // a member light per cluster for the training targets
constexpr int kRis = 4;               // RIS candidates
constexpr int kMaxClusters = 32;

// Word i of the stream (id, frame, view, tag).
__device__ __forceinline__ uint32_t stream_word(uint32_t id, uint32_t frame, uint32_t view,
                                                uint32_t tag, int i, uint32_t k0, uint32_t k1) {
  const uint4 r = philox4x32_10(make_uint4(id, frame, view, ((uint32_t)(i >> 2) << 4) | tag), k0, k1);
  const int l = i & 3;
  return l == 0 ? r.x : l == 1 ? r.y : l == 2 ? r.z : r.w;
}

// Member of cluster y chosen by the word r: floor(r m_y / 2^32).
__device__ __forceinline__ int member_of(const int32_t* off, const int32_t* mem, int y, uint32_t r) {
  const uint32_t m = (uint32_t)(off[y + 1] - off[y]);
  return mem[off[y] + (int)(((uint64_t)r * m) >> 32)];
}

__global__ void __launch_bounds__(256) cluster_targets_kernel(
    const float* __restrict__ lights, const float* __restrict__ spheres, int n_sph,
    const float* __restrict__ boxes, int n_box, const int32_t* __restrict__ off,
    const int32_t* __restrict__ mem, int k, const float* __restrict__ pos, int64_t n,
    uint32_t k0, uint32_t k1, uint32_t frame, float* __restrict__ target) {
  extern __shared__ float4 s_occ[];
  const Occluders occ =
      stage_occluders(spheres, n_sph, boxes, n_box, s_occ, threadIdx.x, blockDim.x);
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t b = t / k;
  const int y = (int)(t - b * k);
  float v = 0.0f;
  if (off[y + 1] > off[y]) {
    const int x = member_of(off, mem, y, stream_word((uint32_t)b, frame, 0u, kTagCluster, y, k0, k1));
    const float4 l = reinterpret_cast<const float4*>(lights)[x];
    const float px = pos[3 * b], py = pos[3 * b + 1], pz = pos[3 * b + 2];
    v = segment_blocked(px, py, pz, l.x, l.y, l.z, occ) ? 0.0f : 1.0f;
  }
  target[t] = v;
}

// Integer reservoir over the first n of N float32 weights w (>= 0) with the
// words r_i: candidate i replaces the pick when r_i Q_i < q_i 2^32, Q_i the
// running sum of the quantised weights (< 2^32).  Loops run over N so the
// arrays stay in registers.
template <int N>
__device__ __forceinline__ int integer_reservoir(const float (&w)[N], int n, const uint32_t (&r)[N]) {
  float wmax = 0.0f;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) wmax = fmaxf(wmax, w[i]);
  if (!(wmax > 0.0f)) return -1;
  const int e = ilogbf(wmax);
  uint32_t Q = 0;
  int sel = -1;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i < n) {
      const uint32_t q = quantize_weight(w[i], e);
      Q += q;
      if (q > 0u && __umulhi(r[i], Q) < q) sel = i;
    }
  }
  return sel;
}

// Light e with I / pi in .w: from the shared copy, or from global memory
// (scaled here, the same rounding) when the lights do not fit on chip.
template <bool kSmemLights>
__device__ __forceinline__ float4 light_at(const float4* s_lt, const float* lights, int e) {
  if (kSmemLights) return s_lt[e];
  float4 l = __ldg(reinterpret_cast<const float4*>(lights) + e);
  l.w = __fmul_rn(l.w, bits_f(kInvPiBits));
  return l;
}

// Integer reservoir over the k cluster weights w with the words of stream
// (pixel, frame, view, kTagWrs), drawn four at a time as the scan reaches
// them: the same picks as integer_reservoir with r[y] = word y.
__device__ __forceinline__ int cluster_reservoir(const float (&w)[kMaxClusters], int k,
                                                 uint32_t pixel, uint32_t frame, uint32_t view,
                                                 uint32_t k0, uint32_t k1) {
  float wmax = 0.0f;
#pragma unroll
  for (int y = 0; y < kMaxClusters; ++y)
    if (y < k) wmax = fmaxf(wmax, w[y]);
  if (!(wmax > 0.0f)) return -1;
  const int e = ilogbf(wmax);
  uint32_t Q = 0;
  int sel = -1;
#pragma unroll
  for (int g = 0; g < kMaxClusters / 4; ++g) {
    if (4 * g < k) {
      const uint4 r4 = philox4x32_10(make_uint4(pixel, frame, view, ((uint32_t)g << 4) | kTagWrs), k0, k1);
      const uint32_t r[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int y = 4 * g + l;
        if (y < k) {
          const uint32_t q = quantize_weight(w[y], e);
          Q += q;
          if (q > 0u && __umulhi(r[l], Q) < q) sel = y;
        }
      }
    }
  }
  return sel;
}

// Lights per shared-memory tile of the tiled step 1 (16 KB).
constexpr int kLightTile = 1024;

// Shared-memory layout: [the lights in cluster-table order, I / pi in .w
// (kSmemLights: all of them; kTiled: one tile of kLightTile)] [spheres]
// [offsets k + 1, as float4 slots] [boxes].  With the lights in table order
// the members of cluster y are the contiguous slots offsets[y] ..
// offsets[y + 1] - 1.
// kSum: first-step weights max(v, 0.001) * c_hat (else max(v, 0.001) alone,
// and no light loop).
// kTiled (with kSum, for light sets too large to stage whole): the CTA's
// threads walk the table in tiles of kLightTile lights staged together in
// shared memory, each thread carrying its pixel's running cluster sum across
// tiles -- the same additions in the same order as the whole-set loop.
template <bool kSmemLights, bool kSum, bool kTiled = false>
__global__ void __launch_bounds__(1024) sample_clustered_kernel(
    const float* __restrict__ lights, int n_lights, const float* __restrict__ spheres, int n_sph,
    const float* __restrict__ boxes, int n_box, const int32_t* __restrict__ off,
    const int32_t* __restrict__ mem, int k, const float* __restrict__ vis,
    const float* __restrict__ pos, const float* __restrict__ nrm, int64_t n,
    int64_t pixel_offset, uint32_t k0, uint32_t k1, uint32_t frame, uint32_t view,
    int32_t* __restrict__ light_out, float* __restrict__ weight_out, float* __restrict__ estimate,
    bool vis_vec4) {
  extern __shared__ float4 s_scene4[];
  const int n_lt_s = kSmemLights ? n_lights : kTiled ? kLightTile : 0;
  float4* s_lt = s_scene4;
  int32_t* s_off = reinterpret_cast<int32_t*>(s_lt + n_lt_s);
  const Occluders occ = stage_occluders(spheres, n_sph, boxes, n_box,
                                        s_lt + n_lt_s + (kMaxClusters + 4) / 4, threadIdx.x,
                                        blockDim.x);
  if (kSmemLights) {
    for (int e = threadIdx.x; e < n_lt_s; e += blockDim.x) {
      float4 l = reinterpret_cast<const float4*>(lights)[mem[e]];
      l.w = __fmul_rn(l.w, bits_f(kInvPiBits));
      s_lt[e] = l;
    }
  }
  for (int e = threadIdx.x; e <= k; e += blockDim.x) s_off[e] = off[e];
  __syncthreads();
  // the CTA walks its pixel batches together (the tiled step 1 has block
  // barriers); a thread past the end takes part in them and writes nothing
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = base + threadIdx.x;
    const bool live = p < n;
    if (!kTiled && !live) continue;
    const int64_t pl = live ? p : 0;
    const float px = pos[3 * pl], py = pos[3 * pl + 1], pz = pos[3 * pl + 2];
    const float nx = nrm[3 * pl], ny = nrm[3 * pl + 1], nz = nrm[3 * pl + 2];
    const uint32_t pixel = (uint32_t)(pixel_offset + p);
    // step 1: the clusters' weights, then the reservoir over them.  The
    // cluster loop stays a loop (one copy of the member loop in the code, so
    // warps at different clusters share the instruction cache); the weights
    // stay in registers through compare-and-select writes.
    float w[kMaxClusters];
    float wsum = 0.0f;
    const float* vrow = vis + pl * k;
    if (kTiled) {
#pragma unroll
      for (int t = 0; t < kMaxClusters; ++t) w[t] = 0.0f;
      int y = 0;
      float ch = 0.0f;
      // cluster y is complete: its weight, in cluster order
      auto finish = [&]() {
        const float wy = __fmul_rn(fmaxf(__ldg(vrow + y), bits_f(kVisClampBits)), ch);
#pragma unroll
        for (int t = 0; t < kMaxClusters; ++t)
          if (t == y) w[t] = wy;
        wsum = __fadd_rn(wsum, wy);
        ch = 0.0f;
        ++y;
      };
      for (int c0 = 0; c0 < n_lights; c0 += kLightTile) {
        const int cn = n_lights - c0 < kLightTile ? n_lights - c0 : kLightTile;
        __syncthreads();   // the previous tile is read by every thread
        for (int e = threadIdx.x; e < cn; e += blockDim.x) {
          float4 l = __ldg(reinterpret_cast<const float4*>(lights) + mem[c0 + e]);
          l.w = __fmul_rn(l.w, bits_f(kInvPiBits));
          s_lt[e] = l;
        }
        __syncthreads();
        if (live) {
#pragma unroll 4
          for (int i = 0; i < cn; ++i) {
            while (c0 + i >= s_off[y + 1]) finish();
            const float4 l = s_lt[i];
            ch = __fadd_rn(ch, contribution(px, py, pz, nx, ny, nz, l.x, l.y, l.z, l.w));
          }
        }
      }
      if (live)
        while (y < k) finish();
    } else if (!kSum) {
      // visibility weights: no member loop, so the row's loads are issued
      // together (16-byte loads when the row allows) into the weights'
      // registers, and the short cluster loop is unrolled
      if (vis_vec4) {
#pragma unroll
        for (int g = 0; g < kMaxClusters / 4; ++g) {
          float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          if (4 * g < k) v = __ldg(reinterpret_cast<const float4*>(vrow) + g);
          w[4 * g] = v.x;
          w[4 * g + 1] = v.y;
          w[4 * g + 2] = v.z;
          w[4 * g + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int t = 0; t < kMaxClusters; ++t) w[t] = t < k ? __ldg(vrow + t) : 0.0f;
      }
#pragma unroll
      for (int t = 0; t < kMaxClusters; ++t) {
        if (t < k) {
          w[t] = s_off[t + 1] > s_off[t] ? fmaxf(w[t], bits_f(kVisClampBits)) : 0.0f;
          wsum = __fadd_rn(wsum, w[t]);
        } else {
          w[t] = 0.0f;
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < kMaxClusters; ++t) w[t] = 0.0f;
#pragma unroll 1
      for (int y = 0; y < k; ++y) {
        const float v = __ldg(vrow + y);
        const int begin = s_off[y], end = s_off[y + 1];
        float ch = 0.0f;
#pragma unroll 4
        for (int i = begin; i < end; ++i) {
          const float4 l = kSmemLights ? s_lt[i] : light_at<false>(s_lt, lights, mem[i]);
          ch = __fadd_rn(ch, contribution(px, py, pz, nx, ny, nz, l.x, l.y, l.z, l.w));
        }
        const float wy = __fmul_rn(fmaxf(v, bits_f(kVisClampBits)), ch);
#pragma unroll
        for (int t = 0; t < kMaxClusters; ++t)
          if (t == y) w[t] = wy;
        wsum = __fadd_rn(wsum, wy);
      }
    }
    if (!live) continue;   // the last batch: nothing to pick, no barrier follows
    const int y = cluster_reservoir(w, k, pixel, frame, view, k0, k1);
    int sel_light = -1;
    float W = 0.0f, cx = 0.0f;
    if (y >= 0) {
      float w_y = 0.0f;
#pragma unroll
      for (int t = 0; t < kMaxClusters; ++t)
        if (t == y) w_y = w[t];
      // step 2: streaming RIS among kRis uniform members of cluster y
      const int base = s_off[y];
      const uint32_t m_y = (uint32_t)(s_off[y + 1] - base);
      const uint4 u = philox4x32_10(make_uint4(pixel, frame, view, (0u << 4) | kTagRis), k0, k1);
      const uint4 v = philox4x32_10(make_uint4(pixel, frame, view, (1u << 4) | kTagRis), k0, k1);
      const uint32_t ru[kRis] = {u.x, u.y, u.z, u.w};
      const uint32_t rr[kRis] = {v.x, v.y, v.z, v.w};
      int slot[kRis];
      float cc[kRis];
#pragma unroll
      for (int t = 0; t < kRis; ++t) {
        slot[t] = base + (int)(((uint64_t)ru[t] * m_y) >> 32);
        const float4 l = kSmemLights ? s_lt[slot[t]] : light_at<false>(s_lt, lights, mem[slot[t]]);
        cc[t] = contribution(px, py, pz, nx, ny, nz, l.x, l.y, l.z, l.w);
      }
      const int j = integer_reservoir(cc, kRis, rr);
      if (j >= 0) {
        float sum = 0.0f;
#pragma unroll
        for (int t = 0; t < kRis; ++t) sum = __fadd_rn(sum, cc[t]);
        float c_j = 0.0f;
        int s_j = 0;
#pragma unroll
        for (int t = 0; t < kRis; ++t)
          if (t == j) {
            c_j = cc[t];
            s_j = slot[t];
          }
        const float mean = __fdiv_rn(sum, (float)kRis);
        const float pr = __fdiv_rn(__fdiv_rn(w_y, wsum), (float)m_y);
        W = __fdiv_rn(mean, __fmul_rn(pr, c_j));
        sel_light = mem[s_j];
        cx = c_j;
      }
    }
    if (light_out) light_out[p] = sel_light;
    if (weight_out) weight_out[p] = W;
    if (estimate) {
      float e = 0.0f;
      if (sel_light >= 0) {
        const float4 l = reinterpret_cast<const float4*>(lights)[sel_light];
        if (!segment_blocked(px, py, pz, l.x, l.y, l.z, occ)) e = __fmul_rn(cx, W);
      }
      estimate[p] = e;
    }
  }
}

// ---- temporal resampling of the cache's reservoirs (ReSTIR, Section 4.2) -----
constexpr uint32_t kTagTemporal = 6;   // the pick between current and previous reservoir
constexpr int kTemporalMCap = 20;      // the previous reservoir counts at most 20x the new one

// p_hat(y) = c_y at the pixel, the correctly rounded float32 contribution
// (0 for y outside [0, n_lights)).
__device__ __forceinline__ float target_of(const float* lights, int n_lights, int y, float px,
                                           float py, float pz, float nx, float ny, float nz) {
  if (y < 0 || y >= n_lights) return 0.0f;
  const float4 l = __ldg(reinterpret_cast<const float4*>(lights) + y);
  return contribution(px, py, pz, nx, ny, nz, l.x, l.y, l.z, __fmul_rn(l.w, bits_f(kInvPiBits)));
}

__global__ void __launch_bounds__(256) temporal_merge_kernel(
    const float* __restrict__ lights, int n_lights, const float* __restrict__ spheres, int n_sph,
    const float* __restrict__ boxes, int n_box, const float* __restrict__ pos,
    const float* __restrict__ nrm, int64_t n, int64_t pixel_offset, uint32_t k0, uint32_t k1,
    uint32_t frame, uint32_t view, const int32_t* __restrict__ cur_light,
    const float* __restrict__ cur_W, const int32_t* __restrict__ prev_light,
    const float* __restrict__ prev_W, const int32_t* __restrict__ prev_M,
    int32_t* __restrict__ light_out, float* __restrict__ W_out, int32_t* __restrict__ M_out,
    float* __restrict__ estimate) {
  extern __shared__ float4 s_occ[];
  Occluders occ = staged_occluders(s_occ, 0, 0);
  if (estimate) {
    occ = stage_occluders(spheres, n_sph, boxes, n_box, s_occ, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float px = pos[3 * p], py = pos[3 * p + 1], pz = pos[3 * p + 2];
    const float nx = nrm[3 * p], ny = nrm[3 * p + 1], nz = nrm[3 * p + 2];
    int yc = cur_light[p];
    int yp = prev_light ? prev_light[p] : -1;
    int Mp = prev_M ? prev_M[p] : 0;
    Mp = Mp < 0 ? 0 : (Mp > kTemporalMCap ? kTemporalMCap : Mp);   // min(M_p, 20 M_c), M_c = 1
    if (yc >= n_lights) yc = -1;
    if (yp >= n_lights || Mp == 0) yp = -1;
    const float pc = target_of(lights, n_lights, yc, px, py, pz, nx, ny, nz);
    const float pp = target_of(lights, n_lights, yp, px, py, pz, nx, ny, nz);
    float w[2];
    w[0] = yc >= 0 ? __fmul_rn(__fmul_rn(1.0f, pc), cur_W[p]) : 0.0f;
    w[1] = yp >= 0 ? __fmul_rn(__fmul_rn((float)Mp, pp), prev_W[p]) : 0.0f;
    const uint4 r4 = philox4x32_10(make_uint4((uint32_t)(pixel_offset + p), frame, view, kTagTemporal),
                                   k0, k1);
    const uint32_t r[2] = {r4.x, r4.y};
    const int j = integer_reservoir(w, 2, r);
    const int y = j == 0 ? yc : j == 1 ? yp : -1;
    const int M = 1 + Mp;
    float W = 0.0f;
    if (y >= 0) W = __fdiv_rn(__fadd_rn(w[0], w[1]), __fmul_rn((float)M, j == 0 ? pc : pp));
    if (light_out) light_out[p] = y;
    if (W_out) W_out[p] = W;
    if (M_out) M_out[p] = M;
    if (estimate) {
      float e = 0.0f;
      if (y >= 0) {
        const float4 l = __ldg(reinterpret_cast<const float4*>(lights) + y);
        if (!segment_blocked(px, py, pz, l.x, l.y, l.z, occ)) e = __fmul_rn(j == 0 ? pc : pp, W);
      }
      estimate[p] = e;
    }
  }
}

}  // namespace

cudaError_t launch_temporal_merge(const nvc_scene* sc, const float* pos, const float* nrm,
                                  int64_t n, int64_t pixel_offset, uint64_t seed, uint32_t frame,
                                  uint32_t view, const int32_t* cur_light, const float* cur_W,
                                  const int32_t* prev_light, const float* prev_W,
                                  const int32_t* prev_M, int32_t* light, float* W, int32_t* M,
                                  float* estimate, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t smem = estimate ? occluder_bytes(sc->n_spheres, sc->n_boxes) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(temporal_merge_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms * 8;
  temporal_merge_kernel<<<(unsigned)(want < cap ? want : cap), 256, smem, s>>>(
      sc->lights, sc->n_lights, sc->spheres, sc->n_spheres, sc->boxes, sc->n_boxes, pos, nrm, n,
      pixel_offset, (uint32_t)seed, (uint32_t)(seed >> 32), frame, view, cur_light, cur_W,
      prev_light, prev_W, prev_M, light, W, M, estimate);
  return cudaGetLastError();
}

cudaError_t launch_cluster_targets(const nvc_scene* sc, const nvc_clusters* cl, const float* pos,
                                   int64_t n, uint64_t seed, uint32_t frame, float* target,
                                   cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t total = n * cl->k;
  const size_t smem = occluder_bytes(sc->n_spheres, sc->n_boxes);
  cluster_targets_kernel<<<(unsigned)((total + 255) / 256), 256, smem, s>>>(
      sc->lights, sc->spheres, sc->n_spheres, sc->boxes, sc->n_boxes, cl->offsets, cl->members,
      cl->k, pos, n, (uint32_t)seed, (uint32_t)(seed >> 32), frame, target);
  return cudaGetLastError();
}

// Shared memory of the sampler: the occluders, plus the lights when they fit
// in the 227 KB a block may opt into (about 14,000 lights); beyond that the
// lights are read through the read-only cache.
constexpr size_t kSmemOptin = 227 * 1024;

size_t sample_clustered_smem(const nvc_scene* sc, const nvc_clusters* cl) {
  const size_t occ =
      occluder_bytes(sc->n_spheres, sc->n_boxes) + sizeof(float4) * ((kMaxClusters + 4) / 4);
  if (cl->weights == NVC_CLUSTER_WEIGHT_VISIBILITY) return occ;   // no light loop
  const size_t lt = sizeof(float) * 4 * (size_t)sc->n_lights;
  return occ + lt <= kSmemOptin ? occ + lt : occ + sizeof(float4) * kLightTile;
}

cudaError_t launch_sample_clustered(const nvc_scene* sc, const nvc_clusters* cl, const float* vis,
                                    const float* pos, const float* nrm, int64_t n,
                                    int64_t pixel_offset, uint64_t seed, uint32_t frame,
                                    uint32_t view, int32_t* light, float* weight, float* estimate,
                                    int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t smem = sample_clustered_smem(sc, cl);
  const bool lights_on_chip =
      occluder_bytes(sc->n_spheres, sc->n_boxes) + sizeof(float4) * ((kMaxClusters + 4) / 4) +
          sizeof(float) * 4 * (size_t)sc->n_lights <=
      kSmemOptin;
  auto kern = cl->weights == NVC_CLUSTER_WEIGHT_VISIBILITY ? sample_clustered_kernel<false, false>
              : lights_on_chip                             ? sample_clustered_kernel<true, true>
                                                           : sample_clustered_kernel<false, true, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // The staged lights are shared by a CTA's threads: take the smallest CTA
  // (128 .. 1024 threads) that keeps the most threads resident per SM, so a
  // large light set does not cut residency.  One wave of resident CTAs
  // strides over the pixels.
  int threads = 128, best = 0;
  for (int t = 128; t <= 1024; t *= 2) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, t, smem);
    if (e != cudaSuccess) return e;
    if (per_sm * t > best) {
      best = per_sm * t;
      threads = t;
    }
  }
  if (best == 0) return cudaErrorInvalidConfiguration;
  const int64_t want = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * (best / threads);
  const int grid = (int)(want < cap ? want : cap);
  // 16-byte loads of a pixel's visibilities need rows of a multiple of 4
  // floats on a 16-byte aligned base
  const bool vis_vec4 = (cl->k & 3) == 0 && (reinterpret_cast<uintptr_t>(vis) & 15) == 0;
  kern<<<grid, threads, smem, s>>>(sc->lights, sc->n_lights, sc->spheres, sc->n_spheres, sc->boxes,
                                   sc->n_boxes, cl->offsets, cl->members, cl->k, vis, pos, nrm, n,
                                   pixel_offset, (uint32_t)seed, (uint32_t)(seed >> 32), frame,
                                   view, light, weight, estimate, vis_vec4);
  return cudaGetLastError();
}

// Lloyd's k-means in float64, the same steps as the oracle: squared
// distances (dx^2 + dy^2) + dz^2, the first nearest centroid, centroids the
// mean of their members summed in light order, empty clusters unchanged.
void kmeans_host(const float* lights, int n, const int32_t* init, int k, int iters,
                 int32_t* assign, double* centroids_out) {
  std::vector<double> C(3 * (size_t)k);
  for (int y = 0; y < k; ++y)
    for (int d = 0; d < 3; ++d) C[3 * y + d] = (double)lights[4 * (size_t)init[y] + d];
  auto assign_all = [&]() {
    for (int i = 0; i < n; ++i) {
      double best = 0.0;
      int arg = 0;
      for (int y = 0; y < k; ++y) {
        const double dx = (double)lights[4 * (size_t)i] - C[3 * y];
        const double dy = (double)lights[4 * (size_t)i + 1] - C[3 * y + 1];
        const double dz = (double)lights[4 * (size_t)i + 2] - C[3 * y + 2];
        const double d2 = (dx * dx + dy * dy) + dz * dz;
        if (y == 0 || d2 < best) {
          best = d2;
          arg = y;
        }
      }
      assign[i] = arg;
    }
  };
  std::vector<double> S(3 * (size_t)k);
  std::vector<int> cnt((size_t)k);
  for (int it = 0; it < iters; ++it) {
    assign_all();
    std::fill(S.begin(), S.end(), 0.0);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int i = 0; i < n; ++i) {
      const int y = assign[i];
      for (int d = 0; d < 3; ++d) S[3 * y + d] = S[3 * y + d] + (double)lights[4 * (size_t)i + d];
      ++cnt[y];
    }
    for (int y = 0; y < k; ++y)
      if (cnt[y] > 0)
        for (int d = 0; d < 3; ++d) C[3 * y + d] = S[3 * y + d] / (double)cnt[y];
  }
  assign_all();
  if (centroids_out)
    for (size_t i = 0; i < C.size(); ++i) centroids_out[i] = C[i];
}

}  // namespace nvc
