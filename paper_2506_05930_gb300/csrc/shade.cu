// Light weights, weighted reservoir sampling and Neural DI (Sections 3.1
// and 3.2 of the paper) on float32 visibility already in memory: the
// separate-kernel path and the stand-alone sampler.
//
// WRS runs in integers so that its decision does not depend on the order
// of floating-point sums: per pixel, e = ilogb(max w), q_i = max(1,
// floor(w_i 2^(23-e))) for w_i > 0, Q_i = q_1 + ... + q_i, and candidate i
// replaces the reservoir iff r_i Q_i < q_i 2^32 (r_i a 32-bit Philox word),
// which is the streaming reservoir rule "keep i with probability
// q_i / Q_i".  One thread per pixel streams over the lights in order.
#include "nvc_internal.cuh"

namespace nvc {

namespace {

struct SceneLights {
  const float* lights;
  int n;
};

// Streaming reservoir over weights produced by `wfn(i)`; the caller has
// already computed wmax.  Returns the selected index or -1.
template <typename WFn>
__device__ __forceinline__ int wrs_stream(WFn wfn, int L, float wmax, uint32_t pixel,
                                          uint32_t frame, uint32_t view, uint32_t k0,
                                          uint32_t k1) {
  if (!(wmax > 0.0f)) return -1;
  const int e = ilogbf(wmax);
  uint64_t Q = 0;
  int sel = -1;
  uint4 r = make_uint4(0, 0, 0, 0);
  for (int i = 0; i < L; ++i) {
    if ((i & 3) == 0)
      r = philox4x32_10(make_uint4(pixel, frame, view, ((uint32_t)(i >> 2) << 4) | kTagWrs), k0, k1);
    const uint32_t ri = (i & 3) == 0 ? r.x : (i & 3) == 1 ? r.y : (i & 3) == 2 ? r.z : r.w;
    const uint32_t q = quantize_weight(wfn(i), e);
    Q += q;
    if (q != 0u && (uint64_t)ri * Q < ((uint64_t)q << 32)) sel = i;
  }
  return sel;
}

__global__ void light_weights_kernel(const float* __restrict__ lights, int L,
                                     const float* __restrict__ pos, const float* __restrict__ nrm,
                                     const float* __restrict__ vis, int64_t n,
                                     float* __restrict__ c_out, float* __restrict__ w_out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * L) return;
  const int64_t p = t / L;
  const int i = (int)(t - p * L);
  const float4 lt = reinterpret_cast<const float4*>(lights)[i];
  const float i_over_pi = __fmul_rn(lt.w, bits_f(kInvPiBits));
  const float c = contribution(pos[3 * p], pos[3 * p + 1], pos[3 * p + 2], nrm[3 * p],
                               nrm[3 * p + 1], nrm[3 * p + 2], lt.x, lt.y, lt.z, i_over_pi);
  if (c_out) c_out[t] = c;
  if (w_out) w_out[t] = __fmul_rn(fmaxf(vis[t], bits_f(kVisClampBits)), c);
}

__global__ void wrs_from_weights_kernel(const float* __restrict__ w, int64_t n, int L,
                                        uint32_t k0, uint32_t k1, uint32_t frame, uint32_t view,
                                        int64_t pixel_offset, int32_t* __restrict__ idx,
                                        float* __restrict__ pdf, float* __restrict__ wsum) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float* wp = w + p * L;
  float wmax = 0.0f, sum = 0.0f;
  for (int i = 0; i < L; ++i) {
    const float wi = wp[i];
    wmax = fmaxf(wmax, wi);
    sum += wi;
  }
  const int sel = wrs_stream([&](int i) { return wp[i]; }, L, wmax,
                             (uint32_t)(pixel_offset + p), frame, view, k0, k1);
  if (idx) idx[p] = sel;
  if (pdf) pdf[p] = sel >= 0 ? wp[sel] / sum : 0.0f;
  if (wsum) wsum[p] = sum;
}

// Separate-kernel shading: visibility already in memory (vis [n][L]).
__global__ void __launch_bounds__(128) shade_from_vis_kernel(
    const float* __restrict__ lights, int L, const float* __restrict__ pos,
    const float* __restrict__ nrm, const float* __restrict__ vis, int64_t n, uint32_t k0,
    uint32_t k1, uint32_t frame, uint32_t view, int64_t pixel_offset, int32_t* __restrict__ idx,
    float* __restrict__ pdf, float* __restrict__ wsum, float* __restrict__ radiance) {
  extern __shared__ float4 s_lights[];   // x, y, z, I/pi
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    float4 lt = reinterpret_cast<const float4*>(lights)[i];
    lt.w = __fmul_rn(lt.w, bits_f(kInvPiBits));
    s_lights[i] = lt;
  }
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float px = pos[3 * p], py = pos[3 * p + 1], pz = pos[3 * p + 2];
  const float nx = nrm[3 * p], ny = nrm[3 * p + 1], nz = nrm[3 * p + 2];
  const float* vp = vis + p * L;
  auto weight = [&](int i) {
    const float4 lt = s_lights[i];
    const float c = contribution(px, py, pz, nx, ny, nz, lt.x, lt.y, lt.z, lt.w);
    return __fmul_rn(fmaxf(vp[i], bits_f(kVisClampBits)), c);
  };
  float wmax = 0.0f, sum = 0.0f, di = 0.0f;
  for (int i = 0; i < L; ++i) {
    const float4 lt = s_lights[i];
    const float c = contribution(px, py, pz, nx, ny, nz, lt.x, lt.y, lt.z, lt.w);
    const float v = vp[i];
    const float wi = __fmul_rn(fmaxf(v, bits_f(kVisClampBits)), c);
    wmax = fmaxf(wmax, wi);
    sum += wi;
    di = fmaf(v, c, di);
  }
  const int sel = wrs_stream(weight, L, wmax, (uint32_t)(pixel_offset + p), frame, view, k0, k1);
  if (idx) idx[p] = sel;
  if (pdf) pdf[p] = sel >= 0 ? weight(sel) / sum : 0.0f;
  if (wsum) wsum[p] = sum;
  if (radiance) radiance[p] = di;
}

}  // namespace

cudaError_t launch_light_weights(const nvc_scene* sc, const float* pos, const float* nrm,
                                 const float* vis, int64_t n, float* c, float* w,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t total = n * sc->n_lights;
  light_weights_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(sc->lights, sc->n_lights,
                                                                     pos, nrm, vis, n, c, w);
  return cudaGetLastError();
}

cudaError_t launch_wrs_from_weights(const float* w, int64_t n, int L, uint64_t seed,
                                    uint32_t frame, uint32_t view, int64_t pixel_offset,
                                    int32_t* idx, float* pdf, float* wsum, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  wrs_from_weights_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(
      w, n, L, (uint32_t)seed, (uint32_t)(seed >> 32), frame, view, pixel_offset, idx, pdf, wsum);
  return cudaGetLastError();
}

cudaError_t launch_shade_from_vis(const nvc_scene* sc, const float* pos, const float* nrm,
                                  const float* vis, int64_t n, uint64_t seed, uint32_t frame,
                                  uint32_t view, int64_t pixel_offset, int32_t* idx,
                                  float* pdf, float* wsum, float* radiance, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t smem = sizeof(float4) * sc->n_lights;
  shade_from_vis_kernel<<<(unsigned)((n + 127) / 128), 128, smem, s>>>(
      sc->lights, sc->n_lights, pos, nrm, vis, n, (uint32_t)seed, (uint32_t)(seed >> 32), frame,
      view, pixel_offset, idx, pdf, wsum, radiance);
  return cudaGetLastError();
}

}  // namespace nvc
