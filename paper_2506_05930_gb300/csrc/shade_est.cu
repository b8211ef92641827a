// The shading pass and the all-lights reference.
//
// Shading (Section 3.1): every pixel casts one shadow ray towards the light
// its reservoir picked and forms the one-sample estimate of Eq. 1,
// V_s c_s / p_s, which is unbiased because the sampler gives every light
// with c_i > 0 a nonzero probability.  A running mean over frames
// (a <- a + (e - a) / k for frame k) accumulates it.
//
// Exact direct illumination (the comparison in Section 4.4): a shadow ray
// from every pixel to every light, sum_i V_i c_i.
//
// Both use the shading path's correctly rounded float32 contribution and
// the shadow-ray tests of the training targets, so each binary decision and
// each float32 result is reproducible operation by operation: the estimate
// is c / p (one division), the running mean three correctly rounded steps,
// and the exact DI a sum over lights in order.
#include "nvc_internal.cuh"
#include "shadow.cuh"

namespace nvc {

namespace {

// Stage the lights with I/pi (when given; float4) and then the occluders
// (stage_occluders' layout) in shared memory.
__device__ __forceinline__ Occluders stage_scene(float* s, const float* spheres, int n_sph,
                                                 const float* boxes, int n_box,
                                                 const float* lights, int n_lights) {
  float4* s_lt = reinterpret_cast<float4*>(s);
  for (int e = threadIdx.x; e < n_lights; e += blockDim.x) {
    float4 l = reinterpret_cast<const float4*>(lights)[e];
    l.w = __fmul_rn(l.w, bits_f(kInvPiBits));
    s_lt[e] = l;
  }
  const Occluders occ =
      stage_occluders(spheres, n_sph, boxes, n_box, s + 4 * n_lights, threadIdx.x, blockDim.x);
  __syncthreads();
  return occ;
}

__global__ void __launch_bounds__(256) shade_estimate_kernel(
    const float* __restrict__ lights, const float* __restrict__ spheres, int n_sph,
    const float* __restrict__ boxes, int n_box, const float* __restrict__ pos,
    const float* __restrict__ nrm, int64_t n, const int32_t* __restrict__ idx,
    const float* __restrict__ pdf, float* __restrict__ estimate, float* __restrict__ accum,
    uint32_t count) {
  extern __shared__ float4 s_scene4[];
  const Occluders occ = stage_scene(reinterpret_cast<float*>(s_scene4), spheres, n_sph, boxes,
                                    n_box, lights, 0);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    float e = 0.0f;
    const int32_t s = idx[p];
    const float pr = pdf[p];
    if (s >= 0 && pr > 0.0f) {
      const float4 l = reinterpret_cast<const float4*>(lights)[s];
      const float px = pos[3 * p], py = pos[3 * p + 1], pz = pos[3 * p + 2];
      const float c = contribution(px, py, pz, nrm[3 * p], nrm[3 * p + 1], nrm[3 * p + 2], l.x,
                                   l.y, l.z, __fmul_rn(l.w, bits_f(kInvPiBits)));
      if (c > 0.0f && !segment_blocked(px, py, pz, l.x, l.y, l.z, occ))
        e = __fdiv_rn(c, pr);
    }
    if (estimate) estimate[p] = e;
    if (accum) {
      const float a = accum[p];
      accum[p] = count <= 1u ? e : __fadd_rn(a, __fdiv_rn(__fsub_rn(e, a), (float)count));
    }
  }
}

// kSmemLights: the lights (with I / pi) are staged after the spheres;
// otherwise they are read through the read-only cache and scaled here (the
// same rounding), for scenes whose lights do not fit on chip.
template <bool kSmemLights>
__global__ void __launch_bounds__(256) exact_di_kernel(
    const float* __restrict__ lights, int L, const float* __restrict__ spheres, int n_sph,
    const float* __restrict__ boxes, int n_box, const float* __restrict__ pos,
    const float* __restrict__ nrm, int64_t n, float* __restrict__ di) {
  extern __shared__ float4 s_scene4[];
  const int L_s = kSmemLights ? L : 0;
  const Occluders occ = stage_scene(reinterpret_cast<float*>(s_scene4), spheres, n_sph, boxes,
                                    n_box, lights, L_s);
  const float4* s_lt = s_scene4;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float px = pos[3 * p], py = pos[3 * p + 1], pz = pos[3 * p + 2];
    const float nx = nrm[3 * p], ny = nrm[3 * p + 1], nz = nrm[3 * p + 2];
    float sum = 0.0f;
    for (int i = 0; i < L; ++i) {
      float4 l;
      if (kSmemLights) {
        l = s_lt[i];
      } else {
        l = __ldg(reinterpret_cast<const float4*>(lights) + i);
        l.w = __fmul_rn(l.w, bits_f(kInvPiBits));
      }
      const float c = contribution(px, py, pz, nx, ny, nz, l.x, l.y, l.z, l.w);
      if (c > 0.0f && !segment_blocked(px, py, pz, l.x, l.y, l.z, occ))
        sum = __fadd_rn(sum, c);
    }
    di[p] = sum;
  }
}

int grid_for(int64_t n, int num_sms) {
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms * 8;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_shade_estimate(const nvc_scene* sc, const float* pos, const float* nrm,
                                  int64_t n, const int32_t* idx, const float* pdf,
                                  float* estimate, float* accum, uint32_t count, int num_sms,
                                  cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t smem = occluder_bytes(sc->n_spheres, sc->n_boxes);
  shade_estimate_kernel<<<grid_for(n, num_sms), 256, smem, s>>>(
      sc->lights, sc->spheres, sc->n_spheres, sc->boxes, sc->n_boxes, pos, nrm, n, idx, pdf,
      estimate, accum, count);
  return cudaGetLastError();
}

cudaError_t launch_exact_di(const nvc_scene* sc, const float* pos, const float* nrm, int64_t n,
                            float* di, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t occ = occluder_bytes(sc->n_spheres, sc->n_boxes);
  const size_t lt = sizeof(float) * 4 * (size_t)sc->n_lights;
  const bool on_chip = occ + lt <= 227 * 1024;
  const size_t smem = on_chip ? occ + lt : occ;
  auto kern = on_chip ? exact_di_kernel<true> : exact_di_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid_for(n, num_sms), 256, smem, s>>>(sc->lights, sc->n_lights, sc->spheres,
                                               sc->n_spheres, sc->boxes, sc->n_boxes, pos, nrm,
                                               n, di);
  return cudaGetLastError();
}

}  // namespace nvc
