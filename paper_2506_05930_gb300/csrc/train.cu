// Online training (Section 3.4 of the paper): training positions, binary
// shadow-ray targets, the loss and its gradient at the logits, and Adam.
#include "nvc_internal.cuh"
#include "shadow.cuh"

namespace nvc {

namespace {

// ---- training positions (training_position in shadow.cuh) -----------------
__global__ void training_positions_kernel(PosGen g, int64_t batch, float* __restrict__ pos) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  const float3 q = training_position(j, g);
  pos[3 * j] = q.x;
  pos[3 * j + 1] = q.y;
  pos[3 * j + 2] = q.z;
}

// ---- shadow rays (occluder tests in shadow.cuh) -------------------------------
// GEN: the kernel also makes the training positions (training_position),
// the lane of light 0 storing each; otherwise it reads them from pos.
template <bool GEN>
__global__ void __launch_bounds__(256) trace_visibility_kernel(
    const float* __restrict__ lights, int L, const float* __restrict__ spheres, int n_sph,
    const float* __restrict__ boxes, int n_box, float* __restrict__ pos, int64_t n,
    float* __restrict__ vis, PosGen gen) {
  extern __shared__ float4 s_occ[];
  const Occluders occ =
      stage_occluders(spheres, n_sph, boxes, n_box, s_occ, threadIdx.x, blockDim.x);
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * L) return;
  const int64_t p = t / L;
  const int i = (int)(t - p * L);
  float px, py, pz;
  if constexpr (GEN) {
    const float3 q = training_position(p, gen);
    px = q.x;
    py = q.y;
    pz = q.z;
    if (i == 0) {
      pos[3 * p] = px;
      pos[3 * p + 1] = py;
      pos[3 * p + 2] = pz;
    }
  } else {
    px = pos[3 * p];
    py = pos[3 * p + 1];
    pz = pos[3 * p + 2];
  }
  const float4 lt = reinterpret_cast<const float4*>(lights)[i];
  const bool blocked = segment_blocked(px, py, pz, lt.x, lt.y, lt.z, occ);
  vis[t] = blocked ? 0.0f : 1.0f;
}

// ---- loss and its gradient at the logits ------------------------------------
// L2: mean (s - y)^2, d/dz = 2 (s - y) s (1 - s) / n.  BCE: mean softplus(z)
// - y z, d/dz = (s - y) / n.  The gradient is multiplied by the loss scale;
// the loss value is reduced in double, one partial per block.
__global__ void __launch_bounds__(256) loss_grad_kernel(const float* __restrict__ logits,
                                                        const float* __restrict__ target,
                                                        int64_t count, int loss_kind,
                                                        float grad_scale,
                                                        float* __restrict__ dlogits,
                                                        double* __restrict__ partials,
                                                        int32_t* status) {
  __shared__ double s_red[8];
  double acc = 0.0;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float z = logits[e], y = target[e];
    const float s = 1.0f / (1.0f + expf(-z));
    float g;
    if (loss_kind == NVC_LOSS_BCE) {
      acc += (double)(fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - y * z);
      g = s - y;
    } else {
      const float r = s - y;
      acc += (double)r * (double)r;
      g = 2.0f * r * s * (1.0f - s);
    }
    g *= grad_scale;
    bad = bad || !isfinite(z) || !isfinite(g);
    dlogits[e] = g;
  }
  if (bad) atomicOr(status + kStNonFinite, 1);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_red[w];
    partials[blockIdx.x] = sum;
  }
}

constexpr int kLossBlocks = 256;

// ---- Adam -------------------------------------------------------------------
// b^t by repeated squaring: at most 2 log2(t) double multiplications, each
// correctly rounded, so a relative error of a few ulps of a double -- far
// below the float32 the results are stored in.  (A library pow in double is
// several microseconds of dependent FP64 work on this part.)
__device__ __forceinline__ double pow_int(double b, int t) {
  double r = 1.0;
  while (t > 0) {
    if (t & 1) r *= b;
    b *= b;
    t >>= 1;
  }
  return r;
}

// The step's constants, read from the loss partials and the status words
// (not changed here): loss = sum of partials (lane-strided over one warp,
// then a shuffle tree) x inv_count; whether the step applies (all gradients
// finite); step t, bias corrections and the scheduled learning rate.
struct StepPlan {
  AdamScalars sc;
  double loss_sum;
  int t;
  bool nonfinite;
};

struct StepArgs {
  const double* partials;
  int n_partials;
  int schedule, ramp;
  float lr0, lr_end, inv_scale;
  double beta1, beta2;
};

// Called by all 32 lanes of one warp; lane 0's result is the plan.
__device__ __forceinline__ StepPlan plan_step(const StepArgs& a, const int32_t* status) {
  StepPlan pl{};
  double s = 0.0;
  for (int i = threadIdx.x & 31; i < a.n_partials; i += 32) s += a.partials[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  pl.loss_sum = s;
  pl.nonfinite = status[kStNonFinite] != 0;
  pl.t = status[kStStep] + 1;
  double lr = a.lr0;
  if (a.schedule == NVC_LR_RAMP) {
    const int k = pl.t - 1 < a.ramp ? pl.t - 1 : a.ramp;
    lr = (double)a.lr0 + ((double)a.lr_end - (double)a.lr0) * (double)k / (double)a.ramp;
  }
  pl.sc.lr_over_bc1 = (float)(lr / (1.0 - pow_int(a.beta1, pl.t)));
  pl.sc.inv_bc2 = (float)(1.0 / (1.0 - pow_int(a.beta2, pl.t)));
  pl.sc.inv_scale = a.inv_scale;
  pl.sc.skip = pl.nonfinite ? 1 : 0;
  return pl;
}

// The step's bookkeeping, once: the loss, the non-finite flag cleared for
// the next step, and either the step count or the skip count and flag.
__device__ __forceinline__ void commit_step(const StepPlan& pl, bool apply, double inv_count,
                                            double* loss_out, int32_t* status) {
  if (loss_out) *loss_out = pl.loss_sum * inv_count;
  status[kStNonFinite] = 0;
  if (!apply) return;
  if (pl.nonfinite) {
    status[kStSkipped] += 1;
    status[kStFlags] |= kFlagNonFinite;
  } else {
    status[kStStep] = pl.t;
  }
}

// Prologue alone (one warp), for the gradient-only calls: the loss and the
// non-finite flag, no update.
__global__ void adam_prologue_kernel(StepArgs a, double inv_count, double* loss_out,
                                     int32_t* status) {
  const StepPlan pl = plan_step(a, status);
  if (threadIdx.x == 0) commit_step(pl, false, inv_count, loss_out, status);
}

// theta -= (lr / bc1) m / (sqrt(v / bc2) + eps), after m, v updates with the
// unscaled gradient; the gradient buffer is cleared for the next step.
// HBM-bound: each thread issues all loads of two float4 groups before any
// arithmetic; m and v stream (evict-first), theta and its half-precision
// copy are stored normally so the table the shading kernel gathers from is
// still in L2, and gradient entries already zero (table rows no sample
// touched) are not rewritten.
__device__ __forceinline__ void adam_scalar(float& th, float g, float& mm, float& vv,
                                            const AdamScalars& sc, float beta1, float beta2,
                                            float eps) {
  g *= sc.inv_scale;
  mm = fmaf(beta1, mm, (1.0f - beta1) * g);
  vv = fmaf(beta2, vv, (1.0f - beta2) * g * g);
  float s;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(s) : "f"(vv * sc.inv_bc2));
  th -= __fdividef(sc.lr_over_bc1 * mm, s + eps);
}

__device__ __forceinline__ bool nonzero4(float4 g) {
  return g.x != 0.0f || g.y != 0.0f || g.z != 0.0f || g.w != 0.0f;
}

// Element j (an MLP weight) of the 16-bit weight image, set to v.
__device__ __forceinline__ void set_image(const MlpImageMap& mp, uint8_t* img, int64_t j, float v) {
  int k = 0;
  while (k + 1 < mp.n_layers && j >= mp.w_off[k + 1]) ++k;
  const int64_t lj = j - mp.w_off[k];
  const int n = (int)(lj / mp.K_real[k]), kk = (int)(lj - (int64_t)n * mp.K_real[k]);
  const int local = ((((n >> 3) * (mp.K[k] >> 3)) + (kk >> 3)) << 6) + ((n & 7) << 3) + (kk & 7);
  if (mp.bf16)
    reinterpret_cast<__nv_bfloat16*>(img + mp.byte_off[k])[local] = __float2bfloat16_rn(v);
  else
    reinterpret_cast<__half*>(img + mp.byte_off[k])[local] = __float2half_rn(v);
}

// A thread loads kAdamGroups float4 groups (e, e + stride, ...) before any
// arithmetic; the launch keeps at most kAdamCtaCap CTAs of 256 threads per
// SM (0: all that fit).  Two groups and two CTAs (16 warps per SM) was the
// fastest point of the 1080p table's update: 1 to 8 groups at 8 to 32 warps
// per SM all took longer.
constexpr int kAdamGroups = 2;
constexpr int kAdamCtaCap = 2;

struct AdamGroups {
  float4 g[kAdamGroups], th[kAdamGroups], mm[kAdamGroups], vv[kAdamGroups];
};

__device__ __forceinline__ void adam_load(AdamGroups& q, const float4* g4, const float4* th4,
                                          const float4* m4, const float4* v4, int64_t e,
                                          int64_t stride, int64_t n4) {
#pragma unroll
  for (int u = 0; u < kAdamGroups; ++u) {
    const int64_t eu = e + u * stride;
    if (u > 0 && eu >= n4) break;
    q.g[u] = __ldcs(g4 + eu);
    q.th[u] = th4[eu];
    q.mm[u] = __ldcs(m4 + eu);
    q.vv[u] = __ldcs(v4 + eu);
  }
}

// The update proper (sc.skip == 0): grid-stride over float4 groups,
// kAdamGroups at a time, then the tail scalars.  q holds the first
// iteration's groups (e = t0), loaded by the caller before the step's
// scalars were known.
__device__ __forceinline__ void adam_update(float* __restrict__ theta, float* __restrict__ grad,
                                            float* __restrict__ m, float* __restrict__ v,
                                            int64_t n4, int64_t n, float beta1, float beta2,
                                            float eps, const AdamScalars& sc,
                                            uint2* __restrict__ table16, int64_t n_table4,
                                            const MlpImageMap& mp, uint8_t* __restrict__ img,
                                            int64_t t0, int64_t stride, AdamGroups& q) {
  float4* g4 = reinterpret_cast<float4*>(grad);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4* th4 = reinterpret_cast<float4*>(theta);
  float4* m4 = reinterpret_cast<float4*>(m);
  float4* v4 = reinterpret_cast<float4*>(v);
  for (int64_t e = t0; e < n4; e += kAdamGroups * stride) {
    if (e != t0) adam_load(q, g4, th4, m4, v4, e, stride, n4);
    float4 (&g)[kAdamGroups] = q.g;
    float4 (&th)[kAdamGroups] = q.th;
    float4 (&mm)[kAdamGroups] = q.mm;
    float4 (&vv)[kAdamGroups] = q.vv;
#pragma unroll
    for (int u = 0; u < kAdamGroups; ++u) {
      const int64_t ee = e + u * stride;
      if (u > 0 && ee >= n4) break;
      adam_scalar(th[u].x, g[u].x, mm[u].x, vv[u].x, sc, beta1, beta2, eps);
      adam_scalar(th[u].y, g[u].y, mm[u].y, vv[u].y, sc, beta1, beta2, eps);
      adam_scalar(th[u].z, g[u].z, mm[u].z, vv[u].z, sc, beta1, beta2, eps);
      adam_scalar(th[u].w, g[u].w, mm[u].w, vv[u].w, sc, beta1, beta2, eps);
      th4[ee] = th[u];
      if (table16 != nullptr && ee < n_table4) {
        const __half2 a = __floats2half2_rn(th[u].x, th[u].y);
        const __half2 b = __floats2half2_rn(th[u].z, th[u].w);
        table16[ee] = make_uint2(*reinterpret_cast<const uint32_t*>(&a),
                                 *reinterpret_cast<const uint32_t*>(&b));
      }
      if (img != nullptr && 4 * ee >= mp.w_off[0] && 4 * ee < mp.w_off[mp.n_layers]) {
        const float tv[4] = {th[u].x, th[u].y, th[u].z, th[u].w};
        for (int c = 0; c < 4; ++c)
          if (4 * ee + c < mp.w_off[mp.n_layers]) set_image(mp, img, 4 * ee + c, tv[c]);
      }
      __stcs(m4 + ee, mm[u]);
      __stcs(v4 + ee, vv[u]);
      if (nonzero4(g[u])) __stcs(g4 + ee, zero);
    }
  }
  for (int64_t e = 4 * n4 + t0; e < n; e += stride) {
    const float g = grad[e];
    grad[e] = 0.0f;
    adam_scalar(theta[e], g, m[e], v[e], sc, beta1, beta2, eps);
    if (img != nullptr && e >= mp.w_off[0] && e < mp.w_off[mp.n_layers])
      set_image(mp, img, e, theta[e]);
  }
}

// table16 (may be NULL): the half-precision copy of the first 4 n_table4
// parameters (the hash table), rewritten from the updated values.  img (may
// be NULL): the tensor cores' 16-bit weight image, whose MLP weights are
// rewritten from the updated values (the separate packing pass's job).
__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ theta,
                                                   float* __restrict__ grad,
                                                   float* __restrict__ m, float* __restrict__ v,
                                                   int64_t n4, int64_t n, float beta1,
                                                   float beta2, float eps,
                                                   StepArgs step, double inv_count,
                                                   double* loss_out, int32_t* status,
                                                   uint2* __restrict__ table16, int64_t n_table4,
                                                   MlpImageMap mp, uint8_t* __restrict__ img) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float4* g4 = reinterpret_cast<float4*>(grad);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  // the first iteration's loads go out before the step is planned, so the
  // planning warp's latency hides behind them
  AdamGroups q;
  if (t0 < n4)
    adam_load(q, g4, reinterpret_cast<const float4*>(theta), reinterpret_cast<const float4*>(m),
              reinterpret_cast<const float4*>(v), t0, stride, n4);
  // every CTA plans the step from the same inputs (warp 0); the last CTA to
  // finish commits its bookkeeping, after every CTA has read the status
  __shared__ StepPlan s_plan;
  if (threadIdx.x < 32) {
    const StepPlan pl = plan_step(step, status);
    if (threadIdx.x == 0) s_plan = pl;
  }
  __syncthreads();
  const AdamScalars sc = s_plan.sc;
  if (sc.skip) {
    for (int64_t e = t0; e < n4; e += stride)
      if (nonzero4(g4[e])) g4[e] = zero;
    for (int64_t e = 4 * n4 + t0; e < n; e += stride) grad[e] = 0.0f;
  } else {
    adam_update(theta, grad, m, v, n4, n, beta1, beta2, eps, sc, table16, n_table4, mp, img,
                t0, stride, q);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    uint32_t* done = reinterpret_cast<uint32_t*>(status + kStAdamDone);
    if (atomicAdd(done, 1u) == gridDim.x - 1) {
      commit_step(s_plan, true, inv_count, loss_out, status);
      atomicExch(done, 0u);
    }
  }
}


// Copy (and unscale) the accumulated gradient out, clearing it.
__global__ void take_gradient_kernel(float* __restrict__ grad, float* __restrict__ out, int64_t n,
                                     float inv_scale) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    out[e] = grad[e] * inv_scale;
    grad[e] = 0.0f;
  }
}

}  // namespace

PosGen pos_gen(const nvc_scene* sc, const float* screen_pos, int64_t n_screen,
               int64_t batch, uint64_t seed, uint32_t frame, int64_t n_world) {
  const bool have_screen = screen_pos != nullptr && n_screen > 0;
  PosGen g;
  g.lo = make_float3(sc->world_min[0], sc->world_min[1], sc->world_min[2]);
  g.ext = make_float3(sc->world_max[0] - sc->world_min[0], sc->world_max[1] - sc->world_min[1],
                      sc->world_max[2] - sc->world_min[2]);
  g.screen = screen_pos;
  g.n_screen = have_screen ? n_screen : 0;
  g.n_world = !have_screen ? batch : n_world < 0 ? batch - batch / 2
                                                 : (n_world < batch ? n_world : batch);
  g.k0 = (uint32_t)seed;
  g.k1 = (uint32_t)(seed >> 32);
  g.frame = frame;
  return g;
}

cudaError_t launch_training_positions(const nvc_scene* sc, const float* screen_pos,
                                      int64_t n_screen, int64_t batch, uint64_t seed,
                                      uint32_t frame, float* pos, cudaStream_t s,
                                      int64_t n_world) {
  if (batch == 0) return cudaSuccess;
  training_positions_kernel<<<(unsigned)((batch + 255) / 256), 256, 0, s>>>(
      pos_gen(sc, screen_pos, n_screen, batch, seed, frame, n_world), batch, pos);
  return cudaGetLastError();
}

cudaError_t launch_training_data(const nvc_scene* sc, const float* screen_pos, int64_t n_screen,
                                 int64_t batch, uint64_t seed, uint32_t frame, float* pos,
                                 float* vis, cudaStream_t s, int64_t n_world) {
  if (batch == 0) return cudaSuccess;
  if (sc->n_lights < 1)
    return launch_training_positions(sc, screen_pos, n_screen, batch, seed, frame, pos, s, n_world);
  const int64_t total = batch * sc->n_lights;
  const size_t smem = occluder_bytes(sc->n_spheres, sc->n_boxes);
  trace_visibility_kernel<true><<<(unsigned)((total + 255) / 256), 256, smem, s>>>(
      sc->lights, sc->n_lights, sc->spheres, sc->n_spheres, sc->boxes, sc->n_boxes, pos, batch,
      vis, pos_gen(sc, screen_pos, n_screen, batch, seed, frame, n_world));
  return cudaGetLastError();
}

cudaError_t launch_trace_visibility(const nvc_scene* sc, const float* pos, int64_t n, float* vis,
                                    cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t total = n * sc->n_lights;
  const size_t smem = occluder_bytes(sc->n_spheres, sc->n_boxes);
  trace_visibility_kernel<false><<<(unsigned)((total + 255) / 256), 256, smem, s>>>(
      sc->lights, sc->n_lights, sc->spheres, sc->n_spheres, sc->boxes, sc->n_boxes,
      const_cast<float*>(pos), n, vis, PosGen{});
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(nvc_handle* h, int64_t n, cudaStream_t s) {
  h->loss_blocks = kLossBlocks;
  const int64_t count = n * h->L;
  const int top = h->n_layers - 1;
  const int maxdim = h->width > h->L ? h->width : h->L;
  float* dtop = h->t_delta + (int64_t)top * h->B * maxdim;
  const float scale = h->cfg.loss_scale / (float)count;
  loss_grad_kernel<<<kLossBlocks, 256, 0, s>>>(h->t_logits, h->t_target, count, h->cfg.loss, scale,
                                               dtop, h->loss_partials, h->status);
  return cudaGetLastError();
}

cudaError_t launch_adam(nvc_handle* h, double* loss_out, bool apply, cudaStream_t s) {
  const nvc_config& c = h->cfg;
  const double inv_count = 1.0 / ((double)h->B * (double)h->L);
  StepArgs a{};
  a.partials = h->loss_partials;
  a.n_partials = h->loss_blocks > 0 ? h->loss_blocks : kLossBlocks;
  a.schedule = c.lr_schedule;
  a.ramp = c.lr_ramp_steps;
  a.lr0 = c.lr;
  a.lr_end = c.lr_end;
  a.inv_scale = 1.0f / c.loss_scale;
  a.beta1 = (double)c.beta1;
  a.beta2 = (double)c.beta2;
  if (!apply) {
    adam_prologue_kernel<<<1, 32, 0, s>>>(a, inv_count, loss_out, h->status);
    return cudaGetLastError();
  }
  // the step's loss, skip decision and scalars are derived inside the
  // update kernel (one launch)
  const int64_t n4 = h->n_params / 4;
  // kAdamGroups float4 groups per thread and pass: no more CTAs than that
  // covers (a small table would otherwise pay for CTAs that each plan the
  // step and find no work), and no more than one resident wave, so every CTA
  // plans the step once, at the start, while its first loads are in flight
  const int64_t want = (n4 + kAdamGroups * 256 - 1) / (kAdamGroups * 256);
  int per_sm = h->adam_ctas_per_sm > 0 ? h->adam_ctas_per_sm : 1;
  if (kAdamCtaCap > 0 && per_sm > kAdamCtaCap) per_sm = kAdamCtaCap;
  const int64_t cap = (int64_t)h->num_sms * per_sm;
  const int blocks = (int)(want < 1 ? 1 : want < cap ? want : cap);
  MlpImageMap mp{};
  uint8_t* img = mlp_image_map(h, &mp) ? static_cast<uint8_t*>(h->mlp_packed) : nullptr;
  adam_kernel<<<blocks, 256, 0, s>>>(h->params, h->grad, h->adam_m, h->adam_v, n4, h->n_params,
                                     c.beta1, c.beta2, c.eps, a, inv_count, loss_out, h->status,
                                     reinterpret_cast<uint2*>(h->table16), h->n_table / 4, mp, img);
  return cudaGetLastError();
}

cudaError_t adam_occupancy(int* ctas_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, adam_kernel, 256, 0);
}

cudaError_t launch_finish_gradient(nvc_handle* h, float* grad_out, double* loss_out,
                                   cudaStream_t s) {
  cudaError_t e = launch_adam(h, loss_out, false, s);
  if (e != cudaSuccess) return e;
  take_gradient_kernel<<<h->num_sms * 4, 256, 0, s>>>(h->grad, grad_out, h->n_params,
                                                      1.0f / h->cfg.loss_scale);
  return cudaGetLastError();
}

}  // namespace nvc
