// C ABI of libnvc: argument checks, device-state lifetime and the order in
// which the kernels of each entry point are queued.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "nvc_internal.cuh"
#include "shadow.cuh"

using namespace nvc;

namespace {

thread_local std::string g_create_error;

nvc_status fail(nvc_handle* h, nvc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return st;
}

nvc_status cuda_fail(nvc_handle* h, cudaError_t e, const char* what) {
  cudaGetLastError();   // the error is reported here; do not leave it for the next call
  return fail(h, NVC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define NVC_CUDA(h, expr)                                   \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #expr); \
  } while (0)

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int level_res(const nvc_config* c, int l) {
  return (int)std::floor((double)c->base_resolution * std::pow(c->growth, (double)l));
}

nvc_status check_config(const nvc_config* c, std::string* why) {
  auto bad = [&](const char* m) {
    *why = m;
    return NVC_ERR_INVALID_ARG;
  };
  if (!c) return bad("config is NULL");
  if (c->n_levels < 1 || c->n_levels > NVC_MAX_LEVELS) return bad("n_levels out of range");
  if (c->n_features != 1 && c->n_features != 2 && c->n_features != 4 && c->n_features != 8)
    return bad("n_features must be 1, 2, 4 or 8");
  if (c->log2_table_size < 4 || c->log2_table_size > 24) return bad("log2_table_size out of range");
  if (c->base_resolution < 1) return bad("base_resolution must be >= 1");
  if (!(c->growth >= 1.0) || !std::isfinite(c->growth)) return bad("growth must be >= 1");
  if (level_res(c, c->n_levels - 1) > (1 << 22)) return bad("finest level resolution above 2^22");
  if (c->n_hidden < 1 || c->n_hidden > NVC_MAX_HIDDEN_LAYERS) return bad("n_hidden out of range");
  if (c->hidden_width < 16 || c->hidden_width > NVC_MAX_WIDTH || c->hidden_width % 16)
    return bad("hidden_width must be a multiple of 16 in [16, 128]");
  if (c->n_outputs < 1 || c->n_outputs > NVC_MAX_LIGHTS) return bad("n_outputs out of range");
  if (c->n_levels * c->n_features > NVC_MAX_WIDTH) return bad("encoded width above 128");
  if (!(c->leaky_slope >= 0.0f && c->leaky_slope < 1.0f)) return bad("leaky_slope not in [0,1)");
  if (c->precision < NVC_PREC_FP32 || c->precision > NVC_PREC_FP8) return bad("bad precision");
  if (c->train_precision != NVC_PREC_FP32 && c->train_precision != NVC_PREC_FP16)
    return bad("train_precision must be FP32 or FP16");
  if (c->loss != NVC_LOSS_L2 && c->loss != NVC_LOSS_BCE) return bad("bad loss");
  if (c->lr_schedule != NVC_LR_CONSTANT && c->lr_schedule != NVC_LR_RAMP)
    return bad("bad lr_schedule");
  if (c->lr_schedule == NVC_LR_RAMP && c->lr_ramp_steps < 1) return bad("lr_ramp_steps < 1");
  if (!(c->lr > 0.0f) || !std::isfinite(c->lr)) return bad("lr must be > 0");
  if (!(c->beta1 >= 0.0f && c->beta1 < 1.0f) || !(c->beta2 >= 0.0f && c->beta2 < 1.0f))
    return bad("betas must be in [0,1)");
  if (!(c->eps >= 0.0f)) return bad("eps must be >= 0");
  if (!(c->loss_scale > 0.0f) || !std::isfinite(c->loss_scale)) return bad("loss_scale must be > 0");
  if (c->batch_positions < 1 || c->batch_positions > (1 << 24)) return bad("batch_positions out of range");
  for (int d = 0; d < 3; ++d)
    if (!(c->bounds_max[d] > c->bounds_min[d]) || !std::isfinite(c->bounds_max[d]) ||
        !std::isfinite(c->bounds_min[d]))
      return bad("bounds_max must exceed bounds_min");
  return NVC_OK;
}

// Scene checks.  Calls with a per-light output or network neuron take at
// most NVC_MAX_LIGHTS lights; those that only loop over the lights (the
// clustered cache, the shading estimate, the exact DI, the training
// positions) pass kAnyLights.
constexpr int kAnyLights = 0x7fffffff;

nvc_status check_scene(nvc_handle* h, const nvc_scene* sc, int expect_lights,
                       int max_lights = NVC_MAX_LIGHTS) {
  if (!sc) return fail(h, NVC_ERR_INVALID_ARG, "scene is NULL");
  if (!sc->lights || !aligned(sc->lights, 16))
    return fail(h, NVC_ERR_INVALID_ARG, "scene lights NULL or not 16-byte aligned");
  if (sc->n_lights < 1 || sc->n_lights > max_lights)
    return fail(h, NVC_ERR_INVALID_ARG, "n_lights out of range");
  if (expect_lights > 0 && sc->n_lights != expect_lights)
    return fail(h, NVC_ERR_INVALID_ARG, "n_lights (%d) != n_outputs (%d)", sc->n_lights,
                expect_lights);
  if (sc->n_spheres < 0 || sc->n_boxes < 0 ||
      sc->n_spheres + sc->n_boxes > NVC_MAX_OCCLUDERS)
    return fail(h, NVC_ERR_INVALID_ARG, "occluder counts out of range");
  if (sc->n_spheres > 0 && (!sc->spheres || !aligned(sc->spheres, 16)))
    return fail(h, NVC_ERR_INVALID_ARG, "spheres NULL or not 16-byte aligned");
  if (sc->n_boxes > 0 && (!sc->boxes || !aligned(sc->boxes, 4)))
    return fail(h, NVC_ERR_INVALID_ARG, "boxes NULL or misaligned");
  for (int d = 0; d < 3; ++d)
    if (!(sc->world_max[d] >= sc->world_min[d]))
      return fail(h, NVC_ERR_INVALID_ARG, "world_max below world_min");
  return NVC_OK;
}

nvc_status check_ptr(nvc_handle* h, const void* p, const char* name, size_t align = 4) {
  if (!p) return fail(h, NVC_ERR_INVALID_ARG, "%s is NULL", name);
  if (!aligned(p, align)) return fail(h, NVC_ERR_INVALID_ARG, "%s is misaligned", name);
  return NVC_OK;
}

#define NVC_TRY(expr)              \
  do {                             \
    nvc_status st_ = (expr);       \
    if (st_ != NVC_OK) return st_; \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e == cudaSuccess) e = cudaMemset(*p, 0, sizeof(T) * count);
  return e;
}

__global__ void set_status_kernel(int32_t* status, int step) {
  status[kStStep] = step;
  status[kStNonFinite] = 0;
}

__global__ void bump_frames_kernel(int32_t* status) { status[kStFrames] += 1; }

// ---- profiling: event pairs resolved when the caller asks ------------------
struct ProfEvents {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, int>> open;  // (stage, index of start event)
  size_t next = 0;
};

}  // namespace

// Per-handle profiling state lives beside the handle (kept out of the struct
// shared with the kernels' translation units).
namespace {
struct ProfTable {
  nvc_handle* h;
  ProfEvents ev;
};
std::vector<ProfTable*> g_prof;
ProfEvents* prof_of(nvc_handle* h) {
  for (auto* t : g_prof)
    if (t->h == h) return &t->ev;
  return nullptr;
}

struct StageScope {
  nvc_handle* h;
  cudaStream_t s;
  int stage;
  int start = -1;
  StageScope(nvc_handle* hh, cudaStream_t ss, int st) : h(hh), s(ss), stage(st) {
    if (!h->profiling) return;
    ProfEvents* pe = prof_of(h);
    if (!pe || pe->next + 2 > pe->pool.size()) return;
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    start = (int)pe->next;
    pe->next += 2;
    cudaEventRecord(pe->pool[start], s);
  }
  ~StageScope() {
    if (start < 0) return;
    ProfEvents* pe = prof_of(h);
    cudaEventRecord(pe->pool[start + 1], s);
    pe->open.push_back({stage, start});
  }
};

void count_launches(nvc_handle* h, int n) { h->launches += n; }

}  // namespace

namespace nvc {

void record_error(const char* msg) { g_create_error = msg; }

nvc_status validate_config(const nvc_config* c, std::string* why) { return check_config(c, why); }

int blocks_per_sm(const void* func, int block, size_t dyn_smem) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) return 1;
  int dev = 0, regs_sm = 65536, smem_sm = 0, thr_sm = 2048, blk_sm = 32, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int warps = (block + 31) / 32;
  int lim = blk_sm;
  lim = std::min(lim, thr_sm / (warps * 32));
  // registers are allocated per warp in units of 256
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
  if (regs_warp > 0) lim = std::min(lim, regs_sm / (regs_warp * warps));
  const size_t smem = fa.sharedSizeBytes + dyn_smem + (size_t)reserved;
  if (smem > 0) lim = std::min(lim, (int)((size_t)smem_sm / smem));
  return lim < 1 ? 1 : lim;
}

}  // namespace nvc

// ============================================================================
extern "C" {

int64_t nvc_param_count(const nvc_config* cfg) {
  std::string why;
  if (check_config(cfg, &why) != NVC_OK) return -1;
  const int64_t din = (int64_t)cfg->n_levels * cfg->n_features;
  int64_t n = (int64_t)cfg->n_levels * ((int64_t)1 << cfg->log2_table_size) * cfg->n_features;
  n += din * cfg->hidden_width;
  n += (int64_t)(cfg->n_hidden - 1) * cfg->hidden_width * cfg->hidden_width;
  n += (int64_t)cfg->n_outputs * cfg->hidden_width;
  return n;
}

int32_t nvc_level_resolution(const nvc_config* cfg, int32_t level) {
  std::string why;
  if (check_config(cfg, &why) != NVC_OK || level < 0 || level >= cfg->n_levels) return -1;
  return level_res(cfg, level);
}

const char* nvc_last_error(const nvc_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

nvc_status nvc_create(const nvc_config* cfg, nvc_handle** out) {
  if (!out) return fail(nullptr, NVC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::string why;
  if (check_config(cfg, &why) != NVC_OK) return fail(nullptr, NVC_ERR_INVALID_ARG, "%s", why.c_str());
  nvc_handle* h = new (std::nothrow) nvc_handle();
  if (!h) return fail(nullptr, NVC_ERR_CUDA, "out of host memory");
  h->cfg = *cfg;
  h->L = cfg->n_outputs;
  h->F = cfg->n_features;
  h->T = 1 << cfg->log2_table_size;
  h->din = cfg->n_levels * cfg->n_features;
  h->width = cfg->hidden_width;
  h->n_hidden = cfg->n_hidden;
  h->n_layers = cfg->n_hidden + 1;
  for (int l = 0; l < cfg->n_levels; ++l) h->res[l] = level_res(cfg, l);
  h->n_table = (int64_t)cfg->n_levels * h->T * h->F;
  int64_t off = h->n_table;
  for (int k = 0; k < h->n_layers; ++k) {
    h->w_in[k] = k == 0 ? h->din : h->width;
    h->w_out[k] = k == h->n_layers - 1 ? h->L : h->width;
    h->w_off[k] = off;
    off += (int64_t)h->w_in[k] * h->w_out[k];
  }
  h->n_params = off;
  h->B = cfg->batch_positions;

  auto cleanup_fail = [&](cudaError_t e, const char* what) {
    nvc_status st = fail(nullptr, NVC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    nvc_destroy(h);
    return st;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return cleanup_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) !=
      cudaSuccess)
    return cleanup_fail(e, "cudaDeviceGetAttribute");
  if ((e = adam_occupancy(&h->adam_ctas_per_sm)) != cudaSuccess)
    return cleanup_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (mlp_fwd_smem_bytes(h) > (size_t)smem_optin) {
    nvc_status st = fail(nullptr, NVC_ERR_UNSUPPORTED,
                         "MLP of this shape needs %zu B of shared memory (limit %d)",
                         mlp_fwd_smem_bytes(h), smem_optin);
    nvc_destroy(h);
    return st;
  }
  const size_t np4 = (size_t)((h->n_params + 3) / 4) * 4;
  const int maxdim = h->width > h->L ? h->width : h->L;
  const size_t B = (size_t)h->B;
  if ((e = dalloc(&h->params, np4)) || (e = dalloc(&h->grad, np4)) ||
      (e = dalloc(&h->adam_m, np4)) || (e = dalloc(&h->adam_v, np4)) ||
      (e = dalloc(&h->t_pos, B * 3)) || (e = dalloc(&h->t_target, B * h->L)) ||
      (e = dalloc(&h->t_feat, B * h->din)) ||
      (e = dalloc(&h->t_act, (size_t)h->n_hidden * B * h->width)) ||
      (e = dalloc(&h->t_logits, B * h->L)) ||
      (e = dalloc(&h->t_delta, (size_t)h->n_layers * B * maxdim)) ||
      (e = dalloc(&h->t_dfeat, B * h->din)) || (e = dalloc(&h->loss_partials, 256)) ||
      (e = dalloc(&h->status, kStWords)) ||
      (e = dalloc(&h->phase_cycles, 4)))
    return cleanup_fail(e, "cudaMalloc");
  h->n_loss_partials = 256;
  {
    float ones[2 * (NVC_MAX_HIDDEN_LAYERS + 1)];
    for (float& o : ones) o = 1.0f;
    if ((e = dalloc(&h->fp8_scales, 2 * (NVC_MAX_HIDDEN_LAYERS + 1))) ||
        (e = cudaMemcpy(h->fp8_scales, ones, sizeof(ones), cudaMemcpyHostToDevice)))
      return cleanup_fail(e, "cudaMalloc");
  }
  h->mlp_packed_bytes = mlp_packed_bytes(h);
  if (h->mlp_packed_bytes) {
    if ((e = cudaMalloc(&h->mlp_packed, h->mlp_packed_bytes)) != cudaSuccess)
      return cleanup_fail(e, "cudaMalloc");
    cudaMemset(h->mlp_packed, 0, h->mlp_packed_bytes);
  }
  if (cfg->train_precision == NVC_PREC_FP16) {
    std::string why;
    if (cfg->precision == NVC_PREC_FP8) {
      nvc_status st = fail(nullptr, NVC_ERR_UNSUPPORTED,
                           "FP16 training shares the 16-bit weight image: with FP8 inference "
                           "train in FP32");
      nvc_destroy(h);
      return st;
    }
    if (!train_tc_supported(h, &why)) {
      nvc_status st = fail(nullptr, NVC_ERR_UNSUPPORTED, "FP16 training: %s", why.c_str());
      nvc_destroy(h);
      return st;
    }
  }
  h->stage_pixels = 65536;
  if ((e = dalloc(&h->s_feat, (size_t)h->stage_pixels * h->din)) ||
      (e = dalloc(&h->s_vis, (size_t)h->stage_pixels * h->L)))
    return cleanup_fail(e, "cudaMalloc");
  if ((e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cleanup_fail(e, "cudaStreamCreate");
  ProfTable* pt = new ProfTable{h, {}};
  g_prof.push_back(pt);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup_fail(e, "cudaDeviceSynchronize");
  *out = h;
  return NVC_OK;
}

void nvc_destroy(nvc_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  cudaFree(h->params);
  cudaFree(h->grad);
  cudaFree(h->adam_m);
  cudaFree(h->adam_v);
  cudaFree(h->mlp_packed);
  cudaFree(h->table16);
  cudaFree(h->t_pos);
  cudaFree(h->t_target);
  cudaFree(h->t_feat);
  cudaFree(h->t_act);
  cudaFree(h->t_logits);
  cudaFree(h->t_delta);
  cudaFree(h->t_dfeat);
  cudaFree(h->loss_partials);
  cudaFree(h->status);
  cudaFree(h->phase_cycles);
  cudaFree(h->fp8_scales);
  cudaFree(h->s_feat);
  cudaFree(h->s_vis);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (auto& sl : h->host_slot) {
    cudaFree(sl.pos);
    cudaFree(sl.nrm);
    cudaFree(sl.idx);
    cudaFree(sl.out);
    if (sl.up) cudaEventDestroy(sl.up);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.down) cudaEventDestroy(sl.down);
  }
  if (h->up_stream) cudaStreamDestroy(h->up_stream);
  if (h->down_stream) cudaStreamDestroy(h->down_stream);
  for (size_t i = 0; i < g_prof.size(); ++i)
    if (g_prof[i]->h == h) {
      for (cudaEvent_t ev : g_prof[i]->ev.pool) cudaEventDestroy(ev);
      delete g_prof[i];
      g_prof.erase(g_prof.begin() + i);
      break;
    }
  delete h;
}

nvc_status nvc_set_staging(nvc_handle* h, int64_t max_pixels) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (max_pixels < 128 || max_pixels > ((int64_t)1 << 26))
    return fail(h, NVC_ERR_INVALID_ARG, "max_pixels out of range");
  NVC_CUDA(h, cudaDeviceSynchronize());
  cudaFree(h->s_feat);
  cudaFree(h->s_vis);
  h->s_feat = h->s_vis = nullptr;
  h->stage_pixels = 0;
  NVC_CUDA(h, dalloc(&h->s_feat, (size_t)max_pixels * h->din));
  NVC_CUDA(h, dalloc(&h->s_vis, (size_t)max_pixels * h->L));
  h->stage_pixels = max_pixels;
  return NVC_OK;
}

nvc_status nvc_set_state(nvc_handle* h, const float* params, const float* adam_m,
                         const float* adam_v, int32_t step, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  NVC_TRY(check_ptr(h, params, "params"));
  if (step < 0) return fail(h, NVC_ERR_INVALID_ARG, "step < 0");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(float) * (size_t)h->n_params;
  NVC_CUDA(h, cudaMemcpyAsync(h->params, params, bytes, cudaMemcpyDeviceToDevice, s));
  if (adam_m)
    NVC_CUDA(h, cudaMemcpyAsync(h->adam_m, adam_m, bytes, cudaMemcpyDeviceToDevice, s));
  else
    NVC_CUDA(h, cudaMemsetAsync(h->adam_m, 0, bytes, s));
  if (adam_v)
    NVC_CUDA(h, cudaMemcpyAsync(h->adam_v, adam_v, bytes, cudaMemcpyDeviceToDevice, s));
  else
    NVC_CUDA(h, cudaMemsetAsync(h->adam_v, 0, bytes, s));
  NVC_CUDA(h, cudaMemsetAsync(h->grad, 0, bytes, s));
  set_status_kernel<<<1, 1, 0, s>>>(h->status, step);
  NVC_CUDA(h, cudaGetLastError());
  NVC_CUDA(h, launch_pack_mlp(h, s));
  NVC_CUDA(h, launch_pack_table(h, s));
  return NVC_OK;
}

nvc_status nvc_set_params(nvc_handle* h, const float* params, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  NVC_TRY(check_ptr(h, params, "params"));
  cudaStream_t s = (cudaStream_t)stream;
  NVC_CUDA(h, cudaMemcpyAsync(h->params, params, sizeof(float) * (size_t)h->n_params,
                              cudaMemcpyDeviceToDevice, s));
  NVC_CUDA(h, launch_pack_mlp(h, s));
  NVC_CUDA(h, launch_pack_table(h, s));
  return NVC_OK;
}

nvc_status nvc_set_table_precision(nvc_handle* h, int32_t precision, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (precision != NVC_PREC_FP32 && precision != NVC_PREC_FP16)
    return fail(h, NVC_ERR_INVALID_ARG, "table precision must be NVC_PREC_FP32 or NVC_PREC_FP16");
  cudaStream_t s = (cudaStream_t)stream;
  NVC_CUDA(h, cudaStreamSynchronize(s));
  if (precision == NVC_PREC_FP32) {
    NVC_CUDA(h, cudaDeviceSynchronize());
    cudaFree(h->table16);
    h->table16 = nullptr;
    return NVC_OK;
  }
  if (!h->table16) {
    void* p = nullptr;
    NVC_CUDA(h, cudaMalloc(&p, sizeof(__half) * (size_t)h->n_table));
    h->table16 = static_cast<__half*>(p);
  }
  NVC_CUDA(h, launch_pack_table(h, s));
  NVC_CUDA(h, cudaStreamSynchronize(s));
  return NVC_OK;
}

nvc_status nvc_get_state(nvc_handle* h, float* params, float* adam_m, float* adam_v,
                         void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(float) * (size_t)h->n_params;
  if (params) NVC_CUDA(h, cudaMemcpyAsync(params, h->params, bytes, cudaMemcpyDeviceToDevice, s));
  if (adam_m) NVC_CUDA(h, cudaMemcpyAsync(adam_m, h->adam_m, bytes, cudaMemcpyDeviceToDevice, s));
  if (adam_v) NVC_CUDA(h, cudaMemcpyAsync(adam_v, h->adam_v, bytes, cudaMemcpyDeviceToDevice, s));
  return NVC_OK;
}

nvc_status nvc_sync_status(nvc_handle* h, void* stream, nvc_counters* out) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (!out) return fail(h, NVC_ERR_INVALID_ARG, "out is NULL");
  NVC_CUDA(h, cudaStreamSynchronize((cudaStream_t)stream));
  int32_t st[kStWords];
  NVC_CUDA(h, cudaMemcpy(st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
  out->step = st[kStStep];
  out->skipped = st[kStSkipped];
  out->error_flags = st[kStFlags];
  out->frames = st[kStFrames];
  return NVC_OK;
}

nvc_status nvc_encode(nvc_handle* h, const float* pos, int64_t n, float* feat, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(h, NVC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(h, pos, "pos"));
  NVC_TRY(check_ptr(h, feat, "feat", h->F % 2 == 0 ? 8 : 4));
  NVC_CUDA(h, launch_encode_fwd(h, pos, n, feat, (cudaStream_t)stream));
  count_launches(h, 1);
  return NVC_OK;
}

nvc_status nvc_infer(nvc_handle* h, const float* pos, int64_t n, float* vis, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(h, NVC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(h, pos, "pos"));
  NVC_TRY(check_ptr(h, vis, "vis"));
  cudaStream_t s = (cudaStream_t)stream;
  if (h->cfg.precision != NVC_PREC_FP32) {
    std::string why;
    if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
    const int keep = h->shade_variant;
    if (h->infer_variant >= 0) h->shade_variant = h->infer_variant;
    const cudaError_t e = launch_shade_fused(h, nullptr, pos, nullptr, n, 0, 0, 0, 0, nullptr,
                                             nullptr, nullptr, nullptr, vis, s);
    h->shade_variant = keep;
    NVC_CUDA(h, e);
    count_launches(h, 1);
    return NVC_OK;
  }
  for (int64_t o = 0; o < n; o += h->stage_pixels) {
    const int64_t m = n - o < h->stage_pixels ? n - o : h->stage_pixels;
    NVC_CUDA(h, launch_encode_fwd(h, pos + 3 * o, m, h->s_feat, s));
    NVC_CUDA(h, launch_mlp_fwd_fp32(h, h->s_feat, m, vis + o * h->L, true, nullptr, s));
    count_launches(h, 2);
  }
  return NVC_OK;
}

nvc_status nvc_mlp_infer_features(nvc_handle* h, const void* feat, int64_t n, int32_t k0,
                                  float* vis, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (h->cfg.precision != NVC_PREC_FP16 && h->cfg.precision != NVC_PREC_BF16)
    return fail(h, NVC_ERR_UNSUPPORTED, "feature inference needs FP16 or BF16 operands");
  if (h->L > 32) return fail(h, NVC_ERR_UNSUPPORTED, "feature inference needs n_outputs <= 32");
  if (k0 != (h->din + 15) / 16 * 16)
    return fail(h, NVC_ERR_INVALID_ARG, "feat rows must hold %d operands", (h->din + 15) / 16 * 16);
  if (n < 0) return fail(h, NVC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(h, feat, "feat", 16));
  NVC_TRY(check_ptr(h, vis, "vis"));
  std::string why;
  if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
  const FusedView v{nullptr, nullptr, n, 0, 0, nullptr, nullptr, nullptr, nullptr, vis, nullptr};
  NVC_CUDA(h, launch_shade_fused_views(h, nullptr, &v, 1, 0, 0, (cudaStream_t)stream, nullptr,
                                       static_cast<const uint16_t*>(feat)));
  count_launches(h, 1);
  return NVC_OK;
}

nvc_status nvc_light_weights(const nvc_scene* scene, const float* pos, const float* nrm,
                             const float* vis, int64_t n, float* c, float* w, void* stream) {
  NVC_TRY(check_scene(nullptr, scene, 0));
  if (n < 0) return fail(nullptr, NVC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, pos, "pos"));
  NVC_TRY(check_ptr(nullptr, nrm, "nrm"));
  if (w) NVC_TRY(check_ptr(nullptr, vis, "vis"));
  NVC_CUDA(nullptr, launch_light_weights(scene, pos, nrm, vis, n, c, w, (cudaStream_t)stream));
  return NVC_OK;
}

nvc_status nvc_wrs_from_weights(const float* w, int64_t n, int32_t n_lights, uint64_t seed,
                                uint32_t frame, uint32_t view, int64_t pixel_offset,
                                int32_t* idx, float* pdf, float* wsum, void* stream) {
  if (n < 0 || pixel_offset < 0) return fail(nullptr, NVC_ERR_INVALID_ARG, "n or offset < 0");
  if (n_lights < 1 || n_lights > NVC_MAX_LIGHTS)
    return fail(nullptr, NVC_ERR_INVALID_ARG, "n_lights out of range");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, w, "w"));
  NVC_CUDA(nullptr, launch_wrs_from_weights(w, n, n_lights, seed, frame, view, pixel_offset, idx,
                                            pdf, wsum, (cudaStream_t)stream));
  return NVC_OK;
}

static nvc_status shade_impl(nvc_handle* h, const nvc_scene* scene, const float* pos,
                             const float* nrm, int64_t n, uint64_t seed, uint32_t frame,
                             uint32_t view, int64_t pixel_offset, int32_t* idx, float* pdf,
                             float* wsum, float* radiance, int fused, cudaStream_t s) {
  if (fused) {
    std::string why;
    if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
    StageScope sc(h, s, 3);
    NVC_CUDA(h, launch_shade_fused(h, scene, pos, nrm, n, seed, frame, view, pixel_offset, idx,
                                   pdf, wsum, radiance, nullptr, s));
    count_launches(h, 1);
    return NVC_OK;
  }
  StageScope sc(h, s, 3);
  for (int64_t o = 0; o < n; o += h->stage_pixels) {
    const int64_t m = n - o < h->stage_pixels ? n - o : h->stage_pixels;
    NVC_CUDA(h, launch_encode_fwd(h, pos + 3 * o, m, h->s_feat, s));
    NVC_CUDA(h, launch_mlp_fwd_fp32(h, h->s_feat, m, h->s_vis, true, nullptr, s));
    NVC_CUDA(h, launch_shade_from_vis(scene, pos + 3 * o, nrm + 3 * o, h->s_vis, m, seed, frame,
                                      view, pixel_offset + o, idx ? idx + o : nullptr,
                                      pdf ? pdf + o : nullptr, wsum ? wsum + o : nullptr,
                                      radiance ? radiance + o : nullptr, s));
    count_launches(h, 3);
  }
  return NVC_OK;
}

static nvc_status shade_checks(nvc_handle* h, const nvc_scene* scene, const float* pos,
                               const float* nrm, int64_t n, int64_t pixel_offset) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  NVC_TRY(check_scene(h, scene, h->L));
  if (n < 0 || pixel_offset < 0) return fail(h, NVC_ERR_INVALID_ARG, "n or offset < 0");
  if (pixel_offset + n > ((int64_t)1 << 32))
    return fail(h, NVC_ERR_INVALID_ARG, "pixel ids must fit in 32 bits");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(h, pos, "pos"));
  NVC_TRY(check_ptr(h, nrm, "nrm"));
  return NVC_OK;
}

nvc_status nvc_shade(nvc_handle* h, const nvc_scene* scene, const float* pos, const float* nrm,
                     int64_t n, uint64_t seed, uint32_t frame, uint32_t view,
                     int64_t pixel_offset, int32_t* idx, float* pdf, float* wsum,
                     float* radiance, int32_t fused, void* stream) {
  NVC_TRY(shade_checks(h, scene, pos, nrm, n, pixel_offset));
  if (n == 0) return NVC_OK;
  return shade_impl(h, scene, pos, nrm, n, seed, frame, view, pixel_offset, idx, pdf, wsum,
                    radiance, fused, (cudaStream_t)stream);
}

nvc_status nvc_wrs_sample(nvc_handle* h, const nvc_scene* scene, const float* pos,
                          const float* nrm, int64_t n, uint64_t seed, uint32_t frame,
                          uint32_t view, int64_t pixel_offset, int32_t* idx, float* pdf,
                          float* wsum, void* stream) {
  NVC_TRY(shade_checks(h, scene, pos, nrm, n, pixel_offset));
  if (n == 0) return NVC_OK;
  return shade_impl(h, scene, pos, nrm, n, seed, frame, view, pixel_offset, idx, pdf, wsum,
                    nullptr, h->cfg.precision != NVC_PREC_FP32, (cudaStream_t)stream);
}

nvc_status nvc_direct_illum(nvc_handle* h, const nvc_scene* scene, const float* pos,
                            const float* nrm, int64_t n, float* radiance, void* stream) {
  NVC_TRY(shade_checks(h, scene, pos, nrm, n, 0));
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(h, radiance, "radiance"));
  return shade_impl(h, scene, pos, nrm, n, 0, 0, 0, 0, nullptr, nullptr, nullptr, radiance,
                    h->cfg.precision != NVC_PREC_FP32, (cudaStream_t)stream);
}

nvc_status nvc_sampler_weights(nvc_handle* h, const nvc_scene* scene, const float* pos,
                               const float* nrm, int64_t n, float* w, void* stream) {
  NVC_TRY(shade_checks(h, scene, pos, nrm, n, 0));
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(h, w, "w"));
  cudaStream_t s = (cudaStream_t)stream;
  if (h->cfg.precision != NVC_PREC_FP32) {
    std::string why;
    if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
    NVC_CUDA(h, launch_shade_fused(h, scene, pos, nrm, n, 0, 0, 0, 0, nullptr, nullptr, nullptr,
                                   nullptr, nullptr, s, w));
    return NVC_OK;
  }
  for (int64_t o = 0; o < n; o += h->stage_pixels) {
    const int64_t m = n - o < h->stage_pixels ? n - o : h->stage_pixels;
    NVC_CUDA(h, launch_encode_fwd(h, pos + 3 * o, m, h->s_feat, s));
    NVC_CUDA(h, launch_mlp_fwd_fp32(h, h->s_feat, m, h->s_vis, true, nullptr, s));
    NVC_CUDA(h, launch_light_weights(scene, pos + 3 * o, nrm + 3 * o, h->s_vis, m, nullptr,
                                     w + o * h->L, s));
  }
  return NVC_OK;
}

// max |x| over each of the layer inputs of a calibration batch -> E4M3 scale
__global__ void activation_scales_kernel(const float* __restrict__ feat, int64_t feat_n,
                                         const float* __restrict__ act, int64_t act_stride,
                                         int64_t act_n, float* scales) {
  const int k = blockIdx.x;
  const float* x = k == 0 ? feat : act + (int64_t)(k - 1) * act_stride;
  const int64_t n = k == 0 ? feat_n : act_n;
  __shared__ float s_max[32];
  float m = 0.0f;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) m = fmaxf(m, fabsf(x[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_max[w]);
    m = fmaxf(m, s_max[0]);
    scales[k] = m > 0.0f ? 448.0f / m : 1.0f;
  }
}

nvc_status nvc_calibrate(nvc_handle* h, const float* pos, int64_t n, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (n < 1 || n > h->B) return fail(h, NVC_ERR_INVALID_ARG, "n must be in [1, batch_positions]");
  NVC_TRY(check_ptr(h, pos, "pos"));
  cudaStream_t s = (cudaStream_t)stream;
  NVC_CUDA(h, launch_encode_fwd(h, pos, n, h->t_feat, s));
  NVC_CUDA(h, launch_mlp_fwd_fp32(h, h->t_feat, n, h->t_logits, false, h->t_act, s));
  activation_scales_kernel<<<h->n_layers, 256, 0, s>>>(h->t_feat, n * h->din, h->t_act,
                                                        (int64_t)h->B * h->width,
                                                        n * h->width, h->fp8_scales);
  NVC_CUDA(h, cudaGetLastError());
  h->fp8_calibrated = true;
  return NVC_OK;
}

nvc_status nvc_shade_phases(nvc_handle* h, const nvc_scene* scene, const float* pos,
                            const float* nrm, int64_t n, uint64_t seed, uint32_t frame,
                            int32_t* idx, float* pdf, float* wsum, float* radiance,
                            double* cycles_out, void* stream) {
  NVC_TRY(shade_checks(h, scene, pos, nrm, n, 0));
  if (n == 0) return fail(h, NVC_ERR_INVALID_ARG, "need n > 0");
  if (!cycles_out) return fail(h, NVC_ERR_INVALID_ARG, "cycles_out is NULL");
  std::string why;
  if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
  if ((h->shade_variant != kShadeMulti2 && h->shade_variant != kShadeMulti4) || h->L > 32)
    return fail(h, NVC_ERR_UNSUPPORTED,
                "the phase profile instruments the tile-stream variants (6, 7) only");
  cudaStream_t s = (cudaStream_t)stream;
  NVC_CUDA(h, cudaMemsetAsync(h->phase_cycles, 0, 4 * sizeof(unsigned long long), s));
  FusedView v{pos, nrm, n, 0, 0, idx, pdf, wsum, radiance, nullptr, nullptr};
  NVC_CUDA(h, launch_shade_fused_views(h, scene, &v, 1, seed, frame, s, h->phase_cycles));
  unsigned long long c[4];
  NVC_CUDA(h, cudaMemcpyAsync(c, h->phase_cycles, sizeof(c), cudaMemcpyDeviceToHost, s));
  NVC_CUDA(h, cudaStreamSynchronize(s));
  for (int i = 0; i < 4; ++i) cycles_out[i] = (double)c[i];
  count_launches(h, 1);
  return NVC_OK;
}

static nvc_status check_variant(nvc_handle* h, int32_t variant) {
  if (variant < 0 || variant >= kShadeVariants)
    return fail(h, NVC_ERR_INVALID_ARG, "variant out of range");
  if (variant != kShadeMono && variant != kShadePair && h->cfg.precision == NVC_PREC_FP8)
    return fail(h, NVC_ERR_UNSUPPORTED, "E4M3 operands run variants 0 and 5 only");
  if (variant != kShadeMono && variant != kShadePair && h->L > 32)
    return fail(h, NVC_ERR_UNSUPPORTED, "variants 1-4, 6 and 7 need n_outputs <= 32");
  return NVC_OK;
}

nvc_status nvc_set_shade_plan(nvc_handle* h, const nvc_shade_plan* plan) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (!plan) return fail(h, NVC_ERR_INVALID_ARG, "plan is NULL");
  NVC_TRY(check_variant(h, plan->variant));
  if (plan->ctas_per_sm < 0 || plan->ctas_per_sm > 64)
    return fail(h, NVC_ERR_INVALID_ARG, "ctas_per_sm out of range");
  h->shade_variant = plan->variant;
  h->shade_ctas_per_sm = plan->ctas_per_sm;
  return NVC_OK;
}

nvc_status nvc_autotune_shade_plan(nvc_handle* h, const nvc_scene* scene, const float* pos,
                                   const float* nrm, int64_t n, int32_t* idx, float* pdf,
                                   float* wsum, float* radiance, int32_t reps,
                                   nvc_shade_plan* chosen, nvc_shade_plan* points, double* ms,
                                   int32_t max_points, int32_t* n_points, void* stream) {
  NVC_TRY(shade_checks(h, scene, pos, nrm, n, 0));
  if (n == 0 || reps < 1) return fail(h, NVC_ERR_INVALID_ARG, "need n > 0 and reps >= 1");
  if ((points || ms) && max_points < 1) return fail(h, NVC_ERR_INVALID_ARG, "max_points < 1");
  std::string why;
  if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  NVC_CUDA(h, cudaEventCreate(&e0));
  NVC_CUDA(h, cudaEventCreate(&e1));
  const int keep_v = h->shade_variant, keep_c = h->shade_ctas_per_sm;
  nvc_shade_plan best{keep_v, keep_c};
  double best_ms = -1.0;
  int np = 0;
  cudaError_t err = cudaSuccess;
  static const int kCtas[] = {0, 1, 2, 3};
  for (int v = 0; v < kShadeVariants && err == cudaSuccess; ++v) {
    if (check_variant(h, v) != NVC_OK) continue;
    for (int c : kCtas) {
      h->shade_variant = v;
      h->shade_ctas_per_sm = c;
      if (launch_shade_fused(h, scene, pos, nrm, n, 1, 0, 0, 0, idx, pdf, wsum, radiance, nullptr,
                             s) != cudaSuccess) {
        cudaGetLastError();
        break;                         // the layout does not fit this configuration
      }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r)
        launch_shade_fused(h, scene, pos, nrm, n, 1, (uint32_t)r, 0, 0, idx, pdf, wsum, radiance,
                           nullptr, s);
      cudaEventRecord(e1, s);
      if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      const double per = (double)t / reps;
      if (np < max_points) {
        if (points) points[np] = nvc_shade_plan{v, c};
        if (ms) ms[np] = per;
      }
      ++np;
      if (best_ms < 0.0 || per < best_ms) {
        best_ms = per;
        best = nvc_shade_plan{v, c};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    h->shade_variant = keep_v;
    h->shade_ctas_per_sm = keep_c;
    return cuda_fail(h, err, "autotune");
  }
  h->shade_variant = best.variant;
  h->shade_ctas_per_sm = best.ctas_per_sm;
  if (chosen) *chosen = best;
  if (n_points) *n_points = np;
  return NVC_OK;
}

nvc_status nvc_set_shade_variant(nvc_handle* h, int32_t variant) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (variant < 0 || variant >= kShadeVariants)
    return fail(h, NVC_ERR_INVALID_ARG, "variant out of range");
  if (variant != kShadeMono && variant != kShadePair && h->cfg.precision == NVC_PREC_FP8)
    return fail(h, NVC_ERR_UNSUPPORTED, "E4M3 operands run variants 0 and 5 only");
  if (variant != kShadeMono && variant != kShadePair && h->L > 32)
    return fail(h, NVC_ERR_UNSUPPORTED, "variants 1-4, 6 and 7 need n_outputs <= 32");
  h->shade_variant = variant;
  return NVC_OK;
}

nvc_status nvc_autotune_infer(nvc_handle* h, const float* pos, int64_t n, float* vis,
                              int32_t reps, int32_t* chosen, double* ms_out, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (n <= 0 || reps < 1) return fail(h, NVC_ERR_INVALID_ARG, "need n > 0 and reps >= 1");
  NVC_TRY(check_ptr(h, pos, "pos"));
  NVC_TRY(check_ptr(h, vis, "vis"));
  for (int v = 0; v < kShadeVariants; ++v)
    if (ms_out) ms_out[v] = -1.0;
  if (h->cfg.precision == NVC_PREC_FP32) {   // the float32 path has no variants
    if (chosen) *chosen = -1;
    return NVC_OK;
  }
  std::string why;
  if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  NVC_CUDA(h, cudaEventCreate(&e0));
  NVC_CUDA(h, cudaEventCreate(&e1));
  const int keep = h->shade_variant;
  int best = -1;
  double best_ms = 0.0;
  cudaError_t err = cudaSuccess;
  for (int v = 0; v < kShadeVariants && err == cudaSuccess; ++v) {
    if (v != kShadeMono && v != kShadePair && h->cfg.precision == NVC_PREC_FP8) continue;
    if (v != kShadeMono && v != kShadePair && h->L > 32) continue;
    h->shade_variant = v;
    if (launch_shade_fused(h, nullptr, pos, nullptr, n, 0, 0, 0, 0, nullptr, nullptr, nullptr,
                           nullptr, vis, s) != cudaSuccess) {
      cudaGetLastError();
      continue;                       // variant does not fit this configuration
    }
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r)
      launch_shade_fused(h, nullptr, pos, nullptr, n, 0, 0, 0, 0, nullptr, nullptr, nullptr,
                         nullptr, vis, s);
    cudaEventRecord(e1, s);
    if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = (double)ms / reps;
    if (ms_out) ms_out[v] = per;
    if (best < 0 || per < best_ms) {
      best = v;
      best_ms = per;
    }
  }
  h->shade_variant = keep;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(h, err, "autotune");
  if (best >= 0) h->infer_variant = best;
  if (chosen) *chosen = h->infer_variant;
  return NVC_OK;
}

nvc_status nvc_autotune_shade(nvc_handle* h, const nvc_scene* scene, const float* pos,
                              const float* nrm, int64_t n, int32_t* idx, float* pdf,
                              float* wsum, float* radiance, int32_t reps, int32_t* chosen,
                              double* ms_out, void* stream) {
  NVC_TRY(shade_checks(h, scene, pos, nrm, n, 0));
  if (n == 0 || reps < 1) return fail(h, NVC_ERR_INVALID_ARG, "need n > 0 and reps >= 1");
  std::string why;
  if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  NVC_CUDA(h, cudaEventCreate(&e0));
  NVC_CUDA(h, cudaEventCreate(&e1));
  const int keep = h->shade_variant;
  int best = -1;
  double best_ms = 0.0;
  for (int v = 0; v < kShadeVariants; ++v) {
    if (ms_out) ms_out[v] = -1.0;
    if (v != kShadeMono && v != kShadePair && h->cfg.precision == NVC_PREC_FP8) continue;
    if (v != kShadeMono && v != kShadePair && h->L > 32) continue;
    h->shade_variant = v;
    cudaError_t e = launch_shade_fused(h, scene, pos, nrm, n, 1, 0, 0, 0, idx, pdf, wsum,
                                       radiance, nullptr, s);
    if (e != cudaSuccess) continue;   // variant does not fit this configuration
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r)
      launch_shade_fused(h, scene, pos, nrm, n, 1, (uint32_t)r, 0, 0, idx, pdf, wsum, radiance,
                         nullptr, s);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      h->shade_variant = keep;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(h, e, "autotune");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = (double)ms / reps;
    if (ms_out) ms_out[v] = per;
    if (best < 0 || per < best_ms) {
      best = v;
      best_ms = per;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->shade_variant = best < 0 ? keep : best;
  if (chosen) *chosen = h->shade_variant;
  return NVC_OK;
}

nvc_status nvc_trace_visibility(const nvc_scene* scene, const float* pos, int64_t n, float* vis,
                                void* stream) {
  NVC_TRY(check_scene(nullptr, scene, 0));
  if (n < 0) return fail(nullptr, NVC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, pos, "pos"));
  NVC_TRY(check_ptr(nullptr, vis, "vis"));
  NVC_CUDA(nullptr, launch_trace_visibility(scene, pos, n, vis, (cudaStream_t)stream));
  return NVC_OK;
}

static cudaError_t current_sms(int* n) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  return cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev);
}

nvc_status nvc_shade_estimate(const nvc_scene* scene, const float* pos, const float* nrm,
                              int64_t n, const int32_t* idx, const float* pdf, float* estimate,
                              float* accum, uint32_t count, void* stream) {
  NVC_TRY(check_scene(nullptr, scene, 0, kAnyLights));
  if (n < 0) return fail(nullptr, NVC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, pos, "pos"));
  NVC_TRY(check_ptr(nullptr, nrm, "nrm"));
  NVC_TRY(check_ptr(nullptr, idx, "idx"));
  NVC_TRY(check_ptr(nullptr, pdf, "pdf"));
  if (!estimate && !accum) return fail(nullptr, NVC_ERR_INVALID_ARG, "estimate and accum both NULL");
  if (estimate) NVC_TRY(check_ptr(nullptr, estimate, "estimate"));
  if (accum) {
    NVC_TRY(check_ptr(nullptr, accum, "accum"));
    if (count < 1) return fail(nullptr, NVC_ERR_INVALID_ARG, "count must be >= 1");
  }
  int sms = 0;
  NVC_CUDA(nullptr, current_sms(&sms));
  NVC_CUDA(nullptr, launch_shade_estimate(scene, pos, nrm, n, idx, pdf, estimate, accum, count,
                                          sms, (cudaStream_t)stream));
  return NVC_OK;
}

nvc_status nvc_exact_di(const nvc_scene* scene, const float* pos, const float* nrm, int64_t n,
                        float* di, void* stream) {
  NVC_TRY(check_scene(nullptr, scene, 0, kAnyLights));
  if (n < 0) return fail(nullptr, NVC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, pos, "pos"));
  NVC_TRY(check_ptr(nullptr, nrm, "nrm"));
  NVC_TRY(check_ptr(nullptr, di, "di"));
  int sms = 0;
  NVC_CUDA(nullptr, current_sms(&sms));
  NVC_CUDA(nullptr, launch_exact_di(scene, pos, nrm, n, di, sms, (cudaStream_t)stream));
  return NVC_OK;
}

nvc_status nvc_training_positions_split(const nvc_scene* scene, const float* screen_pos,
                                        int64_t n_screen, int64_t batch, int64_t n_world,
                                        uint64_t seed, uint32_t frame, float* pos, void* stream) {
  NVC_TRY(check_scene(nullptr, scene, 0, kAnyLights));
  if (batch < 0 || n_screen < 0 || n_screen > ((int64_t)1 << 32))
    return fail(nullptr, NVC_ERR_INVALID_ARG, "batch or n_screen out of range");
  if (batch > ((int64_t)1 << 32)) return fail(nullptr, NVC_ERR_INVALID_ARG, "batch above 2^32");
  if (n_world < -1 || n_world > batch)
    return fail(nullptr, NVC_ERR_INVALID_ARG, "n_world must be -1 or 0..batch");
  if (batch == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, pos, "pos"));
  if (n_screen > 0 && screen_pos) NVC_TRY(check_ptr(nullptr, screen_pos, "screen_pos"));
  NVC_CUDA(nullptr, launch_training_positions(scene, screen_pos, n_screen, batch, seed, frame, pos,
                                              (cudaStream_t)stream, n_world));
  return NVC_OK;
}

nvc_status nvc_training_positions(const nvc_scene* scene, const float* screen_pos,
                                  int64_t n_screen, int64_t batch, uint64_t seed, uint32_t frame,
                                  float* pos, void* stream) {
  return nvc_training_positions_split(scene, screen_pos, n_screen, batch, -1, seed, frame, pos,
                                      stream);
}

nvc_status nvc_set_training_data_fused(nvc_handle* h, int32_t fused) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (fused && h->cfg.train_precision != NVC_PREC_FP16)
    return fail(h, NVC_ERR_UNSUPPORTED, "the fused training data needs FP16 training");
  h->fused_training_data = fused != 0;
  return NVC_OK;
}

nvc_status nvc_training_batch(nvc_handle* h, float* pos, float* target, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (pos) {
    NVC_TRY(check_ptr(h, pos, "pos"));
    NVC_CUDA(h, cudaMemcpyAsync(pos, h->t_pos, sizeof(float) * 3 * (size_t)h->B,
                                cudaMemcpyDeviceToDevice, s));
  }
  if (target) {
    NVC_TRY(check_ptr(h, target, "target"));
    NVC_CUDA(h, cudaMemcpyAsync(target, h->t_target, sizeof(float) * (size_t)h->B * h->L,
                                cudaMemcpyDeviceToDevice, s));
  }
  return NVC_OK;
}

nvc_status nvc_set_training_placement(nvc_handle* h, int64_t n_world) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (n_world < -1 || n_world > h->B)
    return fail(h, NVC_ERR_INVALID_ARG, "n_world must be -1 or 0..batch_positions");
  h->n_world = n_world;
  return NVC_OK;
}

// Forward + backward of one training batch into h->grad (scaled by the loss
// scale); positions are generated unless `given_pos` is set.
static nvc_status train_forward_backward(nvc_handle* h, const nvc_scene* scene,
                                         const float* screen_pos, int64_t n_screen,
                                         uint64_t seed, uint32_t frame, cudaStream_t s,
                                         const nvc_clusters* clusters = nullptr) {
  const int64_t B = h->B;
  if (!clusters && h->fused_training_data && h->cfg.train_precision == NVC_PREC_FP16 &&
      train_tc_gen_supported(h, scene)) {
    // positions, shadow-ray targets, forward, loss, backward and the hash
    // scatter in one tensor-core launch
    StageScope sc(h, s, 1);
    const PosGen g = pos_gen(scene, screen_pos, n_screen, B, seed, frame, h->n_world);
    int blocks = 0;
    NVC_CUDA(h, launch_train_tc(h, B, &blocks, s, scene, &g));
    h->loss_blocks = blocks;
    count_launches(h, 1);
    return NVC_OK;
  }
  {
    StageScope sc(h, s, 0);
    if (clusters) {
      // positions, then one member's visibility per cluster (Section 3.6)
      NVC_CUDA(h, launch_training_positions(scene, screen_pos, n_screen, B, seed, frame, h->t_pos, s,
                                            h->n_world));
      NVC_CUDA(h, launch_cluster_targets(scene, clusters, h->t_pos, B, seed, frame, h->t_target, s));
      count_launches(h, 2);
    } else {
      // positions and their shadow-ray targets in one kernel
      NVC_CUDA(h, launch_training_data(scene, screen_pos, n_screen, B, seed, frame, h->t_pos,
                                       h->t_target, s, h->n_world));
      count_launches(h, 1);
    }
  }
  StageScope sc(h, s, 1);
  if (h->cfg.train_precision == NVC_PREC_FP16) {
    // encode, forward, loss, backward and the hash scatter in one tensor-core kernel
    int blocks = 0;
    NVC_CUDA(h, launch_train_tc(h, B, &blocks, s));
    h->loss_blocks = blocks;
    count_launches(h, 1);
    return NVC_OK;
  }
  NVC_CUDA(h, launch_encode_fwd(h, h->t_pos, B, h->t_feat, s));
  NVC_CUDA(h, launch_mlp_fwd_fp32(h, h->t_feat, B, h->t_logits, false, h->t_act, s));
  NVC_CUDA(h, launch_loss_grad(h, B, s));
  NVC_CUDA(h, launch_mlp_bwd_fp32(h, B, nullptr, h->grad, h->status, s));
  NVC_CUDA(h, launch_encode_bwd(h, h->t_pos, B, h->t_dfeat, h->grad, h->status, s));
  count_launches(h, 4 + 1 + h->n_layers);
  return NVC_OK;
}

static nvc_status train_checks(nvc_handle* h, const nvc_scene* scene, const float* screen_pos,
                               int64_t n_screen) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  NVC_TRY(check_scene(h, scene, h->L));
  if (n_screen < 0 || n_screen > ((int64_t)1 << 32))
    return fail(h, NVC_ERR_INVALID_ARG, "n_screen out of range");
  if (n_screen > 0 && screen_pos) NVC_TRY(check_ptr(h, screen_pos, "screen_pos"));
  return NVC_OK;
}

static nvc_status train_step_impl(nvc_handle* h, const nvc_scene* scene, const float* screen_pos,
                                  int64_t n_screen, uint64_t seed, uint32_t frame,
                                  double* loss_out, cudaStream_t s,
                                  const nvc_clusters* clusters = nullptr) {
  NVC_TRY(train_forward_backward(h, scene, screen_pos, n_screen, seed, frame, s, clusters));
  StageScope sc(h, s, 2);
  NVC_CUDA(h, launch_adam(h, loss_out, true, s));
  // the Adam kernel rewrites a 16-bit weight image itself; E4M3 repacks
  MlpImageMap mp;
  const bool in_adam = mlp_image_map(h, &mp);
  if (!in_adam) NVC_CUDA(h, launch_pack_mlp(h, s));
  count_launches(h, 1 + (h->mlp_packed && !in_adam ? 1 : 0));
  return NVC_OK;
}

nvc_status nvc_train_step(nvc_handle* h, const nvc_scene* scene, const float* screen_pos,
                          int64_t n_screen, uint64_t seed, uint32_t frame, double* loss_out,
                          void* stream) {
  NVC_TRY(train_checks(h, scene, screen_pos, n_screen));
  if (loss_out) NVC_TRY(check_ptr(h, loss_out, "loss_out", 8));
  return train_step_impl(h, scene, screen_pos, n_screen, seed, frame, loss_out,
                         (cudaStream_t)stream);
}

static nvc_status check_clusters(nvc_handle* h, const nvc_scene* scene, const nvc_clusters* cl,
                                 int expect_k) {
  if (!cl) return fail(h, NVC_ERR_INVALID_ARG, "clusters is NULL");
  if (cl->k < 1 || cl->k > 32) return fail(h, NVC_ERR_INVALID_ARG, "clusters: k must be 1..32");
  if (expect_k > 0 && cl->k != expect_k)
    return fail(h, NVC_ERR_INVALID_ARG, "clusters: k must equal n_outputs");
  if (!cl->offsets || !cl->members) return fail(h, NVC_ERR_INVALID_ARG, "clusters: NULL table");
  if (cl->weights != NVC_CLUSTER_WEIGHT_SUM && cl->weights != NVC_CLUSTER_WEIGHT_VISIBILITY)
    return fail(h, NVC_ERR_INVALID_ARG, "clusters: unknown weight mode");
  NVC_TRY(check_ptr(h, cl->offsets, "clusters.offsets"));
  NVC_TRY(check_ptr(h, cl->members, "clusters.members"));
  if (scene->n_lights < 1) return fail(h, NVC_ERR_INVALID_ARG, "clustered scene without lights");
  return NVC_OK;
}

nvc_status nvc_kmeans_lights(const float* lights, int32_t n_lights, const int32_t* init,
                             int32_t k, int32_t iters, int32_t* assign, double* centroids) {
  if (!lights || !init || !assign) return fail(nullptr, NVC_ERR_INVALID_ARG, "NULL argument");
  if (n_lights < 1 || k < 1 || k > n_lights || iters < 0)
    return fail(nullptr, NVC_ERR_INVALID_ARG, "need 1 <= k <= n_lights and iters >= 0");
  for (int y = 0; y < k; ++y)
    if (init[y] < 0 || init[y] >= n_lights)
      return fail(nullptr, NVC_ERR_INVALID_ARG, "init[%d] out of range", y);
  kmeans_host(lights, n_lights, init, k, iters, assign, centroids);
  return NVC_OK;
}

nvc_status nvc_train_step_clustered(nvc_handle* h, const nvc_scene* scene,
                                    const nvc_clusters* clusters, const float* screen_pos,
                                    int64_t n_screen, uint64_t seed, uint32_t frame,
                                    double* loss_out, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  NVC_TRY(check_scene(h, scene, 0, kAnyLights));
  NVC_TRY(check_clusters(h, scene, clusters, h->L));
  if (n_screen < 0 || n_screen > ((int64_t)1 << 32))
    return fail(h, NVC_ERR_INVALID_ARG, "n_screen out of range");
  if (n_screen > 0 && screen_pos) NVC_TRY(check_ptr(h, screen_pos, "screen_pos"));
  if (loss_out) NVC_TRY(check_ptr(h, loss_out, "loss_out", 8));
  return train_step_impl(h, scene, screen_pos, n_screen, seed, frame, loss_out,
                         (cudaStream_t)stream, clusters);
}

nvc_status nvc_cluster_targets(const nvc_scene* scene, const nvc_clusters* clusters,
                               const float* pos, int64_t n, uint64_t seed, uint32_t frame,
                               float* target, void* stream) {
  NVC_TRY(check_scene(nullptr, scene, 0, kAnyLights));
  NVC_TRY(check_clusters(nullptr, scene, clusters, 0));
  // sample ids are 32-bit Philox counters
  if (n < 0 || n > ((int64_t)1 << 32)) return fail(nullptr, NVC_ERR_INVALID_ARG, "n out of range");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, pos, "pos"));
  NVC_TRY(check_ptr(nullptr, target, "target"));
  NVC_CUDA(nullptr, launch_cluster_targets(scene, clusters, pos, n, seed, frame, target,
                                           (cudaStream_t)stream));
  return NVC_OK;
}

nvc_status nvc_sample_clustered(const nvc_scene* scene, const nvc_clusters* clusters,
                                const float* vis, const float* pos, const float* nrm, int64_t n,
                                int64_t pixel_offset, uint64_t seed, uint32_t frame,
                                uint32_t view, int32_t* light, float* weight, float* estimate,
                                void* stream) {
  NVC_TRY(check_scene(nullptr, scene, 0, kAnyLights));
  NVC_TRY(check_clusters(nullptr, scene, clusters, 0));
  if (n < 0 || pixel_offset < 0 || pixel_offset + n > ((int64_t)1 << 32))
    return fail(nullptr, NVC_ERR_INVALID_ARG, "n or pixel ids out of range");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, vis, "vis"));
  NVC_TRY(check_ptr(nullptr, pos, "pos"));
  NVC_TRY(check_ptr(nullptr, nrm, "nrm"));
  if (!light && !weight && !estimate) return fail(nullptr, NVC_ERR_INVALID_ARG, "no output");
  if (light) NVC_TRY(check_ptr(nullptr, light, "light"));
  if (weight) NVC_TRY(check_ptr(nullptr, weight, "weight"));
  if (estimate) NVC_TRY(check_ptr(nullptr, estimate, "estimate"));
  if (sample_clustered_smem(scene, clusters) > 227 * 1024)
    return fail(nullptr, NVC_ERR_UNSUPPORTED, "too many occluders for shared memory");
  int sms = 0;
  NVC_CUDA(nullptr, current_sms(&sms));
  NVC_CUDA(nullptr, launch_sample_clustered(scene, clusters, vis, pos, nrm, n, pixel_offset, seed,
                                            frame, view, light, weight, estimate, sms,
                                            (cudaStream_t)stream));
  return NVC_OK;
}

nvc_status nvc_temporal_merge(const nvc_scene* scene, const float* pos, const float* nrm,
                              int64_t n, int64_t pixel_offset, uint64_t seed, uint32_t frame,
                              uint32_t view, const int32_t* cur_light, const float* cur_W,
                              const int32_t* prev_light, const float* prev_W,
                              const int32_t* prev_M, int32_t* light, float* W, int32_t* M,
                              float* estimate, void* stream) {
  NVC_TRY(check_scene(nullptr, scene, 0, kAnyLights));
  if (n < 0 || pixel_offset < 0 || pixel_offset + n > ((int64_t)1 << 32))
    return fail(nullptr, NVC_ERR_INVALID_ARG, "n or pixel ids out of range");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(nullptr, pos, "pos"));
  NVC_TRY(check_ptr(nullptr, nrm, "nrm"));
  NVC_TRY(check_ptr(nullptr, cur_light, "cur_light"));
  NVC_TRY(check_ptr(nullptr, cur_W, "cur_W"));
  if ((prev_light == nullptr) != (prev_W == nullptr) || (prev_light == nullptr) != (prev_M == nullptr))
    return fail(nullptr, NVC_ERR_INVALID_ARG, "prev_light, prev_W and prev_M go together");
  if (prev_light) {
    NVC_TRY(check_ptr(nullptr, prev_light, "prev_light"));
    NVC_TRY(check_ptr(nullptr, prev_W, "prev_W"));
    NVC_TRY(check_ptr(nullptr, prev_M, "prev_M"));
  }
  if (!light && !W && !M && !estimate) return fail(nullptr, NVC_ERR_INVALID_ARG, "no output");
  if (occluder_bytes(scene->n_spheres, scene->n_boxes) > 227 * 1024)
    return fail(nullptr, NVC_ERR_UNSUPPORTED, "too many occluders for shared memory");
  int sms = 0;
  NVC_CUDA(nullptr, current_sms(&sms));
  NVC_CUDA(nullptr, launch_temporal_merge(scene, pos, nrm, n, pixel_offset, seed, frame, view,
                                          cur_light, cur_W, prev_light, prev_W, prev_M, light, W, M,
                                          estimate, sms, (cudaStream_t)stream));
  return NVC_OK;
}

nvc_status nvc_train_gradient(nvc_handle* h, const nvc_scene* scene, const float* screen_pos,
                              int64_t n_screen, uint64_t seed, uint32_t frame, float* grad,
                              double* loss_out, void* stream) {
  NVC_TRY(train_checks(h, scene, screen_pos, n_screen));
  NVC_TRY(check_ptr(h, grad, "grad"));
  if (loss_out) NVC_TRY(check_ptr(h, loss_out, "loss_out", 8));
  cudaStream_t s = (cudaStream_t)stream;
  NVC_TRY(train_forward_backward(h, scene, screen_pos, n_screen, seed, frame, s));
  NVC_CUDA(h, launch_finish_gradient(h, grad, loss_out, s));
  return NVC_OK;
}

nvc_status nvc_mlp_forward(nvc_handle* h, const float* pos, int64_t n, float* logits,
                           void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0 || n > h->B) return fail(h, NVC_ERR_INVALID_ARG, "n must be in [0, batch_positions]");
  if (n == 0) return NVC_OK;
  NVC_TRY(check_ptr(h, pos, "pos"));
  NVC_TRY(check_ptr(h, logits, "logits"));
  cudaStream_t s = (cudaStream_t)stream;
  NVC_CUDA(h, launch_encode_fwd(h, pos, n, h->t_feat, s));
  NVC_CUDA(h, launch_mlp_fwd_fp32(h, h->t_feat, n, logits, false, h->t_act, s));
  return NVC_OK;
}

__global__ void copy_rows_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

__global__ void take_grad_unscaled_kernel(float* __restrict__ grad, float* __restrict__ out,
                                          int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    out[e] = grad[e];
    grad[e] = 0.0f;
  }
}

nvc_status nvc_mlp_backward(nvc_handle* h, const float* pos, int64_t n, const float* dlogits,
                            float* grad, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0 || n > h->B) return fail(h, NVC_ERR_INVALID_ARG, "n must be in [0, batch_positions]");
  NVC_TRY(check_ptr(h, grad, "grad"));
  cudaStream_t s = (cudaStream_t)stream;
  if (n > 0) {
    NVC_TRY(check_ptr(h, pos, "pos"));
    NVC_TRY(check_ptr(h, dlogits, "dlogits"));
    const int maxdim = h->width > h->L ? h->width : h->L;
    float* dtop = h->t_delta + (int64_t)(h->n_layers - 1) * h->B * maxdim;
    copy_rows_kernel<<<h->num_sms * 4, 256, 0, s>>>(dlogits, dtop, n * h->L);
    NVC_CUDA(h, cudaGetLastError());
    NVC_CUDA(h, launch_mlp_bwd_fp32(h, n, nullptr, h->grad, h->status, s));
    NVC_CUDA(h, launch_encode_bwd(h, pos, n, h->t_dfeat, h->grad, h->status, s));
  }
  take_grad_unscaled_kernel<<<h->num_sms * 4, 256, 0, s>>>(h->grad, grad, h->n_params);
  NVC_CUDA(h, cudaGetLastError());
  return NVC_OK;
}

static nvc_status frame_body(nvc_handle* h, const nvc_scene* scene, const nvc_view* views,
                             int32_t n_views, int32_t train_view, uint64_t seed, uint32_t frame,
                             double* loss_out, cudaStream_t s) {
  if (train_view != NVC_FRAME_NO_TRAINING) {
    const nvc_view* tv = train_view >= 0 ? &views[train_view] : nullptr;
    NVC_TRY(train_step_impl(h, scene, tv ? tv->pos : nullptr, tv ? tv->n_pixels : 0, seed,
                            frame, loss_out, s));
  }
  const bool fused = h->cfg.precision != NVC_PREC_FP32;
  if (fused) {
    // every view of the frame in one persistent launch
    std::string why;
    if (!fused_supported(h, &why)) return fail(h, NVC_ERR_UNSUPPORTED, "%s", why.c_str());
    std::vector<FusedView> fv;
    for (int v = 0; v < n_views; ++v) {
      const nvc_view& vw = views[v];
      if (vw.n_pixels == 0) continue;
      fv.push_back(FusedView{vw.pos, vw.nrm, vw.n_pixels, vw.view_id, 0, vw.idx, vw.pdf, vw.wsum,
                             vw.radiance, nullptr, nullptr});
    }
    StageScope sc(h, s, 3);
    NVC_CUDA(h, launch_shade_fused_views(h, scene, fv.data(), (int)fv.size(), seed, frame, s));
    count_launches(h, ((int)fv.size() + 15) / 16);
  } else {
    for (int v = 0; v < n_views; ++v) {
      const nvc_view& vw = views[v];
      if (vw.n_pixels == 0) continue;
      NVC_TRY(shade_impl(h, scene, vw.pos, vw.nrm, vw.n_pixels, seed, frame, vw.view_id, 0,
                         vw.idx, vw.pdf, vw.wsum, vw.radiance, 0, s));
    }
  }
  bump_frames_kernel<<<1, 1, 0, s>>>(h->status);
  NVC_CUDA(h, cudaGetLastError());
  count_launches(h, 1);
  return NVC_OK;
}

nvc_status nvc_frame(nvc_handle* h, const nvc_scene* scene, const nvc_view* views,
                     int32_t n_views, int32_t train_view, uint64_t seed, uint32_t frame,
                     double* loss_out, int32_t use_graph, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  NVC_TRY(check_scene(h, scene, h->L));
  if (n_views < 0 || (n_views > 0 && !views)) return fail(h, NVC_ERR_INVALID_ARG, "bad views");
  if (train_view >= n_views || train_view < NVC_FRAME_NO_TRAINING)
    return fail(h, NVC_ERR_INVALID_ARG, "train_view out of range");
  for (int v = 0; v < n_views; ++v) {
    NVC_TRY(shade_checks(h, scene, views[v].pos, views[v].nrm, views[v].n_pixels, 0));
  }
  if (loss_out) NVC_TRY(check_ptr(h, loss_out, "loss_out", 8));
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return frame_body(h, scene, views, n_views, train_view, seed, frame, loss_out, s);

  const bool was_profiling = h->profiling;
  h->profiling = false;
  NVC_CUDA(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
  nvc_status st = frame_body(h, scene, views, n_views, train_view, seed, frame, loss_out,
                             h->capture_stream);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &g);
  h->profiling = was_profiling;
  if (st != NVC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamEndCapture");
  if (h->graph_exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(h->graph_exec, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(h->graph_exec);
      h->graph_exec = nullptr;
    }
  }
  if (!h->graph_exec) {
    ce = cudaGraphInstantiate(&h->graph_exec, g, 0);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(h, ce, "cudaGraphInstantiate");
    }
  }
  if (h->graph) cudaGraphDestroy(h->graph);
  h->graph = g;
  NVC_CUDA(h, cudaGraphLaunch(h->graph_exec, s));
  return NVC_OK;
}

// Copy streams, events and two device slots of at least `total` pixels for
// nvc_frame_host.  A slot that must grow is first waited for (its frame and
// read-back), then reallocated.
static cudaError_t host_staging(nvc_handle* h, int64_t total) {
  cudaError_t e;
  if (!h->up_stream) {
    if ((e = cudaStreamCreateWithFlags(&h->up_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&h->down_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
    for (auto& sl : h->host_slot) {
      if ((e = cudaEventCreateWithFlags(&sl.up, cudaEventDisableTiming)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&sl.down, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
  }
  for (auto& sl : h->host_slot) {
    if (sl.cap >= total) continue;
    if ((e = cudaEventSynchronize(sl.done)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(sl.down)) != cudaSuccess) return e;
    cudaFree(sl.pos);
    cudaFree(sl.nrm);
    cudaFree(sl.idx);
    cudaFree(sl.out);
    sl.pos = sl.nrm = sl.out = nullptr;
    sl.idx = nullptr;
    sl.cap = 0;
    const int64_t cap = total > 128 ? total : 128;
    if ((e = cudaMalloc(&sl.pos, sizeof(float) * 3 * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&sl.nrm, sizeof(float) * 3 * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&sl.idx, sizeof(int32_t) * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&sl.out, sizeof(float) * 3 * cap)) != cudaSuccess) return e;
    sl.cap = cap;
  }
  return cudaSuccess;
}

nvc_status nvc_frame_host(nvc_handle* h, const nvc_scene* scene, const nvc_view* host_views,
                          int32_t n_views, int32_t train_view, uint64_t seed, uint32_t frame,
                          double* loss_out, int32_t use_graph, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (n_views < 0 || (n_views > 0 && !host_views)) return fail(h, NVC_ERR_INVALID_ARG, "bad views");
  int64_t total = 0;
  for (int v = 0; v < n_views; ++v) {
    const nvc_view& hv = host_views[v];
    if (hv.n_pixels < 0 || hv.n_pixels > ((int64_t)1 << 32))
      return fail(h, NVC_ERR_INVALID_ARG, "view %d: n_pixels out of range", v);
    if (hv.n_pixels > 0 && (!hv.pos || !hv.nrm))
      return fail(h, NVC_ERR_INVALID_ARG, "view %d: pos or nrm is NULL", v);
    total += hv.n_pixels;
  }
  NVC_CUDA(h, host_staging(h, total));
  const int b = h->host_next;
  nvc_handle::HostSlot& sl = h->host_slot[b];
  cudaStream_t s = (cudaStream_t)stream;
  // upload into slot b once the frame that last read it is done
  NVC_CUDA(h, cudaStreamWaitEvent(h->up_stream, sl.done, 0));
  std::vector<nvc_view> dv(n_views > 0 ? n_views : 1);
  int64_t off = 0;
  for (int v = 0; v < n_views; ++v) {
    const nvc_view& hv = host_views[v];
    nvc_view& d = dv[v];
    const int64_t n = hv.n_pixels;
    d = hv;
    d.pos = sl.pos + 3 * off;
    d.nrm = sl.nrm + 3 * off;
    d.idx = hv.idx ? sl.idx + off : nullptr;
    d.pdf = hv.pdf ? sl.out + off : nullptr;
    d.wsum = hv.wsum ? sl.out + sl.cap + off : nullptr;
    d.radiance = hv.radiance ? sl.out + 2 * sl.cap + off : nullptr;
    if (n > 0) {
      NVC_CUDA(h, cudaMemcpyAsync((void*)d.pos, hv.pos, sizeof(float) * 3 * n,
                                  cudaMemcpyHostToDevice, h->up_stream));
      NVC_CUDA(h, cudaMemcpyAsync((void*)d.nrm, hv.nrm, sizeof(float) * 3 * n,
                                  cudaMemcpyHostToDevice, h->up_stream));
    }
    off += n;
  }
  NVC_CUDA(h, cudaEventRecord(sl.up, h->up_stream));
  // the frame: after the upload, and after this slot's previous read-back
  NVC_CUDA(h, cudaStreamWaitEvent(s, sl.up, 0));
  NVC_CUDA(h, cudaStreamWaitEvent(s, sl.down, 0));
  NVC_TRY(nvc_frame(h, scene, dv.data(), n_views, train_view, seed, frame, loss_out, use_graph,
                    stream));
  NVC_CUDA(h, cudaEventRecord(sl.done, s));
  h->host_next = b ^ 1;
  // read-back on the second copy stream
  NVC_CUDA(h, cudaStreamWaitEvent(h->down_stream, sl.done, 0));
  for (int v = 0; v < n_views; ++v) {
    const nvc_view& hv = host_views[v];
    const nvc_view& d = dv[v];
    const int64_t n = hv.n_pixels;
    if (n == 0) continue;
    if (hv.idx)
      NVC_CUDA(h, cudaMemcpyAsync(hv.idx, d.idx, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                  h->down_stream));
    if (hv.pdf)
      NVC_CUDA(h, cudaMemcpyAsync(hv.pdf, d.pdf, sizeof(float) * n, cudaMemcpyDeviceToHost,
                                  h->down_stream));
    if (hv.wsum)
      NVC_CUDA(h, cudaMemcpyAsync(hv.wsum, d.wsum, sizeof(float) * n, cudaMemcpyDeviceToHost,
                                  h->down_stream));
    if (hv.radiance)
      NVC_CUDA(h, cudaMemcpyAsync(hv.radiance, d.radiance, sizeof(float) * n,
                                  cudaMemcpyDeviceToHost, h->down_stream));
  }
  NVC_CUDA(h, cudaEventRecord(sl.down, h->down_stream));
  return NVC_OK;
}

nvc_status nvc_host_frames_wait(nvc_handle* h, void* stream) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  if (!h->down_stream) return NVC_OK;
  for (auto& sl : h->host_slot) NVC_CUDA(h, cudaStreamWaitEvent((cudaStream_t)stream, sl.down, 0));
  return NVC_OK;
}

nvc_status nvc_set_profiling(nvc_handle* h, int32_t enable) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  ProfEvents* pe = prof_of(h);
  if (enable && pe && pe->pool.empty()) {
    pe->pool.resize(8192);
    for (auto& ev : pe->pool) NVC_CUDA(h, cudaEventCreate(&ev));
  }
  h->profiling = enable != 0;
  return NVC_OK;
}

nvc_status nvc_stage_times(nvc_handle* h, double* ms_out, int32_t n_out, int64_t* launches_out) {
  if (!h) return fail(nullptr, NVC_ERR_INVALID_ARG, "handle is NULL");
  ProfEvents* pe = prof_of(h);
  if (pe && !pe->open.empty()) {
    NVC_CUDA(h, cudaEventSynchronize(pe->pool[pe->open.back().second + 1]));
    for (auto& o : pe->open) {
      float ms = 0.f;
      NVC_CUDA(h, cudaEventElapsedTime(&ms, pe->pool[o.second], pe->pool[o.second + 1]));
      h->stage_ms[o.first] += ms;
    }
    pe->open.clear();
    pe->next = 0;
  }
  for (int i = 0; i < n_out && i < 4; ++i) ms_out[i] = h->stage_ms[i];
  if (launches_out) *launches_out = h->launches;
  for (double& v : h->stage_ms) v = 0.0;
  h->launches = 0;
  return NVC_OK;
}

}  // extern "C"
