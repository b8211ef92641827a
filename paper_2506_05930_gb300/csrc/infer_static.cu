// Inference for callers that cannot allocate GPU memory.
//
// Some callers of a visibility cache must not call cudaMalloc: a renderer
// whose frame loop runs under a fixed GPU memory budget (cudaMalloc may
// synchronise the device and stall the frame), or a plugin inside a host
// application that owns every device allocation and hands out only the
// buffers it made.  nvc_infer needs a handle, and nvc_create allocates.
// nvc_infer_noalloc instead takes the parameters from the caller and keeps
// its one intermediate buffer, the encoded features, in a fixed-size array
// in this file that every GPU loading the library holds until the process
// exits.
//
// It runs the float32 separate-kernel path: encode into that array, then
// the float32 MLP with the sigmoid writing the caller's output.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <string>

#include "nvc_internal.cuh"

namespace {

// Encoded features of up to kScratchFloats / (levels * features) positions
// per call: 8 MiB, e.g. 65,536 positions of a 16-level x 2-feature grid.
constexpr size_t kScratchFloats = (size_t)1 << 21;
static __device__ __align__(256) float g_feat_scratch[kScratchFloats];

// Device address of g_feat_scratch per device, found once per device with
// that device current.  In host code the array's name is only a host-side
// stand-in, never a device address.  Atomic slots: host threads making
// their first call on a device at the same time each look the address up
// and store the same value.
constexpr int kMaxDevices = 64;
std::atomic<float*> g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" nvc_status nvc_infer_noalloc(const nvc_config* cfg, const float* params,
                                        const float* pos, int64_t n, float* vis, void* stream) {
  using namespace nvc;
  std::string why;
  if (validate_config(cfg, &why) != NVC_OK) {
    record_error(("nvc_infer_noalloc: " + why).c_str());
    return NVC_ERR_INVALID_ARG;
  }
  if (n < 0) {
    record_error("nvc_infer_noalloc: n < 0");
    return NVC_ERR_INVALID_ARG;
  }
  if (n == 0) return NVC_OK;
  if (!params || !pos || !vis || ((uintptr_t)params & 15) || ((uintptr_t)pos & 3) ||
      ((uintptr_t)vis & 3)) {
    record_error("nvc_infer_noalloc: params (16-byte aligned), pos and vis must be device pointers");
    return NVC_ERR_INVALID_ARG;
  }
  const int64_t din = (int64_t)cfg->n_levels * cfg->n_features;
  const int64_t max_n = (int64_t)(kScratchFloats / (size_t)din);
  if (n > max_n) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "nvc_infer_noalloc: n = %lld exceeds the %lld positions its fixed %zu-float scratch "
             "holds for this grid; split the call",
             (long long)n, (long long)max_n, kScratchFloats);
    record_error(msg);
    return NVC_ERR_INVALID_ARG;
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    record_error("nvc_infer_noalloc: no usable current device");
    return NVC_ERR_CUDA;
  }
  float* scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_feat_scratch);
    if (e != cudaSuccess || !p) {
      record_error("nvc_infer_noalloc: cudaGetSymbolAddress of the scratch array failed");
      return NVC_ERR_CUDA;
    }
    scratch = static_cast<float*>(p);
    g_scratch_addr[dev].store(scratch, std::memory_order_release);
  }

  // A read-only view of the configuration in the handle's form; nothing in
  // it owns memory.
  nvc_handle v;
  v.cfg = *cfg;
  v.L = cfg->n_outputs;
  v.F = cfg->n_features;
  v.T = 1 << cfg->log2_table_size;
  v.din = (int)din;
  v.width = cfg->hidden_width;
  v.n_hidden = cfg->n_hidden;
  v.n_layers = cfg->n_hidden + 1;
  for (int l = 0; l < cfg->n_levels; ++l)
    v.res[l] = (int)std::floor((double)cfg->base_resolution * std::pow(cfg->growth, (double)l));
  v.n_table = (int64_t)cfg->n_levels * v.T * v.F;
  int64_t off = v.n_table;
  for (int k = 0; k < v.n_layers; ++k) {
    v.w_in[k] = k == 0 ? v.din : v.width;
    v.w_out[k] = k == v.n_layers - 1 ? v.L : v.width;
    v.w_off[k] = off;
    off += (int64_t)v.w_in[k] * v.w_out[k];
  }
  v.n_params = off;
  v.params = const_cast<float*>(params);
  v.device = dev;
  if (cudaDeviceGetAttribute(&v.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    record_error("nvc_infer_noalloc: cannot query the device");
    return NVC_ERR_CUDA;
  }
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (mlp_fwd_smem_bytes(&v) > (size_t)smem_optin) {
    record_error("nvc_infer_noalloc: MLP too large for shared memory");
    return NVC_ERR_UNSUPPORTED;
  }

  cudaStream_t s = (cudaStream_t)stream;
  e = launch_encode_fwd(&v, pos, n, scratch, s);
  if (e == cudaSuccess) e = launch_mlp_fwd_fp32(&v, scratch, n, vis, true, nullptr, s);
  if (e != cudaSuccess) {
    record_error(cudaGetErrorString(e));
    return NVC_ERR_CUDA;
  }
  return NVC_OK;
}
