// Internal declarations of libnvc: the handle, device helpers shared by the
// kernels, and the host-side launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>

#include "nvc.h"

namespace nvc {

// ---------------------------------------------------------------------------
// Float32 constants given by bit pattern, so every consumer rounds the same.
// ---------------------------------------------------------------------------
constexpr uint32_t kInvPiBits = 0x3EA2F983u;    // 1/pi
constexpr uint32_t kVisClampBits = 0x3A83126Fu; // 0.001 (Section 3.1 clamp)
constexpr uint32_t kD2MinBits = 0x358637BDu;    // 1e-6
constexpr uint32_t kSegT0Bits = 0x38D1B717u;    // 1e-4
constexpr uint32_t kSegT1Bits = 0x3F7FF972u;    // 1 - 1e-4

__device__ __forceinline__ float bits_f(uint32_t b) { return __uint_as_float(b); }

// a - b, a + b and a * b on both halves of a float2, each a correctly
// rounded float32 operation (the packed sub/add/mul.rn.f32x2 of sm_100 and
// later).  Written as PTX with an explicit .rn so that no product is fused
// into a following sum: code whose decisions must equal a scalar, one-
// rounding-per-operation definition uses these.
#define NVC_PACKED_OP(NAME, OP)                                                  \
  __device__ __forceinline__ float2 NAME(float2 a, float2 b) {                   \
    uint64_t ua, ub, r;                                                          \
    asm("mov.b64 %0, {%1, %2};" : "=l"(ua) : "f"(a.x), "f"(a.y));                \
    asm("mov.b64 %0, {%1, %2};" : "=l"(ub) : "f"(b.x), "f"(b.y));                \
    asm(OP " %0, %1, %2;" : "=l"(r) : "l"(ua), "l"(ub));                         \
    float2 o;                                                                    \
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));                \
    return o;                                                                    \
  }
NVC_PACKED_OP(fsub2, "sub.rn.f32x2")
NVC_PACKED_OP(fadd2_rn, "add.rn.f32x2")
NVC_PACKED_OP(fmul2_rn, "mul.rn.f32x2")
#undef NVC_PACKED_OP

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC 2011): counter-based, one 128-bit block
// per (counter, key).
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;
enum : uint32_t { kTagWrs = 0, kTagWorld = 1, kTagScreen = 2, kTagShade = 3 };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

__device__ __forceinline__ float uniform24(uint32_t r) {
  return __fmul_rn((float)(r >> 8), 5.9604644775390625e-08f);  // 2^-24, exact
}

// ---------------------------------------------------------------------------
// Hash grid: normalisation, cell and spatial hash.
// ---------------------------------------------------------------------------
constexpr uint32_t kPrime1 = 2654435761u, kPrime2 = 805459861u;

__device__ __forceinline__ uint32_t grid_hash(uint32_t x, uint32_t y, uint32_t z) {
  return x ^ (y * kPrime1) ^ (z * kPrime2);
}

// x_hat = clamp((x - lo) / ext, 0, 1), correctly rounded float32.
__device__ __forceinline__ float normalise(float x, float lo, float ext) {
  return fminf(fmaxf(__fdiv_rn(__fsub_rn(x, lo), ext), 0.0f), 1.0f);
}

// Cell corner and fraction of x_hat at resolution n (float32, exact f).
__device__ __forceinline__ void grid_cell(float xh, int n, int& c, float& f) {
  const float p = __fmul_rn(xh, (float)n);
  int ci = (int)floorf(p);
  ci = ci > n - 1 ? n - 1 : ci;
  c = ci;
  f = __fsub_rn(p, (float)ci);
}

struct EncodeParams {
  int n_levels;
  int log2_table;
  float lo[3];
  float ext[3];
  int res[NVC_MAX_LEVELS];
  float resf[NVC_MAX_LEVELS];   // res as float32 (exact: res < 2^24)
};

// ---------------------------------------------------------------------------
// Light contribution (Lambertian, point light), correctly rounded float32.
// c = ((I * (1/pi)) * (n.d)) / (sqrt(d.d) * max(d.d, 1e-6)) for n.d > 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot3_rn(float ax, float ay, float az, float bx, float by,
                                         float bz) {
  return __fadd_rn(__fadd_rn(__fmul_rn(ax, bx), __fmul_rn(ay, by)), __fmul_rn(az, bz));
}

__device__ __forceinline__ float contribution(float px, float py, float pz, float nx, float ny,
                                              float nz, float lx, float ly, float lz,
                                              float i_over_pi) {
  const float dx = __fsub_rn(lx, px), dy = __fsub_rn(ly, py), dz = __fsub_rn(lz, pz);
  const float d2 = dot3_rn(dx, dy, dz, dx, dy, dz);
  const float ndl = dot3_rn(nx, ny, nz, dx, dy, dz);
  if (!(ndl > 0.0f)) return 0.0f;
  const float den = __fmul_rn(__fsqrt_rn(d2), fmaxf(d2, bits_f(kD2MinBits)));
  return __fdiv_rn(__fmul_rn(i_over_pi, ndl), den);
}

// Integer reservoir weight of w >= 0 given e = ilogb(max w):
// q = max(1, floor(w * 2^(23 - e))) for w > 0, else 0.
__device__ __forceinline__ uint32_t quantize_weight(float w, int e) {
  if (!(w > 0.0f)) return 0u;
  const float s = ldexpf(w, 23 - e);
  const uint32_t q = (uint32_t)floorf(s);
  return q > 0u ? q : 1u;
}

// ---------------------------------------------------------------------------
// Device status words (int32 array in the handle).
// ---------------------------------------------------------------------------
enum StatusWord : int {
  kStStep = 0,
  kStSkipped = 1,
  kStFlags = 2,
  kStFrames = 3,
  kStNonFinite = 4,   // set by the gradient kernels of the current step
  kStSkipNow = 5,     // Adam of the current step is skipped
  kStTileNext = 6,    // shading tile scheduler: next tile ticket (0 between launches)
  kStTileDone = 7,    // shading tile scheduler: tile streams finished (0 between launches)
  kStAdamDone = 8,    // Adam CTAs finished (0 between launches)
  kStWords = 16
};
enum : int { kFlagNonFinite = 1, kFlagTimeout = 2 };

// Variants of the fused shading kernel (chosen by nvc_autotune_shade).
enum ShadeVariant : int {
  kShadeMono = 0,   // every warp encodes, multiplies and samples its own tile
  kShadeWs4 = 1,    // 4 producer warps encode, 4 consumer warps run MLP + sampler
  kShadeWs4C = 2,   // as kShadeWs4, producers also precompute the contributions
  kShadeWs8 = 3,    // 8 producer warps (two threads per pixel) + 4 consumers
  kShadeWs8C = 4,   // as kShadeWs8 with precomputed contributions
  kShadePair = 5,   // two threads per pixel: levels, columns and lights split in halves
  kShadeMulti2 = 6, // two tile streams per CTA sharing the weights
  kShadeMulti4 = 7, // four tile streams per CTA sharing the weights
  kShadeVariants = 8
};

// Where each MLP weight sits in the tensor cores' 16-bit weight image (the
// layout pack_mlp_kernel writes): layer k's W[n][kk] (parameter w_off[k] +
// n K_real + kk) is element ((n/8) (K/8) + kk/8) 64 + (n%8) 8 + kk%8 of the
// layer's block at byte_off[k].  The Adam kernel uses it to refresh the
// image from the updated weights in the same pass.
struct MlpImageMap {
  int n_layers;
  int64_t w_off[NVC_MAX_HIDDEN_LAYERS + 2];   // [n_layers] = end of the last layer
  int K_real[NVC_MAX_HIDDEN_LAYERS + 1], K[NVC_MAX_HIDDEN_LAYERS + 1];
  int byte_off[NVC_MAX_HIDDEN_LAYERS + 1];
  int bf16;
};

// Adam scalars written on the device each step.
struct AdamScalars {
  float lr_over_bc1;     // lr / (1 - b1^t)
  float inv_bc2;         // 1 / (1 - b2^t)
  float inv_scale;       // 1 / loss_scale
  int skip;
};

}  // namespace nvc

// ---------------------------------------------------------------------------
// The handle.
// ---------------------------------------------------------------------------
struct nvc_handle {
  nvc_config cfg;
  int L = 0, F = 0, T = 0, din = 0, width = 0, n_hidden = 0, n_layers = 0;
  int res[NVC_MAX_LEVELS] = {};
  int64_t n_params = 0, n_table = 0;
  int64_t w_off[NVC_MAX_HIDDEN_LAYERS + 1] = {};
  int w_out[NVC_MAX_HIDDEN_LAYERS + 1] = {};
  int w_in[NVC_MAX_HIDDEN_LAYERS + 1] = {};
  int device = 0;
  int num_sms = 0;
  int adam_ctas_per_sm = 0;   // resident Adam CTAs per SM (occupancy query at create)

  // parameters and optimiser state (float32, n_params each)
  float* params = nullptr;
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  // half-precision copy of the hash table read by the fused inference
  // kernels (nvc_set_table_precision; NULL: they read `params`)
  __half* table16 = nullptr;
  // tensor-core copies of the MLP weights, packed for the fused kernel
  void* mlp_packed = nullptr;
  size_t mlp_packed_bytes = 0;

  // training workspace, capacity B positions
  int B = 0;
  float* t_pos = nullptr;     // [B][3]
  float* t_target = nullptr;  // [B][L]
  float* t_feat = nullptr;    // [B][din]
  float* t_act = nullptr;     // [n_hidden][B][width]
  float* t_logits = nullptr;  // [B][L]
  float* t_delta = nullptr;   // [n_layers][B][max(width, L)]
  float* t_dfeat = nullptr;   // [B][din]
  // nvc_frame_host: two device slots of G-buffers and outputs, two copy
  // streams, and the events that order uploads, frames and read-backs
  struct HostSlot {
    int64_t cap = 0;          // pixels the slot's buffers hold
    float* pos = nullptr;     // [cap][3]
    float* nrm = nullptr;     // [cap][3]
    int32_t* idx = nullptr;   // [cap]
    float* out = nullptr;     // [3][cap]: pdf, wsum, radiance
    cudaEvent_t up = nullptr, done = nullptr, down = nullptr;
  } host_slot[2];
  int host_next = 0;
  cudaStream_t up_stream = nullptr, down_stream = nullptr;
  double* loss_partials = nullptr;
  int n_loss_partials = 0;
  int loss_blocks = 0;                  // partials written by the last training pass
  int32_t* status = nullptr;            // nvc::kStWords
  unsigned long long* phase_cycles = nullptr;   // [4], nvc_shade_phases

  // staging of the unfused shading path
  int64_t stage_pixels = 0;
  float* s_feat = nullptr;    // [stage][din]
  float* s_vis = nullptr;     // [stage][L]

  // fused shading kernel variant (nvc::ShadeVariant); nvc_infer's own
  // variant (-1: the shading variant), set by nvc_autotune_infer
  int shade_variant = 0;
  int infer_variant = -1;
  // resident CTAs per SM of the fused shading launches (0: as many as fit),
  // the occupancy point of nvc_set_shade_plan / nvc_autotune_shade_plan
  int shade_ctas_per_sm = 0;
  // world-space share of the training positions (nvc_set_training_placement;
  // -1: the default split, ceil(B / 2) world-space)
  int64_t n_world = -1;
  // FP16 training makes its positions and targets inside the tensor-core
  // training kernel instead of a separate launch (nvc_set_training_data_fused)
  bool fused_training_data = false;
  // E4M3 per-tensor scales: [0, 9) activations (set by nvc_calibrate),
  // [9, 18) weights (set by the weight packing)
  float* fp8_scales = nullptr;
  bool fp8_calibrated = false;

  // frame graph
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;

  // profiling
  bool profiling = false;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  double stage_ms[4] = {0, 0, 0, 0};
  int64_t launches = 0;
  std::string err;
};

namespace nvc {

// Records the message nvc_last_error(NULL) returns on this thread.
void record_error(const char* msg);

// The configuration checks of nvc_create: NVC_OK, or NVC_ERR_INVALID_ARG
// with the reason in *why.
nvc_status validate_config(const nvc_config* c, std::string* why);

// Resident blocks per SM of `func` with `block` threads and `dyn_smem`
// dynamic shared memory, from the function's register and shared-memory
// footprint and the device's per-SM limits.
int blocks_per_sm(const void* func, int block, size_t dyn_smem);

// ---- launchers (each returns cudaGetLastError() of its launches) ----------
// encode.cu
cudaError_t launch_encode_fwd(const nvc_handle* h, const float* pos, int64_t n, float* feat,
                              cudaStream_t s);
cudaError_t launch_encode_bwd(const nvc_handle* h, const float* pos, int64_t n,
                              const float* dfeat, float* grad_table, int32_t* status,
                              cudaStream_t s);
EncodeParams encode_params(const nvc_handle* h);

// mlp_simt.cu
cudaError_t launch_mlp_fwd_fp32(const nvc_handle* h, const float* feat, int64_t n, float* out,
                                bool sigmoid_out, float* act_store, cudaStream_t s);
cudaError_t launch_mlp_bwd_fp32(const nvc_handle* h, int64_t n, const float* dlogits,
                                float* grad, int32_t* status, cudaStream_t s);
size_t mlp_fwd_smem_bytes(const nvc_handle* h);

// shade.cu
cudaError_t launch_light_weights(const nvc_scene* sc, const float* pos, const float* nrm,
                                 const float* vis, int64_t n, float* c, float* w,
                                 cudaStream_t s);
cudaError_t launch_wrs_from_weights(const float* w, int64_t n, int L, uint64_t seed,
                                    uint32_t frame, uint32_t view, int64_t pixel_offset,
                                    int32_t* idx, float* pdf, float* wsum, cudaStream_t s);
cudaError_t launch_shade_from_vis(const nvc_scene* sc, const float* pos, const float* nrm,
                                  const float* vis, int64_t n, uint64_t seed, uint32_t frame,
                                  uint32_t view, int64_t pixel_offset, int32_t* idx,
                                  float* pdf, float* wsum, float* radiance, cudaStream_t s);

// train.cu
// n_world: world-space positions in the batch, -1 for ceil(batch / 2); every
// position is world-space when no screen positions are given.
cudaError_t launch_training_positions(const nvc_scene* sc, const float* screen_pos,
                                      int64_t n_screen, int64_t batch, uint64_t seed,
                                      uint32_t frame, float* pos, cudaStream_t s,
                                      int64_t n_world = -1);
cudaError_t launch_trace_visibility(const nvc_scene* sc, const float* pos, int64_t n,
                                    float* vis, cudaStream_t s);
cudaError_t launch_loss_grad(nvc_handle* h, int64_t n, cudaStream_t s);
cudaError_t launch_adam(nvc_handle* h, double* loss_out, bool apply, cudaStream_t s);
// Resident CTAs per SM of the Adam update (256 threads), for a one-wave grid.
cudaError_t adam_occupancy(int* ctas_per_sm);
cudaError_t launch_finish_gradient(nvc_handle* h, float* grad_out, double* loss_out,
                                   cudaStream_t s);

// fused_tc.cu
cudaError_t launch_pack_mlp(nvc_handle* h, cudaStream_t s);
// The image map of the handle's 16-bit weight image; false when there is
// none to keep (float32 inference, or E4M3, whose per-layer scales need
// the whole layer).
bool mlp_image_map(const nvc_handle* h, MlpImageMap* m);
// Refreshes the half-precision table copy from the master (no-op without one).
cudaError_t launch_pack_table(nvc_handle* h, cudaStream_t s);
bool fused_supported(const nvc_handle* h, std::string* why);
cudaError_t launch_shade_fused(const nvc_handle* h, const nvc_scene* sc, const float* pos,
                               const float* nrm, int64_t n, uint64_t seed, uint32_t frame,
                               uint32_t view, int64_t pixel_offset, int32_t* idx, float* pdf,
                               float* wsum, float* radiance, float* vis_out, cudaStream_t s,
                               float* w_out = nullptr);
size_t mlp_packed_bytes(const nvc_handle* h);
// One view of a multi-view fused launch.
struct FusedView {
  const float* pos;
  const float* nrm;
  int64_t n;
  uint32_t view;
  int64_t pixel_offset;
  int32_t* idx;
  float* pdf;
  float* wsum;
  float* radiance;
  float* vis_out;
  float* w_out;
};
// phase_cycles (device [4] uint64, may be NULL): the several-tiles-per-CTA
// variants add their per-phase SM cycles there (nvc_shade_phases).
cudaError_t launch_shade_fused_views(const nvc_handle* h, const nvc_scene* sc,
                                     const FusedView* views, int n_views, uint64_t seed,
                                     uint32_t frame, cudaStream_t s,
                                     unsigned long long* phase_cycles = nullptr,
                                     const uint16_t* feat16 = nullptr);

// train_tc.cu
bool train_tc_supported(const nvc_handle* h, std::string* why);
// The shading pass's one-sample estimate (and running mean) and the
// all-lights exact DI (shade_est.cu).
cudaError_t launch_shade_estimate(const nvc_scene* sc, const float* pos, const float* nrm,
                                  int64_t n, const int32_t* idx, const float* pdf,
                                  float* estimate, float* accum, uint32_t count, int num_sms,
                                  cudaStream_t s);
cudaError_t launch_exact_di(const nvc_scene* sc, const float* pos, const float* nrm, int64_t n,
                            float* di, int num_sms, cudaStream_t s);
// Clustered cache (clusters.cu).
cudaError_t launch_cluster_targets(const nvc_scene* sc, const nvc_clusters* cl, const float* pos,
                                   int64_t n, uint64_t seed, uint32_t frame, float* target,
                                   cudaStream_t s);
size_t sample_clustered_smem(const nvc_scene* sc, const nvc_clusters* cl);
cudaError_t launch_sample_clustered(const nvc_scene* sc, const nvc_clusters* cl, const float* vis,
                                    const float* pos, const float* nrm, int64_t n,
                                    int64_t pixel_offset, uint64_t seed, uint32_t frame,
                                    uint32_t view, int32_t* light, float* weight, float* estimate,
                                    int num_sms, cudaStream_t s);
// Temporal resampling of per-pixel reservoirs (clusters.cu).
cudaError_t launch_temporal_merge(const nvc_scene* sc, const float* pos, const float* nrm,
                                  int64_t n, int64_t pixel_offset, uint64_t seed, uint32_t frame,
                                  uint32_t view, const int32_t* cur_light, const float* cur_W,
                                  const int32_t* prev_light, const float* prev_W,
                                  const int32_t* prev_M, int32_t* light, float* W, int32_t* M,
                                  float* estimate, int num_sms, cudaStream_t s);
void kmeans_host(const float* lights, int n, const int32_t* init, int k, int iters,
                 int32_t* assign, double* centroids_out);
// Training positions and their shadow-ray targets in one launch (the same
// values as launch_training_positions followed by launch_trace_visibility).
cudaError_t launch_training_data(const nvc_scene* sc, const float* screen_pos, int64_t n_screen,
                                 int64_t batch, uint64_t seed, uint32_t frame, float* pos,
                                 float* vis, cudaStream_t s, int64_t n_world = -1);
// gen (with gen_scene): the fused-data variant, which makes the batch's
// positions and shadow-ray targets itself (into t_pos / t_target).
struct PosGen;
cudaError_t launch_train_tc(nvc_handle* h, int64_t n, int* blocks_used, cudaStream_t s,
                            const nvc_scene* gen_scene = nullptr, const PosGen* gen = nullptr);
bool train_tc_gen_supported(const nvc_handle* h, const nvc_scene* sc);

}  // namespace nvc
