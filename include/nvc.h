/*
 * nvc.h -- C ABI of the neural visibility cache hot path (libnvc.so).
 *
 * The method (Bokshansky & Meister, "Neural Visibility Cache for Real-Time
 * Light Sampling", JCGT 14(2), 2025): every shading point is encoded by a
 * multi-resolution hash grid (Sections 3.1, 3.3), a small MLP predicts one
 * sigmoid visibility per light (Section 3.3), weighted reservoir sampling
 * picks one light per pixel with weights visibility x unshadowed
 * contribution (Section 3.1), or the Neural-DI variant sums them
 * (Section 3.2); the network is trained online every frame against
 * shadow-ray targets (Section 3.4).
 *
 * Conventions shared by every entry point:
 *   - Pointers named in the comments as "device" point to GPU memory owned
 *     by the caller, row-major and densely packed, float32 unless stated.
 *     The library never frees or retains them past the call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every
 *     compute call is asynchronous on it, allocates nothing and never
 *     synchronises the host, unless its comment says otherwise.
 *   - Argument errors are detected on the host before any work is queued
 *     and returned as NVC_ERR_INVALID_ARG / NVC_ERR_UNSUPPORTED; launch
 *     failures as NVC_ERR_CUDA.  nvc_last_error() gives a message.  Errors
 *     found on the device (non-finite gradients, a bounded wait that ran
 *     out) are recorded in the handle's device status and read by
 *     nvc_sync_status().
 *   - A handle is not thread-safe: calls on one handle must not overlap on
 *     the host.  Calls on one handle queued on different streams must be
 *     ordered by the caller.
 *   - Positions are in world space; the encoding normalises them with the
 *     configuration's bounds and clamps to [0,1]^3.
 */
#ifndef NVC_H
#define NVC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NVC_VERSION 1

#define NVC_MAX_LEVELS 32
#define NVC_MAX_FEATURES 8
#define NVC_MAX_HIDDEN_LAYERS 8
#define NVC_MAX_WIDTH 128
#define NVC_MAX_LIGHTS 256      /* lights of a per-light cache (outputs); clustered calls take any number */
#define NVC_MAX_OCCLUDERS 2048

typedef enum nvc_status {
  NVC_OK = 0,
  NVC_ERR_INVALID_ARG = 1,
  NVC_ERR_UNSUPPORTED = 2,
  NVC_ERR_CUDA = 3,
  NVC_ERR_NONFINITE = 4,
  NVC_ERR_TIMEOUT = 5
} nvc_status;

typedef enum nvc_precision {
  NVC_PREC_FP32 = 0,   /* SIMT float32 */
  NVC_PREC_FP16 = 1,   /* tensor cores, fp16 operands, fp32 accumulation */
  NVC_PREC_BF16 = 2,   /* tensor cores, bf16 operands, fp32 accumulation */
  NVC_PREC_FP8 = 3     /* tensor cores, e4m3 operands with per-tensor scale */
} nvc_precision;

typedef enum nvc_loss { NVC_LOSS_L2 = 0, NVC_LOSS_BCE = 1 } nvc_loss;

typedef enum nvc_lr_schedule {
  NVC_LR_CONSTANT = 0,
  NVC_LR_RAMP = 1      /* lr -> lr_end linearly over lr_ramp_steps (Section 3.4) */
} nvc_lr_schedule;

/* Hyper-parameters of one cache (Sections 3.3 and 3.4). */
typedef struct nvc_config {
  int32_t n_levels;          /* hash-grid levels, 1..NVC_MAX_LEVELS */
  int32_t n_features;        /* features per level: 1, 2, 4 or 8 */
  int32_t log2_table_size;   /* T = 2^log2_table_size rows per level, 4..24 */
  int32_t base_resolution;   /* N_min >= 1; level l has floor(N_min*growth^l) cells */
  double growth;             /* >= 1 */
  int32_t n_hidden;          /* hidden layers, 1..NVC_MAX_HIDDEN_LAYERS */
  int32_t hidden_width;      /* neurons per hidden layer, multiple of 16, <= 128 */
  int32_t n_outputs;         /* lights = output neurons, 1..NVC_MAX_LIGHTS */
  float leaky_slope;         /* hidden activation slope for z <= 0 (0 = ReLU) */
  int32_t precision;         /* nvc_precision of the inference MLP */
  int32_t train_precision;   /* nvc_precision of training (FP32 or FP16) */
  int32_t loss;              /* nvc_loss */
  int32_t lr_schedule;       /* nvc_lr_schedule */
  float lr;                  /* base / initial learning rate */
  float lr_end;              /* final learning rate of NVC_LR_RAMP */
  int32_t lr_ramp_steps;
  float beta1, beta2, eps;   /* Adam */
  float loss_scale;          /* static loss scale (1 = none) */
  int32_t batch_positions;   /* training positions per step (each traced to every light) */
  float bounds_min[3];       /* encoding domain */
  float bounds_max[3];
} nvc_config;

/* Analytic scene: point lights and occluders (all device pointers). */
typedef struct nvc_scene {
  const float* lights;       /* [n_lights][4]: x, y, z, intensity */
  int32_t n_lights;          /* must equal the configuration's n_outputs */
  const float* spheres;      /* [n_spheres][4]: cx, cy, cz, radius; may be NULL if 0 */
  int32_t n_spheres;
  const float* boxes;        /* [n_boxes][6]: lo x, y, z, hi x, y, z; may be NULL if 0 */
  int32_t n_boxes;
  float world_min[3];        /* box that world-space training positions are drawn from */
  float world_max[3];
} nvc_scene;

/* Device-side status, read by nvc_sync_status. */
typedef struct nvc_counters {
  int32_t step;              /* Adam updates applied */
  int32_t skipped;           /* training steps skipped for non-finite gradients */
  int32_t error_flags;       /* bit 0: non-finite seen; bit 1: bounded wait ran out */
  int32_t frames;            /* nvc_frame calls queued */
} nvc_counters;

typedef struct nvc_handle nvc_handle;

/* ---- lifetime ---------------------------------------------------------- */

/* Validates `cfg`, allocates the handle's device state (FP32 master
 * parameters, Adam moments, gradients, low-precision copies, training
 * workspace for cfg->batch_positions positions) on the current device and
 * zero-initialises it.  Parameters must then be set with nvc_set_state.
 * Synchronous.  On failure *out is NULL and nvc_last_error(NULL) explains. */
nvc_status nvc_create(const nvc_config* cfg, nvc_handle** out);

/* Frees everything nvc_create allocated; waits for the device first.
 * NULL is ignored. */
void nvc_destroy(nvc_handle* h);

/* Message of the last failed call on `h`, or of the last failed
 * nvc_create on this thread when h is NULL.  Never NULL. */
const char* nvc_last_error(const nvc_handle* h);

/* Number of float32 parameters of a configuration (the flat layout is
 * [table: levels x T x F][W_1: width x n_in][W_2..][W_out: L x width], every
 * matrix row-major [out][in], no biases), or -1 if `cfg` is invalid. */
int64_t nvc_param_count(const nvc_config* cfg);

/* Level resolution N_l = floor(N_min * growth^l) (computed in double), or
 * -1 for an invalid level.  Exposed so callers can check the encoding. */
int32_t nvc_level_resolution(const nvc_config* cfg, int32_t level);

/* ---- state ------------------------------------------------------------- */

/* Copies parameters (device [n_params]) into the handle and refreshes the
 * low-precision copies.  adam_m / adam_v (device [n_params]) may be NULL,
 * meaning zero moments; `step` is the number of updates already applied. */
nvc_status nvc_set_state(nvc_handle* h, const float* params, const float* adam_m,
                         const float* adam_v, int32_t step, void* stream);

/* Copies parameters (device [n_params]) into the handle and refreshes the
 * low-precision weight copies, leaving the Adam moments, the step counter
 * and the gradient as they are: for callers that optimise the parameters
 * themselves (the torch.autograd bridge).  Asynchronous. */
nvc_status nvc_set_params(nvc_handle* h, const float* params, void* stream);

/* Precision of the hash-table features the fused inference kernels read
 * (the tables of Section 3.3): NVC_PREC_FP32 (the default) reads the float32
 * master parameters; NVC_PREC_FP16 keeps a half-precision copy (levels x T
 * x F halves, round to nearest even), written now and refreshed after every
 * parameter change -- nvc_set_state, nvc_set_params and every Adam step of
 * nvc_train_step / nvc_frame -- and the fused kernels (nvc_shade fused = 1,
 * nvc_infer, nvc_sampler_weights and the frames in FP16, BF16 or FP8
 * precision) read it instead.  Training always reads and updates the
 * float32 master; the float32 inference path always reads the master.
 * Synchronous (waits for `stream`); allocates the copy, or frees it when
 * going back to NVC_PREC_FP32.  NVC_ERR_INVALID_ARG for other precisions. */
nvc_status nvc_set_table_precision(nvc_handle* h, int32_t precision, void* stream);

/* Copies parameters and moments out (device [n_params] each; any may be
 * NULL).  Asynchronous; the step count is read by nvc_sync_status. */
nvc_status nvc_get_state(nvc_handle* h, float* params, float* adam_m, float* adam_v,
                         void* stream);

/* Capacity, in pixels, of the buffers the separate-kernel shading path
 * (nvc_shade with fused = 0, and FP32 nvc_infer) stages encoded features and
 * visibility in; larger inputs are processed in chunks of this size.  The
 * default is 65,536.  Synchronous; reallocates. */
nvc_status nvc_set_staging(nvc_handle* h, int64_t max_pixels);

/* Synchronises `stream`, then reads the device status into *out (host). */
nvc_status nvc_sync_status(nvc_handle* h, void* stream, nvc_counters* out);

/* ---- inference (Sections 3.1, 3.3) -------------------------------------- */

/* Hash-grid encoding: feat (device [n][levels*F], level-major) of pos
 * (device [n][3]).  Per level, the 8 corners of the cell containing
 * x_hat * N_l are hashed (x*1 ^ y*2654435761 ^ z*805459861 mod 2^32, mod T)
 * and trilinearly blended.  n = 0 is a no-op. */
nvc_status nvc_encode(nvc_handle* h, const float* pos, int64_t n, float* feat,
                      void* stream);

/* Predicted visibility (device [n][L]) = sigmoid(MLP(encode(pos))), in the
 * configuration's inference precision. */
nvc_status nvc_infer(nvc_handle* h, const float* pos, int64_t n, float* vis,
                     void* stream);

/* The network alone on given encodings (Section 3.3's MLP, sigmoid
 * outputs), on the tensor cores: feat (device, 16-byte aligned) holds
 * [n][k0] 16-bit operands in the handle's precision (FP16 or BF16), k0 =
 * levels*F rounded up to a multiple of 16 (columns past levels*F zero;
 * another k0 is NVC_ERR_INVALID_ARG); vis
 * (device [n][L]) receives the visibilities.  The tile-stream shading
 * kernel runs with its encode replaced by a read of feat: this measures the
 * MLP's tensor-core throughput apart from the encode and the sampler.
 * NVC_ERR_UNSUPPORTED for FP32 or E4M3 operands or n_outputs > 32. */
nvc_status nvc_mlp_infer_features(nvc_handle* h, const void* feat, int64_t n, int32_t k0,
                                  float* vis, void* stream);

/* ---- light sampling (Sections 3.1, 3.2) -------------------------------- */

/* Light weights: c (device [n][L]) = unshadowed contribution of each point
 * light to a Lambertian (albedo 1) point with normal nrm,
 * c = I * max(0, n.w) / (pi * max(|d|^2, 1e-6)), d = light - pos,
 * w = d / |d|; evaluated as ((I * (1/pi)) * (n.d)) / (sqrt(d.d) *
 * max(d.d, 1e-6)) for n.d > 0 (else 0), every operation a correctly
 * rounded float32 one, dot products summed x, y then z.  w (device
 * [n][L], may be NULL) = max(vis, 0.001) * c, the weights the sampler uses
 * (the Section 3.1 clamp).  vis may be NULL when w is NULL. */
nvc_status nvc_light_weights(const nvc_scene* scene, const float* pos, const float* nrm,
                             const float* vis, int64_t n, float* c, float* w,
                             void* stream);

/* Weighted reservoir sampling of one light per row of w (device [n][n_lights],
 * float32 >= 0).  Integer form: q_i = max(1, floor(w_i * 2^(23-e))) for
 * w_i > 0 (e = floor(log2 max w)), Q_i = q_1 + .. + q_i; candidate i
 * replaces the reservoir iff r_i * Q_i < q_i * 2^32 with r_i word i of the
 * Philox-4x32-10 stream counter (pixel_offset + row, frame, view,
 * (i/4) << 4 | 0), key (seed low, seed high).  Outputs (device [n], any may
 * be NULL): idx (-1 if all weights are 0), pdf = w_idx / sum w, wsum. */
nvc_status nvc_wrs_from_weights(const float* w, int64_t n, int32_t n_lights, uint64_t seed,
                                uint32_t frame, uint32_t view, int64_t pixel_offset,
                                int32_t* idx, float* pdf, float* wsum, void* stream);

/* Inference + light weights + WRS for n pixels (pos, nrm device [n][3]). */
nvc_status nvc_wrs_sample(nvc_handle* h, const nvc_scene* scene, const float* pos,
                          const float* nrm, int64_t n, uint64_t seed, uint32_t frame,
                          uint32_t view, int64_t pixel_offset, int32_t* idx, float* pdf,
                          float* wsum, void* stream);

/* Neural direct illumination (Section 3.2): radiance (device [n]) =
 * sum_i vis_i * c_i with the raw predicted visibility, no shadow rays. */
nvc_status nvc_direct_illum(nvc_handle* h, const nvc_scene* scene, const float* pos,
                            const float* nrm, int64_t n, float* radiance, void* stream);

/* The per-pixel hot path in one pass: inference, WRS and Neural DI.
 * Outputs (device [n], any may be NULL) as nvc_wrs_sample and
 * nvc_direct_illum.  fused != 0 runs the single fused kernel of the
 * configuration's precision; fused == 0 runs the separate FP32 kernels
 * (encode, MLP, sampling) with visibility staged in the handle. */
nvc_status nvc_shade(nvc_handle* h, const nvc_scene* scene, const float* pos,
                     const float* nrm, int64_t n, uint64_t seed, uint32_t frame,
                     uint32_t view, int64_t pixel_offset, int32_t* idx, float* pdf,
                     float* wsum, float* radiance, int32_t fused, void* stream);

/* The float32 light weights w (device [n][L]) exactly as the sampler of
 * this configuration's shading path (nvc_shade with fused = 1 for FP16 /
 * BF16, fused = 0 for FP32) computes them for these pixels, so that a
 * caller can re-run the reservoir decision on identical weights. */
nvc_status nvc_sampler_weights(nvc_handle* h, const nvc_scene* scene, const float* pos,
                               const float* nrm, int64_t n, float* w, void* stream);

/* Activation scales of the FP8 (E4M3) path: runs the float32 network on
 * pos (device [n][3], 1 <= n <= batch_positions) and sets each layer
 * input's per-tensor scale to 448 / max |value| (the weights' scales are
 * set the same way from the weights whenever they change).  Required once
 * before FP8 inference; asynchronous. */
nvc_status nvc_calibrate(nvc_handle* h, const float* pos, int64_t n, void* stream);

/* Variants of the fused shading kernel (nvc_shade with fused = 1):
 *   0  every warp encodes, multiplies and samples its own 128-pixel tile;
 *   1  warp-specialised: 4 producer warps encode the next tile while 4
 *      consumer warps run the MLP and the sampler on the current one;
 *   2  as 1, with the producers also computing the light contributions;
 *   3  as 1 with 8 producer warps (two threads per pixel, half the levels
 *      each);
 *   4  as 3 with the contributions computed by the producers;
 *   5  two threads per pixel (256-thread CTAs): the halves split the
 *      encode's levels, the hidden layers' columns and the lights, and meet
 *      in shared memory for the weight maximum, sums and the pick;
 *   6  two tile streams per CTA (256 threads) sharing one copy of the
 *      weights, the light weights kept in shared memory between the
 *      sampler's passes;
 *   7  as 6 with four tile streams per CTA (512 threads).
 * 1-4, 6 and 7 need n_outputs <= 32; 1-7 need FP16/BF16.  All make the same
 * picks from the same float32 weights; all but 5 give bit-identical
 * outputs, 5 sums w and the Neural DI terms over lights [0, H) and [H, L)
 * separately (H = ceil(ceil(L / 2) / 16) * 16), which can change the last
 * bits of wsum, pdf and radiance. */
#define NVC_SHADE_VARIANTS 8

/* Chooses the fused-kernel variant that nvc_infer runs (the variants give
 * bit-identical visibilities; the fastest for exporting them need not be the
 * fastest for shading): times each variant that supports the configuration,
 * `reps` calls of nvc_infer on pos (device [n][3]) into vis (device [n][L],
 * scratch), and keeps the fastest for this handle's nvc_infer.  ms_out (host,
 * NVC_SHADE_VARIANTS doubles, may be NULL) receives each variant's time
 * (-1 where skipped); chosen (host, may be NULL) the variant.  Synchronous.
 * With FP32 inference there are no variants: chosen = -1. */
nvc_status nvc_autotune_infer(nvc_handle* h, const float* pos, int64_t n, float* vis,
                              int32_t reps, int32_t* chosen, double* ms_out, void* stream);

/* Times every applicable variant on these pixels (CUDA events on `stream`,
 * a warm-up then `reps` launches each; synchronises) and keeps the fastest
 * for this handle.  Outputs as nvc_shade (any may be NULL).  chosen (host,
 * may be NULL) receives the variant; ms_out (host [NVC_SHADE_VARIANTS], may
 * be NULL) the mean milliseconds per launch, -1 for a variant not run. */
nvc_status nvc_autotune_shade(nvc_handle* h, const nvc_scene* scene, const float* pos,
                              const float* nrm, int64_t n, int32_t* idx, float* pdf,
                              float* wsum, float* radiance, int32_t reps, int32_t* chosen,
                              double* ms_out, void* stream);

/* Phase profile of the fused shading kernel: one nvc_shade (fused = 1)
 * launch of the handle's variant, which must be 6 or 7 (the tile-stream
 * kernels; NVC_ERR_UNSUPPORTED otherwise), in an instantiation whose first
 * thread of every 128-pixel tile group reads the SM clock at the phase
 * boundaries of each tile.  cycles_out (host [4]) receives the SM cycles
 * summed over all groups and tiles of [0] the hash-grid encode into the
 * operand tile (Section 3.3), [1] the MLP layers up to the output
 * accumulator's read (Section 3.3), [2] the sigmoid, contributions,
 * reservoir pick and Neural DI with the stores (Sections 3.1, 3.2), and
 * [3] every group's whole tile loop; the shares [i] / [3] say where a
 * group's time goes.  Outputs as nvc_shade (pixel ids 0..n-1, view 0).
 * A measurement aid with no counterpart in the paper.  Synchronous. */
nvc_status nvc_shade_phases(nvc_handle* h, const nvc_scene* scene, const float* pos,
                            const float* nrm, int64_t n, uint64_t seed, uint32_t frame,
                            int32_t* idx, float* pdf, float* wsum, float* radiance,
                            double* cycles_out, void* stream);

/* A point of the fused shading kernel's tuning space (nvc_autotune_shade_plan):
 *   variant      the kernel layout, 0 .. NVC_SHADE_VARIANTS-1: tile streams
 *                per CTA (1, 2 or 4 -- 128, 256 or 512 pixels in flight per
 *                CTA: variants 0, 6, 7), the levels of a pixel encoded by one
 *                thread or split between two (variant 5, and variants 3, 4
 *                with producer warps), producer/consumer warp specialisation
 *                (1-4);
 *   ctas_per_sm  how many CTAs of that layout an SM holds at once (the grid
 *                is ctas_per_sm x SMs persistent CTAs); 0 = as many as its
 *                registers, shared memory and TMEM allow.
 * Every point shades identically (the same picks from the same weights;
 * variant 5's sums as stated above). */
typedef struct nvc_shade_plan {
  int32_t variant;
  int32_t ctas_per_sm;
} nvc_shade_plan;

/* Sets the handle's shading point (variant as nvc_set_shade_variant;
 * ctas_per_sm >= 0). */
nvc_status nvc_set_shade_plan(nvc_handle* h, const nvc_shade_plan* plan);

/* The autotuner over the whole tuning space: every applicable variant at
 * ctas_per_sm 0 (all that fit), 1, 2 and 3, each timed as
 * nvc_autotune_shade times a variant (CUDA events on `stream`, a warm-up
 * then `reps` launches; synchronises); keeps the fastest point for the
 * handle.  chosen (host, may be NULL) receives it; points (host
 * [max_points], may be NULL) and ms (host [max_points], may be NULL) every
 * point tried and its mean milliseconds per launch, *n_points (may be
 * NULL) their number.  Outputs as nvc_shade. */
nvc_status nvc_autotune_shade_plan(nvc_handle* h, const nvc_scene* scene, const float* pos,
                                   const float* nrm, int64_t n, int32_t* idx, float* pdf,
                                   float* wsum, float* radiance, int32_t reps,
                                   nvc_shade_plan* chosen, nvc_shade_plan* points, double* ms,
                                   int32_t max_points, int32_t* n_points, void* stream);

/* Selects the fused shading kernel variant (0 .. NVC_SHADE_VARIANTS-1).
 * NVC_ERR_UNSUPPORTED for variants 1-4, 6 and 7 with n_outputs > 32, and for
 * any but 0 and 5 with E4M3 operands. */
nvc_status nvc_set_shade_variant(nvc_handle* h, int32_t variant);

/* ---- the shading pass (Section 3.1) and exact direct illumination -------- */

/* The one-sample estimate of Eq. 1 for the light each pixel's reservoir
 * picked (Section 3.1): one shadow ray from pos[p] to light idx[p] (same
 * segment and occluder tests as nvc_trace_visibility) and
 *     estimate[p] = V c / pdf[p]   (0 when idx[p] < 0, pdf[p] <= 0, c = 0
 *                                   or the ray is blocked),
 * c the light's unshadowed contribution in the float32 order of
 * nvc_light_weights, the division correctly rounded.  idx / pdf as
 * nvc_wrs_sample or nvc_shade write them.  estimate (device [n], may be
 * NULL) receives the estimate; accum (device [n], may be NULL) the running
 * mean over frames: with count = the frame's number k >= 1,
 *     accum[p] = e                               for k = 1,
 *     accum[p] = accum[p] + (e - accum[p]) / k   otherwise (float32, each
 *                                                 step correctly rounded).
 * The scene may hold any number of lights.  Asynchronous on `stream`. */
nvc_status nvc_shade_estimate(const nvc_scene* scene, const float* pos, const float* nrm,
                              int64_t n, const int32_t* idx, const float* pdf, float* estimate,
                              float* accum, uint32_t count, void* stream);

/* Direct illumination with a shadow ray from every pixel to every light:
 * di[p] = sum over lights i in order of c_i for the unblocked ones (float32
 * additions in light order; c_i as in nvc_shade_estimate).  The brute-force
 * reference that the paper's Section 4.4 times against the cache's
 * inference.  pos, nrm device [n][3]; di device [n].  Any number of
 * lights: staged in shared memory when they fit beside the occluders,
 * else read from global memory.  Asynchronous. */
nvc_status nvc_exact_di(const nvc_scene* scene, const float* pos, const float* nrm, int64_t n,
                        float* di, void* stream);

/* ---- clustered cache (Section 3.6) -------------------------------------- */

/* Lights grouped into k clusters, in CSR form (device pointers): the members
 * of cluster y are members[offsets[y] .. offsets[y + 1] - 1] (light indices
 * into nvc_scene.lights, increasing).  The caller owns both arrays and
 * keeps them valid: offsets[0] = 0, non-decreasing, offsets[k] = n_lights,
 * every member in [0, n_lights).  The library does not read the table back
 * to check it (that would cost a synchronisation per call); an invalid
 * table makes the kernels read out of bounds.  With a clustered cache the
 * configuration's n_outputs is k (at most 32) and each output is a
 * cluster's average visibility; the scene may hold any number of lights. */
/* Weights of the first sampling step (nvc_sample_clustered):
 *   NVC_CLUSTER_WEIGHT_SUM         w_y = max(v_y, 0.001) * sum of the members'
 *                                  contributions (one contribution per light
 *                                  and pixel);
 *   NVC_CLUSTER_WEIGHT_VISIBILITY  w_y = max(v_y, 0.001), the inferred average
 *                                  visibility alone (cost independent of the
 *                                  light count).
 * Empty clusters weigh 0 in both; both estimators are unbiased. */
#define NVC_CLUSTER_WEIGHT_SUM 0
#define NVC_CLUSTER_WEIGHT_VISIBILITY 1

typedef struct nvc_clusters {
  int32_t k;
  const int32_t* offsets;    /* [k + 1] */
  const int32_t* members;    /* [n_lights] */
  int32_t weights;           /* NVC_CLUSTER_WEIGHT_*; 0 (zero-initialised) = SUM */
} nvc_clusters;

/* Lloyd's k-means of the light positions (host memory; Section 3.6), in
 * float64: centroids start at the lights init[0..k-1]; each of `iters`
 * iterations assigns every light to its nearest centroid (squared distance
 * (dx^2 + dy^2) + dz^2, ties to the lower cluster) and moves each centroid to
 * the mean of its members summed in light order (an empty cluster keeps its
 * centroid); assign[i] (host [n]) is the final assignment; centroids (host
 * [k][3], may be NULL) the final centroids.  Synchronous, host only. */
nvc_status nvc_kmeans_lights(const float* lights, int32_t n_lights, const int32_t* init,
                             int32_t k, int32_t iters, int32_t* assign, double* centroids);

/* One training step of a clustered cache (Section 3.6): as nvc_train_step,
 * but the target of output y at a training position is the binary
 * visibility of one member of cluster y drawn uniformly (word y of the
 * Philox stream (sample, frame, 0, tag 5)), so the network learns each
 * cluster's average visibility.  clusters->k must equal n_outputs. */
nvc_status nvc_train_step_clustered(nvc_handle* h, const nvc_scene* scene,
                                    const nvc_clusters* clusters, const float* screen_pos,
                                    int64_t n_screen, uint64_t seed, uint32_t frame,
                                    double* loss_out, void* stream);

/* Training targets of a clustered cache for given positions (device [n][3])
 * into target (device [n][k]), sample ids 0..n-1 (n <= 2^32): the data step
 * of nvc_train_step_clustered.  Asynchronous. */
nvc_status nvc_cluster_targets(const nvc_scene* scene, const nvc_clusters* clusters,
                               const float* pos, int64_t n, uint64_t seed, uint32_t frame,
                               float* target, void* stream);

/* Two-step light sampling with a clustered cache (Section 3.6), per pixel:
 *   1. the cluster weights of clusters->weights (for SUM, c_hat_y = sum of
 *      the members' contributions in float32 member order and
 *      w_y = max(vis[p][y], 0.001) c_hat_y), and cluster y picked by the
 *      integer reservoir of nvc_wrs_sample (Philox tag 0, word y);
 *   2. four members of y drawn uniformly (words 0-3 of tag 4), one kept by
 *      the integer reservoir on their contributions (words 4-7), with the
 *      unbiased contribution weight of streaming RIS
 *        W = (sum_j c_j / 4) / (p(x) c(x)),  p(x) = (w_y / sum w) / m_y.
 * vis: device [n][k], the cache's cluster visibilities (nvc_infer).
 * light (device [n], -1 when nothing contributes), weight (W) and estimate
 * (V(x) c(x) W with one shadow ray, 0 when blocked) may each be NULL.
 * Pixel ids are pixel_offset + p.  The scene's lights are staged in shared
 * memory when they fit beside the occluders (about 14,000 lights), else
 * read from global memory; step 1 costs one contribution per light and
 * pixel.  Asynchronous. */
nvc_status nvc_sample_clustered(const nvc_scene* scene, const nvc_clusters* clusters,
                                const float* vis, const float* pos, const float* nrm, int64_t n,
                                int64_t pixel_offset, uint64_t seed, uint32_t frame,
                                uint32_t view, int32_t* light, float* weight, float* estimate,
                                void* stream);

/* ---- the cache as ReSTIR's initial-candidate generator (Sections 3.1, 4.2)
 *
 * Temporal resampling of one reservoir per pixel: the frame's
 * initial-candidate reservoir, made by the cache's sampler (cur_light with
 * its unbiased contribution weight cur_W: 1 / pdf from nvc_wrs_sample /
 * nvc_shade, or W from nvc_sample_clustered), counts M_c = 1 candidate and
 * needs no shadow ray of its own (the cache already weighs visibility);
 * the previous frame's reservoir at the same pixel (prev_light, prev_W,
 * prev_M; prev_M = 0 where the pixel is disoccluded, so the cache's
 * candidate stands alone) counts M_p' = min(prev_M, 20) (the previous
 * reservoir counts at most 20x the new one).  With the target p_hat(y) =
 * c_y, the float32 contribution of nvc_light_weights:
 *     w_c = (1 * p_hat(y_c)) * W_c,   w_p = (M_p' * p_hat(y_p)) * W_p,
 * the integer reservoir of nvc_wrs_sample picks y from (y_c, y_p) with
 * words 0, 1 of the Philox stream (pixel_offset + p, frame, view, 6), and
 *     M = 1 + M_p',   W = (w_c + w_p) / (M * p_hat(y))
 * (float32, each operation correctly rounded in that order; y = -1, W = 0
 * when both weights are 0; a light index outside [0, n_lights) counts as
 * no sample).  Outputs (device [n], any may be NULL, not all): light, W,
 * M and estimate = V(y) p_hat(y) W with one shadow ray (0 when blocked or
 * empty).  The output reservoir is next frame's previous reservoir.
 * prev_* (device [n]) may all be NULL: every pixel disoccluded.  Any
 * number of lights.  Asynchronous. */
nvc_status nvc_temporal_merge(const nvc_scene* scene, const float* pos, const float* nrm,
                              int64_t n, int64_t pixel_offset, uint64_t seed, uint32_t frame,
                              uint32_t view, const int32_t* cur_light, const float* cur_W,
                              const int32_t* prev_light, const float* prev_W,
                              const int32_t* prev_M, int32_t* light, float* W, int32_t* M,
                              float* estimate, void* stream);

/* ---- training (Section 3.4) -------------------------------------------- */

/* Binary visibility vis (device [n][n_lights], 0 or 1) of every light from
 * every position: the segment x + t (l - x), t in [1e-4, 1 - 1e-4], is
 * blocked by a sphere whose centre is closer than its radius to the segment
 * or by a box the segment touches (slab test); float32 arithmetic. */
nvc_status nvc_trace_visibility(const nvc_scene* scene, const float* pos, int64_t n,
                                float* vis, void* stream);

/* Training positions (device [batch][3]; the scene may hold any number of
 * lights, only its world box is used), Section 3.4: positions j < n_w are
 * uniform in the scene's world box, x = lo + u * (hi - lo), u the top 24
 * bits of the words of Philox stream (j, frame, 0, 1) times 2^-24; the rest
 * are G-buffer pixels screen_pos[floor(r * n_screen / 2^32)], r word 0 of
 * stream (j - n_w, frame, 0, 2).  n_w = ceil(batch / 2), the paper's equal
 * world/screen split; n_w = batch when screen_pos is NULL or n_screen = 0. */
nvc_status nvc_training_positions(const nvc_scene* scene, const float* screen_pos,
                                  int64_t n_screen, int64_t batch, uint64_t seed,
                                  uint32_t frame, float* pos, void* stream);

/* nvc_training_positions with a chosen split (the placement options of
 * Section 3.4): n_world world-space positions (0 = screen space only,
 * batch = world space only, -1 = the default ceil(batch / 2)), the rest
 * screen space.  Without screen positions every position is world space.
 * NVC_ERR_INVALID_ARG unless -1 <= n_world <= batch. */
nvc_status nvc_training_positions_split(const nvc_scene* scene, const float* screen_pos,
                                        int64_t n_screen, int64_t batch, int64_t n_world,
                                        uint64_t seed, uint32_t frame, float* pos, void* stream);

/* Placement of the handle's training positions for the following training
 * steps and frames (per-light and clustered): n_world of the
 * batch_positions positions in world space, as nvc_training_positions_split
 * (-1 restores the default split).  Host only; takes effect at the next
 * step, including captured frame graphs (they are recaptured per frame). */
nvc_status nvc_set_training_placement(nvc_handle* h, int64_t n_world);

/* Where an FP16 (tensor-core) training step makes its batch (Section 4.4
 * runs data generation fused into the training pass): fused = 0 (the
 * default) makes the positions and their shadow-ray targets in a launch of
 * their own over all SMs before the training kernel; fused != 0 makes them
 * inside the training kernel, each CTA its own 128-position tiles, the rays
 * traced slice by slice while the forward layers' MMAs run.  Both give the
 * same positions and targets bit for bit (nvc_training_positions /
 * nvc_trace_visibility arithmetic) and so the same loss.  Per-light steps
 * only (clustered steps keep their own targets); the fused form falls back
 * to the separate one when the scene's occluders and lights do not fit in
 * shared memory beside the training tiles.  Host only.
 * NVC_ERR_UNSUPPORTED with FP32 training. */
nvc_status nvc_set_training_data_fused(nvc_handle* h, int32_t fused);

/* The batch of the last training step: positions (device [batch_positions]
 * [3], may be NULL) and binary targets (device [batch_positions][n_outputs],
 * may be NULL) as the step made them.  Asynchronous copies on `stream`. */
nvc_status nvc_training_batch(nvc_handle* h, float* pos, float* target, void* stream);

/* One online training step: batch_positions positions (as
 * nvc_training_positions), shadow-ray targets, forward, loss (L2 or BCE,
 * mean over positions x lights), hand-written backward, Adam (bias
 * corrected; lr from the schedule).  A non-finite gradient skips the
 * update and is counted.  loss_out (device double, may be NULL) receives
 * the unscaled loss. */
nvc_status nvc_train_step(nvc_handle* h, const nvc_scene* scene, const float* screen_pos,
                          int64_t n_screen, uint64_t seed, uint32_t frame, double* loss_out,
                          void* stream);

/* The training step without the update: grad (device [n_params]) receives
 * d loss / d params (unscaled) for the same batch nvc_train_step would use. */
nvc_status nvc_train_gradient(nvc_handle* h, const nvc_scene* scene, const float* screen_pos,
                              int64_t n_screen, uint64_t seed, uint32_t frame, float* grad,
                              double* loss_out, void* stream);

/* Differentiable forward for autograd wrappers: logits (device [n][L]) of
 * pos (device [n][3]), n <= batch_positions; activations are kept in the
 * handle for the next nvc_mlp_backward. */
nvc_status nvc_mlp_forward(nvc_handle* h, const float* pos, int64_t n, float* logits,
                           void* stream);

/* Adjoint of the last nvc_mlp_forward: grad (device [n_params]) receives
 * sum_{b,i} dlogits[b][i] * d logits[b][i] / d params (overwritten). */
nvc_status nvc_mlp_backward(nvc_handle* h, const float* pos, int64_t n,
                            const float* dlogits, float* grad, void* stream);

/* ---- one frame ---------------------------------------------------------- */

/* One view of a frame: its G-buffer and its outputs (device [n_pixels];
 * idx/pdf/wsum/radiance may be NULL). */
typedef struct nvc_view {
  const float* pos;
  const float* nrm;
  int64_t n_pixels;
  uint32_t view_id;
  int32_t* idx;
  float* pdf;
  float* wsum;
  float* radiance;
} nvc_view;

#define NVC_FRAME_WORLD_ONLY (-1) /* train_view: world-space training positions only */
#define NVC_FRAME_NO_TRAINING (-2) /* train_view: no training step this frame */

/* One frame: a training step (Section 3.4: one step per frame) whose
 * screen-space positions come from view `train_view` (or see the two
 * constants above), then inference + WRS + Neural DI of every view.
 * use_graph != 0 records the frame's launches as a CUDA graph and replays
 * it, updating the recorded graph in place when arguments change. */
nvc_status nvc_frame(nvc_handle* h, const nvc_scene* scene, const nvc_view* views,
                     int32_t n_views, int32_t train_view, uint64_t seed, uint32_t frame,
                     double* loss_out, int32_t use_graph, void* stream);

/* One frame from and to host memory: as nvc_frame, with every view's pos,
 * nrm, idx, pdf, wsum and radiance pointing to host memory (page-locked,
 * e.g. cudaHostAlloc; outputs may be NULL).  No counterpart in the paper:
 * it is the upload / read-back a renderer wraps around Section 4's passes.
 *
 * Asynchronous and pipelined: the library stages the G-buffers in one of two
 * device slots (alternating per call; grown with cudaMalloc when a frame has
 * more pixels than any before), uploads on its own copy stream, runs the
 * frame on `stream` once the upload is done, and reads the outputs back on a
 * second copy stream once the frame is done.  So frame f's compute overlaps
 * frame f + 1's upload and frame f - 1's read-back.  The host inputs must
 * stay unchanged, and the host outputs unread, until the frame's read-back
 * has completed: nvc_host_frames_wait orders `stream` after every read-back
 * issued so far.  Errors as nvc_frame. */
nvc_status nvc_frame_host(nvc_handle* h, const nvc_scene* scene, const nvc_view* host_views,
                          int32_t n_views, int32_t train_view, uint64_t seed, uint32_t frame,
                          double* loss_out, int32_t use_graph, void* stream);

/* Makes `stream` wait for every read-back nvc_frame_host has issued
 * (asynchronous: synchronise `stream` to wait on the host). */
nvc_status nvc_host_frames_wait(nvc_handle* h, void* stream);

/* ---- inference without allocation ---------------------------------------- */

/* The paper has no counterpart of this entry point.  It exists for callers
 * that cannot call cudaMalloc: a renderer whose frame loop runs under a
 * fixed GPU memory budget (cudaMalloc can synchronise the device and stall
 * a frame), or a plugin inside an application that owns every device
 * allocation.  Everything else here needs a handle, and nvc_create
 * allocates.
 *
 * Same result as nvc_infer on a float32 handle holding `params`: vis
 * (device [n][n_outputs]) = sigmoid(MLP(encode(pos))) with the float32
 * kernels, for pos (device [n][3]) and params (device [nvc_param_count],
 * 16-byte aligned, the layout of nvc_set_state).  cfg->precision is
 * ignored.  No memory is allocated: the encoded features go to a fixed
 * array of 2^21 floats (8 MiB) inside the library, which every GPU that
 * loads the library holds until the process exits; n * n_levels *
 * n_features above 2^21 is rejected with NVC_ERR_INVALID_ARG and a message
 * in nvc_last_error(NULL).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call on a device
 * uses the same array: calls whose kernels overlap on the GPU (other
 * streams, other host threads) race on it and must be ordered by the
 * caller. */
nvc_status nvc_infer_noalloc(const nvc_config* cfg, const float* params, const float* pos,
                             int64_t n, float* vis, void* stream);

/* ---- profiling ---------------------------------------------------------- */

/* Random-row gather microbenchmark: the roofline denominator of the
 * hash-grid encode, which reads 8 rows of a level's table per position at
 * hashed, effectively random rows (Section 3.3).  n_threads threads each
 * load rows_per_thread (a multiple of 8) rows of row_bytes (4, 8 or 16)
 * bytes from table (device, 16-byte aligned, table_bytes / row_bytes a
 * power of two up to 2^31), eight independent loads in flight before they
 * are summed, row indices from a per-thread linear congruential sequence
 * started from `seed`; sink (device [n_threads]) receives each thread's
 * sum so that no load is dead.  The caller times the launch on `stream`;
 * rows gathered = n_threads * rows_per_thread.  A measurement aid with no
 * counterpart in the paper.  Asynchronous. */
nvc_status nvc_gather_bench(const void* table, int64_t table_bytes, int32_t row_bytes,
                            int64_t n_threads, int32_t rows_per_thread, uint32_t seed,
                            float* sink, void* stream);


/* When enabled, the handle records CUDA events around each stage it
 * launches; nvc_stage_times (synchronising) returns the summed milliseconds
 * per stage since the last reset: [0] training data, [1] training
 * forward+backward, [2] Adam, [3] shade (inference+WRS+DI). */
nvc_status nvc_set_profiling(nvc_handle* h, int32_t enable);
nvc_status nvc_stage_times(nvc_handle* h, double* ms_out, int32_t n_out, int64_t* launches_out);

#ifdef __cplusplus
}
#endif
#endif /* NVC_H */
