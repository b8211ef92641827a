// Plain float32 MLP (Section 3.3: hidden layers with leaky ReLU, sigmoid
// output, no biases) on the CUDA cores: the reference GPU path the tensor-
// core kernels are measured against, and the float32 training forward and
// backward.
//
// Forward: one sample per thread, 128 threads per block, persistent over
// 128-row tiles.  All weight matrices live in shared memory transposed to
// [in][out] so 8 consecutive outputs are two broadcast float4 loads; the
// activations of the tile live in shared memory as [feature][row] with a
// row stride of 129 floats (bank-conflict free for both the per-thread
// reads and the cooperative tile loads).
//
// Backward (the hand-written adjoint): delta_out -> for each layer from the
// top, g = delta W (rows of W are contiguous, so the original [out][in]
// layout is the broadcast-friendly one here), delta = g * act'(a) with
// act'(a) = 1 for a > 0 else the slope; the weight gradients
// dW = delta^T a are a separate tiled reduction over the batch.
#include "nvc_internal.cuh"

namespace nvc {

namespace {

// Samples per tile = threads per block: 128, or 32 when a batch has fewer
// 128-row tiles than SMs (so a small training batch still spreads over the
// GPU).  Shared activation rows are padded to R + 1 floats (no bank
// conflicts between the threads' columns).
constexpr int kRows = 128;
constexpr int kRowsSmall = 32;

struct MlpDims {
  int n_layers;
  int in[NVC_MAX_HIDDEN_LAYERS + 1];
  int out[NVC_MAX_HIDDEN_LAYERS + 1];
  int pad_out[NVC_MAX_HIDDEN_LAYERS + 1];  // out rounded up to 8
  int pad_in[NVC_MAX_HIDDEN_LAYERS + 1];   // in rounded up to 8
  int64_t w_off[NVC_MAX_HIDDEN_LAYERS + 1];
  int s_off[NVC_MAX_HIDDEN_LAYERS + 1];    // smem float offset of each layer
  int s_weights;                           // total smem floats for weights
  int maxdim;
  float slope;
};

__host__ __device__ inline int round8(int x) { return (x + 7) & ~7; }

MlpDims make_dims(const nvc_handle* h, bool transposed) {
  MlpDims d{};
  d.n_layers = h->n_layers;
  d.slope = h->cfg.leaky_slope;
  int off = 0;
  // the shared activation buffers hold the encoded input and hidden layers;
  // the output layer goes straight to global memory (and, in the backward,
  // its delta is read from there)
  d.maxdim = h->din > h->width ? h->din : h->width;
  for (int k = 0; k < h->n_layers; ++k) {
    d.in[k] = h->w_in[k];
    d.out[k] = h->w_out[k];
    d.pad_out[k] = round8(h->w_out[k]);
    d.pad_in[k] = round8(h->w_in[k]);
    d.w_off[k] = h->w_off[k];
    d.s_off[k] = off;
    off += transposed ? d.in[k] * d.pad_out[k] : d.out[k] * d.pad_in[k];
  }
  d.s_weights = off;
  return d;
}

size_t smem_bytes(const MlpDims& d, int rows = kRows) {
  return sizeof(float) * ((size_t)d.s_weights + 2 * (size_t)round8(d.maxdim) * (rows + 1));
}

__device__ __forceinline__ float act_fn(float z, float slope) { return z > 0.0f ? z : slope * z; }

__device__ __forceinline__ float sigmoid_f(float z) { return 1.0f / (1.0f + expf(-z)); }

template <int R>
__global__ void __launch_bounds__(R) mlp_fwd_kernel(const float* __restrict__ feat, int64_t n,
                                                        const float* __restrict__ params,
                                                        MlpDims d, float* __restrict__ y,
                                                        int sigmoid_out,
                                                        float* __restrict__ act_store,
                                                        int64_t act_layer_stride) {
  extern __shared__ float smem[];
  float* sw = smem;
  float* buf0 = smem + d.s_weights;
  float* buf1 = buf0 + round8(d.maxdim) * (R + 1);
  const int t = threadIdx.x;

  // weights, transposed to [in][pad_out] with zero padding
  for (int k = 0; k < d.n_layers; ++k) {
    const int in = d.in[k], out = d.out[k], po = d.pad_out[k];
    for (int e = t; e < in * po; e += R) {
      const int i = e / po, j = e - i * po;
      sw[d.s_off[k] + e] = j < out ? __ldg(params + d.w_off[k] + (int64_t)j * in + i) : 0.0f;
    }
  }
  __syncthreads();

  const int din = d.in[0];
  const int64_t n_tiles = (n + R - 1) / R;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * R;
    const int rows = (int)(n - row0 < R ? n - row0 : R);
    // cooperative, coalesced load of the tile's inputs into buf0[k][row]
    for (int e = t; e < R * din; e += R) {
      const int r = e / din, k = e - r * din;
      buf0[k * (R + 1) + r] = r < rows ? __ldg(feat + (row0 + r) * din + k) : 0.0f;
    }
    __syncthreads();
    float* src = buf0;
    float* dst = buf1;
    const int64_t row = row0 + t;
    const bool live = t < rows;
    for (int k = 0; k < d.n_layers; ++k) {
      const int in = d.in[k], nout = d.out[k], po = d.pad_out[k];
      const float* wk = sw + d.s_off[k];
      const bool last = k == d.n_layers - 1;
      for (int jb = 0; jb < po; jb += 8) {
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < in; ++i) {
          const float x = src[i * (R + 1) + t];
          const float4 w0 = *reinterpret_cast<const float4*>(wk + i * po + jb);
          const float4 w1 = *reinterpret_cast<const float4*>(wk + i * po + jb + 4);
          acc[0] = fmaf(w0.x, x, acc[0]);
          acc[1] = fmaf(w0.y, x, acc[1]);
          acc[2] = fmaf(w0.z, x, acc[2]);
          acc[3] = fmaf(w0.w, x, acc[3]);
          acc[4] = fmaf(w1.x, x, acc[4]);
          acc[5] = fmaf(w1.y, x, acc[5]);
          acc[6] = fmaf(w1.z, x, acc[6]);
          acc[7] = fmaf(w1.w, x, acc[7]);
        }
        if (!last) {
          float* a_row = act_store ? act_store + k * act_layer_stride + row * nout : nullptr;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = jb + q;
            if (j < nout) {
              const float a = act_fn(acc[q], d.slope);
              dst[j * (R + 1) + t] = a;
              if (a_row && live) a_row[j] = a;
            }
          }
        } else if (live) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = jb + q;
            if (j < nout) y[row * nout + j] = sigmoid_out ? sigmoid_f(acc[q]) : acc[q];
          }
        }
      }
      __syncthreads();
      float* tmp = src;
      src = dst;
      dst = tmp;
    }
  }
}

template <int R>
__global__ void __launch_bounds__(R) mlp_bwd_kernel(int64_t n, const float* __restrict__ params,
                                                        MlpDims d, const float* __restrict__ act,
                                                        int64_t act_layer_stride,
                                                        float* __restrict__ delta,
                                                        int64_t delta_layer_stride,
                                                        float* __restrict__ dfeat) {
  extern __shared__ float smem[];
  float* sw = smem;
  float* buf0 = smem + d.s_weights;
  float* buf1 = buf0 + round8(d.maxdim) * (R + 1);
  const int t = threadIdx.x;
  // weights in [out][pad_in] (rows contiguous), zero padding
  for (int k = 0; k < d.n_layers; ++k) {
    const int in = d.in[k], out = d.out[k], pi = d.pad_in[k];
    for (int e = t; e < out * pi; e += R) {
      const int j = e / pi, i = e - j * pi;
      sw[d.s_off[k] + e] = i < in ? __ldg(params + d.w_off[k] + (int64_t)j * in + i) : 0.0f;
    }
  }
  __syncthreads();
  const int top = d.n_layers - 1;
  const int L = d.out[top];
  const int64_t n_tiles = (n + R - 1) / R;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * R;
    const int rows = (int)(n - row0 < R ? n - row0 : R);
    const float* dtop = delta + top * delta_layer_stride;
    float* src = buf0;
    float* dst = buf1;
    const int64_t row = row0 + t;
    const bool live = t < rows;
    for (int k = top; k >= 0; --k) {
      const int in = d.in[k], out = d.out[k], pi = d.pad_in[k];
      const float* wk = sw + d.s_off[k];
      const float* g_row = dtop + (live ? row : 0) * L;   // top layer: delta from global
      for (int ib = 0; ib < pi; ib += 8) {
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int j = 0; j < out; ++j) {
          const float g = k == top ? (live ? g_row[j] : 0.0f) : src[j * (R + 1) + t];
          const float4 w0 = *reinterpret_cast<const float4*>(wk + j * pi + ib);
          const float4 w1 = *reinterpret_cast<const float4*>(wk + j * pi + ib + 4);
          acc[0] = fmaf(w0.x, g, acc[0]);
          acc[1] = fmaf(w0.y, g, acc[1]);
          acc[2] = fmaf(w0.z, g, acc[2]);
          acc[3] = fmaf(w0.w, g, acc[3]);
          acc[4] = fmaf(w1.x, g, acc[4]);
          acc[5] = fmaf(w1.y, g, acc[5]);
          acc[6] = fmaf(w1.z, g, acc[6]);
          acc[7] = fmaf(w1.w, g, acc[7]);
        }
        if (k > 0) {
          // input of layer k is hidden layer k-1's activation a: delta = g * act'(a)
          const float* a_row = act + (int64_t)(k - 1) * act_layer_stride + row * in;
          float* d_row = delta + (int64_t)(k - 1) * delta_layer_stride + row * in;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int i = ib + q;
            if (i < in) {
              const float a = live ? a_row[i] : 0.0f;
              const float dv = a > 0.0f ? acc[q] : d.slope * acc[q];
              dst[i * (R + 1) + t] = dv;
              if (live) d_row[i] = dv;
            }
          }
        } else if (live) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int i = ib + q;
            if (i < in) dfeat[row * in + i] = acc[q];
          }
        }
      }
      __syncthreads();
      float* tmp = src;
      src = dst;
      dst = tmp;
    }
  }
}

// dW[j][i] += sum_b D[b][j] * A[b][i] over a `chunk`-row slice of the batch
// (a multiple of kWgSub), one 32 x 32 tile of dW per CTA.
constexpr int kWgTile = 32, kWgSub = 32;

__global__ void __launch_bounds__(256) weight_grad_kernel(const float* __restrict__ D, int ldd,
                                                          const float* __restrict__ A, int lda,
                                                          int64_t n, int n_out, int n_in,
                                                          int chunk, float* __restrict__ dW,
                                                          int32_t* status) {
  __shared__ float sD[kWgSub][kWgTile + 1];
  __shared__ float sA[kWgSub][kWgTile + 1];
  const int j0 = blockIdx.x * kWgTile, i0 = blockIdx.y * kWgTile;
  const int64_t b0 = (int64_t)blockIdx.z * chunk;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[2][2] = {{0, 0}, {0, 0}};
  for (int sb = 0; sb < chunk && b0 + sb < n; sb += kWgSub) {
    for (int e = threadIdx.x; e < kWgSub * kWgTile; e += 256) {
      const int r = e / kWgTile, c = e - r * kWgTile;
      const int64_t b = b0 + sb + r;
      sD[r][c] = (b < n && j0 + c < n_out) ? D[b * ldd + j0 + c] : 0.0f;
      sA[r][c] = (b < n && i0 + c < n_in) ? A[b * lda + i0 + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < kWgSub; ++r) {
      const float d0 = sD[r][ty], d1 = sD[r][ty + 16];
      const float a0 = sA[r][tx], a1 = sA[r][tx + 16];
      acc[0][0] = fmaf(d0, a0, acc[0][0]);
      acc[0][1] = fmaf(d0, a1, acc[0][1]);
      acc[1][0] = fmaf(d1, a0, acc[1][0]);
      acc[1][1] = fmaf(d1, a1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = j0 + ty + 16 * p, i = i0 + tx + 16 * q;
      if (j < n_out && i < n_in) {
        if (!isfinite(acc[p][q])) atomicOr(status + kStNonFinite, 1);
        atomicAdd(dW + (int64_t)j * n_in + i, acc[p][q]);
      }
    }
}

int small_rows(const nvc_handle* h, int64_t n) { return (n + kRows - 1) / kRows < h->num_sms; }

template <int R>
cudaError_t launch_fwd(const nvc_handle* h, const MlpDims& d, const float* feat, int64_t n,
                       float* out, bool sigmoid_out, float* act_store, cudaStream_t s) {
  const size_t smem = smem_bytes(d, R);
  cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel<R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t n_tiles = (n + R - 1) / R;
  const int per_sm = blocks_per_sm((const void*)mlp_fwd_kernel<R>, R, smem);
  const int64_t cap = (int64_t)per_sm * h->num_sms;
  const int blocks = (int)(n_tiles < cap ? n_tiles : cap);
  mlp_fwd_kernel<R><<<blocks, R, smem, s>>>(feat, n, h->params, d, out, sigmoid_out ? 1 : 0,
                                            act_store, (int64_t)h->B * h->width);
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_bwd(const nvc_handle* h, const MlpDims& d, int64_t n, cudaStream_t s) {
  const size_t smem = smem_bytes(d, R);
  cudaError_t e = cudaFuncSetAttribute(mlp_bwd_kernel<R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t n_tiles = (n + R - 1) / R;
  const int per_sm = blocks_per_sm((const void*)mlp_bwd_kernel<R>, R, smem);
  const int64_t cap = (int64_t)per_sm * h->num_sms;
  const int blocks = (int)(n_tiles < cap ? n_tiles : cap);
  const int maxdim = h->width > h->L ? h->width : h->L;
  mlp_bwd_kernel<R><<<blocks, R, smem, s>>>(n, h->params, d, h->t_act,
                                            (int64_t)h->B * h->width, h->t_delta,
                                            (int64_t)h->B * maxdim, h->t_dfeat);
  return cudaGetLastError();
}

}  // namespace

size_t mlp_fwd_smem_bytes(const nvc_handle* h) { return smem_bytes(make_dims(h, true)); }

cudaError_t launch_mlp_fwd_fp32(const nvc_handle* h, const float* feat, int64_t n, float* out,
                                bool sigmoid_out, float* act_store, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const MlpDims d = make_dims(h, true);
  return small_rows(h, n) ? launch_fwd<kRowsSmall>(h, d, feat, n, out, sigmoid_out, act_store, s)
                          : launch_fwd<kRows>(h, d, feat, n, out, sigmoid_out, act_store, s);
}

cudaError_t launch_mlp_bwd_fp32(const nvc_handle* h, int64_t n, const float* dlogits_unused,
                                float* grad, int32_t* status, cudaStream_t s) {
  (void)dlogits_unused;
  if (n == 0) return cudaSuccess;
  const MlpDims d = make_dims(h, false);
  cudaError_t e = small_rows(h, n) ? launch_bwd<kRowsSmall>(h, d, n, s) : launch_bwd<kRows>(h, d, n, s);
  if (e != cudaSuccess) return e;
  const int maxdim = h->width > h->L ? h->width : h->L;
  const int64_t act_stride = (int64_t)h->B * h->width;
  const int64_t delta_stride = (int64_t)h->B * maxdim;
  // weight gradients: layer k's input is t_feat (k = 0) or hidden activation k-1
  for (int k = 0; k < h->n_layers; ++k) {
    const float* D = h->t_delta + (int64_t)k * delta_stride;
    const float* A = k == 0 ? h->t_feat : h->t_act + (int64_t)(k - 1) * act_stride;
    const int lda = h->w_in[k];
    // split the batch so the layer's tiles give about two CTAs per SM: a
    // small batch is otherwise a handful of CTAs walking it serially
    const int tx = (h->w_out[k] + kWgTile - 1) / kWgTile, ty = (h->w_in[k] + kWgTile - 1) / kWgTile;
    const int64_t want = 2 * (int64_t)h->num_sms;
    int64_t chunk = (n * tx * ty + want - 1) / want;
    chunk = (chunk + kWgSub - 1) / kWgSub * kWgSub;
    if (chunk < kWgSub) chunk = kWgSub;
    dim3 grid(tx, ty, (unsigned)((n + chunk - 1) / chunk));
    weight_grad_kernel<<<grid, 256, 0, s>>>(D, h->w_out[k], A, lda, n, h->w_out[k], h->w_in[k],
                                            (int)chunk, grad + h->w_off[k], status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nvc
