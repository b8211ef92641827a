// Random-row gather microbenchmark: the rate at which the SMs fetch rows
// of 4, 8 or 16 bytes at uniformly random places of a table that stays in
// L2.  It is the roofline denominator of the hash-grid encode (Section 3.3
// of the paper): an encode reads 8 table rows per (pixel, level) at hashed,
// effectively random addresses, each row F features wide.
//
// The access pattern follows the encode's: every thread issues 8
// independent row loads (one cell's corners) before it consumes any of
// them, then blends them into a running sum so that no load is dead.  Row
// indices come from a 32-bit linear congruential sequence per thread, top
// bits taken, which costs two instructions a row -- less than the encode's
// hash, so the rate measured is the memory system's, not the index
// arithmetic's.
#include "nvc_internal.cuh"

namespace nvc {
namespace {

template <int ROW>
struct RowT;
template <>
struct RowT<4> {
  using T = float;
  __device__ static float first(float v) { return v; }
};
template <>
struct RowT<8> {
  using T = float2;
  __device__ static float first(float2 v) { return v.x + v.y; }
};
template <>
struct RowT<16> {
  using T = float4;
  __device__ static float first(float4 v) { return (v.x + v.y) + (v.z + v.w); }
};

template <int ROW>
__global__ void __launch_bounds__(256) gather_bench_kernel(const void* __restrict__ table,
                                                           int row_shift, int groups,
                                                           uint32_t seed, float* __restrict__ sink,
                                                           int64_t n_threads) {
  using T = typename RowT<ROW>::T;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= n_threads) return;
  const T* rows = reinterpret_cast<const T*>(table);
  // a distinct, well-mixed start per thread (one multiply-xorshift round)
  uint32_t s = (uint32_t)tid * 0x9E3779B1u ^ seed;
  s ^= s >> 16;
  s *= 0x85EBCA6Bu;
  s ^= s >> 13;
  float acc = 0.0f;
  for (int g = 0; g < groups; ++g) {
    uint32_t r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      s = s * 1664525u + 1013904223u;
      r[k] = s >> row_shift;
    }
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldg(rows + r[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc += RowT<ROW>::first(v[k]);
  }
  sink[tid] = acc;
}

}  // namespace
}  // namespace nvc

extern "C" nvc_status nvc_gather_bench(const void* table, int64_t table_bytes, int32_t row_bytes,
                                       int64_t n_threads, int32_t rows_per_thread, uint32_t seed,
                                       float* sink, void* stream) {
  using namespace nvc;
  if (row_bytes != 4 && row_bytes != 8 && row_bytes != 16) {
    record_error("nvc_gather_bench: row_bytes must be 4, 8 or 16");
    return NVC_ERR_INVALID_ARG;
  }
  const int64_t n_rows = table_bytes / row_bytes;
  if (table_bytes <= 0 || table_bytes % row_bytes != 0 || (n_rows & (n_rows - 1)) != 0 ||
      n_rows < 2 || n_rows > ((int64_t)1 << 31)) {
    record_error("nvc_gather_bench: table_bytes / row_bytes must be a power of two in [2, 2^31]");
    return NVC_ERR_INVALID_ARG;
  }
  if (n_threads < 1 || rows_per_thread < 8 || rows_per_thread % 8 != 0) {
    record_error("nvc_gather_bench: need n_threads >= 1 and rows_per_thread a positive multiple of 8");
    return NVC_ERR_INVALID_ARG;
  }
  if (!table || ((uintptr_t)table & 15) || !sink || ((uintptr_t)sink & 3)) {
    record_error("nvc_gather_bench: table (16-byte aligned) and sink must be device pointers");
    return NVC_ERR_INVALID_ARG;
  }
  int log2_rows = 0;
  while (((int64_t)1 << log2_rows) < n_rows) ++log2_rows;
  const int shift = 32 - log2_rows;   // top log2_rows bits of the sequence: an index < n_rows
  const int groups = rows_per_thread / 8;
  const int64_t blocks = (n_threads + 255) / 256;
  if (blocks > 0x7FFFFFFFLL) {
    record_error("nvc_gather_bench: too many threads");
    return NVC_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  switch (row_bytes) {
    case 4:
      gather_bench_kernel<4><<<(unsigned)blocks, 256, 0, s>>>(table, shift, groups, seed, sink, n_threads);
      break;
    case 8:
      gather_bench_kernel<8><<<(unsigned)blocks, 256, 0, s>>>(table, shift, groups, seed, sink, n_threads);
      break;
    default:
      gather_bench_kernel<16><<<(unsigned)blocks, 256, 0, s>>>(table, shift, groups, seed, sink, n_threads);
      break;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    record_error(cudaGetErrorString(e));
    return NVC_ERR_CUDA;
  }
  return NVC_OK;
}
