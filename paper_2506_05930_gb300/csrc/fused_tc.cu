// Fused tensor-core shading kernel (placeholder until the tcgen05 path lands).
#include "nvc_internal.cuh"

namespace nvc {

size_t mlp_packed_bytes(const nvc_handle*) { return 0; }

cudaError_t launch_pack_mlp(nvc_handle*, cudaStream_t) { return cudaSuccess; }

bool fused_supported(const nvc_handle*, std::string* why) {
  *why = "fused tensor-core kernel not available";
  return false;
}

cudaError_t launch_shade_fused(const nvc_handle*, const nvc_scene*, const float*, const float*,
                               int64_t, uint64_t, uint32_t, uint32_t, int64_t, int32_t*, float*,
                               float*, float*, float*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace nvc
