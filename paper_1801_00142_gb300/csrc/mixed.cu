// Tensor-core contraction path (placeholder until the tcgen05 kernels land):
// creating a context with a tensor-core precision fails loudly.
#include "mixed.cuh"

struct MixedCtx { int unused; };

size_t mixed_workspace_bytes(int, int, int) { return 256; }
cudaError_t mixed_create(MixedCtx** out, char*, size_t, int, int, int) {
  *out = nullptr;
  return cudaErrorNotSupported;
}
cudaError_t mixed_prepare(MixedCtx*, const int*, double* const*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t mixed_gemm(MixedCtx*, const GemmF64&, cudaStream_t) { return cudaErrorNotSupported; }
void mixed_destroy(MixedCtx*) {}
