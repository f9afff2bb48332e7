// xtrg_tc_gemm_static: the tensor-core contraction primitive for callers that
// cannot allocate device memory.
//
// xtrg_tc_gemm needs device scratch for the BF16 planes of its operands and
// for the FP32 partial sums, which its caller passes in as a workspace.  Some
// callers have no way to provide one: code running inside a framework or a
// plugin that owns every device allocation and exposes no allocator, and
// small tools that must not grow the device footprint per call.  This entry
// point takes only the inputs and the output and places all of its scratch in
// one file-scope device array of fixed size (XTRG_TC_STATIC_SCRATCH_BYTES),
// which every GPU that loads this library holds until the process exits.
//
// The host cannot use the array's name as a device address (in host code it
// names a host-side shadow), so the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on it; that first call should therefore come before any stream
// capture.  All calls share the one array: the error flag is cleared on every
// call, everything else is overwritten before it is read, and calls whose
// work overlaps on the GPU (on different streams, or from different threads
// without ordering) race on it.  Like xtrg_tc_gemm, every call synchronises
// the stream it is given before returning.
#include "../../include/xtrg.h"
#include "common.cuh"
#include "tc_gemm_entry.cuh"

#define XTRG_TC_STATIC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_tc_static_scratch[XTRG_TC_STATIC_SCRATCH_BYTES];

namespace {

struct ScratchAddr {
  cudaError_t err;
  void* ptr;
};
PerDevice<ScratchAddr> g_scratch_addr;

// Device address of the static scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  ScratchAddr a{cudaSuccess, nullptr};
  cudaError_t e = g_scratch_addr.get(
      [](int) {
        ScratchAddr r{cudaSuccess, nullptr};
        r.err = cudaGetSymbolAddress(&r.ptr, g_tc_static_scratch);
        return r;
      },
      &a);
  if (e != cudaSuccess) return e;
  if (a.err != cudaSuccess) return a.err;
  *out = a.ptr;
  return cudaSuccess;
}

}  // namespace

extern "C" xtrg_status xtrg_tc_gemm_static(const double* A, const double* B, double* C, int M,
                                           int N, int K, int batch, int planes, int nprod,
                                           int splitk, void* stream) {
  const xtrg_status s = tc_gemm_check_args(A, B, C, M, N, K, batch, planes, nprod, splitk);
  if (s != XTRG_OK) return s;
  // the layout is the workspace variant's own, so the bound follows any change to it
  if (tc_gemm_scratch(M, N, K, batch, planes, splitk).total > XTRG_TC_STATIC_SCRATCH_BYTES)
    return XTRG_ENOMEM;
  char* base = nullptr;
  if (scratch_address((void**)&base) != cudaSuccess) return XTRG_ECUDA;
  return tc_gemm_run(A, B, C, M, N, K, batch, planes, nprod, splitk, base, (cudaStream_t)stream);
}
