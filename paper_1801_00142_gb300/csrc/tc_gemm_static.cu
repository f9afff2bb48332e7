// xtrg_tc_gemm_static: the tensor-core contraction primitive for callers that
// cannot allocate device memory.
//
// xtrg_tc_gemm needs device scratch for the BF16 planes of its operands and
// for the FP32 partial sums, which its caller passes in as a workspace.  Some
// callers have no way to provide one: code running inside a framework or a
// plugin that owns every device allocation and exposes no allocator, code
// inside a captured region or a callback where cudaMalloc is not allowed, and
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
// without ordering) race on it.
#include <cstring>
#include <mutex>

#include "../../include/xtrg.h"
#include "common.cuh"
#include "mixed_ops.cuh"
#include "tc_gemm.cuh"

#define XTRG_TC_STATIC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_tc_static_scratch[XTRG_TC_STATIC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the static scratch on the current device (set up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_tc_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" xtrg_status xtrg_tc_gemm_static(const double* A, const double* B, double* C, int M,
                                           int N, int K, int batch, int planes, int nprod,
                                           int splitk, void* stream) {
  if (!A || !B || !C) return XTRG_EINVAL;
  if (M < 1 || N < 1 || K < 1 || batch < 1 || planes < 2 || planes > 3 || splitk < 1)
    return XTRG_EINVAL;
  if (!(nprod == 1 || nprod == 3 || (nprod == 6 && planes == 3))) return XTRG_EINVAL;
  const long long ld = tc_ld(K);
  const size_t a_bytes = up256((size_t)planes * batch * M * ld * 2);
  const size_t b_bytes = up256((size_t)planes * batch * N * ld * 2);
  const size_t p_bytes = up256((size_t)splitk * batch * M * N * 4);
  if (a_bytes + b_bytes + p_bytes + 256 > XTRG_TC_STATIC_SCRATCH_BYTES) return XTRG_ENOMEM;
  char* base = nullptr;
  if (scratch_address((void**)&base) != cudaSuccess) return XTRG_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  __nv_bfloat16* pa = (__nv_bfloat16*)base;
  __nv_bfloat16* pb = (__nv_bfloat16*)(base + a_bytes);
  float* part = (float*)(base + a_bytes + b_bytes);
  int* err = (int*)(base + a_bytes + b_bytes + p_bytes);
  const long long psA = (long long)batch * M * ld, psB = (long long)batch * N * ld;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return XTRG_ECUDA;
  if (to_planes(A, idx_plain(K), idx_plain(1), (long long)M * K, M, K, batch, pa, ld,
                (long long)M * ld, planes, psA, st) != cudaSuccess)
    return XTRG_ECUDA;
  if (to_planes(B, idx_plain(K), idx_plain(1), (long long)N * K, N, K, batch, pb, ld,
                (long long)N * ld, planes, psB, st) != cudaSuccess)
    return XTRG_ECUDA;
  TcOperand oa{pa, planes, M, K, ld, (long long)M * ld, psA, batch};
  TcOperand ob{pb, planes, N, K, ld, (long long)N * ld, psB, batch};
  TcOutput out;
  memset(&out, 0, sizeof out);
  out.mode = TC_OUT_PARTIAL;
  out.f32 = part;
  out.alpha = 1.0;
  if (tc_gemm(oa, ob, M, N, K, batch, nprod, splitk, out, err, st) != cudaSuccess)
    return XTRG_ECUDA;
  if (reduce_partials(part, splitk, (long long)batch * M * N, C, st) != cudaSuccess)
    return XTRG_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return XTRG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return XTRG_ECUDA;
  return h ? XTRG_ETIMEOUT : XTRG_OK;
}
