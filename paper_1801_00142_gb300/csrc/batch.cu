// Many independent XTRG runs on one GPU (see xtrg_batch_run in xtrg.h).
//
// The instances of a batch are independent problems: interleaved tau0 grids
// of one Hamiltonian (Eq. zshift) or different (L, Delta, D*) chains.  One
// instance alone leaves most of the GPU idle at small bonds and waits on the
// host at every truncation, so several run at once: the caller's workspace is
// cut into equal slots, each driven by a host thread with its own stream, and
// the threads take instances from a shared queue (largest first, so the
// uneven sizes balance).  Results are written to the caller's host array.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "xtrg.h"

namespace {

std::mutex g_batch_mu;
std::string g_batch_err;

void set_batch_error(const std::string& s) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  g_batch_err = s;
}

constexpr size_t kAlign = 256;
inline size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

__attribute__((visibility("hidden"))) const char* xtrg_batch_last_error() {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  return g_batch_err.c_str();
}

extern "C" xtrg_status xtrg_batch_plan(int n, const xtrg_mpo* H, const xtrg_config* cfg,
                                       size_t workspace_bytes, int max_concurrent, int* n_slots,
                                       size_t* slot_bytes) {
  if (n < 1 || !H || !cfg || !n_slots || !slot_bytes) {
    set_batch_error("xtrg_batch_plan: bad arguments");
    return XTRG_EINVAL;
  }
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    const size_t b = xtrg_workspace_bytes(&H[i], &cfg[i]);
    if (b == 0) {
      set_batch_error("xtrg_batch_plan: instance " + std::to_string(i) +
                      " has a bad Hamiltonian or configuration");
      return XTRG_EINVAL;
    }
    need = std::max(need, round_up(b));
  }
  const int cap = max_concurrent > 0 ? max_concurrent : 8;
  const size_t fit = workspace_bytes / need;
  *slot_bytes = need;
  *n_slots = (int)std::min<size_t>(std::min<size_t>((size_t)n, (size_t)cap), fit);
  if (*n_slots < 1) {
    set_batch_error("xtrg_batch_plan: the workspace holds no instance (" +
                    std::to_string(need) + " bytes needed)");
    return XTRG_ENOMEM;
  }
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_batch_run(int n, const xtrg_mpo* H, const xtrg_config* cfg,
                                      const int* n_doublings, xtrg_obs* out, void* workspace,
                                      size_t workspace_bytes, int max_concurrent,
                                      void* cuda_stream) {
  if (!n_doublings || !out || !workspace || ((uintptr_t)workspace % kAlign) != 0) {
    set_batch_error("xtrg_batch_run: bad arguments (workspace must be 256-byte aligned)");
    return XTRG_EINVAL;
  }
  for (int i = 0; i < n; ++i)
    if (n_doublings[i] < 0) {
      set_batch_error("xtrg_batch_run: negative n_doublings");
      return XTRG_EINVAL;
    }
  int slots = 0;
  size_t slot_bytes = 0;
  xtrg_status st = xtrg_batch_plan(n, H, cfg, workspace_bytes, max_concurrent, &slots, &slot_bytes);
  if (st != XTRG_OK) return st;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) {
    set_batch_error(std::string("xtrg_batch_run: ") + cudaGetErrorString(ce));
    return XTRG_ECUDA;
  }
  cudaStream_t caller = (cudaStream_t)cuda_stream;
  cudaEvent_t start = nullptr;
  if ((ce = cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventRecord(start, caller)) != cudaSuccess) {
    set_batch_error(std::string("xtrg_batch_run: ") + cudaGetErrorString(ce));
    if (start) cudaEventDestroy(start);
    return XTRG_ECUDA;
  }
  // row offsets of each instance in out, and the order of the queue
  std::vector<long long> off(n + 1, 0);
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + n_doublings[i] + 1;
  std::vector<size_t> bytes(n);
  for (int i = 0; i < n; ++i) bytes[i] = xtrg_workspace_bytes(&H[i], &cfg[i]);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)bytes[a] * (n_doublings[a] + 1) > (long long)bytes[b] * (n_doublings[b] + 1);
  });
  std::atomic<int> next(0);
  std::atomic<int> failed(0);
  std::vector<xtrg_status> status(slots, XTRG_OK);
  std::vector<cudaEvent_t> done(slots, nullptr);
  auto worker = [&](int t) {
    cudaStream_t s = nullptr;
    auto fail = [&](xtrg_status code, const std::string& msg) {
      status[t] = code;
      failed.store(1);
      set_batch_error(msg);
    };
    cudaError_t e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, start, 0);
    if (e != cudaSuccess) {
      fail(XTRG_ECUDA, std::string("xtrg_batch_run: ") + cudaGetErrorString(e));
      if (s) cudaStreamDestroy(s);
      return;
    }
    char* base = (char*)workspace + (size_t)t * slot_bytes;
    while (!failed.load()) {
      const int q = next.fetch_add(1);
      if (q >= n) break;
      const int i = order[q];
      xtrg_ctx* ctx = nullptr;
      xtrg_status r = xtrg_create(&ctx, &H[i], &cfg[i], base, slot_bytes, s);
      if (r == XTRG_OK) r = xtrg_init(ctx);
      if (r == XTRG_OK) r = xtrg_observables(ctx, &out[off[i]]);
      for (int d = 1; r == XTRG_OK && d <= n_doublings[i]; ++d) {
        r = xtrg_double(ctx);
        if (r == XTRG_OK) r = xtrg_observables(ctx, &out[off[i] + d]);
      }
      if (r != XTRG_OK)
        fail(r, "xtrg_batch_run: instance " + std::to_string(i) + ": " +
                    (ctx ? xtrg_last_error(ctx) : "context creation failed"));
      if (ctx) xtrg_destroy(ctx);
    }
    if (cudaEventCreateWithFlags(&done[t], cudaEventDisableTiming) == cudaSuccess)
      cudaEventRecord(done[t], s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < slots; ++t) pool.emplace_back(worker, t);
  for (auto& th : pool) th.join();
  // the caller's stream is ordered after every instance's work
  for (int t = 0; t < slots; ++t)
    if (done[t]) {
      cudaStreamWaitEvent(caller, done[t], 0);
      cudaEventDestroy(done[t]);
    }
  cudaEventDestroy(start);
  for (int t = 0; t < slots; ++t)
    if (status[t] != XTRG_OK) return status[t];
  return XTRG_OK;
}
