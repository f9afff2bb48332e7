// Internal declarations shared by the XTRG CUDA sources (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

// Number of kernels this library has launched (all contexts, all streams);
// every launch site calls note_launch().
extern unsigned long long g_xtrg_launches;
// launches made by the calling host thread (a graph capture's own count)
extern thread_local unsigned long long t_xtrg_launches;
static inline void note_launch() {
  __atomic_add_fetch(&g_xtrg_launches, 1ull, __ATOMIC_RELAXED);
  ++t_xtrg_launches;
}

// One-time set-up per device (kernel attributes, SM counts, occupancy): the
// first call on a device runs make(dev) with that device current and keeps
// its result; later calls on the same device return the kept value.  Safe to
// call from several host threads.  Function attributes set by cudaFuncSetAttribute
// belong to the device that was current, so they must be set once on each.
constexpr int XTRG_MAX_DEVICES = 64;
template <typename T>
struct PerDevice {
  std::once_flag once[XTRG_MAX_DEVICES];
  T val[XTRG_MAX_DEVICES];
  template <typename F>
  cudaError_t get(F make, T* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= XTRG_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&]() { val[dev] = make(dev); });
    *out = val[dev];
    return cudaSuccess;
  }
};

// A strided view of one GEMM index.  The index idx in [0, n2*n1*n0) is split
// as idx = (i2*n1 + i1)*n0 + i0 and lands at element offset
// i2*s2 + i1*s1 + i0*s0.  A plain stride s is {1, 1, s, 0, 0}.
struct Idx3 {
  int n1, n0;
  long long s2, s1, s0;
};

static inline Idx3 idx_plain(long long s) { return Idx3{1, 1, s, 0, 0}; }
// idx = i2*n0 + i0
static inline Idx3 idx_split2(int n0, long long s_outer, long long s_inner) {
  return Idx3{1, n0, s_outer, 0, s_inner};
}
// idx = (i2*n1 + i1)*n0 + i0
static inline Idx3 idx_split3(int n1, int n0, long long s2, long long s1, long long s0) {
  return Idx3{n1, n0, s2, s1, s0};
}

__host__ __device__ inline long long idx_off(const Idx3& d, long long idx) {
  long long i0 = idx % d.n0;
  long long t = idx / d.n0;
  long long i1 = t % d.n1;
  long long i2 = t / d.n1;
  return i2 * d.s2 + i1 * d.s1 + i0 * d.s0;
}

// C[b](m, n) = alpha * sum_k A[b](m, k) * B[b](k, n) + beta * C[b](m, n)
// with A[b](m, k) at A + b*sab + off(am, m) + off(ak, k), and likewise for B, C.
struct GemmF64 {
  int M, N, K, batch;
  const double* A; Idx3 am, ak; long long sab;
  const double* B; Idx3 bk, bn; long long sbb;
  double* C; Idx3 cm, cn; long long scb;
  double alpha, beta;
};

cudaError_t gemm_f64(const GemmF64& g, cudaStream_t st);


// ---------------------------------------------------------------- SVD split
// One-sided (Hestenes) Jacobi SVD of a row-major m x n matrix M in FP64,
// with selection of the largest singular values.  See svd_jacobi.cu.
struct SvdBuffers {
  double* W;       // len x ncols, column j contiguous
  double* V;       // ncols x ncols, column j contiguous
  double* sig;     // ncols
  int* perm;       // ncols: perm[r] = column with the r-th largest sigma
  int* counter;    // rotations in the current sweep
  double* stats;   // [0] = total weight, [1] = discarded fraction, [2] = sigma_max, [3] = rank
  int* kept;       // number kept
  size_t max_elems;   // capacity of W and of V in doubles
  int max_cols;
};

// Mode of the two output factors: M ~= Left * Right with Left m x k and Right
// k x n.  SPLIT_RIGHT: Left = U, Right = Sigma V^T (left-to-right sweep).
// SPLIT_LEFT: Left = U Sigma, Right = V^T (right-to-left sweep).
enum SplitMode { SPLIT_RIGHT = 0, SPLIT_LEFT = 1 };

struct SvdResult {
  int k;              // kept singular values
  int rank;           // singular values above rel_tol * sigma_max (before the cap)
  int sweeps;         // Jacobi sweeps used
  double discarded;   // discarded weight / total weight
  double sigma_max;
};

// Returns cudaSuccess or an error; *converged is false if the sweep limit was hit.
cudaError_t svd_split_f64(const double* M, int m, int n, int kcap, double rel_tol,
                          SplitMode mode, double* left, double* right,
                          const SvdBuffers& buf, cudaStream_t st, SvdResult* res,
                          bool* converged);

// The same split decided on the device, with no host read: the kernel runs
// only if *run_if > thresh (or *run_if is not finite) and keeps exactly
// min(kcap, m, n) columns (numerically zero ones included, as zero columns
// of the orthonormal factor).  It then raises acc->disc_max to its
// discarded weight (non-negative doubles, compared by bit pattern), counts
// itself in acc->runs and records a timeout (1) or a sweep limit (2) in
// acc->status (maximum).  Buffers of acc are device memory.
struct SvdDeviceAcc {
  double* disc_max;
  unsigned long long* runs;
  int* status;
};
cudaError_t svd_split_f64_if(const double* M, int m, int n, int kcap, SplitMode mode,
                             double* left, double* right, const SvdBuffers& buf, cudaStream_t st,
                             const double* run_if, double thresh, const SvdDeviceAcc& acc);

// ---------------------------------------------------------------- MPO kernels
cudaError_t mpo_exact_product(const double* A, int la, int ra, const double* B, int lb, int rb,
                              double* G, cudaStream_t st);
cudaError_t mpo_direct_sum_site(const double* P, int pl, int pr, double alpha, const double* Q,
                                int ql, int qr, int pos, int L, double* out, cudaStream_t st);
cudaError_t dev_fill(double* p, double v, long long n, cudaStream_t st);
cudaError_t dev_scale(double* p, double v, long long n, cudaStream_t st);
cudaError_t dev_sumsq(const double* p, long long n, double* out, cudaStream_t st);
// p *= 1 / sqrt(*ss) (ss: device scalar), unless *ss is not positive and finite
cudaError_t dev_scale_rsqrt(double* p, const double* ss, long long n, cudaStream_t st);
cudaError_t dev_identity_site(double* p, cudaStream_t st);
