// FP64 one-sided (Hestenes) Jacobi SVD and the two-site split of Fig. VMPO(d).
//
// The generalised overlap C_E (Eq. LSEProd) is factorised C_E = U Lambda V^T
// and truncated by *number*: the largest min(D*, numerical rank) singular
// values are kept (Sec. II D: truncation by discarded weight is avoided; only
// singular values at or below rel_tol * sigma_max, i.e. numerically zero, are
// dropped).  Left-to-right the left factor is U and the right factor
// Lambda V^T; right-to-left Lambda goes with U (App. D.1).
//
// One-sided Jacobi orthogonalises the min(m, n) columns of M (or of M^T) by
// plane rotations; it resolves small singular values to high relative
// accuracy, which the series initialisation needs (its higher-order terms sit
// 1e-10 .. 1e-15 below the leading singular value).  The rotations of one
// round of the round-robin ordering act on disjoint column pairs and run as
// one CTA per pair.
#include <math.h>

#include "common.cuh"

namespace {

constexpr int RT = 256;

__global__ void svd_load_kernel(const double* __restrict__ M, int m, int n, int trans,
                                double* __restrict__ W, double* __restrict__ V, int len,
                                int ncols) {
  long long total = (long long)len * ncols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int j = (int)(e / len), i = (int)(e % len);
    // column j of M (trans = 0, len = m) or of M^T (trans = 1, len = n)
    W[e] = trans ? M[(long long)j * n + i] : M[(long long)i * n + j];
  }
  long long vt = (long long)ncols * ncols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < vt;
       e += (long long)gridDim.x * blockDim.x) {
    int j = (int)(e / ncols), i = (int)(e % ncols);
    V[e] = (i == j) ? 1.0 : 0.0;
  }
}

__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += red[i];
  return s;
}

__global__ void __launch_bounds__(RT) svd_round_kernel(double* __restrict__ W, double* __restrict__ V,
                                                       int len, int ncols, int nn, int round,
                                                       double tol, int* counter) {
  __shared__ double red[3][RT / 32];
  const int i = blockIdx.x;
  const int mod = nn - 1;
  int p, q;
  if (i == 0) {
    p = round;
    q = nn - 1;
  } else {
    p = (round + i) % mod;
    q = (round - i + mod) % mod;
  }
  if (p > q) { int t = p; p = q; q = t; }
  if (q >= ncols) return;  // the padding column of an odd count
  double* wp = W + (long long)p * len;
  double* wq = W + (long long)q * len;
  double a = 0.0, b = 0.0, g = 0.0;
  for (int e = threadIdx.x; e < len; e += RT) {
    double x = wp[e], y = wq[e];
    a = fma(x, x, a);
    b = fma(y, y, b);
    g = fma(x, y, g);
  }
  a = block_sum(a, red[0]);
  b = block_sum(b, red[1]);
  g = block_sum(g, red[2]);
  if (!(fabs(g) > tol * sqrt(a) * sqrt(b)) || a == 0.0 || b == 0.0) return;
  // rotation zeroing the (p, q) Gram entry: tan = sign(z)/(|z| + sqrt(1+z^2))
  double z = (b - a) / (2.0 * g);
  double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + hypot(1.0, z));
  double c = 1.0 / sqrt(1.0 + t * t);
  double s = c * t;
  for (int e = threadIdx.x; e < len; e += RT) {
    double x = wp[e], y = wq[e];
    wp[e] = c * x - s * y;
    wq[e] = s * x + c * y;
  }
  double* vp = V + (long long)p * ncols;
  double* vq = V + (long long)q * ncols;
  for (int e = threadIdx.x; e < ncols; e += RT) {
    double x = vp[e], y = vq[e];
    vp[e] = c * x - s * y;
    vq[e] = s * x + c * y;
  }
  if (threadIdx.x == 0) atomicAdd(counter, 1);
}

__global__ void svd_colnorm_kernel(const double* __restrict__ W, int len, double* __restrict__ sig) {
  __shared__ double red[RT / 32];
  const double* w = W + (long long)blockIdx.x * len;
  double a = 0.0;
  for (int e = threadIdx.x; e < len; e += RT) a = fma(w[e], w[e], a);
  a = block_sum(a, red);
  if (threadIdx.x == 0) sig[blockIdx.x] = sqrt(a);
}

// One CTA: rank the singular values (descending, ties by column index),
// choose k = max(1, min(kcap, #{sigma > rel_tol * sigma_max})) and the
// discarded weight.  Non-negative doubles order like their bit patterns.
__global__ void svd_select_kernel(const double* __restrict__ sig, int ncols, int kcap,
                                  double rel_tol, int* __restrict__ perm, int* __restrict__ kept,
                                  double* __restrict__ stats) {
  __shared__ double smax, stot;
  __shared__ int scount;
  if (threadIdx.x == 0) { smax = 0.0; stot = 0.0; scount = 0; }
  __syncthreads();
  for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
    long long bj = __double_as_longlong(sig[j]);
    int r = 0;
    for (int i = 0; i < ncols; ++i) {
      long long bi = __double_as_longlong(sig[i]);
      r += (bi > bj) || (bi == bj && i < j);
    }
    perm[r] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0, tot = 0.0;
    for (int j = 0; j < ncols; ++j) { mx = fmax(mx, sig[j]); tot += sig[j] * sig[j]; }
    smax = mx;
    stot = tot;
  }
  __syncthreads();
  int cnt = 0;
  for (int j = threadIdx.x; j < ncols; j += blockDim.x) cnt += sig[j] > rel_tol * smax;
  atomicAdd(&scount, cnt);
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = scount;
    if (k > kcap) k = kcap;
    if (k < 1) k = 1;
    double keptw = 0.0;
    for (int r = 0; r < k; ++r) { double s = sig[perm[r]]; keptw += s * s; }
    *kept = k;
    stats[0] = stot;
    stats[1] = stot > 0.0 ? fmax(0.0, (stot - keptw) / stot) : 0.0;
    stats[2] = smax;
    stats[3] = (double)scount;
  }
}

// Left (m x k) and Right (k x n) factors from the converged rotation.
// trans = 0: W = M V = U Sigma (len = m), V holds V.
// trans = 1: W = M^T V' = V Sigma (len = n), V' holds U.
__global__ void svd_emit_kernel(const double* __restrict__ W, const double* __restrict__ V,
                                const double* __restrict__ sig, const int* __restrict__ perm,
                                int k, int len, int ncols, int m, int n, int trans, int mode,
                                double* __restrict__ left, double* __restrict__ right) {
  long long nl = (long long)m * k, nr = (long long)k * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nl + nr;
       e += (long long)gridDim.x * blockDim.x) {
    bool isleft = e < nl;
    int r, x;
    if (isleft) { x = (int)(e / k); r = (int)(e % k); }
    else { r = (int)((e - nl) / n); x = (int)((e - nl) % n); }
    int j = perm[r];
    double s = sig[j];
    // is the stored column the Sigma-scaled vector (W) or a unit vector (V)?
    bool fromW = isleft ? (trans == 0) : (trans == 1);
    double base = fromW ? W[(long long)j * len + x] : V[(long long)j * ncols + x];
    bool want_sigma = isleft ? (mode == SPLIT_LEFT) : (mode == SPLIT_RIGHT);
    double v;
    if (want_sigma == fromW) v = base;
    else if (want_sigma) v = base * s;
    else v = (s > 0.0) ? base / s : 0.0;
    if (isleft) left[(long long)x * k + r] = v;
    else right[(long long)r * n + x] = v;
  }
}

inline int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t svd_split_f64(const double* M, int m, int n, int kcap, double rel_tol, SplitMode mode,
                          double* left, double* right, const SvdBuffers& buf, cudaStream_t st,
                          SvdResult* res, bool* converged) {
  const int trans = (m < n) ? 1 : 0;
  const int len = trans ? n : m;
  const int ncols = trans ? m : n;
  *converged = true;
  if ((size_t)len * ncols > buf.max_elems || (size_t)ncols * ncols > buf.max_elems ||
      ncols > buf.max_cols)
    return cudaErrorInvalidValue;
  cudaError_t e;
  svd_load_kernel<<<grid_for((long long)len * ncols), 256, 0, st>>>(M, m, n, trans, buf.W, buf.V,
                                                                   len, ncols);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nn = ncols + (ncols & 1);
  const double tol = sqrt((double)len) * 2.220446049250313e-16;
  const int max_sweeps = 60;
  int sweeps = 0;
  if (ncols > 1) {
    for (; sweeps < max_sweeps; ++sweeps) {
      if ((e = cudaMemsetAsync(buf.counter, 0, sizeof(int), st)) != cudaSuccess) return e;
      for (int r = 0; r < nn - 1; ++r) {
        svd_round_kernel<<<nn / 2, RT, 0, st>>>(buf.W, buf.V, len, ncols, nn, r, tol, buf.counter);
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      int h = 0;
      if ((e = cudaMemcpyAsync(&h, buf.counter, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      if (h == 0) { ++sweeps; break; }
    }
    if (sweeps >= max_sweeps) *converged = false;
  }
  svd_colnorm_kernel<<<ncols, RT, 0, st>>>(buf.W, len, buf.sig);
  svd_select_kernel<<<1, 1024, 0, st>>>(buf.sig, ncols, kcap, rel_tol, buf.perm, buf.kept,
                                        buf.stats);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int k = 0;
  double stats[4];
  if ((e = cudaMemcpyAsync(&k, buf.kept, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(stats, buf.stats, 4 * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  svd_emit_kernel<<<grid_for((long long)(m + n) * k), 256, 0, st>>>(
      buf.W, buf.V, buf.sig, buf.perm, k, len, ncols, m, n, trans, (int)mode, left, right);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  res->k = k;
  res->sweeps = sweeps;
  res->discarded = stats[1];
  res->sigma_max = stats[2];
  res->rank = (int)stats[3];
  return cudaSuccess;
}
