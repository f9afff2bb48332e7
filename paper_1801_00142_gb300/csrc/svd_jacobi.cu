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
// 1e-10 .. 1e-15 below the leading singular value).
//
// GPU mapping: one persistent cooperative kernel per split.  Each round of
// the round-robin ordering rotates disjoint column pairs, one warp per pair
// (shuffle reductions, no block barriers); rounds are separated by a grid
// barrier whose wait is bounded (on expiry the kernel records a timeout and
// every CTA leaves).  Convergence, the column norms, the selection of the
// kept singular values and the emission of the two factors all happen inside
// the same launch, so the host synchronises once per split to read k.
#include <math.h>

#include "common.cuh"

namespace {

constexpr int WPB = 4;                  // warps per CTA
constexpr int NT = WPB * 32;
constexpr long long SPIN_LIMIT = 1LL << 22;

struct SvdArgs {
  const double* M;
  int m, n, trans, len, ncols, nn, kcap, mode, max_sweeps;
  double tol, rel_tol;
  double *W, *V, *sig;
  int* perm;
  double *left, *right;
  unsigned* bar;      // [0] arrivals, [1] generation
  int* rot;           // [3] rotations per sweep (ring)
  int* out;           // [0] k, [1] rank, [2] sweeps, [3] status (0 ok, 1 timeout, 2 not converged)
  double* stats;      // [0] total weight, [1] discarded fraction, [2] sigma_max,
                      // [3] ||M||_F^2 (accumulated while loading)
  // device-decided mode (all null otherwise): run only if *run_if > thresh
  // or is not finite; keep exactly min(kcap, ncols); report into acc
  const double* run_if;
  double thresh;
  SvdDeviceAcc acc;
};

// Grid barrier with a bounded wait.  Returns false if the wait expired or
// another CTA already recorded a timeout (then every CTA returns).
__device__ bool grid_barrier(const SvdArgs& a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vb = a.bar;
    volatile int* st = a.out + 3;
    if (*st == 1) {
      ok = 0;
    } else {
      unsigned gen = vb[1];
      __threadfence();
      unsigned arrived = atomicAdd(a.bar, 1u);
      if (arrived == gridDim.x - 1) {
        vb[0] = 0;
        __threadfence();
        atomicAdd(a.bar + 1, 1u);
      } else {
        long long it = 0;
        while (vb[1] == gen) {
          if (++it > SPIN_LIMIT || *st == 1) {
            atomicExch(a.out + 3, 1);
            if (a.acc.status) atomicMax(a.acc.status, 1);
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
  return ok != 0;
}

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(NT) svd_persistent(SvdArgs a) {
  // device-decided mode: every CTA leaves before the first barrier
  if (a.run_if && *a.run_if <= a.thresh) return;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * WPB + (threadIdx.x >> 5);
  const int TW = gridDim.x * WPB;
  const long long gt = blockIdx.x * (long long)NT + threadIdx.x;
  const long long GT = (long long)gridDim.x * NT;

  // load: column j of M (trans = 0) or of M^T (trans = 1); V = I
  const long long tot = (long long)a.len * a.ncols;
  double ss = 0.0;
  for (long long e = gt; e < tot; e += GT) {
    int j = (int)(e / a.len), i = (int)(e % a.len);
    const double x = a.trans ? a.M[(long long)j * a.n + i] : a.M[(long long)i * a.n + j];
    a.W[e] = x;
    ss = fma(x, x, ss);
  }
  ss = warp_sum(ss);
  if (lane == 0) atomicAdd(a.stats + 3, ss);
  for (long long e = gt; e < (long long)a.ncols * a.ncols; e += GT) {
    int j = (int)(e / a.ncols), i = (int)(e % a.ncols);
    a.V[e] = (i == j) ? 1.0 : 0.0;
  }
  if (gt < 3) a.rot[gt] = 0;
  if (!grid_barrier(a)) return;
  // Gram entries below eps^2 ||M||_F^2 are beneath the resolution of the
  // whole problem: pairs of numerically-zero columns are not rotated (without
  // this floor, columns of pure rounding noise can rotate without end)
  const double gfloor = 4.930380657631324e-32 * ((volatile double*)a.stats)[3];

  const int mod = a.nn - 1;
  const int npairs = a.nn / 2;
  int sweeps = 0;
  bool converged = a.ncols < 2;
  for (int s = 0; s < a.max_sweeps && !converged; ++s) {
    if (gt == 0) a.rot[(s + 1) % 3] = 0;
    int myrot = 0;
    for (int r = 0; r < mod; ++r) {
      for (int i = gw; i < npairs; i += TW) {
        int p, q;
        if (i == 0) { p = r; q = a.nn - 1; }
        else { p = (r + i) % mod; q = (r - i + mod) % mod; }
        if (p > q) { int t = p; p = q; q = t; }
        if (q >= a.ncols) continue;
        double* wp = a.W + (long long)p * a.len;
        double* wq = a.W + (long long)q * a.len;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int e = lane; e < a.len; e += 32) {
          double x = wp[e], y = wq[e];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (!(fabs(ga) > a.tol * sqrt(al) * sqrt(be)) || !(fabs(ga) > gfloor) || al == 0.0 ||
            be == 0.0)
          continue;
        // rotation zeroing the (p, q) Gram entry: t = sign(z)/(|z| + sqrt(1+z^2))
        double z = (be - al) / (2.0 * ga);
        double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + hypot(1.0, z));
        double c = 1.0 / sqrt(1.0 + t * t);
        double sn = c * t;
        for (int e = lane; e < a.len; e += 32) {
          double x = wp[e], y = wq[e];
          wp[e] = c * x - sn * y;
          wq[e] = sn * x + c * y;
        }
        double* vp = a.V + (long long)p * a.ncols;
        double* vq = a.V + (long long)q * a.ncols;
        for (int e = lane; e < a.ncols; e += 32) {
          double x = vp[e], y = vq[e];
          vp[e] = c * x - sn * y;
          vq[e] = sn * x + c * y;
        }
        ++myrot;
      }
      if (!grid_barrier(a)) return;
    }
    if (lane == 0 && myrot) atomicAdd(a.rot + (s % 3), myrot);
    if (!grid_barrier(a)) return;
    sweeps = s + 1;
    converged = ((volatile int*)a.rot)[s % 3] == 0;
  }

  // column norms = singular values
  for (int j = gw; j < a.ncols; j += TW) {
    const double* w = a.W + (long long)j * a.len;
    double s2 = 0.0;
    for (int e = lane; e < a.len; e += 32) s2 = fma(w[e], w[e], s2);
    s2 = warp_sum(s2);
    if (lane == 0) a.sig[j] = sqrt(s2);
  }
  if (!grid_barrier(a)) return;

  // rank the singular values (descending; ties by column index; non-negative
  // doubles order like their bit patterns) and select k
  for (int j = (int)gt; j < a.ncols; j += (int)GT) {
    long long bj = __double_as_longlong(a.sig[j]);
    int rk = 0;
    for (int i = 0; i < a.ncols; ++i) {
      long long bi = __double_as_longlong(a.sig[i]);
      rk += (bi > bj) || (bi == bj && i < j);
    }
    a.perm[rk] = j;
  }
  if (!grid_barrier(a)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double mx = 0.0, totw = 0.0;
    for (int j = 0; j < a.ncols; ++j) { mx = fmax(mx, a.sig[j]); totw += a.sig[j] * a.sig[j]; }
    int cnt = 0;
    for (int j = 0; j < a.ncols; ++j) cnt += a.sig[j] > a.rel_tol * mx;
    int k = cnt < a.kcap ? cnt : a.kcap;
    if (a.run_if) k = a.kcap < a.ncols ? a.kcap : a.ncols;
    if (k < 1) k = 1;
    double keptw = 0.0;
    for (int r = 0; r < k; ++r) { double s = a.sig[a.perm[r]]; keptw += s * s; }
    a.out[0] = k;
    a.out[1] = cnt;
    a.out[2] = sweeps;
    if (!converged) a.out[3] = 2;
    a.stats[0] = totw;
    a.stats[1] = totw > 0.0 ? fmax(0.0, (totw - keptw) / totw) : 0.0;
    a.stats[2] = mx;
    if (a.run_if) {
      if (a.acc.disc_max)
        atomicMax(reinterpret_cast<unsigned long long*>(a.acc.disc_max),
                  (unsigned long long)__double_as_longlong(a.stats[1]));
      if (a.acc.runs) atomicAdd(a.acc.runs, 1ull);
      if (a.acc.status && !converged) atomicMax(a.acc.status, 2);
      if (a.acc.status && !isfinite(mx)) atomicMax(a.acc.status, 3);
    }
  }
  if (!grid_barrier(a)) return;

  // emit Left (m x k) and Right (k x n).
  // trans = 0: W = M V = U Sigma (len = m), V holds V.
  // trans = 1: W = M^T V' = V Sigma (len = n), V' holds U.
  const int k = ((volatile int*)a.out)[0];
  const long long nl = (long long)a.m * k, nr = (long long)k * a.n;
  for (long long e = gt; e < nl + nr; e += GT) {
    bool isleft = e < nl;
    int r, x;
    if (isleft) { x = (int)(e / k); r = (int)(e % k); }
    else { r = (int)((e - nl) / a.n); x = (int)((e - nl) % a.n); }
    int j = a.perm[r];
    double s = a.sig[j];
    bool fromW = isleft ? (a.trans == 0) : (a.trans == 1);   // W holds Sigma-scaled vectors
    double base = fromW ? a.W[(long long)j * a.len + x] : a.V[(long long)j * a.ncols + x];
    bool want_sigma = isleft ? (a.mode == SPLIT_LEFT) : (a.mode == SPLIT_RIGHT);
    double v;
    if (want_sigma == fromW) v = base;
    else if (want_sigma) v = base * s;
    else v = (s > 0.0) ? base / s : 0.0;
    if (isleft) a.left[(long long)x * k + r] = v;
    else a.right[(long long)r * a.n + x] = v;
  }
}

// CTAs of the cooperative launch (once per device, thread-safe)
struct SvdSetup {
  cudaError_t err;
  int max_ctas;
};
PerDevice<SvdSetup> g_svd_setup;

SvdSetup svd_setup() {
  SvdSetup s{cudaSuccess, 0};
  cudaError_t e = g_svd_setup.get(
      [](int dev) {
        SvdSetup r{cudaSuccess, 0};
        int sms = 0, per = 0;
        r.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (r.err == cudaSuccess)
          r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, svd_persistent, NT, 0);
        r.max_ctas = sms * (per < 2 ? per : 2);
        if (r.err == cudaSuccess && r.max_ctas < 1) r.err = cudaErrorLaunchOutOfResources;
        return r;
      },
      &s);
  if (e != cudaSuccess) s.err = e;
  return s;
}

cudaError_t svd_launch(const double* M, int m, int n, int kcap, double rel_tol, SplitMode mode,
                       double* left, double* right, const SvdBuffers& buf, cudaStream_t st,
                       const double* run_if, double thresh, const SvdDeviceAcc& acc) {
  const int trans = (m < n) ? 1 : 0;
  const int len = trans ? n : m;
  const int ncols = trans ? m : n;
  if ((size_t)len * ncols > buf.max_elems || (size_t)ncols * ncols > buf.max_elems ||
      ncols > buf.max_cols)
    return cudaErrorInvalidValue;
  cudaError_t e;
  const SvdSetup setup = svd_setup();
  if (setup.err != cudaSuccess) return setup.err;
  const int max_ctas = setup.max_ctas;
  SvdArgs a;
  a.M = M; a.m = m; a.n = n; a.trans = trans; a.len = len; a.ncols = ncols;
  a.nn = ncols + (ncols & 1);
  a.kcap = kcap; a.mode = (int)mode; a.max_sweeps = 60;
  a.tol = sqrt((double)len) * 2.220446049250313e-16;
  a.rel_tol = rel_tol;
  a.W = buf.W; a.V = buf.V; a.sig = buf.sig; a.perm = buf.perm;
  a.left = left; a.right = right;
  a.bar = (unsigned*)buf.counter;      // 2 words
  a.rot = buf.counter + 2;             // 3 words
  a.out = buf.kept;                    // 4 words
  a.stats = buf.stats;
  a.run_if = run_if;
  a.thresh = thresh;
  a.acc = acc;
  if ((e = cudaMemsetAsync(buf.counter, 0, 8 * sizeof(int), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(buf.kept, 0, 4 * sizeof(int), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(buf.stats, 0, 4 * sizeof(double), st)) != cudaSuccess) return e;
  int pairs = a.nn / 2;
  int grid = (pairs + WPB - 1) / WPB;
  long long work = (long long)len * ncols / (NT * 8);
  if (work > grid) grid = (int)work;
  if (grid > max_ctas) grid = max_ctas;
  if (grid < 1) grid = 1;
  void* args[] = {&a};
  note_launch();
  return cudaLaunchCooperativeKernel((void*)svd_persistent, dim3(grid), dim3(NT), args, 0, st);
}

}  // namespace

cudaError_t svd_split_f64_if(const double* M, int m, int n, int kcap, SplitMode mode,
                             double* left, double* right, const SvdBuffers& buf, cudaStream_t st,
                             const double* run_if, double thresh, const SvdDeviceAcc& acc) {
  if (!run_if) return cudaErrorInvalidValue;
  return svd_launch(M, m, n, kcap, 0.0, mode, left, right, buf, st, run_if, thresh, acc);
}

cudaError_t svd_split_f64(const double* M, int m, int n, int kcap, double rel_tol, SplitMode mode,
                          double* left, double* right, const SvdBuffers& buf, cudaStream_t st,
                          SvdResult* res, bool* converged) {
  *converged = true;
  cudaError_t e = svd_launch(M, m, n, kcap, rel_tol, mode, left, right, buf, st, nullptr, 0.0,
                             SvdDeviceAcc{nullptr, nullptr, nullptr});
  if (e != cudaSuccess) return e;
  int out[4];
  double stats[3];
  if ((e = cudaMemcpyAsync(out, buf.kept, sizeof out, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(stats, buf.stats, sizeof stats, cudaMemcpyDeviceToHost, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  if (out[3] == 1) return cudaErrorLaunchTimeout;
  if (out[3] == 2) *converged = false;
  res->k = out[0];
  res->rank = out[1];
  res->sweeps = out[2];
  res->discarded = stats[1];
  res->sigma_max = stats[2];
  return cudaSuccess;
}
