// Truncation of the tensor-core path: one warm-started subspace step with
// block Gram-Schmidt orthonormalisation.
//
// The two-site update keeps the dominant rank-k subspace of C_E (Fig.
// VMPO(d)).  The FP64 path computes it exactly by Jacobi SVD; here, where
// C_E itself carries FP32-level errors, one step of subspace iteration from
// the previous sweep's basis is used instead: left-to-right,
//   Y = C_E V_prev (+ eta R),  U = orth(Y),  C_i = U,  C_{i+1} = U^T C_E,
// and mirrored right-to-left.  V_prev are the orthonormal rows of the current
// C_{i+1} (right-canonical guess, or V^T of the previous right-to-left pass),
// padded with pseudo-random columns when the bond grows.  The tiny random
// term eta R keeps every column of Y away from exact zero; directions it adds
// carry weight below eta^2 relative.
//
// orth() is first tried as a scaled CholeskyQR2 of the whole block (tensor-core
// Gram, one-CTA FP32 Cholesky, all-SM triangular solve; see below), which is
// exact in the subspace and fast when the columns, scaled to unit norm, are
// well conditioned, as they are once the warm start has converged.  When a
// pivot shows that they are not, the fallback is block classical
// Gram-Schmidt over panels of 32 columns: two FP32
// projection passes against the earlier panels, then CholeskyQR2 inside the
// panel with the 32 x 32 Gram and its Cholesky factor in FP64 (or, in the
// cluster kernel below, a double-float Gram and FP64 Cholesky).  Columns whose
// Cholesky pivot sits at the FP64 noise floor carry no weight and are set to
// zero instead of being divided by that pivot.  Up to 16 x 64 rows it runs in
// one thread-block cluster (orth_cluster); beyond that, or where such a
// cluster cannot be resident, as one persistent cooperative kernel: every
// CTA keeps its slab of rows in shared memory, reductions over rows go
// through per-CTA partials in global memory (summed in a fixed order, so
// results are deterministic), and phases are separated by bounded grid
// barriers.  The caller checks max |U^T U - I| over the live
// columns and takes the exact split when the FP32 projections lost
// orthogonality (steep, rank-deficient spectra).
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include <atomic>

#include "common.cuh"
#include "mixed_ops.cuh"
#include "subspace_split.cuh"
#include "tc_gemm.cuh"

namespace {

inline int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

// counter-based pseudo-random value in [-1, 1) (splitmix64 finaliser)
__device__ inline float hash_uniform(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

// Q[r][j] (rows x k) = src(j, r) for j < kold (src FP64 with strides), else
// pseudo-random.  src(j, r) = S[j*sj + r*sr].
__global__ void warm_start_kernel(const double* __restrict__ S, long long sj, long long sr,
                                  int kold, int rows, int k, unsigned long long seed0,
                                  const unsigned long long* __restrict__ base,
                                  float* __restrict__ Q) {
  const unsigned long long seed = seed0 ^ (*base * 0x9E3779B97F4A7C15ull);
  const long long total = (long long)rows * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / k), j = (int)(e % k);
    Q[e] = j < kold ? (float)S[j * sj + r * sr] : hash_uniform(seed * 0x100000001B3ull + e);
  }
}

// Y += eta R with eta = 1e-5 * rms(C_E), rms from ||C_E||^2 on the device
__global__ void add_noise_kernel(float* __restrict__ Y, long long n, const double* __restrict__ tot,
                                 double inv_mn, unsigned long long seed0,
                                 const unsigned long long* __restrict__ base) {
  const unsigned long long seed = seed0 ^ (*base * 0x9E3779B97F4A7C15ull);
  const float eta = (float)(1e-5 * sqrt(*tot * inv_mn));
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    Y[e] += eta * hash_uniform(seed ^ (0xD1B54A32D192ED03ull * (e + 1)));
}

__global__ void copy_f2d_kernel(const float* __restrict__ a, long long n, double* __restrict__ b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    b[e] = (double)a[e];
}

// out[c][r] = in[r][c] (rows x cols -> cols x rows), FP32 -> FP64
__global__ void transpose_f2d_kernel(const float* __restrict__ a, int rows, int cols,
                                     double* __restrict__ b) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / rows), r = (int)(e % rows);
    b[e] = (double)a[(long long)r * cols + c];
  }
}

// sum of squares in FP64 (grid-stride, one atomic per CTA)
__global__ void sumsq_f64_kernel(const double* __restrict__ a, long long n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    s = fma(a[e], a[e], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
    atomicAdd(out, t);
  }
}

constexpr int PANEL = 32;
constexpr int ORTH_NT = 256;
constexpr int ROWS_PER_CTA = 8;
constexpr int MAX_K = SUBSPACE_BLOCK_K;
constexpr long long ORTH_SPIN_LIMIT = 1LL << 22;

struct OrthArgs {
  float* Y;          // rows x k, row-major
  int rows, k;
  float* part;       // [G][MAX_K * PANEL] per-CTA partial sums
  float* red;        // [MAX_K * PANEL] reduced sums
  double* partd;     // [G][PANEL * PANEL] per-CTA partial Grams (FP64)
  double* redd;      // [PANEL * PANEL] reduced Gram (FP64)
  unsigned* bar;     // [0] arrivals, [1] generation
  int* status;       // 0 ok, 1 barrier timeout
  const int* run_if; // null, or run only if *run_if != 0 (the fast path broke down)
};

// grid barrier with a bounded wait (false: timed out, every CTA leaves)
__device__ bool orth_barrier(const OrthArgs& a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vb = a.bar;
    volatile int* stp = a.status;
    if (*stp) {
      ok = 0;
    } else {
      const unsigned gen = vb[1];
      __threadfence();
      const unsigned arrived = atomicAdd(a.bar, 1u);
      if (arrived == gridDim.x - 1) {
        vb[0] = 0;
        __threadfence();
        atomicAdd(a.bar + 1, 1u);
      } else {
        long long it = 0;
        while (vb[1] == gen) {
          if (++it > ORTH_SPIN_LIMIT || *stp) {
            atomicExch(a.status, 1);
            ok = 0;
            break;
          }
          if (it > 64) __nanosleep(32);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
  return ok != 0;
}

// Sum of the per-CTA partials of n entries into a.red (a.redd): each CTA
// takes chunks of 32 consecutive entries; its warps split the G partials
// (coalesced 128-byte rows), and a fixed-order sum over the warps in shared
// memory combines them, so the result is deterministic.  The loop bounds
// depend on blockIdx only, so every thread of a CTA takes the same branches
// through the __syncthreads().
// scratch: ORTH_NT values of T in shared memory (the caller's Ss, which is
// not live during a reduction)
template <typename T>
__device__ void reduce_partials_grid_t(const T* __restrict__ part, long long part_stride,
                                       T* __restrict__ red, int n, T* scratch) {
  T (*red_s)[32] = reinterpret_cast<T (*)[32]>(scratch);
  const int G = gridDim.x, lane = threadIdx.x % 32, w = threadIdx.x / 32;
  constexpr int NW = ORTH_NT / 32;
  for (int e0 = blockIdx.x * 32; e0 < n; e0 += gridDim.x * 32) {
    const int e = e0 + lane;
    T s = T(0);
    if (e < n) {
#pragma unroll 4
      for (int g = w; g < G; g += NW) s += part[(long long)g * part_stride + e];
    }
    red_s[w][lane] = s;
    __syncthreads();
    if (w == 0 && e < n) {
      T t = T(0);
#pragma unroll
      for (int q = 0; q < NW; ++q) t += red_s[q][lane];
      red[e] = t;
    }
    __syncthreads();
  }
}

__device__ void reduce_partials_grid(const OrthArgs& a, int n, float* scratch) {
  reduce_partials_grid_t<float>(a.part, (long long)MAX_K * PANEL, a.red, n, scratch);
}

__device__ void reduce_partials_grid_f64(const OrthArgs& a, int n, float* scratch) {
  reduce_partials_grid_t<double>(a.partd, (long long)PANEL * PANEL, a.redd, n,
                                 reinterpret_cast<double*>(scratch));
}

__global__ void __launch_bounds__(ORTH_NT) orth_persistent(OrthArgs a) {
  if (a.run_if) {
    if (*a.run_if == 0) return;   // every CTA leaves before any barrier
    // run_if[1] counts the orthonormalisations the fast path handed over
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(const_cast<int*>(a.run_if) + 1, 1);
  }
  __shared__ float Ys[ROWS_PER_CTA][MAX_K + 1];
  __shared__ __align__(16) float Ss[MAX_K * PANEL];
  __shared__ double Ld[PANEL][PANEL + 1];
  __shared__ double Linv[PANEL];   // reciprocals of the Cholesky pivots (0 for dead columns)
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * ROWS_PER_CTA;
  const int nr = min(ROWS_PER_CTA, a.rows - r0);
  const int k = a.k;
  float* mypart = a.part + (long long)blockIdx.x * MAX_K * PANEL;
  for (int e = tid; e < ROWS_PER_CTA * k; e += ORTH_NT) {
    const int r = e / k, c = e % k;
    Ys[r][c] = r < nr ? a.Y[(long long)(r0 + r) * k + c] : 0.f;
  }
  __syncthreads();
  for (int j0 = 0; j0 < k; j0 += PANEL) {
    const int w = min(PANEL, k - j0);
    // ---- two projection passes against columns [0, j0)
    for (int pass = 0; pass < 2 && j0 > 0; ++pass) {
      for (int e = tid; e < j0 * w; e += ORTH_NT) {
        const int j = e / w, c = e % w;
        float s = 0.f;
        for (int r = 0; r < nr; ++r) s = fmaf(Ys[r][j], Ys[r][j0 + c], s);
        mypart[e] = s;
      }
      if (!orth_barrier(a)) return;
      reduce_partials_grid(a, j0 * w, Ss);
      if (!orth_barrier(a)) return;
      for (int e = tid; e < j0 * w; e += ORTH_NT) Ss[e] = a.red[e];
      __syncthreads();
      for (int e = tid; e < nr * w; e += ORTH_NT) {
        const int r = e / w, c = e % w;
        float v = Ys[r][j0 + c];
        for (int j = 0; j < j0; ++j) v = fmaf(-Ys[r][j], Ss[j * w + c], v);
        Ys[r][j0 + c] = v;
      }
      // No grid barrier here: the next reduction writes a.red only after
      // the next phase's first barrier, which every CTA reaches after its
      // copy of a.red; and the partials are rewritten only after the barrier
      // that ended this reduction.  The CTA barrier orders this CTA's row
      // updates before the next phase reads them.
      __syncthreads();
    }
    // ---- CholeskyQR2 inside the panel with an FP64 Gram and Cholesky;
    // columns whose pivot is at the FP64 noise floor carry no weight and are
    // set to zero (dead) instead of being divided by that pivot
    for (int pass = 0; pass < 2; ++pass) {
      double* mypd = a.partd + (long long)blockIdx.x * PANEL * PANEL;
      for (int e = tid; e < w * w; e += ORTH_NT) {
        const int c = e / w, d = e % w;
        double s = 0.0;
        for (int r = 0; r < nr; ++r) s = fma((double)Ys[r][j0 + c], (double)Ys[r][j0 + d], s);
        mypd[e] = s;
      }
      if (!orth_barrier(a)) return;
      reduce_partials_grid_f64(a, w * w, Ss);
      if (!orth_barrier(a)) return;
      for (int e = tid; e < w * w; e += ORTH_NT) Ld[e / w][e % w] = a.redd[e];
      __syncthreads();
      if (tid < 32) {
        const int lane = tid;
        double dmax = 0.0;
        for (int c = 0; c < w; ++c) dmax = fmax(dmax, Ld[c][c]);
        const double thr = 1e-13 * dmax;
        for (int j = 0; j < w; ++j) {
          const double pj = Ld[j][j];
          const bool dead = !(pj > thr) || !(dmax > 0.0);
          // one FP64 square root and reciprocal per pivot (lane j), then
          // multiplications: FP64 division is a long instruction sequence
          if (lane == j) {
            const double d = dead ? 0.0 : sqrt(pj);
            Ld[j][j] = d;
            Linv[j] = dead ? 0.0 : 1.0 / d;
          }
          __syncwarp();
          if (lane > j && lane < w) Ld[lane][j] = Ld[lane][j] * Linv[j];
          __syncwarp();
          if (lane > j && lane < w)
            for (int c = j + 1; c <= lane; ++c) Ld[lane][c] -= Ld[lane][j] * Ld[c][j];
          __syncwarp();
        }
      }
      __syncthreads();
      // rows <- rows L^{-T} (dead columns -> 0)
      for (int r = tid; r < nr; r += ORTH_NT) {
        double x[PANEL];
        for (int c = 0; c < w; ++c) {
          double v = (double)Ys[r][j0 + c];
          for (int d = 0; d < c; ++d) v = fma(-x[d], Ld[c][d], v);
          x[c] = v * Linv[c];
        }
        for (int c = 0; c < w; ++c) Ys[r][j0 + c] = (float)x[c];
      }
      // (no grid barrier: the same argument as for the projection passes)
      __syncthreads();
    }
  }
  for (int e = tid; e < nr * k; e += ORTH_NT) {
    const int r = e / k, c = e % k;
    a.Y[(long long)(r0 + r) * k + c] = Ys[r][c];
  }
}


// ---------------------------------------------------------------------------
// The same block Gram-Schmidt inside one thread-block cluster of OC_NC CTAs
// (rows <= OC_NC * OC_RMAX).  Each CTA keeps its slab of rows in shared
// memory; every reduction over rows is a reduce-scatter and an all-gather
// through distributed shared memory between two cluster barriers, instead
// of two grid-wide barriers and a pass through L2.  The in-panel work is
// spread over the CTA: the panel Gram is accumulated in double-float FP32
// (exact products, compensated sums: FP32 pipes, about 44 significant bits),
// the 32 x 32 Cholesky runs right-looking on all threads in FP64, and the
// triangular solve is a product with L^{-1} (FP64, split into two floats)
// in double-float arithmetic.  Dead columns are handled as in the grid
// kernel.  Every CTA runs the same sequence of cluster barriers (no early
// exit), and a last barrier keeps each CTA's shared memory alive until its
// peers have read it.
namespace cg = cooperative_groups;

constexpr int OC_NC = 16;
constexpr int OC_RMAX = 64;
constexpr int OC_NT = 256;
constexpr int OC_BUF = MAX_K * PANEL;           // floats per exchange buffer
constexpr int OC_OUT = OC_RMAX * PANEL / OC_NT;  // panel outputs per thread

struct OrthClusterArgs {
  float* Y;
  int rows, k, rpc;   // rpc: rows per CTA (<= OC_RMAX)
  const int* run_if;  // null, or run only if *run_if != 0 (the fast path broke down)
};

// s + e = a + b exactly (round-to-nearest adds, never contracted)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += a * b with the product exact (fma residual)
__device__ __forceinline__ void df_fma(float a, float b, float& hi, float& lo) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  float t, e;
  two_sum(hi, p, t, e);
  hi = t;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

size_t orth_cluster_smem(int k) {
  return (size_t)OC_RMAX * (k + 1) * 4      // Ys
         + 3 * (size_t)OC_BUF * 4           // Pf, Rf, Ss
         + 3 * (size_t)PANEL * (PANEL + 1) * 8   // Ld, Lf, Li
         + 2 * (size_t)PANEL * (PANEL + 1) * 4   // Lh, Ll
         + PANEL * 8 + 64;                  // Linv, alignment slack
}

__global__ void __launch_bounds__(OC_NT, 1) orth_cluster(OrthClusterArgs a) {
  // every CTA of the cluster reads the same flag and leaves before any barrier
  if (a.run_if) {
    if (*a.run_if == 0) return;
    // run_if[1] counts the orthonormalisations the fast path handed over
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(const_cast<int*>(a.run_if) + 1, 1);
  }
  extern __shared__ __align__(16) unsigned char oc_smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x;
  const int rank = (int)cluster.block_rank();
  const int k = a.k, ld = k + 1;
  double* Ld = reinterpret_cast<double*>(oc_smem);              // working Gram [PANEL][PANEL+1]
  double* Lf = Ld + PANEL * (PANEL + 1);                        // Cholesky factor
  double* Li = Lf + PANEL * (PANEL + 1);                        // its inverse
  double* Linv = Li + PANEL * (PANEL + 1);                      // reciprocal pivots
  float* Pf = reinterpret_cast<float*>(Linv + PANEL);           // partials (peers read)
  float* Rf = Pf + OC_BUF;                                      // owned sums (peers read)
  float* Ss = Rf + OC_BUF;                                      // gathered coefficients
  float* Lh = Ss + OC_BUF;                                      // L^{-1} high part
  float* Ll = Lh + PANEL * (PANEL + 1);                         // L^{-1} low part
  float* Ys = Ll + PANEL * (PANEL + 1);                         // rows x ld
  double* Pd = reinterpret_cast<double*>(Pf);
  double* Rd = reinterpret_cast<double*>(Rf);
  const int r0 = rank * a.rpc;
  const int nr = max(0, min(a.rpc, a.rows - r0));
  for (int e = tid; e < OC_RMAX * ld; e += OC_NT) {
    const int r = e / ld, c = e % ld;
    Ys[e] = (r < nr && c < k) ? a.Y[(long long)(r0 + r) * k + c] : 0.f;
  }
  __syncthreads();
  for (int j0 = 0; j0 < k; j0 += PANEL) {
    const int w = min(PANEL, k - j0);
    // ---- two projection passes against columns [0, j0)
    for (int pass = 0; pass < 2 && j0 > 0; ++pass) {
      const int n = j0 * w;
      for (int e = tid; e < n; e += OC_NT) {
        const int j = e / w, c = e % w;
        float sacc = 0.f;
        for (int r = 0; r < nr; ++r) sacc = fmaf(Ys[r * ld + j], Ys[r * ld + j0 + c], sacc);
        Pf[e] = sacc;
      }
      cluster.sync();
      const int sl = (n + OC_NC - 1) / OC_NC;
      const int lo = rank * sl, hi = min(n, lo + sl);
      for (int e = lo + tid; e < hi; e += OC_NT) {
        float sacc = 0.f;
        for (int q = 0; q < OC_NC; ++q) sacc += cluster.map_shared_rank(Pf, q)[e];
        Rf[e] = sacc;
      }
      cluster.sync();
      for (int e = tid; e < n; e += OC_NT) Ss[e] = cluster.map_shared_rank(Rf, e / sl)[e];
      __syncthreads();
      for (int e = tid; e < nr * w; e += OC_NT) {
        const int r = e / w, c = e % w;
        float v = Ys[r * ld + j0 + c];
        for (int j = 0; j < j0; ++j) v = fmaf(-Ys[r * ld + j], Ss[j * w + c], v);
        Ys[r * ld + j0 + c] = v;
      }
      __syncthreads();
    }
    // ---- CholeskyQR2 inside the panel
    for (int pass = 0; pass < 2; ++pass) {
      const int n2 = w * w;
      for (int e = tid; e < n2; e += OC_NT) {
        const int c = e / w, d = e % w;
        float h = 0.f, l = 0.f;
        for (int r = 0; r < nr; ++r) df_fma(Ys[r * ld + j0 + c], Ys[r * ld + j0 + d], h, l);
        Pd[e] = (double)h + (double)l;
      }
      cluster.sync();
      const int sl = (n2 + OC_NC - 1) / OC_NC;
      const int lo = rank * sl, hi = min(n2, lo + sl);
      for (int e = lo + tid; e < hi; e += OC_NT) {
        double sacc = 0.0;
        for (int q = 0; q < OC_NC; ++q) sacc += cluster.map_shared_rank(Pd, q)[e];
        Rd[e] = sacc;
      }
      cluster.sync();
      for (int e = tid; e < n2; e += OC_NT)
        Ld[(e / w) * (PANEL + 1) + e % w] = cluster.map_shared_rank(Rd, e / sl)[e];
      for (int e = tid; e < PANEL * (PANEL + 1); e += OC_NT) {
        Lf[e] = 0.0;
        Li[e] = 0.0;
      }
      __syncthreads();
      double dmax = 0.0;
      for (int c = 0; c < w; ++c) dmax = fmax(dmax, Ld[c * (PANEL + 1) + c]);
      const double thr = 1e-13 * dmax;
      // right-looking Cholesky: the working Gram's column j stays unscaled
      // during step j, the factor goes to Lf (no read/write overlap)
      for (int j = 0; j < w; ++j) {
        if (tid == 0) {
          const double pj = Ld[j * (PANEL + 1) + j];
          const bool dead = !(pj > thr) || !(dmax > 0.0);
          const double dg = dead ? 0.0 : sqrt(pj);
          Lf[j * (PANEL + 1) + j] = dg;
          Linv[j] = dead ? 0.0 : 1.0 / dg;
        }
        __syncthreads();
        const double lj = Linv[j];
        const int t = w - 1 - j;
        for (int i = j + 1 + tid; i < w; i += OC_NT) Lf[i * (PANEL + 1) + j] = Ld[i * (PANEL + 1) + j] * lj;
        const double lj2 = lj * lj;
        for (int e = tid; e < t * t; e += OC_NT) {
          const int ii = j + 1 + e / t, cc = j + 1 + e % t;
          if (cc <= ii)
            Ld[ii * (PANEL + 1) + cc] -= Ld[ii * (PANEL + 1) + j] * Ld[cc * (PANEL + 1) + j] * lj2;
        }
        __syncthreads();
      }
      // L^{-1}: lane i builds column i by forward substitution
      if (tid < w) {
        const int i = tid;
        Li[i * (PANEL + 1) + i] = Linv[i];
        for (int j = i + 1; j < w; ++j) {
          double sacc = 0.0;
          for (int m = i; m < j; ++m) sacc = fma(Lf[j * (PANEL + 1) + m], Li[m * (PANEL + 1) + i], sacc);
          Li[j * (PANEL + 1) + i] = -Linv[j] * sacc;
        }
      }
      __syncthreads();
      for (int e = tid; e < n2; e += OC_NT) {
        const int c = e / w, d = e % w;
        const double x = Li[c * (PANEL + 1) + d];
        const float xh = (float)x;
        Lh[c * (PANEL + 1) + d] = xh;
        Ll[c * (PANEL + 1) + d] = (float)(x - (double)xh);
      }
      __syncthreads();
      // rows <- rows L^{-T}: x[r][c] = sum_{d <= c} L^{-1}[c][d] y[r][d]
      float outv[OC_OUT];
#pragma unroll
      for (int t = 0; t < OC_OUT; ++t) {
        const int e = tid + t * OC_NT;
        float h = 0.f, l = 0.f;
        if (e < nr * w) {
          const int r = e / w, c = e % w;
          for (int d = 0; d <= c; ++d) {
            const float y = Ys[r * ld + j0 + d];
            df_fma(y, Lh[c * (PANEL + 1) + d], h, l);
            l = __fmaf_rn(y, Ll[c * (PANEL + 1) + d], l);
          }
        }
        outv[t] = h + l;
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < OC_OUT; ++t) {
        const int e = tid + t * OC_NT;
        if (e < nr * w) Ys[(e / w) * ld + j0 + e % w] = outv[t];
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < nr * k; e += OC_NT) {
    const int r = e / k, c = e % k;
    a.Y[(long long)(r0 + r) * k + c] = Ys[r * ld + c];
  }
  // peers may still be reading this CTA's exchange buffers
  cluster.sync();
}

// cleared when a cluster launch fails: the grid-wide kernel is used from then on
std::atomic<int> g_orth_cluster_ok{1};

// Launch configuration of orth_cluster (one cluster of OC_NC CTAs).
cudaLaunchConfig_t orth_cluster_config(size_t smem, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(OC_NC);
  cfg.blockDim = dim3(OC_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = OC_NC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Whether one cluster of OC_NC CTAs with the largest shared-memory request
// can be resident on the current device (asked once per device; no kernel
// runs for it).
PerDevice<bool> g_orth_cluster_avail;

bool orth_cluster_available() {
  bool avail = false;
  if (g_orth_cluster_avail.get(
          [](int) {
            const size_t smem = orth_cluster_smem(MAX_K);
            if (cudaFuncSetAttribute(orth_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                     1) != cudaSuccess ||
                cudaFuncSetAttribute(orth_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess) {
              cudaGetLastError();
              return false;
            }
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = orth_cluster_config(smem, 0, attr);
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, orth_cluster, &cfg) != cudaSuccess) {
              cudaGetLastError();
              return false;
            }
            return nclusters >= 1;
          },
          &avail) != cudaSuccess)
    return false;
  return avail && g_orth_cluster_ok.load(std::memory_order_relaxed) != 0;
}

// CTAs of the grid-wide kernel's cooperative launch (once per device, thread-safe)
struct OrthSetup {
  cudaError_t err;
  int max_ctas;
};
PerDevice<OrthSetup> g_orth_setup;

OrthSetup orth_setup() {
  OrthSetup s{cudaSuccess, 0};
  cudaError_t e = g_orth_setup.get(
      [](int dev) {
        OrthSetup r{cudaSuccess, 0};
        int sms = 0, per = 0;
        r.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (r.err == cudaSuccess)
          r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, orth_persistent, ORTH_NT, 0);
        r.max_ctas = sms * per;
        return r;
      },
      &s);
  if (e != cudaSuccess) s.err = e;
  return s;
}

// C[m][n] (row stride ldc) = sum over s of part[s][m][n]
__global__ void sum_partials_kernel(const float* __restrict__ part, int splitk, int M, int N,
                                    float* __restrict__ C, long long ldc) {
  const long long MN = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MN;
       e += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < splitk; ++s) acc += part[s * MN + e];
    C[(e / N) * ldc + e % N] = acc;
  }
}

#define RET(x)                                 \
  do {                                         \
    cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) return _e;          \
  } while (0)

// C (M x N, FP32 row-major, ldc) = A B^T on the tensor cores (3 planes, 6
// products).  Each operand is either given as BF16 planes already (p: row
// stride pld, plane stride pps) or as an FP32 view split by to_planes_f32.
struct View {
  const float* f;
  Idx3 rv, kv;
  const __nv_bfloat16* p;
  long long pld, pps;
};

View planes_view(const __nv_bfloat16* p, long long pld, long long pps) {
  return View{nullptr, idx_plain(0), idx_plain(0), p, pld, pps};
}
View f32_view(const float* f, Idx3 rv, Idx3 kv) { return View{f, rv, kv, nullptr, 0, 0}; }

cudaError_t tc_product(const View& a, const View& b, int M, int N, int K, float* C, long long ldc,
                       const SubspaceBuffers& buf, cudaStream_t st) {
  const long long ld = tc_ld(K);
  const long long psa = (long long)M * ld, psb = (long long)N * ld;
  if (psa > buf.psa || psb > buf.psb) return cudaErrorInvalidValue;
  TcOperand A{buf.pa, 3, M, K, ld, 0, buf.psa, 1};
  TcOperand B{buf.pb, 3, N, K, ld, 0, buf.psb, 1};
  if (a.p) A = TcOperand{a.p, 3, M, K, a.pld, 0, a.pps, 1};
  else RET(to_planes_f32(a.f, a.rv, a.kv, 0, M, K, 1, buf.pa, ld, 0, 3, buf.psa, st));
  // a Gram (the same FP32 view on both sides) converts its operand once
  const bool same = !a.p && !b.p && a.f == b.f && M == N && !memcmp(&a.rv, &b.rv, sizeof(Idx3)) &&
                    !memcmp(&a.kv, &b.kv, sizeof(Idx3));
  if (b.p) B = TcOperand{b.p, 3, N, K, b.pld, 0, b.pps, 1};
  else if (same) B = A;
  else RET(to_planes_f32(b.f, b.rv, b.kv, 0, N, K, 1, buf.pb, ld, 0, 3, buf.psb, st));
  TcOutput o;
  memset(&o, 0, sizeof o);
  o.alpha = 1.0;
  // products with few output tiles (the k x k Grams, the k-wide factors)
  // split K so that about one wave of CTAs runs, partials summed after
  const int kb = (K + 63) / 64, tiles = ((M + 127) / 128) * ((N + 127) / 128);
  int splitk = 1;
  if (buf.part && tiles < 76) {
    int sk = 152 / tiles;
    sk = sk < kb ? sk : kb;
    sk = sk < 32 ? sk : 32;
    const int per = (kb + sk - 1) / sk;
    sk = (kb + per - 1) / per;
    if ((size_t)sk * M * N <= buf.part_floats) splitk = sk;
  }
  if (splitk == 1) {
    o.mode = TC_OUT_F32;
    o.f32 = C;
    o.cm = idx_plain(ldc);
    o.cn = idx_plain(1);
    return tc_gemm(A, B, M, N, K, 1, 6, 1, o, buf.err, st);
  }
  o.mode = TC_OUT_PARTIAL;
  o.f32 = buf.part;
  RET(tc_gemm(A, B, M, N, K, 1, 6, splitk, o, buf.err, st));
  note_launch();
  sum_partials_kernel<<<grid_for((long long)M * N), 256, 0, st>>>(buf.part, splitk, M, N, C, ldc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fast path of the orthonormalisation: scaled CholeskyQR2.
//
// Y = C_E V_prev + eta R has columns of very different norms (they follow
// the singular values of C_E), but once the warm start has converged they
// are close to orthogonal.  With the column scaling D = diag(1/||y_j||) the
// Gram G = D Y^T Y D is then well conditioned, and two CholeskyQR passes
// (G = L L^T, U = Y D L^{-T}) give an orthonormal U to FP32 level.  The
// Gram runs on the tensor cores (tc_product, 24-bit products, unbiased
// FP32 accumulation), the k x k Cholesky on one CTA in FP32 (blocked
// right-looking, packed lower triangle in shared memory), and the
// triangular solve on every SM (one warp per row, blocks of 32 columns).
// A scaled pivot below tau means Y is ill conditioned (a warm start far
// from converged, a growing bond): the factor kernel raises *flag and the
// block Gram-Schmidt kernels, launched after it, orthonormalise the
// untouched Y instead (they return at once when *flag is 0).  A column
// whose norm is zero is dead: its output column is zero, as in the block
// Gram-Schmidt kernels.
constexpr int CQ_NT = 384;        // threads of the factor kernel (12 warps: up to 170 registers)
constexpr int CQ_SOLVE_NT = 256;  // threads of the solve kernel (8 warps, one row each)

__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }

// shared memory of the factor kernel: the packed lower triangle, the
// transposed panel copy Pt[32][MAX_K], the scaling and the reciprocal pivots
constexpr int CQ_LD = 36;   // row stride of the factored diagonal block copy (16-byte rows)

size_t cholqr_factor_smem(int k) {
  const size_t packed = ((size_t)k * (k + 1) / 2 + 3) / 4 * 4;
  return (packed + (size_t)32 * MAX_K + 32 * CQ_LD + 2 * MAX_K) * 4;
}

// G (k x k FP32 row-major, symmetric; lower triangle read) -> Lout (packed
// lower Cholesky factor of D G D), dout (the scaling d_j; 0 for a dead
// column), linv_out (1 / L_jj, 0 for a dead column); *flag = 1 if a live
// scaled pivot falls below tau (never cleared here), or, with deflate set,
// that column is dropped as dead instead (its part orthogonal to the columns
// before it is below sqrt(tau) of its norm: numerically dependent) and
// counted in flag[4].  Right-looking, 32-wide
// panels: the diagonal block in registers of warp 0 (lane = row, shuffles),
// the rows below it one per thread against that block, then the trailing
// update in 4 x 4 register blocks from the transposed panel copy (float4
// reads, conflict-free).  With run_if set, runs only if *run_if != 0 and
// *flag == 0.
__global__ void __launch_bounds__(CQ_NT, 1)
    cholqr_factor(const float* __restrict__ G, int k, float tau, int deflate,
                  float* __restrict__ Lout, float* __restrict__ dout, float* __restrict__ linv_out,
                  int* flag, const int* run_if) {
  if (run_if && (*run_if == 0 || *flag)) return;
  if (run_if && threadIdx.x == 0) atomicAdd(const_cast<int*>(run_if) + 1, 1);
  extern __shared__ __align__(16) float cq[];
  const int np = k * (k + 1) / 2;
  float* A = cq;                                    // packed lower triangle
  float* Pt = cq + ((np + 3) / 4 * 4);              // panel, transposed: Pt[t * MAX_K + row]
  float* Ld = Pt + 32 * MAX_K;                      // factored diagonal block, Ld[r * CQ_LD + c]
  float* d = Ld + 32 * CQ_LD;                       // scaling
  float* li = d + MAX_K;                            // 1 / L_jj
  __shared__ float red[32];
  __shared__ int bad, ndefl;
  __shared__ __align__(16) float colb[32];   // column of the diagonal-block step
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  float gm = 0.f;
  for (int j = tid; j < k; j += CQ_NT) {
    const float g = G[(long long)j * k + j];
    gm = fmaxf(gm, (g == g) ? g : 3.0e38f);
  }
  for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  if (lane == 0) red[warp] = gm;
  if (tid == 0) {
    bad = 0;
    ndefl = 0;
  }
  __syncthreads();
  if (tid < 32) {
    float v = tid < CQ_NT / 32 ? red[tid] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (tid == 0) red[0] = v;
  }
  __syncthreads();
  const float gmax = red[0];
  for (int j = tid; j < k; j += CQ_NT) {
    const float g = G[(long long)j * k + j];
    d[j] = (g > 1e-30f * gmax && g < 3.0e38f) ? 1.f / sqrtf(g) : 0.f;
  }
  __syncthreads();
  // packed load, row by row (one warp per row, coalesced reads of G); the
  // row's eight loads are issued before any is used, so a warp waits on the
  // memory latency once per row rather than once per 32 columns
  for (int i = warp; i < k; i += CQ_NT / 32) {
    const float di = d[i];
    float g[MAX_K / 32];
#pragma unroll
    for (int t = 0; t < MAX_K / 32; ++t) {
      const int j = lane + 32 * t;
      g[t] = j <= i ? G[(long long)i * k + j] : 0.f;
    }
#pragma unroll
    for (int t = 0; t < MAX_K / 32; ++t) {
      const int j = lane + 32 * t;
      if (j <= i) {
        const float v = g[t] * di * d[j];
        A[pk(i, j)] = (v == v) ? v : 0.f;
        if (v != v) bad = 1;
      }
    }
  }
  __syncthreads();
  for (int p0 = 0; p0 < k; p0 += 32) {
    const int pw = min(32, k - p0);
    // (a) the diagonal block: lane r holds row p0 + r (columns p0..p0+31)
    if (warp == 0) {
      float r[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) r[c] = (lane < pw && c <= lane) ? A[pk(p0 + lane, p0 + c)] : 0.f;
      // dead columns of the block (zero scaling) as one bit per lane; pivots
      // that break down, collected the same way (the pivot is warp-uniform)
      const unsigned deadm = __ballot_sync(0xffffffffu, lane < pw && d[p0 + lane] == 0.f);
      unsigned brokem = 0;
      float myinv = 0.f;
      // Per step, the pivot comes by one shuffle; the new column L_.,j goes
      // through shared memory and is read back as float4 broadcasts (a
      // shuffle per trailing column made each step several hundred cycles).
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j < pw) {
          const float piv = __shfl_sync(0xffffffffu, r[j], j);
          const bool dead = (deadm >> j) & 1u;
          const bool broke = !dead && !(piv > tau);
          const float rs = rsqrtf(piv);
          const bool good = !(dead || broke);
          const float ljj = good ? piv * rs : 1.f;
          const float inv = good ? rs : 0.f;
          if (broke) brokem |= 1u << j;
          if (lane == j) myinv = inv;
          const float lj = r[j] * inv;   // L_lane,j (lane > j)
          r[j] = lane == j ? ljj : (lane > j ? lj : r[j]);
          if (j < 31) {
            colb[lane] = lj;
            __syncwarp();
            // trailing part of the block: r[c] -= L_lane,j L_c,j for j < c <= lane
#pragma unroll
            for (int c4 = (j + 1) / 4; c4 < 8; ++c4) {
              const float4 x4 = *reinterpret_cast<const float4*>(colb + 4 * c4);
              const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int c = 4 * c4 + u;
                if (c > j) r[c] = lane >= c ? fmaf(-lj, xs[u], r[c]) : r[c];
              }
            }
            __syncwarp();
          }
        }
      }
      if (lane < pw) li[p0 + lane] = myinv;
      if (lane == 0 && brokem) {
        if (deflate) ndefl += __popc(brokem);
        else bad = 1;
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (lane < pw && c <= lane) A[pk(p0 + lane, p0 + c)] = r[c];
        Ld[lane * CQ_LD + c] = (lane < pw && c <= lane) ? r[c] : 0.f;
      }
    }
    __syncthreads();
    // (b) rows below the block: L_ip = A_ip L_pp^{-T}, one thread per row;
    // the rows of L_pp are read as float4 broadcasts and each dot product
    // runs in four partial sums (short dependency chains)
    for (int i = p0 + pw + tid; i < k; i += CQ_NT) {
      float x[32];
      const int base = pk(i, p0);
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        if (t < pw) {
          float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            if (4 * q4 < t) {
              const float4 l = *reinterpret_cast<const float4*>(Ld + t * CQ_LD + 4 * q4);
              // entries q >= t of row t are zero in Ld (and x[q] for q >= t
              // is not yet defined): only q < t is taken
              s4[0] = fmaf(x[4 * q4], l.x, s4[0]);
              if (4 * q4 + 1 < t) s4[1] = fmaf(x[4 * q4 + 1], l.y, s4[1]);
              if (4 * q4 + 2 < t) s4[2] = fmaf(x[4 * q4 + 2], l.z, s4[2]);
              if (4 * q4 + 3 < t) s4[3] = fmaf(x[4 * q4 + 3], l.w, s4[3]);
            }
          }
          x[t] = (A[base + t] - ((s4[0] + s4[1]) + (s4[2] + s4[3]))) * li[p0 + t];
        }
      }
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < pw) {
          A[base + t] = x[t];
          Pt[t * MAX_K + i] = x[t];
        }
    }
    __syncthreads();
    // (c) trailing update A_ic -= sum_t L_it L_ct for p0+pw <= c <= i
    const int r0 = p0 + pw, n = k - r0;
    if (n > 0) {
      const int nb = (n + 3) / 4, nblk = nb * (nb + 1) / 2;
      for (int bidx = tid; bidx < nblk; bidx += CQ_NT) {
        int bi = (int)((sqrtf(8.f * (float)bidx + 1.f) - 1.f) * 0.5f);
        while (bi * (bi + 1) / 2 > bidx) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= bidx) ++bi;
        const int bc = bidx - bi * (bi + 1) / 2;
        const int i0 = r0 + 4 * bi, c0 = r0 + 4 * bc;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        // i0, c0 are multiples of 4 below MAX_K: whole float4 reads.  Rows
        // of Pt past k hold stale values; they only reach the entries of acc
        // with i >= k or c >= k, which are not stored.
#pragma unroll 8
        for (int t = 0; t < pw; ++t) {
          const float4 a = *reinterpret_cast<const float4*>(Pt + t * MAX_K + i0);
          const float4 b = *reinterpret_cast<const float4*>(Pt + t * MAX_K + c0);
          const float pi[4] = {a.x, a.y, a.z, a.w}, pc[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(pi[u], pc[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int i = i0 + u, c = c0 + v;
            if (i < k && c <= i) A[pk(i, c)] -= acc[u][v];
          }
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < np; e += CQ_NT) Lout[e] = A[e];
  for (int j = tid; j < k; j += CQ_NT) {
    dout[j] = d[j];
    linv_out[j] = li[j];
  }
  if (tid == 0 && bad) atomicExch(flag, 1);
  if (tid == 0 && ndefl) atomicAdd(flag + 4, ndefl);
}

// U[r] = (Y[r] o d) L^{-T} for every row r (one warp per row; rows ldy / ldu
// apart, so a column block of a wider matrix works in place): with u L^T = z,
// u_j = (z_j - sum_{i<j} u_i L_ji) / L_jj, in blocks of 32 columns (earlier
// blocks first, then a sequential solve inside the block).  Does nothing if
// *flag is set (the fast path broke down) or, with run_if set, if *run_if is
// 0.  U may be Y itself (ldu = ldy): each row is read by the lanes that
// write it, column j before U[r][j].
__global__ void __launch_bounds__(CQ_SOLVE_NT)
    cholqr_solve(const float* Y, long long ldy, int rows, int k,
                 const float* __restrict__ Lp, const float* __restrict__ dv,
                 const float* __restrict__ linv, const int* __restrict__ flag,
                 const int* __restrict__ run_if, float* U, long long ldu) {
  if (*flag || (run_if && *run_if == 0)) return;
  extern __shared__ __align__(16) float Ls[];
  const int np = k * (k + 1) / 2;
  // the packed factor (16-byte aligned in global memory), 16 bytes per load
  const int n4 = np / 4;
#pragma unroll 4
  for (int e = threadIdx.x; e < n4; e += CQ_SOLVE_NT)
    reinterpret_cast<float4*>(Ls)[e] = reinterpret_cast<const float4*>(Lp)[e];
  for (int e = 4 * n4 + threadIdx.x; e < np; e += CQ_SOLVE_NT) Ls[e] = Lp[e];
  __syncthreads();
  const int lane = threadIdx.x % 32;
  const int WPB = CQ_SOLVE_NT / 32;
  for (int r = blockIdx.x * WPB + threadIdx.x / 32; r < rows; r += gridDim.x * WPB) {
    float x[MAX_K / 32];
#pragma unroll
    for (int qb = 0; qb < MAX_K / 32; ++qb) {
      x[qb] = 0.f;
      if (qb * 32 < k) {
        const int j = qb * 32 + lane;
        float s = (j < k) ? Y[(long long)r * ldy + j] * dv[j] : 0.f;
        // earlier blocks
#pragma unroll
        for (int q = 0; q < MAX_K / 32; ++q) {
          if (q < qb) {
#pragma unroll 8
            for (int t = 0; t < 32; ++t) {
              const float xt = __shfl_sync(0xffffffffu, x[q], t);
              if (j < k) s = fmaf(-xt, Ls[pk(j, q * 32 + t)], s);
            }
          }
        }
        // inside the block (1 / L_jj read before the chain: a load inside it,
        // one per step, put the memory latency on the chain 32 times)
        const float lij = (j < k) ? linv[j] : 0.f;
        float xj = 0.f;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          if (qb * 32 + t < k) {
            if (lane == t) xj = s * lij;
            const float xt = __shfl_sync(0xffffffffu, xj, t);
            if (lane > t && j < k) s = fmaf(-xt, Ls[pk(j, qb * 32 + t)], s);
          }
        }
        x[qb] = xj;
        if (j < k) U[(long long)r * ldu + j] = xj;
      }
    }
  }
}

// Y (rows x k, row-major FP32) <- orthonormal basis of its column space.
cudaError_t orth_check(const float* Q, int rows, int k, const SubspaceBuffers& b, cudaStream_t st);

cudaError_t block_cgs(float* Y, int rows, int k, const SubspaceBuffers& b, cudaStream_t st,
                      const int* run_if) {
  if (k > MAX_K) return cudaErrorInvalidValue;
  if (rows <= OC_NC * OC_RMAX && orth_cluster_available()) {
    OrthClusterArgs ca;
    ca.Y = Y; ca.rows = rows; ca.k = k; ca.run_if = run_if;
    ca.rpc = (rows + OC_NC - 1) / OC_NC;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = orth_cluster_config(orth_cluster_smem(k), st, attr);
    note_launch();
    if (cudaLaunchKernelEx(&cfg, orth_cluster, ca) == cudaSuccess) {
      __atomic_add_fetch(&g_orth_cluster_calls, 1ull, __ATOMIC_RELAXED);
      ++t_orth_cluster_calls;
      return cudaSuccess;
    }
    // the cluster could not be launched: use the grid-wide kernel from now on
    cudaGetLastError();
    g_orth_cluster_ok.store(0, std::memory_order_relaxed);
  }
  const int G = (rows + ROWS_PER_CTA - 1) / ROWS_PER_CTA;
  const OrthSetup setup = orth_setup();
  RET(setup.err);
  if (G > setup.max_ctas || G > b.orth_max_ctas) return cudaErrorInvalidValue;
  OrthArgs a;
  a.Y = Y; a.rows = rows; a.k = k;
  a.part = b.orth_part; a.red = b.orth_red;
  a.partd = b.orth_partd; a.redd = b.orth_redd;
  a.bar = b.orth_bar; a.status = (int*)(b.orth_bar + 2);
  a.run_if = run_if;
  RET(cudaMemsetAsync(b.orth_bar, 0, 4 * sizeof(unsigned), st));
  void* args[] = {&a};
  note_launch();
  RET(cudaLaunchCooperativeKernel((void*)orth_persistent, dim3(G), dim3(ORTH_NT), args, 0, st));
  return cudaSuccess;
}

// shared-memory opt-in of the two CholeskyQR kernels, once per device
PerDevice<cudaError_t> g_cholqr_setup;

cudaError_t cholqr_setup() {
  cudaError_t r = cudaSuccess;
  cudaError_t e = g_cholqr_setup.get(
      [](int) {
        cudaError_t x = cudaFuncSetAttribute(cholqr_factor,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cholqr_factor_smem(MAX_K));
        if (x == cudaSuccess)
          x = cudaFuncSetAttribute(cholqr_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)((size_t)MAX_K * (MAX_K + 1) / 2 * 4));
        return x;
      },
      &r);
  return e != cudaSuccess ? e : r;
}

// Two scaled CholeskyQR passes on the column block Yb (rows x w, row stride
// ldy): Yb -> U1 (in tmp, row stride w) -> Yb.  A breakdown raises
// b.chol_flag[0] and leaves Yb as it was.
cudaError_t cholqr2_block(float* Yb, long long ldy, int rows, int w, float* tmp,
                          const SubspaceBuffers& b, cudaStream_t st) {
  const size_t fsm = cholqr_factor_smem(w), ssm = (size_t)w * (w + 1) / 2 * 4;
  const int wpb = CQ_SOLVE_NT / 32;
  int grid = (rows + wpb - 1) / wpb;
  if (grid > 152) grid = 152;
  const float* src = Yb;
  long long lds = ldy;
  float* dst = tmp;
  long long ldd = w;
  for (int pass = 0; pass < 2; ++pass) {
    // G = Yb^T Yb (w x w) on the tensor cores
    RET(tc_product(f32_view(src, idx_plain(1), idx_plain(lds)),
                   f32_view(src, idx_plain(1), idx_plain(lds)), w, w, rows, b.out, w, b, st));
    note_launch();
    cholqr_factor<<<1, CQ_NT, fsm, st>>>(b.out, w, pass == 0 ? 1e-6f : 0.25f, pass == 0 ? 1 : 0,
                                         b.chol_L, b.chol_d, b.chol_li, b.chol_flag, nullptr);
    RET(cudaGetLastError());
    note_launch();
    cholqr_solve<<<grid, CQ_SOLVE_NT, ssm, st>>>(src, lds, rows, w, b.chol_L, b.chol_d, b.chol_li,
                                                 b.chol_flag, nullptr, dst, ldd);
    RET(cudaGetLastError());
    src = tmp;
    lds = w;
    dst = Yb;
    ldd = ldy;
  }
  return cudaSuccess;
}

// Yb[r][c] -= Z[r][c] (Yb row stride ldy, Z row stride w), unless *flag
__global__ void subtract_block_kernel(float* __restrict__ Yb, long long ldy,
                                      const float* __restrict__ Z, int rows, int w,
                                      const int* __restrict__ flag) {
  if (*flag) return;
  const long long total = (long long)rows * w;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / w, c = e % w;
    Yb[r * ldy + c] -= Z[e];
  }
}

// The second CholeskyQR pass to first order.  After the first pass the Gram
// of U1 is G2 = I + E with E small; its Cholesky factor is L = I + Phi(E) +
// O(E^2), Phi(E) the strictly lower part of E plus half its diagonal, so
// U2 = U1 L^{-T} = U1 (I - Phi(E)^T) + O(E^2) and U2^T U2 = I + O(E^2).
// Writes B = I - Phi(E) (k x k row-major: U2 = U1 B^T is one tensor-core
// product); dead columns (G2_jj < 1/2, zero columns of U1) keep B's row e_j
// and get zeros elsewhere.  If a live |E_ij| exceeds emax (or is not
// finite), sets *need_full: the full second pass runs instead (and counts
// itself in need_full[1]).
__global__ void cholqr_linear_kernel(const float* __restrict__ G, int k, float emax,
                                     float* __restrict__ B, int* need_full) {
  bool big = false;
  const long long total = (long long)k * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e / k), c = (int)(e % k);
    const float gn = G[(long long)n * k + n], gc = G[(long long)c * k + c];
    const bool ln = gn >= 0.5f, lc = gc >= 0.5f;
    float v = 0.f;
    if (!ln) {
      v = (n == c) ? 1.f : 0.f;
    } else if (lc) {
      const float E = (n == c) ? gn - 1.f : G[e];
      if (!(fabsf(E) <= emax)) big = true;
      v = (n == c) ? 1.f - 0.5f * E : (n > c ? -E : 0.f);
    }
    B[e] = v;
  }
  if (__syncthreads_or(big) && threadIdx.x == 0) atomicExch(need_full, 1);
}

// dst[r][c] = src[r][c] (rows x k, contiguous) if *flag != 0
__global__ void copy_if_flag_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                    long long n, const int* __restrict__ flag) {
  if (*flag == 0) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// Largest |E_ij| of the first-order second pass; above it the full second
// CholeskyQR pass runs.  The neglected O(E^2) terms (up to about 4 k E^2 in
// the max norm, typically ~1e-5 at k = 256) stay below the orthonormality
// check's bound; removing them by one more first-order correction of the
// checked basis was measured not to change the free energy.
constexpr float CQ_LINEAR_EMAX = 1e-3f;

// An orthonormal basis of the columns of Y (rows x k, FP32), written to
// *U (b.Q or Y itself); Y and b.Q are overwritten.  Up to one column block
// (k <= b.orth_block): scaled CholeskyQR2 with its second pass to first order
// (Y -> U1 in place, then U2 = U1 B^T into b.Q, see cholqr_linear_kernel);
// the full second pass runs instead when U1 is too far from orthonormal, and
// the block Gram-Schmidt kernels when a pass breaks down (all chosen on the
// device by flags; see cholqr_factor).  Wider: block classical Gram-Schmidt
// over column blocks, each projected twice against the blocks before it on
// the tensor cores (S = Q^T Y_b, Y_b -= Q S) and then orthonormalised by
// scaled CholeskyQR2, result in Y; a breakdown leaves Y unorthonormal, which
// the caller's orthonormality check turns into the exact split.
cudaError_t orthonormalise(float* Y, int rows, int k, const SubspaceBuffers& b, cudaStream_t st,
                           float** U) {
  if (k > SUBSPACE_MAX_K) return cudaErrorInvalidValue;
  RET(cholqr_setup());
  // chol_flag: [0] breakdown, [1] breakdowns counted by the block Gram-Schmidt
  // kernels, [2] full second pass needed, [3] full second passes counted,
  // [4] columns dropped as numerically dependent by the first pass
  RET(cudaMemsetAsync(b.chol_flag, 0, sizeof(int), st));
  RET(cudaMemsetAsync(b.chol_flag + 2, 0, sizeof(int), st));
  const int B = b.orth_block;
  if (B < 32 || B > MAX_K || B % 32) return cudaErrorInvalidValue;
  if (k <= B) {
    const size_t fsm = cholqr_factor_smem(k), ssm = (size_t)k * (k + 1) / 2 * 4;
    const int wpb = CQ_SOLVE_NT / 32;
    const int grid = (rows + wpb - 1) / wpb < 152 ? (rows + wpb - 1) / wpb : 152;
    float* G = b.out;                          // k x k Grams
    float* Bm = b.out + (size_t)k * k;         // k x k first-order factor
    int* need_full = b.chol_flag + 2;
    // pass 1: G = Y^T Y, scaled Cholesky, Y <- U1 in place (skipped on breakdown)
    RET(tc_product(f32_view(Y, idx_plain(1), idx_plain(k)), f32_view(Y, idx_plain(1), idx_plain(k)),
                   k, k, rows, G, k, b, st));
    note_launch();
    cholqr_factor<<<1, CQ_NT, fsm, st>>>(G, k, 1e-6f, 1, b.chol_L, b.chol_d, b.chol_li,
                                         b.chol_flag, nullptr);
    RET(cudaGetLastError());
    note_launch();
    cholqr_solve<<<grid, CQ_SOLVE_NT, ssm, st>>>(Y, k, rows, k, b.chol_L, b.chol_d, b.chol_li,
                                                 b.chol_flag, nullptr, Y, k);
    RET(cudaGetLastError());
    // pass 2 to first order: G = U1^T U1 = I + E, b.Q <- U1 (I - Phi(E)^T)
    RET(tc_product(f32_view(Y, idx_plain(1), idx_plain(k)), f32_view(Y, idx_plain(1), idx_plain(k)),
                   k, k, rows, G, k, b, st));
    note_launch();
    cholqr_linear_kernel<<<grid_for((long long)k * k), 256, 0, st>>>(G, k, CQ_LINEAR_EMAX, Bm,
                                                                     need_full);
    RET(cudaGetLastError());
    RET(tc_product(f32_view(Y, idx_plain(k), idx_plain(1)), f32_view(Bm, idx_plain(k), idx_plain(1)),
                   rows, k, k, b.Q, k, b, st));
    // the full second pass, only if E was too large: U1 -> b.Q
    note_launch();
    cholqr_factor<<<1, CQ_NT, fsm, st>>>(G, k, 0.25f, 0, b.chol_L, b.chol_d, b.chol_li,
                                         b.chol_flag, need_full);
    RET(cudaGetLastError());
    note_launch();
    cholqr_solve<<<grid, CQ_SOLVE_NT, ssm, st>>>(Y, k, rows, k, b.chol_L, b.chol_d, b.chol_li,
                                                 b.chol_flag, need_full, b.Q, k);
    RET(cudaGetLastError());
    // a breakdown in either pass: block Gram-Schmidt on Y (the input, or U1
    // after a breakdown of the second pass), copied to b.Q
    RET(block_cgs(Y, rows, k, b, st, b.chol_flag));
    note_launch();
    copy_if_flag_kernel<<<grid_for((long long)rows * k), 256, 0, st>>>(Y, b.Q, (long long)rows * k,
                                                                       b.chol_flag);
    RET(cudaGetLastError());
    *U = b.Q;
    return cudaSuccess;
  }
  *U = Y;
  for (int j0 = 0; j0 < k; j0 += B) {
    const int w = k - j0 < B ? k - j0 : B;
    float* Yb = Y + j0;
    for (int pass = 0; pass < 2 && j0 > 0; ++pass) {
      // S (j0 x w, in b.out) = Q^T Y_b with Q = Y[:, :j0]
      RET(tc_product(f32_view(Y, idx_plain(1), idx_plain(k)), f32_view(Yb, idx_plain(1), idx_plain(k)),
                     j0, w, rows, b.out, w, b, st));
      // Z (rows x w, in b.Q) = Q S
      RET(tc_product(f32_view(Y, idx_plain(k), idx_plain(1)), f32_view(b.out, idx_plain(1), idx_plain(w)),
                     rows, w, j0, b.Q, w, b, st));
      note_launch();
      subtract_block_kernel<<<grid_for((long long)rows * w), 256, 0, st>>>(Yb, k, b.Q, rows, w,
                                                                           b.chol_flag);
      RET(cudaGetLastError());
    }
    RET(cholqr2_block(Yb, k, rows, w, b.Q, b, st));
  }
  return cudaSuccess;
}

}  // namespace

unsigned long long g_orth_cluster_calls = 0;
thread_local unsigned long long t_orth_cluster_calls = 0;

size_t subspace_plane_elems_a(int cap) { return 3 * (size_t)(4 * cap) * tc_ld(4 * cap); }
size_t subspace_plane_elems_b(int cap) { return 3 * (size_t)(4 * cap) * tc_ld(4 * cap); }

namespace {
// max over live columns of |Q^T Q - I| (dead columns, norm < 1/2, are skipped)
// into b.dscal[2] (as FP64).  Q^T Q by the tensor cores, 6 products.
__global__ void orth_defect_kernel(const float* __restrict__ G, int k, double* out) {
  __shared__ float red[32];
  float mx = 0.f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e % k;
    const float gi = G[(long long)i * k + i], gj = G[(long long)j * k + j];
    if (gi < 0.5f || gj < 0.5f) continue;
    const float d = fabsf(G[e] - (i == j ? 1.f : 0.f));
    mx = fmaxf(mx, d != d ? 1e30f : d);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t = fmaxf(t, red[i]);
    // non-negative doubles order like their bit patterns (*out starts at +0)
    atomicMax(reinterpret_cast<unsigned long long*>(out),
              (unsigned long long)__double_as_longlong((double)t));
  }
}

cudaError_t orth_check(const float* Q, int rows, int k, const SubspaceBuffers& b, cudaStream_t st) {
  RET(tc_product(f32_view(Q, idx_plain(1), idx_plain(k)), f32_view(Q, idx_plain(1), idx_plain(k)),
                 k, k, rows, b.out, k, b, st));
  note_launch();
  const int g = (k * k + 4095) / 4096;
  orth_defect_kernel<<<g < 152 ? g : 152, 1024, 0, st>>>(b.out, k, b.dscal + 2);
  return cudaGetLastError();
}

}  // namespace

size_t subspace_buffer_floats(int cap) {
  const size_t m = 4 * (size_t)cap;
  const size_t G = (m + ROWS_PER_CTA - 1) / ROWS_PER_CTA;
  return m * cap /*Q*/ + m * cap /*Y*/ + m * m /*out*/ + G * MAX_K * PANEL /*orth partials*/ +
         MAX_K * PANEL /*orth reduced*/ + 64 /*scal*/ + 2 * G * PANEL * PANEL /*FP64 partial Grams*/ +
         2 * PANEL * PANEL /*FP64 Gram*/ + 64;
}

int subspace_orth_ctas(int cap) { return (4 * cap + ROWS_PER_CTA - 1) / ROWS_PER_CTA; }

namespace {
// discarded weight 1 - ||centre||^2 / ||C_E||^2 of an accepted split
// (orthonormality defect <= thresh) raised into *disc_max
__global__ void split_finish_kernel(const double* __restrict__ ce_ss, const double* __restrict__ dscal,
                                    double thresh, double* disc_max) {
  const double tot = *ce_ss, defect = dscal[2];
  const double disc = tot > 0.0 ? fmax(0.0, 1.0 - dscal[1] / tot) : 0.0;
  if (defect <= thresh)
    atomicMax(reinterpret_cast<unsigned long long*>(disc_max),
              (unsigned long long)__double_as_longlong(disc));
}

// After the orthonormality check (G = Q^T Q): the defect is set to +inf if no
// column of Q is live, or if a blocked orthonormalisation (which has no
// Gram-Schmidt fallback) broke down, so that the exact split runs.
__global__ void split_guard_kernel(const float* __restrict__ G, int k, const int* __restrict__ flag,
                                   int blocked, double* defect) {
  __shared__ int live;
  if (threadIdx.x == 0) live = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    if (G[(long long)j * k + j] >= 0.5f) live = 1;
  __syncthreads();
  if (threadIdx.x == 0 && (!live || (blocked && *flag))) *defect = INFINITY;
}

cudaError_t split_guard(int k, const SubspaceBuffers& b, cudaStream_t st) {
  note_launch();
  split_guard_kernel<<<1, 256, 0, st>>>(b.out, k, b.chol_flag, k > b.orth_block ? 1 : 0,
                                        b.dscal + 2);
  return cudaGetLastError();
}
}  // namespace

const double* subspace_defect(const SubspaceBuffers& b) { return b.dscal + 2; }

namespace {
__global__ void bump_kernel(unsigned long long* p) { *p += 1; }
}  // namespace

cudaError_t subspace_next_seed(const SubspaceBuffers& b, cudaStream_t st) {
  note_launch();
  bump_kernel<<<1, 1, 0, st>>>(b.seed_base);
  return cudaGetLastError();
}

cudaError_t subspace_split(const double* CE, int m, int n, int k, int dir_right,
                           const double* warm, int kold, double* left, double* right,
                           unsigned long long seed, const SubspaceBuffers& b, cudaStream_t st,
                           double* disc_max, double thresh) {
  (void)CE;
  if (k > SUBSPACE_MAX_K || k > m || k > n) return cudaErrorInvalidValue;
  const double inv_mn = 1.0 / ((double)m * n);
  const long long ldn = tc_ld(n), ldm = tc_ld(m);
  const View ce = planes_view(b.ce_rm, ldn, b.ce_ps);    // C_E   (m rows, K = n)
  const View cet = planes_view(b.ce_tr, ldm, b.ce_ps);   // C_E^T (n rows, K = m)
  RET(cudaMemsetAsync(b.dscal + 1, 0, 2 * sizeof(double), st));
  if (dir_right) {
    // warm start: rows of the current C_{i+1} (kold x n) -> Q (n x k)
    note_launch();
    warm_start_kernel<<<grid_for((long long)n * k), 256, 0, st>>>(warm, n, 1, kold, n, k, seed,
                                                                  b.seed_base, b.Q);
    // Y = C_E Q (m x k): A = C_E (m rows, K = n), B = Q^T (k rows, K = n)
    RET(tc_product(ce, f32_view(b.Q, idx_plain(1), idx_plain(k)), m, k, n, b.Y, k, b, st));
    note_launch();
    add_noise_kernel<<<grid_for((long long)m * k), 256, 0, st>>>(b.Y, (long long)m * k, b.ce_ss,
                                                                 inv_mn, seed + 7, b.seed_base);
    RET(cudaGetLastError());
    float* U = nullptr;
    RET(orthonormalise(b.Y, m, k, b, st, &U));
    RET(orth_check(U, m, k, b, st));
    RET(split_guard(k, b, st));
    // C_i = U (m x k); C_{i+1} = U^T C_E (k x n)
    note_launch();
    copy_f2d_kernel<<<grid_for((long long)m * k), 256, 0, st>>>(U, (long long)m * k, left);
    // U^T C_E (k x n): A = U^T (k rows, K = m), B = C_E^T (n rows, K = m)
    RET(tc_product(f32_view(U, idx_plain(1), idx_plain(k)), cet, k, n, m, b.out, n, b, st));
    note_launch();
    copy_f2d_kernel<<<grid_for((long long)k * n), 256, 0, st>>>(b.out, (long long)k * n, right);
    RET(cudaGetLastError());
  } else {
    // warm start: columns of the current C_i (m x kold) -> Q (m x k)
    note_launch();
    warm_start_kernel<<<grid_for((long long)m * k), 256, 0, st>>>(warm, 1, kold, kold, m, k, seed,
                                                                  b.seed_base, b.Q);
    // Z = C_E^T Q (n x k): A = C_E^T (n rows, K = m), B = Q^T (k rows, K = m)
    RET(tc_product(cet, f32_view(b.Q, idx_plain(1), idx_plain(k)), n, k, m, b.Y, k, b, st));
    note_launch();
    add_noise_kernel<<<grid_for((long long)n * k), 256, 0, st>>>(b.Y, (long long)n * k, b.ce_ss,
                                                                 inv_mn, seed + 7, b.seed_base);
    RET(cudaGetLastError());
    float* V = nullptr;
    RET(orthonormalise(b.Y, n, k, b, st, &V));
    RET(orth_check(V, n, k, b, st));
    RET(split_guard(k, b, st));
    // C_{i+1} = V^T (k x n); C_i = C_E V (m x k)
    note_launch();
    transpose_f2d_kernel<<<grid_for((long long)n * k), 256, 0, st>>>(V, n, k, right);
    // C_E V (m x k): A = C_E (m rows, K = n), B = V^T (k rows, K = n)
    RET(tc_product(ce, f32_view(V, idx_plain(1), idx_plain(k)), m, k, n, b.out, k, b, st));
    note_launch();
    copy_f2d_kernel<<<grid_for((long long)m * k), 256, 0, st>>>(b.out, (long long)m * k, left);
    RET(cudaGetLastError());
  }
  // ||centre||^2 for the discarded weight 1 - ||centre||^2 / ||C_E||^2
  double* centre = dir_right ? right : left;
  const long long nc = dir_right ? (long long)k * n : (long long)m * k;
  note_launch();
  sumsq_f64_kernel<<<grid_for(nc) < 304 ? grid_for(nc) : 304, 256, 0, st>>>(centre, nc,
                                                                            b.dscal + 1);
  RET(cudaGetLastError());
  if (disc_max) {
    note_launch();
    split_finish_kernel<<<1, 1, 0, st>>>(b.ce_ss, b.dscal, thresh, disc_max);
    RET(cudaGetLastError());
  }
  return cudaSuccess;
}
