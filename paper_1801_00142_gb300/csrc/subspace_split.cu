// Truncation of the tensor-core path: one warm-started subspace step with
// shifted CholeskyQR3 orthonormalisation, in FP32.
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
// carry weight below eta^2 relative.  orth() is block classical Gram-Schmidt
// with reorthogonalisation (panels of 32 columns, three projection passes
// against the earlier panels as FP32 GEMMs, then three in-panel passes in
// shared memory): unlike Cholesky-based QR it does not square the condition
// number, so columns without weight in C_E become arbitrary orthonormal
// completions instead of breaking the factorisation.
#include <math.h>

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
                                  int kold, int rows, int k, unsigned long long seed,
                                  float* __restrict__ Q) {
  const long long total = (long long)rows * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / k), j = (int)(e % k);
    Q[e] = j < kold ? (float)S[j * sj + r * sr] : hash_uniform(seed * 0x100000001B3ull + e);
  }
}

__global__ void add_noise_kernel(float* __restrict__ Y, long long n, float eta,
                                 unsigned long long seed) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    Y[e] += eta * hash_uniform(seed ^ (0xD1B54A32D192ED03ull * (e + 1)));
}

__global__ void copy_d2f_kernel(const double* __restrict__ a, long long n, float* __restrict__ b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    b[e] = (float)a[e];
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

// In-panel orthonormalisation: columns [j0, j0+w) of Y (rows x k, row-major)
// against each other, three passes per column, then normalisation.  One CTA;
// the panel lives in shared memory.
constexpr int PANEL = 32;
constexpr int PSTR = PANEL + 1;   // padded row stride: conflict-free shared-memory columns

__global__ void __launch_bounds__(1024) panel_orth_kernel(float* __restrict__ Y, int rows, int k,
                                                          int j0, int w) {
  extern __shared__ float V[];    // V[r * PSTR + c]
  __shared__ float dots[PANEL];
  __shared__ float red[32];
  const int tid = threadIdx.x, lane = tid % 32, wid = tid / 32, nw = blockDim.x / 32;
  for (int e = tid; e < rows * w; e += blockDim.x) {
    const int r = e / w, c = e % w;
    V[r * PSTR + c] = Y[(long long)r * k + j0 + c];
  }
  __syncthreads();
  for (int c = 0; c < w; ++c) {
    for (int pass = 0; pass < 3; ++pass) {
      if (c > 0) {
        // dots[c'] = <v_c', v_c> for c' < c, one warp per c'
        for (int cp = wid; cp < c; cp += nw) {
          float s = 0.f;
          for (int r = lane; r < rows; r += 32) s = fmaf(V[r * PSTR + cp], V[r * PSTR + c], s);
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) dots[cp] = s;
        }
        __syncthreads();
        for (int r = tid; r < rows; r += blockDim.x) {
          float v = V[r * PSTR + c];
          for (int cp = 0; cp < c; ++cp) v = fmaf(-dots[cp], V[r * PSTR + cp], v);
          V[r * PSTR + c] = v;
        }
        __syncthreads();
      }
    }
    float s = 0.f;
    for (int r = tid; r < rows; r += blockDim.x) s = fmaf(V[r * PSTR + c], V[r * PSTR + c], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[wid] = s;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int i = 0; i < nw; ++i) t += red[i];
      dots[0] = t > 0.f ? rsqrtf(t) : 0.f;
    }
    __syncthreads();
    const float inv = dots[0];
    for (int r = tid; r < rows; r += blockDim.x) V[r * PSTR + c] *= inv;
    __syncthreads();
  }
  for (int e = tid; e < rows * w; e += blockDim.x) {
    const int r = e / w, c = e % w;
    Y[(long long)r * k + j0 + c] = V[r * PSTR + c];
  }
}

GemmF32 g32(int M, int N, int K, const float* A, Idx3 am, Idx3 ak, const float* B, Idx3 bk,
            Idx3 bn, float* C, Idx3 cm, Idx3 cn) {
  GemmF32 g;
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.A = A; g.am = am; g.ak = ak; g.sab = 0;
  g.B = B; g.bk = bk; g.bn = bn; g.sbb = 0;
  g.C = C; g.cm = cm; g.cn = cn; g.scb = 0;
  g.alpha = 1.0; g.beta = 0.0;
  return g;
}

#define RET(x)                                 \
  do {                                         \
    cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) return _e;          \
  } while (0)

// Y (rows x k, row-major FP32) <- orthonormal basis of its column space
// (block classical Gram-Schmidt, three passes).  S: k x PANEL scratch.
cudaError_t block_cgs(float* Y, int rows, int k, float* S, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    RET(cudaFuncSetAttribute(panel_orth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             1028 * PSTR * (int)sizeof(float)));
    attr = true;
  }
  if (rows > 1028) return cudaErrorInvalidValue;
  for (int j0 = 0; j0 < k; j0 += PANEL) {
    const int w = k - j0 < PANEL ? k - j0 : PANEL;
    for (int pass = 0; pass < 3 && j0 > 0; ++pass) {
      // S = Q[:, :j0]^T Y[:, j0:j0+w]
      RET(gemm_f32(g32(j0, w, rows, Y, idx_plain(1), idx_plain(k), Y + j0, idx_plain(k),
                       idx_plain(1), S, idx_plain(w), idx_plain(1)),
                   st));
      // Y[:, j0:j0+w] -= Q[:, :j0] S
      GemmF32 g = g32(rows, w, j0, Y, idx_plain(k), idx_plain(1), S, idx_plain(w), idx_plain(1),
                      Y + j0, idx_plain(k), idx_plain(1));
      g.alpha = -1.0;
      g.beta = 1.0;
      RET(gemm_f32(g, st));
    }
    note_launch();
    panel_orth_kernel<<<1, 1024, (size_t)rows * PSTR * sizeof(float), st>>>(Y, rows, k, j0, w);
    RET(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace

size_t subspace_plane_elems_a(int cap) { return 3 * (size_t)(4 * cap) * tc_ld(4 * cap); }
size_t subspace_plane_elems_b(int cap) { return 3 * (size_t)(4 * cap) * tc_ld(4 * cap); }

namespace {
// C (M x N, FP32 row-major, ldc) = A B^T on the tensor cores, A and B given as
// FP64 or FP32 views through to_planes (3 planes, 6 products).
struct View {
  const double* d;
  const float* f;
  Idx3 rv, kv;
};

cudaError_t tc_product(const View& a, const View& b, int M, int N, int K, float* C, long long ldc,
                       const SubspaceBuffers& buf, cudaStream_t st) {
  const long long ld = tc_ld(K);
  const long long psa = (long long)M * ld, psb = (long long)N * ld;
  if (psa > buf.psa || psb > buf.psb) return cudaErrorInvalidValue;
  if (a.d) RET(to_planes(a.d, a.rv, a.kv, 0, M, K, 1, buf.pa, ld, 0, 3, buf.psa, st));
  else RET(to_planes_f32(a.f, a.rv, a.kv, 0, M, K, 1, buf.pa, ld, 0, 3, buf.psa, st));
  if (b.d) RET(to_planes(b.d, b.rv, b.kv, 0, N, K, 1, buf.pb, ld, 0, 3, buf.psb, st));
  else RET(to_planes_f32(b.f, b.rv, b.kv, 0, N, K, 1, buf.pb, ld, 0, 3, buf.psb, st));
  TcOperand A{buf.pa, 3, M, K, ld, 0, buf.psa, 1};
  TcOperand B{buf.pb, 3, N, K, ld, 0, buf.psb, 1};
  TcOutput o;
  memset(&o, 0, sizeof o);
  o.mode = TC_OUT_F32;
  o.f32 = C;
  o.cm = idx_plain(ldc);
  o.cn = idx_plain(1);
  o.alpha = 1.0;
  return tc_gemm(A, B, M, N, K, 1, 6, 1, o, buf.err, st);
}
}  // namespace

size_t subspace_buffer_floats(int cap) {
  const size_t m = 4 * (size_t)cap;
  return m * m /*CE32*/ + m * cap /*Q*/ + m * cap /*Y*/ + (size_t)cap * cap * 2 /*G, L*/ +
         m * m /*out*/ + 64;
}

cudaError_t subspace_split(const double* CE, int m, int n, int k, int dir_right,
                           const double* warm, int kold, double* left, double* right,
                           unsigned long long seed, const SubspaceBuffers& b, cudaStream_t st,
                           double* discarded) {
  if (k > 256 || k > m || k > n) return cudaErrorInvalidValue;
  const long long mn = (long long)m * n;
  // ||C_E||^2 (FP64)
  RET(cudaMemsetAsync(b.dscal, 0, 2 * sizeof(double), st));
  note_launch();
  sumsq_f64_kernel<<<grid_for(mn) < 304 ? grid_for(mn) : 304, 256, 0, st>>>(CE, mn, b.dscal);
  RET(cudaGetLastError());
  double tot = 0.0;
  RET(cudaMemcpyAsync(&tot, b.dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
  RET(cudaStreamSynchronize(st));
  const float eta = (float)(1e-5 * sqrt(tot / ((double)m * n)));
  if (dir_right) {
    // warm start: rows of the current C_{i+1} (kold x n) -> Q (n x k)
    note_launch();
    warm_start_kernel<<<grid_for((long long)n * k), 256, 0, st>>>(warm, n, 1, kold, n, k, seed,
                                                                  b.Q);
    // Y = C_E Q (m x k): A = C_E (m rows, K = n), B = Q^T (k rows, K = n)
    RET(tc_product(View{CE, nullptr, idx_plain(n), idx_plain(1)},
                   View{nullptr, b.Q, idx_plain(1), idx_plain(k)}, m, k, n, b.Y, k, b, st));
    note_launch();
    add_noise_kernel<<<grid_for((long long)m * k), 256, 0, st>>>(b.Y, (long long)m * k, eta,
                                                                 seed + 7);
    RET(cudaGetLastError());
    RET(block_cgs(b.Y, m, k, b.G, st));
    // C_i = U (m x k); C_{i+1} = U^T C_E (k x n)
    note_launch();
    copy_f2d_kernel<<<grid_for((long long)m * k), 256, 0, st>>>(b.Y, (long long)m * k, left);
    // U^T C_E (k x n): A = U^T (k rows, K = m), B = C_E^T (n rows, K = m)
    RET(tc_product(View{nullptr, b.Y, idx_plain(1), idx_plain(k)},
                   View{CE, nullptr, idx_plain(1), idx_plain(n)}, k, n, m, b.out, n, b, st));
    note_launch();
    copy_f2d_kernel<<<grid_for((long long)k * n), 256, 0, st>>>(b.out, (long long)k * n, right);
    RET(cudaGetLastError());
  } else {
    // warm start: columns of the current C_i (m x kold) -> Q (m x k)
    note_launch();
    warm_start_kernel<<<grid_for((long long)m * k), 256, 0, st>>>(warm, 1, kold, kold, m, k, seed,
                                                                  b.Q);
    // Z = C_E^T Q (n x k): A = C_E^T (n rows, K = m), B = Q^T (k rows, K = m)
    RET(tc_product(View{CE, nullptr, idx_plain(1), idx_plain(n)},
                   View{nullptr, b.Q, idx_plain(1), idx_plain(k)}, n, k, m, b.Y, k, b, st));
    note_launch();
    add_noise_kernel<<<grid_for((long long)n * k), 256, 0, st>>>(b.Y, (long long)n * k, eta,
                                                                 seed + 7);
    RET(cudaGetLastError());
    RET(block_cgs(b.Y, n, k, b.G, st));
    // C_{i+1} = V^T (k x n); C_i = C_E V (m x k)
    note_launch();
    transpose_f2d_kernel<<<grid_for((long long)n * k), 256, 0, st>>>(b.Y, n, k, right);
    // C_E V (m x k): A = C_E (m rows, K = n), B = V^T (k rows, K = n)
    RET(tc_product(View{CE, nullptr, idx_plain(n), idx_plain(1)},
                   View{nullptr, b.Y, idx_plain(1), idx_plain(k)}, m, k, n, b.out, k, b, st));
    note_launch();
    copy_f2d_kernel<<<grid_for((long long)m * k), 256, 0, st>>>(b.out, (long long)m * k, left);
    RET(cudaGetLastError());
  }
  // discarded weight = 1 - ||centre||^2 / ||C_E||^2
  double* centre = dir_right ? right : left;
  const long long nc = dir_right ? (long long)k * n : (long long)m * k;
  note_launch();
  sumsq_f64_kernel<<<grid_for(nc) < 304 ? grid_for(nc) : 304, 256, 0, st>>>(centre, nc,
                                                                            b.dscal + 1);
  RET(cudaGetLastError());
  double kept = 0.0;
  RET(cudaMemcpyAsync(&kept, b.dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  RET(cudaStreamSynchronize(st));
  *discarded = tot > 0.0 ? fmax(0.0, 1.0 - kept / tot) : 0.0;
  return cudaSuccess;
}
