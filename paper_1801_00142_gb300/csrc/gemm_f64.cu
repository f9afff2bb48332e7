// FP64 CUDA-core tensor contraction as a batched GEMM over strided views.
//
// Every contraction of the XTRG compression (the environment substeps of
// Fig. VMPO(c), the two-site overlap C_E of Eq. LSEProd and the transfer
// contractions of the traces) is a batched GEMM whose row, column and
// contraction indices are up to three-level strided views of the stored
// tensors (struct Idx3), so no permutation pass is needed between steps.
//
// This is the FP64 path; it also serves the canonicalisation and the traces
// of the tensor-core path.  On GB300 the FP64 rate
// is a small fraction of the FP32 rate, so the FP64 kernel is bound by FP64
// issue: a 64x64 output tile per 256-thread CTA, 4x4 outputs per thread, k
// staged 16 at a time through shared memory, with the per-tile view offsets
// precomputed once per tile.
#include "common.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T, typename G>
__global__ void __launch_bounds__(NT) gemm_kernel(G g, int a_kfast, int b_kfast) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ long long offAm[BM], offBn[BN], offAk[BK], offBk[BK];

  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long long b = blockIdx.z;
  const T* A = g.A + b * g.sab;
  const T* B = g.B + b * g.sbb;

  if (tid < BM) {
    int m = m0 + tid;
    offAm[tid] = (m < g.M) ? idx_off(g.am, m) : 0;
  } else if (tid < BM + BN) {
    int n = n0 + tid - BM;
    offBn[tid - BM] = (n < g.N) ? idx_off(g.bn, n) : 0;
  }

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    __syncthreads();
    if (tid < BK) {
      int k = k0 + tid;
      offAk[tid] = (k < g.K) ? idx_off(g.ak, k) : 0;
    } else if (tid >= 32 && tid < 32 + BK) {
      int k = k0 + tid - 32;
      offBk[tid - 32] = (k < g.K) ? idx_off(g.bk, k) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      int e = tid + q * NT;
      int mi, ki;
      if (a_kfast) { ki = e % BK; mi = e / BK; } else { mi = e % BM; ki = e / BM; }
      int m = m0 + mi, k = k0 + ki;
      As[ki][mi] = (m < g.M && k < g.K) ? A[offAm[mi] + offAk[ki]] : T(0);
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      int e = tid + q * NT;
      int ni, ki;
      if (b_kfast) { ki = e % BK; ni = e / BK; } else { ni = e % BN; ki = e / BN; }
      int n = n0 + ni, k = k0 + ki;
      Bs[ki][ni] = (n < g.N && k < g.K) ? B[offBk[ki] + offBn[ni]] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
  }

  T* C = g.C + b * g.scb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
    long long om = idx_off(g.cm, m);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      long long o = om + idx_off(g.cn, n);
      T v = (T)g.alpha * acc[i][j];
      if (g.beta != 0.0) v += (T)g.beta * C[o];
      C[o] = v;
    }
  }
}

int innermost_unit(const Idx3& d) {
  // the fastest-varying sub-index of the view has unit stride
  if (d.n0 > 1) return d.s0 == 1;
  if (d.n1 > 1) return d.s1 == 1;
  return d.s2 == 1;
}

template <typename T, typename G>
cudaError_t launch(const G& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.K <= 0 || g.batch > 65535) return cudaErrorInvalidValue;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  int a_kfast = innermost_unit(g.ak) && !innermost_unit(g.am);
  int b_kfast = innermost_unit(g.bk) && !innermost_unit(g.bn);
  note_launch();
  gemm_kernel<T, G><<<grid, NT, 0, st>>>(g, a_kfast, b_kfast);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_f64(const GemmF64& g, cudaStream_t st) { return launch<double>(g, st); }
