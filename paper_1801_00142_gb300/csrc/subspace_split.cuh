// Warm-started subspace truncation of the tensor-core path (subspace_split.cu).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

struct SubspaceBuffers {
  float* Q;         // max(m, n) x k
  float* Y;         // max(m, n) x k
  float* out;       // m x n (k x n or m x k results)
  float* orth_part; // orthonormalisation: per-CTA partial sums
  float* orth_red;  // orthonormalisation: reduced sums
  double* orth_partd;  // orthonormalisation: per-CTA partial panel Grams (FP64)
  double* orth_redd;   // orthonormalisation: reduced panel Gram (FP64)
  unsigned* orth_bar;  // orthonormalisation: grid barrier words + status (4 words)
  int orth_max_ctas;
  float* scal;      // scratch scalars
  double* dscal;    // FP64 scratch scalars (3)
  __nv_bfloat16* pa;   // tensor-core operand planes (3 x 4cap x ld(4cap))
  __nv_bfloat16* pb;   // tensor-core operand planes (3 x 4cap x ld(4cap))
  long long psa, psb;  // their plane strides
  int* err;            // bounded-wait error flag of the tensor-core GEMM
};

// Largest k the orthonormalisation handles; wider splits take the exact path.
constexpr int SUBSPACE_MAX_K = 256;

// Orthonormalisations launched as one thread-block cluster (all contexts).
extern unsigned long long g_orth_cluster_calls;

// BF16 elements of pa and pb for bond capacity cap.
size_t subspace_plane_elems_a(int cap);
size_t subspace_plane_elems_b(int cap);

// Floats needed by the float buffers above for bond capacity cap (m, n <= 4 cap).
size_t subspace_buffer_floats(int cap);
// CTAs of the orthonormalisation kernel for rows <= 4 cap.
int subspace_orth_ctas(int cap);

// Split C_E (m x n, FP64 row-major) into left (m x k) and right (k x n), FP64.
// dir_right = 1 (left-to-right): left = U orthonormal, right = U^T C_E,
// warm = current C_{i+1} (kold x n, orthonormal rows).  dir_right = 0:
// right = V^T orthonormal rows, left = C_E V, warm = current C_i (m x kold).
// *orth_defect: max |Q^T Q - I| over the live columns of the orthonormal
// factor; the caller falls back to the exact split when it is too large.
// Synchronises the stream (reads FP64 norms).
cudaError_t subspace_split(const double* CE, int m, int n, int k, int dir_right,
                           const double* warm, int kold, double* left, double* right,
                           unsigned long long seed, const SubspaceBuffers& b, cudaStream_t st,
                           double* discarded, double* orth_defect);
