// Warm-started subspace truncation of the tensor-core path (subspace_split.cu).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

struct SubspaceBuffers {
  float* CE32;      // m x n
  float* Q;         // max(m, n) x k
  float* Y;         // max(m, n) x k
  float* G;         // k x k
  float* L;         // k x k
  float* out;       // m x n (k x n or m x k results)
  float* scal;      // scratch scalars
  double* dscal;    // FP64 scratch scalars (2)
  __nv_bfloat16* pa;   // tensor-core operand planes (3 x 4cap x ld(4cap))
  __nv_bfloat16* pb;   // tensor-core operand planes (3 x 4cap x ld(4cap))
  long long psa, psb;  // their plane strides
  int* err;            // bounded-wait error flag of the tensor-core GEMM
};

// BF16 elements of pa and pb for bond capacity cap.
size_t subspace_plane_elems_a(int cap);
size_t subspace_plane_elems_b(int cap);

// Floats needed by the buffers above for bond capacity cap (m, n <= 4 cap).
size_t subspace_buffer_floats(int cap);

// Split C_E (m x n, FP64 row-major) into left (m x k) and right (k x n), FP64.
// dir_right = 1 (left-to-right): left = U orthonormal, right = U^T C_E,
// warm = current C_{i+1} (kold x n, orthonormal rows).  dir_right = 0:
// right = V^T orthonormal rows, left = C_E V, warm = current C_i (m x kold).
// Synchronises the stream (reads two FP64 norms).
cudaError_t subspace_split(const double* CE, int m, int n, int k, int dir_right,
                           const double* warm, int kold, double* left, double* right,
                           unsigned long long seed, const SubspaceBuffers& b, cudaStream_t st,
                           double* discarded);
