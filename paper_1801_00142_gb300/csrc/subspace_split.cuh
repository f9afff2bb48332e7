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
  // C_E as BF16 planes in both orientations and its squared Frobenius norm,
  // written by reduce_partials_planes before subspace_split reads them
  __nv_bfloat16* ce_rm;   // [plane][m][tc_ld(n)]
  __nv_bfloat16* ce_tr;   // [plane][n][tc_ld(m)]
  long long ce_ps;        // plane stride of both (elements)
  double* ce_ss;          // ||C_E||_F^2 (device scalar)
  // scaled CholeskyQR2: packed Cholesky factor, column scaling, 1 / L_jj,
  // breakdown flag (0: the fast path succeeded)
  float* chol_L;          // w (w + 1) / 2 for a column block of width w
  float* chol_d;          // SUBSPACE_BLOCK_K
  float* chol_li;         // SUBSPACE_BLOCK_K
  int* chol_flag;         // [0] breakdown flag of the current call, [1] count of breakdowns,
                          // [2] full second pass flag, [3] its count, [4] deflated columns
  int orth_block;         // column-block width of the orthonormalisation (32..SUBSPACE_BLOCK_K)
  unsigned long long* seed_base;   // device counter mixed into the noise seeds (one per product)
  float* part;            // FP32 split-K partials of the small tensor-core products (may be
  size_t part_floats;     // shared with other split-K users: free during a split)
};

// Widest column block the one-block orthonormalisation kernels take, and the
// largest k of the blocked orthonormalisation; wider splits take the exact
// path.
constexpr int SUBSPACE_BLOCK_K = 256;
constexpr int SUBSPACE_MAX_K = 1024;

// Floats of chol_L (one column block).
constexpr size_t SUBSPACE_CHOL_FLOATS = (size_t)SUBSPACE_BLOCK_K * (SUBSPACE_BLOCK_K + 1) / 2;

// Orthonormalisations launched as one thread-block cluster (all contexts; and
// by the calling host thread).
extern unsigned long long g_orth_cluster_calls;
extern thread_local unsigned long long t_orth_cluster_calls;

// BF16 elements of pa and pb for bond capacity cap.
size_t subspace_plane_elems_a(int cap);
size_t subspace_plane_elems_b(int cap);

// Floats needed by the float buffers above for bond capacity cap (m, n <= 4 cap).
size_t subspace_buffer_floats(int cap);
// CTAs of the orthonormalisation kernel for rows <= 4 cap.
int subspace_orth_ctas(int cap);

// Split C_E (m x n) into left (m x k) and right (k x n), FP64.  C_E is read
// from b.ce_rm / b.ce_tr / b.ce_ss (its planes and norm, see above); the
// FP64 array CE itself is not read (the caller's exact fallback uses it).
// dir_right = 1 (left-to-right): left = U orthonormal, right = U^T C_E,
// warm = current C_{i+1} (kold x n, orthonormal rows).  dir_right = 0:
// right = V^T orthonormal rows, left = C_E V, warm = current C_i (m x kold).
// Everything stays on the device (no host read): the orthonormality defect
// max |Q^T Q - I| over the live columns of the orthonormal factor is left in
// *subspace_defect(b), from which the caller's exact fallback decides on the
// device; if disc_max is not null and the defect is <= thresh, the
// discarded weight 1 - ||kept||^2 / ||C_E||^2 is raised into *disc_max.
cudaError_t subspace_split(const double* CE, int m, int n, int k, int dir_right,
                           const double* warm, int kold, double* left, double* right,
                           unsigned long long seed, const SubspaceBuffers& b, cudaStream_t st,
                           double* disc_max, double thresh);
const double* subspace_defect(const SubspaceBuffers& b);
// Advance the device seed counter (once per product, inside a captured graph
// too, so that every doubling draws fresh noise).
cudaError_t subspace_next_seed(const SubspaceBuffers& b, cudaStream_t st);
