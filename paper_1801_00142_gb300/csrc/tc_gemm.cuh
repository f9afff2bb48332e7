// Tensor-core GEMM for sm_103a: tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulation in tensor memory), operands staged by TMA with 128-byte
// swizzle, warp-specialised producer / MMA issuer / epilogue.
//
// Each operand is a 4-D tensor [plane][batch][rows][k] (K-major) or
// [plane][batch][k][rows] (MN-major) of BF16 whose planes hold a split
// x ~= x0 + x1 (+ x2) of a higher-precision value; the
// product is accumulated as sum over the requested (plane_a, plane_b) pairs,
// e.g. x0y0 + x0y1 + x1y0 (3 products, ~16 significant bits) or the six
// products with plane index sum <= 2 (~24 bits).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

enum TcOutMode {
  TC_OUT_F32 = 0,      // FP32 values scattered through (cm, cn, scb)
  TC_OUT_BF16P = 1,    // BF16 split planes scattered through (cm, cn, scb)
  TC_OUT_PARTIAL = 2   // FP32 split-K partials, plain [split][batch][M][N]
};

struct TcOperand {
  const __nv_bfloat16* base;   // plane 0, batch 0, row 0, k 0
  int planes;
  int rows, k;                 // logical sizes (k is the contraction length)
  long long ld;                // leading stride in elements (multiple of 8), see mn_major
  long long batch_stride;      // elements (0: operand shared by all batches)
  long long plane_stride;      // elements
  int batches;                 // 1 if shared
  int mn_major = 0;            // 0: element (r, k) at r*ld + k (K-major);
                               // 1: element (r, k) at k*ld + r (MN-major, rows contiguous)
};

struct TcOutput {
  int mode;
  float* f32;
  __nv_bfloat16* bf16;
  int planes;                  // BF16 planes written (2 or 3)
  long long plane_stride;
  Idx3 cm, cn;
  long long scb;
  double alpha;
};

// C[b] = alpha * sum_products A[b] * B[b]^T (A: M x K, B: N x K, both K-major).
// nprod in {1, 3, 6}; splitk >= 1 (only with TC_OUT_PARTIAL).
cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, int M, int N, int K, int batch,
                    int nprod, int splitk, const TcOutput& out, int* dev_err, cudaStream_t st);

// Rows needed in the padded row stride of an operand buffer with k columns.
static inline long long tc_ld(long long k) { return (k + 7) / 8 * 8; }
