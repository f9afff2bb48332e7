// Internal helpers behind the FP64-in / FP64-out tensor-core GEMM entry points
// (xtrg_tc_gemm with a caller workspace, xtrg_tc_gemm_static with a fixed
// device array): one scratch layout and one code path for both.
#pragma once
#include <stddef.h>

#include <cuda_runtime.h>

#include "../../include/xtrg.h"

// Byte offsets of the scratch of one call: A planes [0, a), B planes
// [a, a + b), FP32 split-K partials [a + b, a + b + part), then an int error
// flag; total includes the flag's 256-byte slot.
struct TcGemmScratch {
  size_t a, b, part, total;
};
// b_kn: B given as batch x K x N (C = A B) instead of batch x N x K (C = A B^T).
TcGemmScratch tc_gemm_scratch(int M, int N, int K, int batch, int planes, int splitk,
                              bool b_kn = false);

// XTRG_EINVAL for arguments xtrg_tc_gemm rejects, else XTRG_OK.
xtrg_status tc_gemm_check_args(const double* A, const double* B, double* C, int M, int N, int K,
                               int batch, int planes, int nprod, int splitk);

// C = A B^T on the tensor cores using the scratch at base (256-byte aligned,
// tc_gemm_scratch(...).total bytes); synchronises st.
xtrg_status tc_gemm_run(const double* A, const double* B, double* C, int M, int N, int K, int batch,
                        int planes, int nprod, int splitk, char* base, cudaStream_t st,
                        bool b_kn = false);
