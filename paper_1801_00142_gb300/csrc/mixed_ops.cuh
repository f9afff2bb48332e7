// Conversions and re-layouts of the tensor-core path (see mixed_ops.cu).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

// out[b][r][k] = split planes of src[b*sbs + off(rv, r) + off(kv, k)] for
// k < K, zero for K <= k < ld; planes = 2 or 3, plane stride ops.
cudaError_t to_planes(const double* src, Idx3 rv, Idx3 kv, long long sbs, int rows, int K,
                      int batch, __nv_bfloat16* out, long long ld, long long obs, int planes,
                      long long ops, cudaStream_t st);
cudaError_t to_planes_f32(const float* src, Idx3 rv, Idx3 kv, long long sbs, int rows, int K,
                          int batch, __nv_bfloat16* out, long long ld, long long obs, int planes,
                          long long ops, cudaStream_t st);
// out[e] = sum_i part[i*n + e] in FP64
cudaError_t reduce_partials(const float* part, int splits, long long n, double* out,
                            cudaStream_t st);
// C = sum of the split-K partials (m x n): FP64 into out, the three BF16
// planes (plane stride ps) row-major into prm [m][ldn] and transposed into
// ptr [n][ldm] (zero padding), and ||C||_F^2 into *ss (device scalar).
cudaError_t reduce_partials_planes(const float* part, int splits, int m, int n, double* out,
                                   __nv_bfloat16* prm, long long ldn, __nv_bfloat16* ptr,
                                   long long ldm, long long ps, double* ss, cudaStream_t st);
