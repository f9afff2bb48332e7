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
// out[p][r][k] = src[p][k * sld + r] (plane-wise transpose), zero for K <= k < ld
cudaError_t transpose_planes(const __nv_bfloat16* src, long long sld, int rows, int K,
                             __nv_bfloat16* out, long long ld, int planes, long long sps,
                             long long ops, cudaStream_t st);
// out[r][k] = src[off(rv, r) + off(kv, k)] for each plane (plane strides sps -> ops)
cudaError_t relayout_planes(const __nv_bfloat16* src, Idx3 rv, Idx3 kv, int rows, int K,
                            __nv_bfloat16* out, long long ld, int planes, long long sps,
                            long long ops, cudaStream_t st);
// out[e] = sum_i part[i*n + e] in FP64
cudaError_t reduce_partials(const float* part, int splits, long long n, double* out,
                            cudaStream_t st);
cudaError_t f32_to_f64(const float* a, long long n, double* b, cudaStream_t st);
