// Tensor-core (tcgen05) contraction path; see mixed.cu.
#pragma once
#include "common.cuh"

struct MixedCtx;

// Device workspace the tensor-core path needs for a chain of L sites with
// bond capacity cap and Hamiltonian bond DH (0 if the path is not available).
size_t mixed_workspace_bytes(int L, int cap, int DH);
cudaError_t mixed_create(MixedCtx** out, char* ws, size_t bytes, int L, int cap, int DH);
// Called once per product before its contractions (site tensors of rho).
cudaError_t mixed_prepare(MixedCtx* m, const int* dims, double* const* sites, cudaStream_t st);
// Same contract as gemm_f64, computed on the tensor cores.
cudaError_t mixed_gemm(MixedCtx* m, const GemmF64& g, cudaStream_t st);
void mixed_destroy(MixedCtx* m);
