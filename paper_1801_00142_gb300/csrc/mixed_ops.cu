// Layout and precision conversions of the tensor-core path: FP64 tensors to
// BF16 split planes through strided views, plane-preserving re-layouts, and
// the FP64 reduction of split-K partial sums.
#include <cuda_bf16.h>

#include "mixed_ops.cuh"

namespace {

inline int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

// out[b][r][k] (row stride ld, batch stride obs, plane stride ops) =
// split(src[b*sbs + off(rv, r) + off(kv, k)]); padding columns k in [K, ld) = 0
template <typename S>
__global__ void to_planes_kernel(const S* __restrict__ src, Idx3 rv, Idx3 kv, long long sbs,
                                 int rows, int K, int batch, __nv_bfloat16* __restrict__ out,
                                 long long ld, long long obs, int planes, long long ops) {
  const long long per = (long long)rows * ld;
  const long long total = per * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / per);
    const long long w = e % per;
    const int r = (int)(w / ld), k = (int)(w % ld);
    double x = 0.0;
    if (k < K) x = (double)src[b * sbs + idx_off(rv, r) + idx_off(kv, k)];
    const __nv_bfloat16 p0 = __double2bfloat16(x);
    const double r1 = x - (double)__bfloat162float(p0);
    const __nv_bfloat16 p1 = __double2bfloat16(r1);
    const long long o = b * obs + (long long)r * ld + k;
    out[o] = p0;
    out[o + ops] = p1;
    if (planes > 2) out[o + 2 * ops] = __double2bfloat16(r1 - (double)__bfloat162float(p1));
  }
}

__global__ void relayout_planes_kernel(const __nv_bfloat16* __restrict__ src, Idx3 rv, Idx3 kv,
                                       int rows, int K, __nv_bfloat16* __restrict__ out,
                                       long long ld, int planes, long long sps, long long ops) {
  const long long per = (long long)rows * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), k = (int)(e % ld);
    const long long so = (k < K) ? idx_off(rv, r) + idx_off(kv, k) : -1;
    for (int p = 0; p < planes; ++p)
      out[e + p * ops] = so >= 0 ? src[so + p * sps] : __float2bfloat16_rn(0.f);
  }
}

// out[p][r][k] = src[p][k][r] for r < rows, k < K (32 x 32 tiles through shared
// memory, coalesced on both sides); padding columns K <= k < ld are zeroed.
__global__ void transpose_planes_kernel(const __nv_bfloat16* __restrict__ src, long long sld,
                                        int rows, int K, __nv_bfloat16* __restrict__ out,
                                        long long ld, long long sps, long long ops) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int p = blockIdx.z;
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const __nv_bfloat16* sp = src + p * sps;
  __nv_bfloat16* op = out + p * ops;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8 threads
  for (int y = ty; y < 32; y += 8) {
    const int k = k0 + y, r = r0 + tx;
    tile[y][tx] = (k < K && r < rows) ? sp[(long long)k * sld + r] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int r = r0 + y, k = k0 + tx;
    if (r < rows && k < ld) op[(long long)r * ld + k] = tile[tx][y];
  }
}

__global__ void reduce_partials_kernel(const float* __restrict__ part, int splits, long long n,
                                       double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < splits; ++i) s += (double)part[i * n + e];
    out[e] = s;
  }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ a, long long n, double* __restrict__ b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    b[e] = (double)a[e];
}

}  // namespace

cudaError_t to_planes(const double* src, Idx3 rv, Idx3 kv, long long sbs, int rows, int K,
                      int batch, __nv_bfloat16* out, long long ld, long long obs, int planes,
                      long long ops, cudaStream_t st) {
  long long total = (long long)rows * ld * batch;
  if (total <= 0) return cudaSuccess;
  note_launch();
  to_planes_kernel<double><<<grid_for(total), 256, 0, st>>>(src, rv, kv, sbs, rows, K, batch, out,
                                                            ld, obs, planes, ops);
  return cudaGetLastError();
}

cudaError_t to_planes_f32(const float* src, Idx3 rv, Idx3 kv, long long sbs, int rows, int K,
                          int batch, __nv_bfloat16* out, long long ld, long long obs, int planes,
                          long long ops, cudaStream_t st) {
  long long total = (long long)rows * ld * batch;
  if (total <= 0) return cudaSuccess;
  note_launch();
  to_planes_kernel<float><<<grid_for(total), 256, 0, st>>>(src, rv, kv, sbs, rows, K, batch, out,
                                                           ld, obs, planes, ops);
  return cudaGetLastError();
}

cudaError_t transpose_planes(const __nv_bfloat16* src, long long sld, int rows, int K,
                             __nv_bfloat16* out, long long ld, int planes, long long sps,
                             long long ops, cudaStream_t st) {
  if (rows <= 0 || ld <= 0) return cudaSuccess;
  dim3 grid((rows + 31) / 32, (int)((ld + 31) / 32), planes);
  note_launch();
  transpose_planes_kernel<<<grid, 256, 0, st>>>(src, sld, rows, K, out, ld, sps, ops);
  return cudaGetLastError();
}

cudaError_t relayout_planes(const __nv_bfloat16* src, Idx3 rv, Idx3 kv, int rows, int K,
                            __nv_bfloat16* out, long long ld, int planes, long long sps,
                            long long ops, cudaStream_t st) {
  long long total = (long long)rows * ld;
  if (total <= 0) return cudaSuccess;
  note_launch();
  relayout_planes_kernel<<<grid_for(total), 256, 0, st>>>(src, rv, kv, rows, K, out, ld, planes,
                                                          sps, ops);
  return cudaGetLastError();
}

cudaError_t reduce_partials(const float* part, int splits, long long n, double* out,
                            cudaStream_t st) {
  note_launch();
  reduce_partials_kernel<<<grid_for(n), 256, 0, st>>>(part, splits, n, out);
  return cudaGetLastError();
}

cudaError_t f32_to_f64(const float* a, long long n, double* b, cudaStream_t st) {
  note_launch();
  f32_to_f64_kernel<<<grid_for(n), 256, 0, st>>>(a, n, b);
  return cudaGetLastError();
}
