// Layout and precision conversions of the tensor-core path: FP64 tensors to
// BF16 split planes through strided views, and the FP64 reduction of split-K
// partial sums (alone, or fused with the planes of the result in both
// orientations).
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

__global__ void reduce_partials_kernel(const float* __restrict__ part, int splits, long long n,
                                       double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < splits; ++i) s += (double)part[i * n + e];
    out[e] = s;
  }
}


// One 32 x 32 tile of C = sum of the split-K partials: the FP64 result, its
// three BF16 planes in both orientations (row-major [m][ldn] and transposed
// [n][ldm], the K-major operands of C x and C^T x), and the tile's sum of
// squares added into *ss.  The transposed planes go through shared memory so
// that both the reads and the writes are coalesced; padding columns of both
// plane layouts are written as zero.
__global__ void reduce_partials_planes_kernel(const float* __restrict__ part, int splits, int m,
                                              int n, double* __restrict__ out,
                                              __nv_bfloat16* __restrict__ prm, long long ldn,
                                              __nv_bfloat16* __restrict__ ptr, long long ldm,
                                              long long ps, double* ss) {
  // the three planes of the tile, kept for the transposed writes (FP64
  // arithmetic is slow on this GPU: the partials are summed in FP32 with a
  // compensation term, which keeps the sum to about FP64 accuracy for the
  // few splits, and the planes are cut from that pair in FP32)
  __shared__ __nv_bfloat16 tp[3][32][34];
  __shared__ double red[8];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8 threads
  const int n0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
  const long long mn = (long long)m * n;
  double acc = 0.0;
  for (int y = ty; y < 32; y += 8) {
    const int r = m0 + y, c = n0 + tx;
    float hi = 0.f, lo = 0.f;
    if (r < m && c < n) {
      const long long e = (long long)r * n + c;
      for (int i = 0; i < splits; ++i) {
        // two-sum: hi + lo = old hi + part exactly, errors gathered in lo
        const float x = part[i * mn + e];
        const float t = hi + x;
        const float bp = t - hi;
        lo += (hi - (t - bp)) + (x - bp);
        hi = t;
      }
      const double v = (double)hi + (double)lo;
      out[e] = v;
      acc = fma(v, v, acc);
    }
    const __nv_bfloat16 p0 = __float2bfloat16_rn(hi);
    const float r1 = (hi - __bfloat162float(p0)) + lo;
    const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
    tp[0][y][tx] = p0;
    tp[1][y][tx] = p1;
    tp[2][y][tx] = p2;
    if (r < m && c < ldn) {
      const long long o = (long long)r * ldn + c;
      prm[o] = p0;
      prm[o + ps] = p1;
      prm[o + 2 * ps] = p2;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (tx == 0) red[ty] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    atomicAdd(ss, t);
  }
  for (int y = ty; y < 32; y += 8) {
    const int r = n0 + y, c = m0 + tx;   // row r of C^T, column c
    if (r < n && c < ldm) {
      const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
      const bool in = c < m;
      const long long o = (long long)r * ldm + c;
      ptr[o] = in ? tp[0][tx][y] : z;
      ptr[o + ps] = in ? tp[1][tx][y] : z;
      ptr[o + 2 * ps] = in ? tp[2][tx][y] : z;
    }
  }
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

cudaError_t reduce_partials(const float* part, int splits, long long n, double* out,
                            cudaStream_t st) {
  note_launch();
  reduce_partials_kernel<<<grid_for(n), 256, 0, st>>>(part, splits, n, out);
  return cudaGetLastError();
}


cudaError_t reduce_partials_planes(const float* part, int splits, int m, int n, double* out,
                                   __nv_bfloat16* prm, long long ldn, __nv_bfloat16* ptr,
                                   long long ldm, long long ps, double* ss, cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ss, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
  note_launch();
  reduce_partials_planes_kernel<<<grid, 256, 0, st>>>(part, splits, m, n, out, prm, ldn, ptr, ldm,
                                                      ps, ss);
  return cudaGetLastError();
}
