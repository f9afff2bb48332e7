// Small MPO kernels: the exact (fat) product used as the initial guess of the
// series products, the direct sum "alpha*P + I" of the Horner steps of
// Eq. RhoTau, and FP64 fill/scale/norm helpers used by the normalisation.
#include "common.cuh"

unsigned long long g_xtrg_launches = 0;
thread_local unsigned long long t_xtrg_launches = 0;

namespace {

inline int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

// G[(a,b)][s][u][(a',b')] = sum_t A[a][t][s][a'] * B[b][t][u][b']   (the
// operator A^T B with Kronecker-fused bonds, bond dimension Da*Db)
__global__ void exact_product_kernel(const double* __restrict__ A, int la, int ra,
                                     const double* __restrict__ B, int lb, int rb,
                                     double* __restrict__ G) {
  const long long R = (long long)ra * rb;
  const long long total = (long long)la * lb * 4 * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long rr = e % R;
    long long t1 = e / R;
    int u = (int)(t1 % 2);
    int s = (int)((t1 / 2) % 2);
    long long ll = t1 / 4;
    int a = (int)(ll / lb), b = (int)(ll % lb);
    int a2 = (int)(rr / rb), b2 = (int)(rr % rb);
    double v = 0.0;
#pragma unroll
    for (int t = 0; t < 2; ++t)
      v += A[(((long long)a * 2 + t) * 2 + s) * ra + a2] * B[(((long long)b * 2 + t) * 2 + u) * rb + b2];
    G[e] = v;
  }
}

// Site pos of alpha*P + Q with block-diagonal bonds; the first site
// concatenates along the right bond, the last along the left bond.
__global__ void direct_sum_kernel(const double* __restrict__ P, int pl, int pr, double alpha,
                                  const double* __restrict__ Q, int ql, int qr, int first,
                                  int last, int ol, int orr, double* __restrict__ out) {
  const long long total = (long long)ol * 4 * orr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e % orr);
    int st = (int)((e / orr) % 4);
    int l = (int)(e / (4LL * orr));
    double v = 0.0;
    // P block occupies rows [0, pl) (or all rows on the first site) and
    // columns [0, pr) (or all columns on the last site)
    bool inP_l = first ? true : (l < pl);
    bool inP_r = last ? true : (r < pr);
    bool inQ_l = first ? true : (l >= pl);
    bool inQ_r = last ? true : (r >= pr);
    if (first && last) {
      // a one-site chain: plain sum
      v = alpha * P[(long long)st * pr + r] + Q[(long long)st * qr + r];
    } else if (first) {
      if (r < pr) v = alpha * P[((long long)l * 4 + st) * pr + r];
      else v = Q[((long long)l * 4 + st) * qr + (r - pr)];
    } else if (last) {
      if (l < pl) v = P[((long long)l * 4 + st) * pr + r];
      else v = Q[((long long)(l - pl) * 4 + st) * qr + r];
    } else if (inP_l && inP_r) {
      v = P[((long long)l * 4 + st) * pr + r];
    } else if (inQ_l && inQ_r) {
      v = Q[((long long)(l - pl) * 4 + st) * qr + (r - pr)];
    }
    out[e] = v;
  }
}

__global__ void fill_kernel(double* p, double v, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    p[e] = v;
}

__global__ void scale_kernel(double* p, double v, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    p[e] *= v;
}

// p *= 1 / sqrt(*ss) if *ss is positive and finite (else p is left as it is)
__global__ void scale_rsqrt_kernel(double* p, const double* __restrict__ ss, long long n) {
  const double v = *ss;
  if (!(v > 0.0) || !isfinite(v)) return;
  const double f = 1.0 / sqrt(v);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    p[e] *= f;
}

// single-CTA sum of squares (the tensors reduced here are small: one site)
__global__ void sumsq_kernel(const double* __restrict__ p, long long n, double* out) {
  __shared__ double red[32];
  double a = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) a = fma(p[e], p[e], a);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += red[i];
    *out = s;
  }
}

__global__ void identity_site_kernel(double* p) {
  if (threadIdx.x < 4) p[threadIdx.x] = (threadIdx.x == 0 || threadIdx.x == 3) ? 1.0 : 0.0;
}

}  // namespace

cudaError_t mpo_exact_product(const double* A, int la, int ra, const double* B, int lb, int rb,
                              double* G, cudaStream_t st) {
  long long total = (long long)la * lb * 4 * ra * rb;
  note_launch();
  exact_product_kernel<<<grid_for(total), 256, 0, st>>>(A, la, ra, B, lb, rb, G);
  return cudaGetLastError();
}

cudaError_t mpo_direct_sum_site(const double* P, int pl, int pr, double alpha, const double* Q,
                                int ql, int qr, int pos, int L, double* out, cudaStream_t st) {
  int first = pos == 0, last = pos == L - 1;
  int ol = first ? 1 : pl + ql;
  int orr = last ? 1 : pr + qr;
  long long total = (long long)ol * 4 * orr;
  note_launch();
  direct_sum_kernel<<<grid_for(total), 256, 0, st>>>(P, pl, pr, alpha, Q, ql, qr, first, last, ol,
                                                     orr, out);
  return cudaGetLastError();
}

cudaError_t dev_fill(double* p, double v, long long n, cudaStream_t st) {
  note_launch();
  fill_kernel<<<grid_for(n), 256, 0, st>>>(p, v, n);
  return cudaGetLastError();
}

cudaError_t dev_scale(double* p, double v, long long n, cudaStream_t st) {
  note_launch();
  scale_kernel<<<grid_for(n), 256, 0, st>>>(p, v, n);
  return cudaGetLastError();
}

cudaError_t dev_scale_rsqrt(double* p, const double* ss, long long n, cudaStream_t st) {
  note_launch();
  scale_rsqrt_kernel<<<grid_for(n), 256, 0, st>>>(p, ss, n);
  return cudaGetLastError();
}

cudaError_t dev_sumsq(const double* p, long long n, double* out, cudaStream_t st) {
  note_launch();
  sumsq_kernel<<<1, 1024, 0, st>>>(p, n, out);
  return cudaGetLastError();
}

cudaError_t dev_identity_site(double* p, cudaStream_t st) {
  note_launch();
  identity_site_kernel<<<1, 32, 0, st>>>(p);
  return cudaGetLastError();
}
