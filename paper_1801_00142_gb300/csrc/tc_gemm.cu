// tcgen05 / TMA GEMM kernel (see tc_gemm.cuh).
//
// CTA tile 128 x 128 (M x N), K-block of 64 BF16 (one 128-byte swizzle row;
// 2 stages at 6 planes); persistent CTAs (one per SM).  Warp 0: TMA producer (one elected thread);
// warp 1: MMA issuer (one elected thread, 4 x UMMA_K=16 per K-block and
// product); warp 2: tensor-memory allocation; warps 4-7: epilogue
// (tcgen05.ld 32x32b, lane quarter = warp % 4).
//
// Accumulation.  The tensor core rounds its FP32 accumulator toward zero, so
// long accumulation chains in tensor memory shrink every output by a
// systematic relative bias that grows with the chain (measured: ~1e-5 after
// 64 K-blocks of positive products).  The leading product x0*y0 of the split
// planes is therefore accumulated one K-block at a time (four MMAs of exact
// BF16 products, which the tensor core sums without loss at this length)
// into a double-buffered "main" accumulator, and the epilogue warps add each
// K-block's result into FP32 registers with round-to-nearest additions while
// the MMAs of the next K-block run.  The correction products (x0*y1, x1*y0,
// ...), about 2^-8 of the leading one and of uncorrelated sign, accumulate
// over the whole K range in a second, per-tile "corr" accumulator that the
// epilogue adds once at the end of the tile.  Tensor memory: main buffers at
// columns [0, 256), corr buffers (double-buffered across tiles) at [256, 512).
//
// Every mbarrier wait is bounded: on expiry the CTA records an error in
// dev_err, drains its own outstanding TMA loads and MMAs (bounded again),
// frees its tensor memory and returns.
#include <stdint.h>
#include <stdlib.h>

#include "tc_gemm.cuh"

namespace {

constexpr int BM = 128, BN = 128;
constexpr int NTHREADS = 256;

// Shared-memory geometry for a K-block of BK BF16 (64: 128-byte swizzle,
// 32: 64-byte swizzle).  K-major tiles are BM rows of SW bytes in 8-row
// groups SBO bytes apart; MN-major tiles are ATOMS atoms of BK MN-elements,
// each BK K-rows of SW bytes (ATOM bytes), ATOM bytes apart.
template <int BK>
struct Geo {
  static constexpr int SW = BK * 2;           // bytes of one swizzled row
  static constexpr int TILE = BM * BK * 2;    // bytes per operand plane and stage
  static constexpr int SWZ = BK == 64 ? 2 : 4;   // descriptor swizzle code: 128 B / 64 B
  static constexpr int SBO = 8 * SW;          // 8-row group stride
  static constexpr int ATOM = BK * SW;        // MN-major atom: BK K-rows x SW bytes
  static constexpr int ATOMS = BM / BK;       // MN-major atoms per 128-wide tile
  static_assert(BK == 64 || BK == 32, "K-block of 32 or 64");
};
constexpr long long WAIT_LIMIT = 1LL << 24;
constexpr int TMEM_COLS = 4 * BN;     // main [0, 2 BN), corr [2 BN, 4 BN)
constexpr int CORR_COL = 2 * BN;

struct KParams {
  int M, N, K, batch, splitk, kb_total, kb_per;
  int pa_planes, pb_planes, nprod;
  int prod_a[6], prod_b[6];
  int a_batched, b_batched;
  int a_mn, b_mn;   // operand staged MN-major (two 64-wide boxes per plane)
  int m_fast;       // tile order: m fastest (fewer m tiles than n tiles) or n fastest
  int stages;
  int chunk_kb;   // K-blocks per main accumulation chunk
  TcOutput out;
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on an mbarrier phase; false (and *err set) on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 256) __nanosleep(64);
    if ((i & 1023) == 1023 && *(volatile int*)err) return false;
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

// K-major operand tile: rows of SW bytes, 8-row groups SBO bytes apart; the
// leading byte offset is unused for swizzled K-major layouts.
template <int BK>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused)
  d |= (uint64_t)(Geo<BK>::SBO >> 4) << 32;        // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                          // descriptor version (sm_100 family)
  d |= (uint64_t)Geo<BK>::SWZ << 61;               // swizzle mode
  return d;
}

// MN-major operand tile: K-rows of BK contiguous MN elements (SW bytes),
// 8-row groups SBO bytes apart along K (stride byte offset), consecutive
// BK-wide MN atoms ATOM bytes apart (leading byte offset).
template <int BK>
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(Geo<BK>::ATOM >> 4) << 16;       // leading byte offset: next MN atom
  d |= (uint64_t)(Geo<BK>::SBO >> 4) << 32;        // stride byte offset: next 8 K-rows
  d |= (uint64_t)1 << 46;                          // descriptor version (sm_100 family)
  d |= (uint64_t)Geo<BK>::SWZ << 61;               // swizzle mode
  return d;
}

// instruction descriptor: kind::f16, A = B = BF16, D = F32, M = 128, N = 128;
// bits 15 / 16 select an MN-major A / B
__host__ __device__ constexpr uint32_t idesc_bf16_128x128(int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a_mn & 1) << 15) |
         ((uint32_t)(b_mn & 1) << 16) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void store_out(const TcOutput& o, long long off, float v) {
  if (o.mode == TC_OUT_BF16P) {
    __nv_bfloat16 p0 = __float2bfloat16_rn(v);
    float r = v - __bfloat162float(p0);
    __nv_bfloat16 p1 = __float2bfloat16_rn(r);
    o.bf16[off] = p0;
    o.bf16[off + o.plane_stride] = p1;
    if (o.planes > 2) {
      float r2 = r - __bfloat162float(p1);
      o.bf16[off + 2 * o.plane_stride] = __float2bfloat16_rn(r2);
    }
  } else {
    o.f32[off] = v;
  }
}

__device__ __forceinline__ uint32_t bf16_bits(__nv_bfloat16 x) {
  return (uint32_t)__bfloat16_as_ushort(x);
}

// Split two values into up to three BF16 planes and pack each plane's pair
// (first value in the low half: the lower address).
__device__ __forceinline__ void split_pack2(float a, float b, uint32_t& w0, uint32_t& w1,
                                            uint32_t& w2) {
  const __nv_bfloat16 a0 = __float2bfloat16_rn(a), b0 = __float2bfloat16_rn(b);
  const float ar = a - __bfloat162float(a0), br = b - __bfloat162float(b0);
  const __nv_bfloat16 a1 = __float2bfloat16_rn(ar), b1 = __float2bfloat16_rn(br);
  const __nv_bfloat16 a2 = __float2bfloat16_rn(ar - __bfloat162float(a1));
  const __nv_bfloat16 b2 = __float2bfloat16_rn(br - __bfloat162float(b1));
  w0 = bf16_bits(a0) | (bf16_bits(b0) << 16);
  w1 = bf16_bits(a1) | (bf16_bits(b1) << 16);
  w2 = bf16_bits(a2) | (bf16_bits(b2) << 16);
}

// Store 32 consecutive output columns of one row (v[0..31] already scaled).
// Column layout of the chunk, decided once per tile: contiguous (32 columns
// at consecutive offsets), paired (columns 2j, 2j+1 adjacent) or scattered.
// Vector stores need the lane's start offset aligned (8 elements for BF16
// planes / 4 for FP32) and the plane stride likewise; otherwise narrower
// stores are used.
__device__ __forceinline__ void store_chunk(const TcOutput& o, long long om,
                                            const long long* col, int layout, int ncols,
                                            const float* v) {
  if (o.mode == TC_OUT_BF16P) {
    const long long ps = o.plane_stride;
    const long long off0 = om + col[0];
    if (layout == 2 && ncols == 32 && ((off0 | ps) & 7) == 0) {
#pragma unroll
      for (int q8 = 0; q8 < 4; ++q8) {
        uint32_t w[3][4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          split_pack2(v[q8 * 8 + 2 * e], v[q8 * 8 + 2 * e + 1], w[0][e], w[1][e], w[2][e]);
        __nv_bfloat16* d = o.bf16 + off0 + q8 * 8;
        *reinterpret_cast<uint4*>(d) = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
        *reinterpret_cast<uint4*>(d + ps) = make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
        if (o.planes > 2)
          *reinterpret_cast<uint4*>(d + 2 * ps) = make_uint4(w[2][0], w[2][1], w[2][2], w[2][3]);
      }
      return;
    }
    if (layout >= 1 && ncols == 32 && ((om + col[0]) & 1) == 0 && (ps & 1) == 0) {
#pragma unroll
      for (int jj = 0; jj < 32; jj += 2) {
        const long long off = om + col[jj];
        uint32_t w0, w1, w2;
        split_pack2(v[jj], v[jj + 1], w0, w1, w2);
        *reinterpret_cast<uint32_t*>(o.bf16 + off) = w0;
        *reinterpret_cast<uint32_t*>(o.bf16 + off + ps) = w1;
        if (o.planes > 2) *reinterpret_cast<uint32_t*>(o.bf16 + off + 2 * ps) = w2;
      }
      return;
    }
  } else {
    const long long off0 = om + col[0];
    if (layout == 2 && ncols == 32 && (off0 & 3) == 0) {
      float4* d = reinterpret_cast<float4*>(o.f32 + off0);
#pragma unroll
      for (int q4 = 0; q4 < 8; ++q4)
        d[q4] = make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
      return;
    }
  }
#pragma unroll
  for (int jj = 0; jj < 32; ++jj)
    if (jj < ncols) store_out(o, om + col[jj], v[jj]);
}

// Tile t -> (m tile, n tile, batch x split).  The smaller of the two output
// dimensions runs fastest, so CTAs working at the same time share the tile
// of the larger operand (read from DRAM once, then from L2).
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int m_fast, int& mt,
                                            int& nt, int& z) {
  const int mn = tiles_m * tiles_n;
  z = t / mn;
  const int r = t - z * mn;
  if (m_fast) {
    mt = r % tiles_m;
    nt = r / tiles_m;
  } else {
    nt = r % tiles_n;
    mt = r / tiles_n;
  }
}

// Persistent kernel: every CTA walks the output tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (tile order: see tile_coords, then batch x
// split).  The main accumulator is double-buffered per chunk of chunk_kb
// K-blocks and the corr accumulator per tile, so the MMAs of the next chunk
// (and of the next tile) run while the epilogue drains and stores; the
// operand stage ring continues across tiles.
//
// The operand layout of B (BMN: MN-major) and the number of plane products
// (NPROD: 1, 3 or 6) are template parameters: the MMA issuer is one thread
// that must issue a 128x128x16 MMA about every 70 cycles, so its loop holds
// no branches on them and its descriptors are the stage's two base
// descriptors plus compile-time offsets (measured: the runtime-selected
// descriptors alone cost 16 % of the kernel's time).
template <int BK, int BMN, int NPROD>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const KParams p) {
  using G = Geo<BK>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  const int stage_bytes = (p.pa_planes + p.pb_planes) * G::TILE;
  uint64_t* full = (uint64_t*)(smem + S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* main_full = empty + S;      // [2] per chunk
  uint64_t* main_empty = main_full + 2; // [2]
  uint64_t* corr_full = main_empty + 2; // [2] per tile
  uint64_t* corr_empty = corr_full + 2; // [2]
  uint64_t* done = corr_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  long long* col_off_all = (long long*)(tmem_slot + 2);   // [4][BN] per-warp column offsets

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tiles_n = (p.N + BN - 1) / BN, tiles_m = (p.M + BM - 1) / BM;
  const int tiles = tiles_n * tiles_m * p.batch * p.splitk;
  const int CK = p.chunk_kb;
  constexpr bool has_corr = NPROD > 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&main_full[b], 1);
      mbar_init(&main_empty[b], 4);
      mbar_init(&corr_full[b], 1);
      mbar_init(&corr_empty[b], 4);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    long long g = 0;   // k-blocks issued by this CTA
    int s = 0;         // stage of k-block g, and the parity of its round
    uint32_t ph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      int mt, nt, z;
      tile_coords(t, tiles_m, tiles_n, p.m_fast, mt, nt, z);
      const int bidx = z / p.splitk, split = z % p.splitk;
      const int kb_begin = split * p.kb_per;
      const int kb_end = min(kb_begin + p.kb_per, p.kb_total);
      const int ba = p.a_batched ? bidx : 0, bb = p.b_batched ? bidx : 0;
      for (int kb = kb_begin; kb < kb_end && ok; ++kb, ++g) {
        if (g >= S) ok = mbar_wait(&empty[s], ph ^ 1u, p.err);
        if (!ok) break;
        uint8_t* st = smem + s * stage_bytes;
        mbar_expect_tx(&full[s], stage_bytes);
        const int k0 = kb * BK;
        for (int q = 0; q < p.pa_planes; ++q)
          tma_load_4d(st + q * G::TILE, &mapA, &full[s], k0, mt * BM, ba, q);
        for (int q = 0; q < p.pb_planes; ++q) {
          uint8_t* dst = st + (p.pa_planes + q) * G::TILE;
          if (BMN) {
#pragma unroll
            for (int a = 0; a < G::ATOMS; ++a)
              tma_load_4d(dst + a * G::ATOM, &mapB, &full[s], nt * BN + a * BK, k0, bb, q);
          } else {
            tma_load_4d(dst, &mapB, &full[s], k0, nt * BN, bb, q);
          }
        }
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    // drain: every load issued must have landed before the CTA may exit
    for (long long i = (g > S ? g - S : 0); i < g; ++i)
      mbar_wait(&full[i % S], (uint32_t)((i / S) & 1), p.err);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    // plane products: (0,0) is the main one, then (0,1) (1,0) (0,2) (1,1) (2,0)
    constexpr int PA[6] = {0, 0, 1, 0, 1, 2}, PB[6] = {0, 1, 0, 2, 1, 0};
    constexpr uint32_t PLANE = G::TILE >> 4;                 // descriptor units per plane
    constexpr uint32_t KSTEP_A = 2;                          // 16 BF16 = 32 B along K
    constexpr uint32_t KSTEP_B = BMN ? (16 * G::SW) >> 4 : 2;   // MN-major: 16 K-rows
    const uint32_t idesc = idesc_bf16_128x128(0, BMN);
    const uint32_t boff = (uint32_t)(p.pa_planes * G::TILE);
    int s = 0;         // stage of the current k-block, and the parity of its round
    uint32_t ph = 0;
    long long h = 0;   // main chunks issued
    int j = 0;         // tiles of this CTA
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++j) {
      const int z = t / (tiles_n * tiles_m);
      const int split = z % p.splitk;
      const int kb_begin = split * p.kb_per;
      const int kb_end = min(kb_begin + p.kb_per, p.kb_total);
      const int cb = j & 1;
      if (has_corr && j >= 2) ok = mbar_wait(&corr_empty[cb], (uint32_t)(((j >> 1) - 1) & 1), p.err);
      if (!ok) break;
      const uint32_t ccol = tmem + (uint32_t)(CORR_COL + cb * BN);
      int ci = 0;   // position inside the main chunk
      for (int kb = kb_begin; kb < kb_end && ok; ++kb) {
        const int mb = (int)(h & 1);
        if (ci == 0 && h >= 2) ok = mbar_wait(&main_empty[mb], (uint32_t)(((h >> 1) - 1) & 1), p.err);
        if (!ok) break;
        ok = mbar_wait(&full[s], ph, p.err);
        if (!ok) break;
        fence_after();
        const uint32_t base = smem_u32(smem + s * stage_bytes);
        const uint64_t dA = smem_desc<BK>(base);
        const uint64_t dB = BMN ? smem_desc_mn<BK>(base + boff) : smem_desc<BK>(base + boff);
        const uint32_t mcol = tmem + (uint32_t)(mb * BN);
        const bool main_acc = ci > 0, corr_acc = kb > kb_begin;
#pragma unroll
        for (int pr = 0; pr < NPROD; ++pr) {
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t da = dA + (uint64_t)(PA[pr] * PLANE + kk * KSTEP_A);
            const uint64_t db = dB + (uint64_t)(PB[pr] * PLANE + kk * KSTEP_B);
            const bool acc = kk > 0 || (pr == 0 ? main_acc : (pr > 1 || corr_acc));
            mma_bf16(pr == 0 ? mcol : ccol, da, db, idesc, acc ? 1u : 0u);
          }
          if (pr == 0 && (ci == CK - 1 || kb == kb_end - 1)) {
            // the chunk's leading products are issued: the epilogue may take it
            mma_commit(&main_full[mb]);
            ++h;
          }
        }
        mma_commit(&empty[s]);
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
        if (++ci == CK) ci = 0;
      }
      // an empty tile (split beyond K) commits nothing it would have to wait for
      if (ok && has_corr) mma_commit(&corr_full[cb]);
    }
    // the done barrier tracks completion of every MMA issued so far
    mma_commit(done);
  } else if (warp >= 4) {
    // ---------------- epilogue (4 warps; warp % 4 selects the TMEM lane quarter)
    const int q = warp % 4;
    const TcOutput& o = p.out;
    long long* col_off = col_off_all + q * BN;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    long long h = 0;   // main chunks drained
    int j = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++j) {
      int mt, nt, z;
      tile_coords(t, tiles_m, tiles_n, p.m_fast, mt, nt, z);
      const int bidx = z / p.splitk, split = z % p.splitk;
      const int kb_begin = split * p.kb_per;
      const int kb_end = min(kb_begin + p.kb_per, p.kb_total);
      const int n0 = nt * BN, m0 = mt * BM;
      const int cb = j & 1;
      // column offsets of this tile, computed once per warp (the 3-level views
      // need divisions); warp-private, so no barrier across warps is needed
      __syncwarp();
      for (int cc = lane; cc < BN; cc += 32) {
        const int n = n0 + cc;
        col_off[cc] = (o.mode == TC_OUT_PARTIAL || n >= p.N) ? (long long)n : idx_off(o.cn, n);
      }
      __syncwarp();
      // layout of each 32-column chunk (2 bits per chunk: 2 contiguous, 1 paired)
      int layouts = 0;
#pragma unroll
      for (int ch = 0; ch < BN / 32; ++ch) {
        const long long mine = col_off[ch * 32 + lane];
        const bool contig = mine == col_off[ch * 32] + lane;
        // paired: every even column's partner follows it, and all pair starts
        // have the parity of the chunk's first column (one alignment test
        // per row then covers the whole chunk)
        const bool paired = (lane & 1) || (col_off[ch * 32 + lane + 1] == mine + 1 &&
                                           ((mine - col_off[ch * 32]) & 1) == 0);
        const unsigned mc = __ballot_sync(0xffffffffu, contig);
        const unsigned mp = __ballot_sync(0xffffffffu, paired);
        layouts |= (mc == 0xffffffffu ? 2 : (mp == 0xffffffffu ? 1 : 0)) << (2 * ch);
      }
      // accumulate the tile: every main chunk, then the corrections, each
      // added with round-to-nearest FP32 additions
      float acc[BN];
#pragma unroll
      for (int jj = 0; jj < BN; ++jj) acc[jj] = 0.f;
      for (int kb = kb_begin; kb < kb_end && ok; kb += CK, ++h) {
        const int mb = (int)(h & 1);
        ok = mbar_wait(&main_full[mb], (uint32_t)((h >> 1) & 1), p.err);
        if (!ok) break;
        fence_after();
#pragma unroll
        for (int c = 0; c < BN; c += 32) {
          float v[32];
          tmem_ld32(lane_base + (uint32_t)(mb * BN + c), v);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) acc[c + jj] = __fadd_rn(acc[c + jj], v[jj]);
        }
        fence_before();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&main_empty[mb]))
                       : "memory");
      }
      if (!ok) break;
      if (has_corr) {
        ok = mbar_wait(&corr_full[cb], (uint32_t)((j >> 1) & 1), p.err);
        if (!ok) break;
        fence_after();
        if (kb_end > kb_begin) {
#pragma unroll
          for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld32(lane_base + (uint32_t)(CORR_COL + cb * BN + c), v);
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) acc[c + jj] = __fadd_rn(acc[c + jj], v[jj]);
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&corr_empty[cb]))
                       : "memory");
      }
      const int m = m0 + q * 32 + lane;
      if (m >= p.M) continue;
      float* dstp = nullptr;
      long long om = 0;
      if (o.mode == TC_OUT_PARTIAL)
        dstp = o.f32 + (((long long)split * p.batch + bidx) * p.M + m) * (long long)p.N;
      else
        om = bidx * o.scb + idx_off(o.cm, m);
      const float alpha = (float)o.alpha;
#pragma unroll
      for (int c = 0; c < BN; c += 32) {
        const int ncols = min(32, p.N - (n0 + c));
        if (ncols <= 0) continue;
        float* v = acc + c;
        if (o.mode == TC_OUT_PARTIAL) {
          float* d = dstp + n0 + c;
          if (ncols == 32 && ((uintptr_t)d & 15) == 0) {
#pragma unroll
            for (int q4 = 0; q4 < 8; ++q4)
              reinterpret_cast<float4*>(d)[q4] =
                  make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
          } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
              if (jj < ncols) d[jj] = v[jj];
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) v[jj] *= alpha;
          store_chunk(o, om, col_off + c, (layouts >> (2 * (c / 32))) & 3, ncols, v);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 2) {
    // all MMAs of this CTA have completed before its tensor memory is freed
    if (lane == 0) mbar_wait(done, 0, p.err);
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

// One-time lookups (function-local statics: initialised once, thread-safe,
// so contexts driven from several host threads share them safely).
EncodeFn get_encode() {
  static const EncodeFn fn = []() -> EncodeFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeFn)p;
    return nullptr;
  }();
  return fn;
}

// the kernel's shared-memory opt-in and the SM count, once per device
struct LaunchSetup {
  cudaError_t err;
  int sms;
};
PerDevice<LaunchSetup> g_launch_setup;

template <int BMN, int NPROD>
cudaError_t opt_in() {
  return cudaFuncSetAttribute(tc_gemm_kernel<64, BMN, NPROD>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

cudaError_t launch_setup(int* sms) {
  LaunchSetup s{cudaSuccess, 0};
  cudaError_t e = g_launch_setup.get(
      [](int dev) {
        LaunchSetup r{cudaSuccess, 0};
        const cudaError_t o[6] = {opt_in<0, 1>(), opt_in<0, 3>(), opt_in<0, 6>(),
                                  opt_in<1, 1>(), opt_in<1, 3>(), opt_in<1, 6>()};
        for (cudaError_t x : o)
          if (r.err == cudaSuccess) r.err = x;
        if (r.err == cudaSuccess)
          r.err = cudaDeviceGetAttribute(&r.sms, cudaDevAttrMultiProcessorCount, dev);
        return r;
      },
      &s);
  if (e != cudaSuccess) return e;
  *sms = s.sms;
  return s.err;
}

// Terms per main accumulation chunk: 64 x XTRG_TC_CHUNK_KB (1..64) if set,
// else 256 (BF16 products per tensor-memory chain, which the tensor core
// sums exactly for same-signed terms of similar size; measured 3 % faster
// than 128 at the same accuracy)
int chunk_terms() {
  static const int v = []() {
    const char* e = getenv("XTRG_TC_CHUNK_KB");
    const int x = e ? atoi(e) : 0;
    return 64 * ((x >= 1 && x <= 64) ? x : 4);
  }();
  return v;
}

// K-block width: 64 BF16 (one 128-byte swizzle row).  A 32-wide K-block
// (64-byte swizzle, twice the stages) computed the same and was slower.
constexpr int K_BLOCK = 64;

// 4-D map with BK-wide boxes (BK = 64: 128-byte swizzle, 32: 64-byte),
// out-of-range elements read as zero.
cudaError_t make_map(CUtensorMap* map, const TcOperand& op, int BK) {
  EncodeFn enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  if (op.ld % 8 != 0 || op.ld < (op.mn_major ? op.rows : op.k) || ((uintptr_t)op.base % 16) != 0)
    return cudaErrorInvalidValue;
  // K-major: (k, rows, batch, plane), box (BK, 128); MN-major: (rows, k,
  // batch, plane), box (BK, BK), loaded 128 / BK times per 128-wide tile
  const long long outer = op.mn_major ? op.k : op.rows;
  const long long bstride = op.batches > 1 ? op.batch_stride : outer * op.ld;
  cuuint64_t dims[4] = {(cuuint64_t)(op.mn_major ? op.rows : op.k),
                        (cuuint64_t)(op.mn_major ? op.k : op.rows), (cuuint64_t)op.batches,
                        (cuuint64_t)op.planes};
  cuuint64_t strides[3] = {(cuuint64_t)op.ld * 2, (cuuint64_t)bstride * 2,
                           (cuuint64_t)op.plane_stride * 2};
  if ((strides[1] % 16) || (strides[2] % 16)) return cudaErrorInvalidValue;
  cuuint32_t box[4] = {(cuuint32_t)BK, (cuuint32_t)(op.mn_major ? BK : BM), 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapSwizzle swz = BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)op.base, dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, int M, int N, int K, int batch,
                    int nprod, int splitk, const TcOutput& out, int* dev_err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (K <= 0 || splitk < 1 || batch * splitk > 65535) return cudaErrorInvalidValue;
  if (A.rows < M || B.rows < N || A.k != K || B.k != K) return cudaErrorInvalidValue;
  if ((A.batches != 1 && A.batches != batch) || (B.batches != 1 && B.batches != batch))
    return cudaErrorInvalidValue;
  if (splitk > 1 && out.mode != TC_OUT_PARTIAL) return cudaErrorInvalidValue;
  // A is staged K-major; B K-major or MN-major
  if (A.mn_major) return cudaErrorInvalidValue;
  const int BK = K_BLOCK;
  KParams p;
  p.M = M; p.N = N; p.K = K; p.batch = batch; p.splitk = splitk;
  p.kb_total = (K + BK - 1) / BK;
  p.kb_per = (p.kb_total + splitk - 1) / splitk;
  p.pa_planes = A.planes;
  p.pb_planes = B.planes;
  static const int pa6[6] = {0, 0, 1, 0, 1, 2}, pb6[6] = {0, 1, 0, 2, 1, 0};
  if (nprod != 1 && nprod != 3 && nprod != 6) return cudaErrorInvalidValue;
  for (int i = 0; i < nprod; ++i) {
    p.prod_a[i] = pa6[i];
    p.prod_b[i] = pb6[i];
    if (pa6[i] >= A.planes || pb6[i] >= B.planes) return cudaErrorInvalidValue;
  }
  p.nprod = nprod;
  p.a_batched = A.batches > 1;
  p.b_batched = B.batches > 1;
  p.a_mn = A.mn_major ? 1 : 0;
  p.b_mn = B.mn_major ? 1 : 0;
  p.m_fast = ((M + BM - 1) / BM) < ((N + BN - 1) / BN) ? 1 : 0;
  // as many stages as fit next to the barriers (up to 6)
  const int stage_bytes = (A.planes + B.planes) * BM * BK * 2;
  int S = (200 * 1024) / stage_bytes;
  if (S > 6) S = 6;
  if (S < 2) return cudaErrorInvalidValue;
  p.stages = S;
  p.chunk_kb = chunk_terms() / BK;
  p.out = out;
  p.err = dev_err;
  CUtensorMap ma, mb;
  cudaError_t e;
  if ((e = make_map(&ma, A, BK)) != cudaSuccess) return e;
  if ((e = make_map(&mb, B, BK)) != cudaSuccess) return e;
  const int smem = S * stage_bytes + 1024 + (2 * S + 9) * 8 + 8 + 4 * BN * 8 + 64;
  int sms = 0;
  if ((e = launch_setup(&sms)) != cudaSuccess) return e;
  const long long tiles =
      (long long)((N + BN - 1) / BN) * ((M + BM - 1) / BM) * (long long)batch * splitk;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)(tiles < sms ? tiles : sms));
  note_launch();
  const int sel = (B.mn_major ? 3 : 0) + (nprod == 1 ? 0 : nprod == 3 ? 1 : 2);
  switch (sel) {
    case 0: tc_gemm_kernel<64, 0, 1><<<grid, NTHREADS, smem, st>>>(ma, mb, p); break;
    case 1: tc_gemm_kernel<64, 0, 3><<<grid, NTHREADS, smem, st>>>(ma, mb, p); break;
    case 2: tc_gemm_kernel<64, 0, 6><<<grid, NTHREADS, smem, st>>>(ma, mb, p); break;
    case 3: tc_gemm_kernel<64, 1, 1><<<grid, NTHREADS, smem, st>>>(ma, mb, p); break;
    case 4: tc_gemm_kernel<64, 1, 3><<<grid, NTHREADS, smem, st>>>(ma, mb, p); break;
    default: tc_gemm_kernel<64, 1, 6><<<grid, NTHREADS, smem, st>>>(ma, mb, p); break;
  }
  return cudaGetLastError();
}
