// C ABI and host driver of the XTRG beta-doubling engine (declared in xtrg.h).
//
// The host drives the sweep; every arithmetic step runs in this library's
// kernels on the caller's stream.  All device memory is carved from the
// caller's workspace.
//
// Method (arXiv:1801.00142):
//   init    rho(tau0) = sum_k (-tau0)^k H^k / k!       Eq. RhoTau (Sec. II C),
//           Horner form Y <- I + (-tau0/k) H Y; each product compressed by the
//           variational scheme of App. D.1 with the exact product as guess,
//           "+I" an exact direct sum.
//   double  rho <- compress(rho^T rho)                  Eq. rho:scale2 (Sec. II B)
//   compress: right-canonical guess, right environments, then full sweeps
//           (L->R, R->L) of two-site updates C_i C_{i+1} = C_E  (Eq. LSEProd)
//           with C_E from the environments of Fig. VMPO(a,c) and the split of
//           Fig. VMPO(d), keeping at most D* singular values.
//   normalise by the centre's Frobenius norm, ln c_{n+1} = 2 ln c_n + ln s.
//   observables: Eq. ThermalQuan (Sec. III A) from Tr rho, Tr(H rho), Tr(H^2 rho).
//
// Storage: an MPO site W[l][s][t][r] is row-major; environments at bond i are
// stored [c][a][b] (c = bond of the compressed MPO C, a/b = bonds of the
// factors A/B); the left half of C_E is stored [c][s][u][a'][b'] and the
// right half [s'][u'][c''][a'][b'], so C_E = Lpart * Rpart^T is one GEMM.
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/xtrg.h"
#include "common.cuh"
#include "mixed_ops.cuh"
#include "subspace_split.cuh"
#include "tc_gemm.cuh"
#include "tc_gemm_entry.cuh"

namespace {

struct DevMpo {
  std::vector<int> dims;        // L+1 bond dimensions
  std::vector<double*> site;    // L device slots
  size_t slot;                  // capacity of each slot, in doubles
};

struct Plan {
  int L, DH, cap, cap_fat, fat_bond, capc;
  size_t n_h, n_site, n_csite, n_fat, n_pp, n_env, n_part, n_ce, n_svd, n_svd_cols, n_usbuf,
      n_obs, n_herm;
  // tensor-core path (per plane, in BF16 elements)
  int planes;
  size_t m_site[4], m_env, m_t1, m_lp, m_ct, m_part;
  size_t mixed_bytes;
  size_t total;
};

constexpr int SPLITK_MAX = 32;

constexpr size_t ALIGN = 256;
inline size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Capacities: rho and the Horner iterate Y have bonds <= cap = D* + 1.  The
// compressed MPO C starts from a right-canonicalised guess whose bonds can
// exceed D* before the sweeps truncate them: for the exact-product guess of
// the series products they are bounded by the fused bond DH * cap_fat, so C
// and everything shaped by C's bonds use capc = max(cap, DH * cap_fat).
bool plan_sizes(int L, int DH, const xtrg_config* cfg, Plan* p) {
  if (L < 2 || DH < 1 || cfg->dstar < 1 || cfg->dstar > 1024) return false;
  if (cfg->orth_block < 0 || cfg->orth_block > SUBSPACE_BLOCK_K || cfg->orth_block % 32) return false;
  p->L = L;
  p->DH = DH;
  p->cap = cfg->dstar + 1;
  p->cap_fat = p->cap < 64 ? p->cap : 64;
  p->fat_bond = DH * p->cap_fat;
  p->capc = p->cap > p->fat_bond ? p->cap : p->fat_bond;
  const size_t cap = p->cap, capc = p->capc, fb = p->fat_bond;
  const size_t da = cap > (size_t)DH ? cap : (size_t)DH;    // bound of A's bonds
  p->n_h = (size_t)DH * 4 * DH;
  p->n_site = cap * 4 * cap;
  p->n_csite = capc * 4 * capc;
  p->n_fat = fb * 4 * fb;
  p->n_pp = capc * 4 * capc;
  p->n_env = da * cap * capc;
  p->n_part = 4 * capc * da * cap;
  p->n_ce = 16 * capc * capc;
  p->n_svd = 16 * capc * capc;
  p->n_svd_cols = 4 * capc;
  p->n_usbuf = capc * capc;
  p->n_obs = (size_t)DH * DH * 4 * cap * 2;
  p->n_herm = cap * cap;   // one transfer matrix of the Hermiticity check (T: 4 of these)
  p->planes = cfg->prec == XTRG_BF16X6 ? 3 : 2;
  {
    const size_t c = cap, l1 = tc_ld(c), l2 = tc_ld(2 * c), lsq = tc_ld(c * c), l4 = tc_ld(4 * c);
    p->m_site[0] = 4 * c * l1;   // rho^T layout for the first left substep
    p->m_site[1] = 2 * c * l2;   // (u,b') x (b,t) layout for the second left substep
    p->m_site[2] = 4 * c * l1;   // (a',t',s') x a'' layout for the first right substep
    p->m_site[3] = 2 * c * l2;   // (b',u') x (t',b'') layout for the second right substep
    p->m_env = c * c * l1;
    p->m_t1 = c * 2 * c * l2;
    p->m_lp = 4 * c * lsq;
    p->m_ct = c * l4;
    p->m_part = (size_t)SPLITK_MAX * 16 * c * c;
    size_t pl = p->planes, mb = 0;
    for (int k = 0; k < 4; ++k) mb += up((size_t)L * pl * p->m_site[k] * 2);
    mb += up((size_t)(L + 1) * pl * p->m_env * 2);
    // the halves of the two-site environment: one of each, or one per site
    // when they stay resident (keep_parts)
    const size_t nparts = cfg->keep_parts ? (size_t)L : 1;
    mb += 2 * up(pl * p->m_t1 * 2) + 2 * up(nparts * pl * p->m_lp * 2);
    mb += up(pl * p->m_ct * 2) + up(p->m_part * 4) + 2 * ALIGN;
    mb += up(subspace_buffer_floats(p->cap) * 4) + 3 * ALIGN;
    mb += up(subspace_plane_elems_a(p->cap) * 2) + up(subspace_plane_elems_b(p->cap) * 2);
    mb += 2 * up(subspace_plane_elems_a(p->cap) * 2) + ALIGN;   // C_E planes, both orientations
    mb += up(SUBSPACE_CHOL_FLOATS * 4) + 2 * up(SUBSPACE_BLOCK_K * 4) + ALIGN;   // CholeskyQR2 factor
    p->mixed_bytes = (cfg->prec == XTRG_FP64) ? 0 : mb;
  }
  size_t t = 0;
  t += up((size_t)L * p->n_h * 8);          // H
  t += up((size_t)L * 4 * 8);               // identity sites
  t += up((size_t)L * p->n_site * 8);       // Y
  t += 2 * up((size_t)L * p->n_csite * 8);  // rho, C (swapped after every product)
  t += up((size_t)L * p->n_fat * 8);        // exact-product guess
  t += 2 * up(p->n_pp * 8);                 // canonicalisation ping-pong
  t += up((size_t)(L + 1) * p->n_env * 8);  // environments
  t += 3 * up(p->n_part * 8);               // T1, Lpart, Rpart
  t += up(p->n_ce * 8);                     // C_E
  t += 2 * up(p->n_svd * 8) + up(p->n_svd_cols * 8) + up(p->n_svd_cols * 4) + 3 * ALIGN;
  t += up(p->n_usbuf * 8);
  t += 3 * up(p->n_obs * 8);
  t += 8 * up(p->n_herm * 8);              // Hermiticity transfers: 2 + 2 ping-pong, T (x4)
  t += up(64 * 8);                          // scalars
  t += p->mixed_bytes;
  p->total = t;
  return true;
}

}  // namespace

struct xtrg_ctx {
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0, used = 0;
  xtrg_config cfg{};
  Plan plan{};
  int L = 0, DH = 0, cap = 0;
  int sms = 152;   // SMs of the device the context was created on
  DevMpo H, rho, C, Y, I, fat;
  double* pp[2] = {nullptr, nullptr};
  std::vector<double*> env;
  double *T1 = nullptr, *Lp = nullptr, *Rp = nullptr, *CE = nullptr, *usbuf = nullptr;
  double *ob[3] = {nullptr, nullptr, nullptr};
  double *hf[2] = {nullptr, nullptr}, *hr[2] = {nullptr, nullptr}, *ht = nullptr;
  double* scal = nullptr;
  SvdBuffers svd{};
  // tensor-core path buffers (BF16 planes)
  struct {
    int P = 0, nprod = 0;
    std::vector<__nv_bfloat16*> site[4];
    std::vector<__nv_bfloat16*> env;
    __nv_bfloat16 *T1 = nullptr, *T1R = nullptr, *Lp = nullptr, *Rp = nullptr, *Ct = nullptr;
    // left half of site i / right half of site j (distinct buffers per site
    // when keep_parts, else all alias Lp / Rp)
    std::vector<__nv_bfloat16*> lpc, rpc;
    float* part = nullptr;
    int* err = nullptr;
    // device-side results of a product's sweeps, read once at its end:
    // [0] largest discarded weight of the last sweep, [1] exact-split
    // fallbacks (u64, cumulative), [2] +inf (run condition of an exact split
    // that always runs), [3] status of the exact splits (int: 1 timeout,
    // 2 sweep limit, 3 non-finite)
    double* acc = nullptr;
    SubspaceBuffers sb{};
  } m;
  bool mixed_ready = false;
  bool use_mixed = false;   // contraction arithmetic of the current product
  double lnc = 0.0, beta = 0.0;
  int nd = 0;
  bool have_rho = false;
  bool rho_canonical = false;   // sites 1..L-1 right-orthonormal (output of init/double)
  double last_trunc = 0.0;
  double flops_contr = 0.0, flops_split = 0.0;
  long long updates = 0;
  // profiling of the tensor-core GEMMs: event pairs resolved per product
  bool profiling = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  double tc_flops = 0.0, tc_ms = 0.0, split_ms = 0.0;
  long long tc_launches = 0;
  std::vector<int> ev_tag;             // call site of each event pair
  double tag_ms[8] = {0}, tag_flops[8] = {0};
  long long tag_n[8] = {0};
  int cur_tag = 0;
  long long fallbacks = 0;   // tensor-core path updates that used the exact split
  // CUDA graphs of saturated tensor-core doublings (one per buffer parity:
  // rho and C swap after every doubling)
  struct DoublingGraph {
    cudaGraphExec_t exec = nullptr;
    const double* rho0 = nullptr;   // rho's first site when captured (the parity)
    std::vector<int> dims;          // rho's bonds when captured
    std::vector<int> out_dims;      // C's bonds after the captured doubling
    // host counters a replay advances by
    long long d_updates = 0;
    unsigned long long d_launches = 0, d_cluster = 0;
    double d_flops_contr = 0.0, d_flops_split = 0.0;
  };
  std::vector<DoublingGraph> graphs;
  cudaStream_t cap_st = nullptr;    // capture stream (created on first use)
  std::vector<int> prev_mixed_dims;  // rho's bonds at the previous tensor-core doubling
  bool graphs_off = false;           // disabled (XTRG_NO_GRAPHS=1) or a capture failed
  bool herm_check = true;            // xtrg_observables computes herm_defect
  long long graph_replays = 0, graph_captures = 0;
  bool tune_splits = true;   // autotune C_E's split-K (see mixed_ce)
  std::string err;
};

namespace {

xtrg_status fail(xtrg_ctx* c, xtrg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(x)                                                                               \
  do {                                                                                      \
    cudaError_t _e = (x);                                                                   \
    if (_e != cudaSuccess)                                                                  \
      return fail(ctx, XTRG_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #x,                  \
                  cudaGetErrorString(_e));                                                  \
  } while (0)
#define TRY(x)                                                                              \
  do {                                                                                      \
    xtrg_status _s = (x);                                                                   \
    if (_s != XTRG_OK) return _s;                                                           \
  } while (0)

char* carve(xtrg_ctx* c, size_t bytes) {
  size_t b = up(bytes);
  if (c->used + b > c->ws_bytes) return nullptr;
  char* p = c->ws + c->used;
  c->used += b;
  return p;
}

bool carve_mpo(xtrg_ctx* c, DevMpo* m, size_t slot) {
  m->slot = slot;
  m->dims.assign(c->L + 1, 1);
  m->site.resize(c->L);
  double* base = (double*)carve(c, (size_t)c->L * slot * 8);
  if (!base) return false;
  for (int i = 0; i < c->L; ++i) m->site[i] = base + (size_t)i * slot;
  return true;
}

size_t site_elems(const DevMpo& m, int i) { return (size_t)m.dims[i] * 4 * m.dims[i + 1]; }

// ------------------------------------------------------------------ GEMMs
xtrg_status gemm(xtrg_ctx* ctx, const GemmF64& g) {
  ctx->flops_contr += 2.0 * g.M * (double)g.N * g.K * g.batch;
  CK(gemm_f64(g, ctx->st));
  return XTRG_OK;
}

// plain FP64 GEMM (bookkeeping contractions: canonicalisation, transfers)
xtrg_status gemm64(xtrg_ctx* ctx, const GemmF64& g) {
  CK(gemm_f64(g, ctx->st));
  return XTRG_OK;
}

GemmF64 mk(int M, int N, int K, int batch, const double* A, Idx3 am, Idx3 ak, long long sab,
           const double* B, Idx3 bk, Idx3 bn, long long sbb, double* C, Idx3 cm, Idx3 cn,
           long long scb) {
  GemmF64 g;
  g.M = M; g.N = N; g.K = K; g.batch = batch;
  g.A = A; g.am = am; g.ak = ak; g.sab = sab;
  g.B = B; g.bk = bk; g.bn = bn; g.sbb = sbb;
  g.C = C; g.cm = cm; g.cn = cn; g.scb = scb;
  g.alpha = 1.0; g.beta = 0.0;
  return g;
}

// ------------------------------------------------------- split (Fig. VMPO(d))
xtrg_status split(xtrg_ctx* ctx, const double* M, int m, int n, int kcap, SplitMode mode,
                  double* left, double* right, SvdResult* r) {
  bool conv = true;
  cudaError_t e = svd_split_f64(M, m, n, kcap, ctx->cfg.svd_rel_tol, mode, left, right, ctx->svd,
                                ctx->st, r, &conv);
  if (e == cudaErrorLaunchTimeout)
    return fail(ctx, XTRG_ETIMEOUT, "svd split %dx%d: a bounded device barrier expired", m, n);
  if (e != cudaSuccess) return fail(ctx, XTRG_ECUDA, "svd split %dx%d: %s", m, n, cudaGetErrorString(e));
  if (!conv) return fail(ctx, XTRG_ENUMERIC, "Jacobi SVD of a %dx%d matrix did not converge", m, n);
  if (!std::isfinite(r->sigma_max)) return fail(ctx, XTRG_ENUMERIC, "non-finite singular value");
  int len = m > n ? m : n, nc = m > n ? n : m;
  ctx->flops_split += (double)r->sweeps * nc * (nc - 1) / 2.0 * (6.0 * len + 4.0 * nc);
  return XTRG_OK;
}

// Right-canonicalise the MPO given by (src_dims, src) into C: for i = L-1..1
// the site is split by an SVD into (U Lambda) V^T, V^T is kept and U Lambda is
// multiplied into site i-1.  Only numerically-zero directions are dropped.
xtrg_status canonicalize(xtrg_ctx* ctx, const std::vector<int>& sdims,
                         const std::vector<double*>& src, DevMpo& C) {
  const int L = ctx->L;
  const double* cur = src[L - 1];
  int cl = sdims[L - 1], cr = 1;
  C.dims[L] = 1;
  for (int i = L - 1; i >= 1; --i) {
    SvdResult r;
    TRY(split(ctx, cur, cl, 4 * cr, ctx->plan.capc, SPLIT_LEFT, ctx->usbuf, C.site[i], &r));
    if (r.rank > ctx->plan.capc)
      return fail(ctx, XTRG_ENOMEM, "canonical bond at site %d exceeds capacity %d", i,
                  ctx->plan.capc);
    C.dims[i] = r.k;
    // site i-1 times (U Lambda): (l' * 4) x cl times cl x k
    int lp = sdims[i - 1];
    double* out = ctx->pp[i & 1];
    GemmF64 g = mk(lp * 4, r.k, cl, 1, src[i - 1], idx_plain(cl), idx_plain(1), 0, ctx->usbuf,
                   idx_plain(r.k), idx_plain(1), 0, out, idx_plain(r.k), idx_plain(1), 0);
    TRY(gemm64(ctx, g));
    cur = out;
    cl = lp;
    cr = r.k;
  }
  C.dims[0] = 1;
  CK(cudaMemcpyAsync(C.site[0], cur, sizeof(double) * 4 * cr, cudaMemcpyDeviceToDevice, ctx->st));
  return XTRG_OK;
}

// Left half of C_E at site i (Fig. VMPO(a,c), substeps 1-2):
//   T1[c][b][t][s][a'] = sum_a V_L[c][a][b] A_i[a][t][s][a']
//   Lp[c][s][u][a'][b'] = sum_{b,t} T1[c][b][t][s][a'] B_i[b][t][u][b']
xtrg_status left_part(xtrg_ctx* ctx, const DevMpo& A, const DevMpo& B, const DevMpo& C, int i,
                      const double* VL) {
  const int a = A.dims[i], a2 = A.dims[i + 1], b = B.dims[i], b2 = B.dims[i + 1], c = C.dims[i];
  TRY(gemm(ctx, mk(b, 4 * a2, a, c, VL, idx_plain(1), idx_plain(b), (long long)a * b, A.site[i],
                   idx_plain(4 * a2), idx_plain(1), 0, ctx->T1, idx_plain(4 * a2), idx_plain(1),
                   (long long)b * 4 * a2)));
  const long long ab2 = (long long)a2 * b2;
  TRY(gemm(ctx, mk(2 * a2, 2 * b2, 2 * b, c, ctx->T1, idx_plain(1), idx_plain(2 * a2),
                   (long long)b * 4 * a2, B.site[i], idx_plain(2 * b2), idx_plain(1), 0, ctx->Lp,
                   idx_split2(a2, 2 * ab2, b2), idx_split2(b2, ab2, 1), 4 * ab2)));
  return XTRG_OK;
}

// Right half of C_E at site j (mirror of the above):
//   T1[c''][a'][t'][s'][b''] = sum_a'' A_j[a'][t'][s'][a''] V_R[c''][a''][b'']
//   Rp[s'][u'][c''][a'][b'] = sum_{t',b''} T1[c''][a'][t'][s'][b''] B_j[b'][t'][u'][b'']
xtrg_status right_part(xtrg_ctx* ctx, const DevMpo& A, const DevMpo& B, const DevMpo& C, int j,
                       const double* VR) {
  const int a1 = A.dims[j], a2 = A.dims[j + 1], b1 = B.dims[j], b2 = B.dims[j + 1];
  const int c2 = C.dims[j + 1];
  TRY(gemm(ctx, mk(4 * a1, b2, a2, c2, A.site[j], idx_plain(a2), idx_plain(1), 0, VR,
                   idx_plain(b2), idx_plain(1), (long long)a2 * b2, ctx->T1, idx_plain(b2),
                   idx_plain(1), (long long)4 * a1 * b2)));
  const long long ab1 = (long long)a1 * b1;
  TRY(gemm(ctx, mk(2 * a1, 2 * b1, 2 * b2, c2, ctx->T1, idx_split2(2, 4LL * b2, b2),
                   idx_split2(b2, 2LL * b2, 1), (long long)4 * a1 * b2, B.site[j],
                   idx_split2(b2, 2LL * b2, 1), idx_split2(2, 4LL * b2, b2), 0, ctx->Rp,
                   idx_split2(2, b1, 2LL * c2 * ab1), idx_split2(2, 1, (long long)c2 * ab1),
                   ab1)));
  return XTRG_OK;
}

// V_L[i+1][c'][a'][b'] = sum_{c,s,u} C_i[c][s][u][c'] Lp[c][s][u][a'][b']   (substep 3)
xtrg_status left_env(xtrg_ctx* ctx, const DevMpo& A, const DevMpo& B, const DevMpo& C, int i,
                     double* out) {
  const int k = C.dims[i + 1], c = C.dims[i];
  const long long ab2 = (long long)A.dims[i + 1] * B.dims[i + 1];
  return gemm(ctx, mk(k, (int)ab2, 4 * c, 1, C.site[i], idx_plain(1), idx_plain(k), 0, ctx->Lp,
                      idx_plain(ab2), idx_plain(1), 0, out, idx_plain(ab2), idx_plain(1), 0));
}

// V_R[j][c'][a'][b'] = sum_{s',u',c''} C_j[c'][s'][u'][c''] Rp[s'][u'][c''][a'][b']
xtrg_status right_env(xtrg_ctx* ctx, const DevMpo& A, const DevMpo& B, const DevMpo& C, int j,
                      double* out) {
  const int k = C.dims[j], c2 = C.dims[j + 1];
  const long long ab1 = (long long)A.dims[j] * B.dims[j];
  return gemm(ctx, mk(k, (int)ab1, 4 * c2, 1, C.site[j], idx_plain(4 * c2), idx_plain(1), 0,
                      ctx->Rp, idx_plain(ab1), idx_plain(1), 0, out, idx_plain(ab1), idx_plain(1),
                      0));
}

#define CKM(x)                                                                              \
  do {                                                                                      \
    cudaError_t _e = (x);                                                                   \
    if (_e != cudaSuccess)                                                                  \
      return fail(ctx, XTRG_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #x,                  \
                  cudaGetErrorString(_e));                                                  \
  } while (0)

// Profiling: a pair of events around a stretch of stream work, tagged with
// its call site (tags 0-4: tensor-core GEMMs, 5: truncation of the
// tensor-core path, 6: one FP64 two-site update, 7: the FP64 initial right
// environments); the first is recorded here, the second by the caller after
// the work.
constexpr int TAG_SPLIT = 5, TAG_UPDATE64 = 6, TAG_ENVPASS64 = 7;
xtrg_status ev_pair(xtrg_ctx* ctx, int tag, cudaEvent_t* e0, cudaEvent_t* e1) {
  if (ctx->ev_used + 2 > ctx->ev.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      CKM(cudaEventCreate(&e));
      ctx->ev.push_back(e);
    }
  }
  *e0 = ctx->ev[ctx->ev_used++];
  *e1 = ctx->ev[ctx->ev_used++];
  ctx->ev_tag.push_back(tag);
  ctx->tag_n[tag]++;
  CKM(cudaEventRecord(*e0, ctx->st));
  return XTRG_OK;
}

// sum the recorded event intervals by tag (the stream has been synchronised)
xtrg_status resolve_events(xtrg_ctx* ctx) {
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float ms = 0.f;
    // a pair left open by a call that failed midway is skipped
    if (cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const int tag = i / 2 < ctx->ev_tag.size() ? ctx->ev_tag[i / 2] : 0;
    if (tag == TAG_SPLIT)
      ctx->split_ms += ms;
    else
      ctx->tc_ms += ms;
    ctx->tag_ms[tag] += ms;
  }
  ctx->ev_used = 0;
  ctx->ev_tag.clear();
  return XTRG_OK;
}

// Variational compression of A^T B into C (App. D.1).  C holds the guess,
// already right-canonical; on return C is the compressed MPO with its
// orthogonality centre at site 0.
xtrg_status compress(xtrg_ctx* ctx, const DevMpo& A, const DevMpo& B, DevMpo& C, int dstar,
                     int sweeps) {
  const int L = ctx->L;
  const int kcap = dstar < ctx->cap ? dstar : ctx->cap;
  CK(dev_fill(ctx->env[0], 1.0, 1, ctx->st));
  CK(dev_fill(ctx->env[L], 1.0, 1, ctx->st));
  cudaEvent_t p0 = nullptr, p1 = nullptr;
  if (ctx->profiling) TRY(ev_pair(ctx, TAG_ENVPASS64, &p0, &p1));
  for (int j = L - 1; j >= 1; --j) {
    TRY(right_part(ctx, A, B, C, j, ctx->env[j + 1]));
    TRY(right_env(ctx, A, B, C, j, ctx->env[j]));
  }
  if (p1) CK(cudaEventRecord(p1, ctx->st));
  double maxdisc = 0.0;
  for (int s = 0; s < sweeps; ++s) {
    const bool last = s == sweeps - 1;
    for (int dir = 0; dir < 2; ++dir) {
      for (int step = 0; step < L - 1; ++step) {
        const int i = dir == 0 ? step : L - 2 - step;
        cudaEvent_t u0 = nullptr, u1 = nullptr;
        if (ctx->profiling) TRY(ev_pair(ctx, TAG_UPDATE64, &u0, &u1));
        TRY(left_part(ctx, A, B, C, i, ctx->env[i]));
        TRY(right_part(ctx, A, B, C, i + 1, ctx->env[i + 2]));
        const int m = 4 * C.dims[i], n = 4 * C.dims[i + 2];
        const long long K = (long long)A.dims[i + 1] * B.dims[i + 1];
        TRY(gemm(ctx, mk(m, n, (int)K, 1, ctx->Lp, idx_plain(K), idx_plain(1), 0, ctx->Rp,
                         idx_plain(1), idx_plain(K), 0, ctx->CE, idx_plain(n), idx_plain(1), 0)));
        SvdResult r;
        TRY(split(ctx, ctx->CE, m, n, kcap, dir == 0 ? SPLIT_RIGHT : SPLIT_LEFT, C.site[i],
                  C.site[i + 1], &r));
        C.dims[i + 1] = r.k;
        if (last && r.discarded > maxdisc) maxdisc = r.discarded;
        if (dir == 0) TRY(left_env(ctx, A, B, C, i, ctx->env[i + 1]));
        else TRY(right_env(ctx, A, B, C, i + 1, ctx->env[i + 1]));
        if (u1) CK(cudaEventRecord(u1, ctx->st));
        ctx->updates++;
      }
    }
  }
  if (ctx->profiling) {
    CK(cudaStreamSynchronize(ctx->st));
    TRY(resolve_events(ctx));
  }
  ctx->last_trunc = maxdisc;
  return XTRG_OK;
}

// ------------------------------------------------ MPO sums (App. D.2)
// Overlap environments of one term T of an MPO sum with the compressed C:
// E[t][c] at each bond (t: T's bond, c: C's bond), left ones filled L->R and
// right ones R->L in one slot per bond, as the product's environments.
struct SumTerm {
  const DevMpo* T;
  double w;
  double* env;        // (L+1) slots of env_slot doubles
};

// G1[(c,s,u)][t'] = sum_t E_L[t][c] T_i[t][(s,u,t')]   (into g, Dc x 4 Dt')
xtrg_status sum_left_part(xtrg_ctx* ctx, const SumTerm& x, const DevMpo& C, int i, size_t slot,
                          double* g) {
  const int dt = x.T->dims[i], dt2 = x.T->dims[i + 1], dc = C.dims[i];
  return gemm64(ctx, mk(dc, 4 * dt2, dt, 1, x.env + (size_t)i * slot, idx_plain(1), idx_plain(dc), 0,
                        x.T->site[i], idx_plain(4 * dt2), idx_plain(1), 0, g, idx_plain(4 * dt2),
                        idx_plain(1), 0));
}

// G2[(t',s',u')][c''] = sum_t'' T_j[(t',s',u')][t''] E_R[t''][c'']   (into g, 4 Dt' x Dc'')
xtrg_status sum_right_part(xtrg_ctx* ctx, const SumTerm& x, const DevMpo& C, int j, size_t slot,
                           double* g) {
  const int dt = x.T->dims[j], dt2 = x.T->dims[j + 1], dc2 = C.dims[j + 1];
  return gemm64(ctx, mk(4 * dt, dc2, dt2, 1, x.T->site[j], idx_plain(dt2), idx_plain(1), 0,
                        x.env + (size_t)(j + 1) * slot, idx_plain(dc2), idx_plain(1), 0, g,
                        idx_plain(dc2), idx_plain(1), 0));
}

// E_L at bond i+1: E'[t'][c'] = sum_(c,s,u) G1[(c,s,u)][t'] C_i[(c,s,u)][c']
xtrg_status sum_left_env(xtrg_ctx* ctx, const SumTerm& x, const DevMpo& C, int i, size_t slot,
                         double* g) {
  TRY(sum_left_part(ctx, x, C, i, slot, g));
  const int dt2 = x.T->dims[i + 1], dc = C.dims[i], dc2 = C.dims[i + 1];
  return gemm64(ctx, mk(dt2, dc2, 4 * dc, 1, g, idx_plain(1), idx_plain(dt2), 0, C.site[i],
                        idx_plain(dc2), idx_plain(1), 0, x.env + (size_t)(i + 1) * slot,
                        idx_plain(dc2), idx_plain(1), 0));
}

// E_R at bond j: E[t][c] = sum_(s,u,c'') G2[t][(s,u,c'')] C_j[c][(s,u,c'')]
xtrg_status sum_right_env(xtrg_ctx* ctx, const SumTerm& x, const DevMpo& C, int j, size_t slot,
                          double* g) {
  TRY(sum_right_part(ctx, x, C, j, slot, g));
  const int dt = x.T->dims[j], dc = C.dims[j], dc2 = C.dims[j + 1];
  return gemm64(ctx, mk(dt, dc, 4 * dc2, 1, g, idx_plain(4 * dc2), idx_plain(1), 0, C.site[j],
                        idx_plain(1), idx_plain(4 * dc2), 0, x.env + (size_t)j * slot,
                        idx_plain(dc), idx_plain(1), 0));
}

// Variational compression of sum_j w_j T_j into C (App. D.2, Eq. LSESum):
// C holds the guess, right-canonical; the two-site solution is
// C_i C_{i+1} = sum_j w_j C_E,j with C_E,j = G1_j G2_j, split as in the
// product compression.  On return the orthogonality centre is site 0.
xtrg_status compress_sum(xtrg_ctx* ctx, std::vector<SumTerm>& terms, DevMpo& C, int dstar,
                         int sweeps, size_t slot) {
  const int L = ctx->L;
  const int kcap = dstar < ctx->cap ? dstar : ctx->cap;
  double* g1 = ctx->T1;
  double* g2 = ctx->Lp;
  for (auto& x : terms) {
    CK(dev_fill(x.env, 1.0, 1, ctx->st));
    CK(dev_fill(x.env + (size_t)L * slot, 1.0, 1, ctx->st));
    for (int j = L - 1; j >= 1; --j) TRY(sum_right_env(ctx, x, C, j, slot, g2));
  }
  double maxdisc = 0.0;
  for (int s = 0; s < sweeps; ++s) {
    const bool last = s == sweeps - 1;
    for (int dir = 0; dir < 2; ++dir) {
      for (int step = 0; step < L - 1; ++step) {
        const int i = dir == 0 ? step : L - 2 - step;
        const int m = 4 * C.dims[i], n = 4 * C.dims[i + 2];
        for (size_t t = 0; t < terms.size(); ++t) {
          const SumTerm& x = terms[t];
          TRY(sum_left_part(ctx, x, C, i, slot, g1));
          TRY(sum_right_part(ctx, x, C, i + 1, slot, g2));
          const int dt = x.T->dims[i + 1];
          GemmF64 g = mk(m, n, dt, 1, g1, idx_plain(dt), idx_plain(1), 0, g2, idx_plain(n),
                         idx_plain(1), 0, ctx->CE, idx_plain(n), idx_plain(1), 0);
          g.alpha = x.w;
          g.beta = t == 0 ? 0.0 : 1.0;
          TRY(gemm(ctx, g));
        }
        SvdResult r;
        TRY(split(ctx, ctx->CE, m, n, kcap, dir == 0 ? SPLIT_RIGHT : SPLIT_LEFT, C.site[i],
                  C.site[i + 1], &r));
        C.dims[i + 1] = r.k;
        if (last && r.discarded > maxdisc) maxdisc = r.discarded;
        for (auto& x : terms) {
          if (dir == 0) TRY(sum_left_env(ctx, x, C, i, slot, g1));
          else TRY(sum_right_env(ctx, x, C, i + 1, slot, g2));
        }
        ctx->updates++;
      }
    }
  }
  ctx->last_trunc = maxdisc;
  return XTRG_OK;
}

// ||C_0||_F for the centre site; C_0 /= s.  Returns ln s.
// Device part: s^2 = ||C_0||_F^2 into ctx->scal[0], C_0 /= s (no host read).
xtrg_status normalize_device(xtrg_ctx* ctx, DevMpo& C) {
  const long long n = (long long)site_elems(C, 0);
  CK(dev_sumsq(C.site[0], n, ctx->scal, ctx->st));
  CK(dev_scale_rsqrt(C.site[0], ctx->scal, n, ctx->st));
  return XTRG_OK;
}

// Host part: reads s^2 (synchronises), *lns = ln s.
xtrg_status normalize_finish(xtrg_ctx* ctx, double* lns) {
  double ss = 0.0;
  CK(cudaMemcpyAsync(&ss, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (!(ss > 0.0) || !std::isfinite(ss))
    return fail(ctx, XTRG_ENUMERIC, "norm of the compressed MPO is %g", ss);
  *lns = std::log(std::sqrt(ss));
  return XTRG_OK;
}

xtrg_status normalize(xtrg_ctx* ctx, DevMpo& C, double* lns) {
  TRY(normalize_device(ctx, C));
  return normalize_finish(ctx, lns);
}

// Debug mode (environment XTRG_DEBUG=1): after each step of a product, scan
// the FP64 result for non-finite values and name the first step that made one.
bool debug_on() {
  static const bool v = []() {
    const char* e = getenv("XTRG_DEBUG");
    return e && e[0] == '1';
  }();
  return v;
}

xtrg_status debug_check(xtrg_ctx* ctx, const char* what, const double* p, long long n, int i) {
  if (!debug_on() || n <= 0) return XTRG_OK;
  CK(dev_sumsq(p, n, ctx->scal + 16, ctx->st));
  double v = 0.0;
  CK(cudaMemcpyAsync(&v, ctx->scal + 16, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (!std::isfinite(v))
    return fail(ctx, XTRG_ENUMERIC, "debug: %s at bond %d is not finite (sum of squares %g)", what,
                i, v);
  return XTRG_OK;
}

bool mixed_for_beta(const xtrg_ctx* ctx, double beta) {
  return ctx->cfg.prec != XTRG_FP64 && ctx->mixed_ready && beta >= ctx->cfg.beta_switch;
}

// ============================================================ tensor-core path
// The doubling product A = B = rho with every contraction on tcgen05.  Layouts
// (all operands K-major, BF16 planes, rows padded to tc_ld):
//   site copies  sT[(s,a',t)][a]   sP[(u,b')][(b,t)]   sN[(a',t',s')][a'']   sQ[(b',u')][(t',b'')]
//   environment  V[c][b][a]                 (left and right alike)
//   left half    T1[c][(s,a')][(b,t)]  ->  Lp[(c,s,u)][(b',a')]
//   right half   T1R[c''][(a',s')][(t',b'')]  ->  Rp[(s',u',c'')][(b',a')]
//   C_E = Lp Rp^T (split-K, FP64 sum); env update V' = C^T-part x (Lp or Rp)
//   with the half read MN-major.

TcOperand opnd(const __nv_bfloat16* base, int P, int rows, int k, long long ld,
               long long batch_stride, long long plane_stride, int batches) {
  TcOperand o;
  o.base = base; o.planes = P; o.rows = rows; o.k = k; o.ld = ld;
  o.batch_stride = batch_stride; o.plane_stride = plane_stride; o.batches = batches;
  return o;
}

TcOutput out_planes(__nv_bfloat16* base, int P, long long ps, Idx3 cm, Idx3 cn, long long scb) {
  TcOutput o;
  memset(&o, 0, sizeof o);
  o.mode = TC_OUT_BF16P; o.bf16 = base; o.planes = P; o.plane_stride = ps;
  o.cm = cm; o.cn = cn; o.scb = scb; o.alpha = 1.0;
  return o;
}

xtrg_status tc(xtrg_ctx* ctx, const TcOperand& A, const TcOperand& B, int M, int N, int K,
               int batch, int splitk, const TcOutput& o) {
  const double fl = 2.0 * M * (double)N * K * batch;
  ctx->flops_contr += fl;
  ctx->tc_flops += fl;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->profiling) {
    TRY(ev_pair(ctx, ctx->cur_tag, &e0, &e1));
    ctx->tag_flops[ctx->cur_tag] += fl;
  }
  CKM(tc_gemm(A, B, M, N, K, batch, ctx->m.nprod, splitk, o, ctx->m.err, ctx->st));
  if (e1) {
    CKM(cudaEventRecord(e1, ctx->st));
    ctx->tc_launches++;
  }
  return XTRG_OK;
}


// BF16-plane copies of rho's sites for the four substep layouts.
xtrg_status mixed_prepare(xtrg_ctx* ctx) {
  const DevMpo& R = ctx->rho;
  const int P = ctx->m.P;
  for (int i = 0; i < ctx->L; ++i) {
    const int l = R.dims[i], r = R.dims[i + 1];
    const double* w = R.site[i];
    // rows (s, a', t): t, which pairs with b in T1's contraction index
    // (b, t), is innermost, so the epilogue writes each (b, t) pair as one
    // 4-byte store per plane
    CKM(to_planes(w, idx_split3(r, 2, r, 1, 2LL * r), idx_plain(4LL * r), 0, 4 * r, l, 1,
                  ctx->m.site[0][i], tc_ld(l), 0, P, ctx->plan.m_site[0], ctx->st));
    CKM(to_planes(w, idx_plain(1), idx_plain(2LL * r), 0, 2 * r, 2 * l, 1, ctx->m.site[1][i],
                  tc_ld(2 * l), 0, P, ctx->plan.m_site[1], ctx->st));
    CKM(to_planes(w, idx_plain(r), idx_plain(1), 0, 4 * l, r, 1, ctx->m.site[2][i], tc_ld(r), 0, P,
                  ctx->plan.m_site[2], ctx->st));
    CKM(to_planes(w, idx_split2(2, 4LL * r, r), idx_split2(r, 2LL * r, 1), 0, 2 * l, 2 * r, 1,
                  ctx->m.site[3][i], tc_ld(2 * r), 0, P, ctx->plan.m_site[3], ctx->st));
  }
  return XTRG_OK;
}

// env slot [c][b][a] from an FP64 scalar 1 (the boundary environments)
xtrg_status mixed_unit_env(xtrg_ctx* ctx, int slot) {
  CK(dev_fill(ctx->scal + 8, 1.0, 1, ctx->st));
  CKM(to_planes(ctx->scal + 8, idx_plain(0), idx_plain(0), 0, 1, 1, 1, ctx->m.env[slot], tc_ld(1),
                0, ctx->m.P, ctx->plan.m_env, ctx->st));
  return XTRG_OK;
}

// Lp from env[i] and site i (left half of Fig. VMPO(a), substeps 1-2)
xtrg_status mixed_left_part(xtrg_ctx* ctx, const DevMpo& C, int i) {
  __nv_bfloat16* Lp = ctx->m.lpc[i];
  const DevMpo& R = ctx->rho;
  const int P = ctx->m.P;
  const int a = R.dims[i], a2 = R.dims[i + 1], c = C.dims[i];
  const long long ldE = tc_ld(a), ld1 = tc_ld(2 * a), ldL = tc_ld((long long)a2 * a2);
  ctx->cur_tag = 1;
  TcOperand Ae = opnd(ctx->m.env[i], P, a, a, ldE, (long long)a * ldE, ctx->plan.m_env, c);
  TcOperand Bs = opnd(ctx->m.site[0][i], P, 4 * a2, a, tc_ld(a), 0, ctx->plan.m_site[0], 1);
  TRY(tc(ctx, Ae, Bs, a, 4 * a2, a, c, 1,
         out_planes(ctx->m.T1, P, ctx->plan.m_t1, idx_plain(2),
                    idx_split3(a2, 2, (long long)a2 * ld1, ld1, 1), 2LL * a2 * ld1)));
  ctx->cur_tag = 2;
  TcOperand At = opnd(ctx->m.T1, P, 2 * a2, 2 * a, ld1, 2LL * a2 * ld1, ctx->plan.m_t1, c);
  TcOperand Bp = opnd(ctx->m.site[1][i], P, 2 * a2, 2 * a, tc_ld(2 * a), 0, ctx->plan.m_site[1], 1);
  TRY(tc(ctx, At, Bp, 2 * a2, 2 * a2, 2 * a, c, 1,
         out_planes(Lp, P, ctx->plan.m_lp, idx_split2(a2, 2 * ldL, 1),
                    idx_split2(a2, ldL, a2), 4 * ldL)));
  return XTRG_OK;
}

// Rp from env[j+1] and site j (right half)
xtrg_status mixed_right_part(xtrg_ctx* ctx, const DevMpo& C, int j) {
  __nv_bfloat16* Rp = ctx->m.rpc[j];
  const DevMpo& R = ctx->rho;
  const int P = ctx->m.P;
  const int a2 = R.dims[j], a3 = R.dims[j + 1], c2 = C.dims[j + 1];
  const long long ldE = tc_ld(a3), ld2 = tc_ld(2 * a3), ldR = tc_ld((long long)a2 * a2);
  ctx->cur_tag = 1;
  TcOperand An = opnd(ctx->m.site[2][j], P, 4 * a2, a3, tc_ld(a3), 0, ctx->plan.m_site[2], 1);
  TcOperand Be = opnd(ctx->m.env[j + 1], P, a3, a3, ldE, (long long)a3 * ldE, ctx->plan.m_env, c2);
  TRY(tc(ctx, An, Be, 4 * a2, a3, a3, c2, 1,
         out_planes(ctx->m.T1R, P, ctx->plan.m_t1, idx_split3(2, 2, 2 * ld2, a3, ld2),
                    idx_plain(1), 2LL * a2 * ld2)));
  ctx->cur_tag = 2;
  TcOperand At = opnd(ctx->m.T1R, P, 2 * a2, 2 * a3, ld2, 2LL * a2 * ld2, ctx->plan.m_t1, c2);
  TcOperand Bq = opnd(ctx->m.site[3][j], P, 2 * a2, 2 * a3, tc_ld(2 * a3), 0, ctx->plan.m_site[3], 1);
  TRY(tc(ctx, At, Bq, 2 * a2, 2 * a2, 2 * a3, c2, 1,
         out_planes(Rp, P, ctx->plan.m_lp, idx_split2(2, 1, 2LL * c2 * ldR),
                    idx_split2(2, a2, (long long)c2 * ldR), ldR)));
  return XTRG_OK;
}

// new environment at slot from a C site (FP64) and the Lp or Rp planes:
//   left:  V'[c'][b'][a'] = sum_{(c,s,u)} C_i[(c,s,u)][c'] Lp[(c,s,u)][(b',a')]
//   right: V'[c'][b'][a'] = sum_{(s',u',c'')} C_j[c'][(s',u',c'')] Rp[(s',u',c'')][(b',a')]
xtrg_status mixed_env(xtrg_ctx* ctx, const double* Csite, int kout, int kin, bool left,
                      const __nv_bfloat16* part, int a, int slot) {
  const int P = ctx->m.P;
  const long long ab = (long long)a * a, ldP = tc_ld(ab), ldK = tc_ld(kin), ldE = tc_ld(a);
  // C^T-part [c'][k]: left reads C_i[k][c'], right reads C_j[c'][k]
  CKM(to_planes(Csite, left ? idx_plain(1) : idx_plain(kin), left ? idx_plain(kout) : idx_plain(1),
                0, kout, kin, 1, ctx->m.Ct, ldK, 0, P, ctx->plan.m_ct, ctx->st));
  ctx->cur_tag = 4;
  TcOperand Ac = opnd(ctx->m.Ct, P, kout, kin, ldK, 0, ctx->plan.m_ct, 1);
  // B(n = (b',a'), k = (c,s,u)) is the half itself, [k][n] with row stride
  // ldP: staged MN-major, no transpose pass
  TcOperand Bt = opnd(part, P, (int)ab, kin, ldP, 0, ctx->plan.m_lp, 1);
  Bt.mn_major = 1;
  return tc(ctx, Ac, Bt, kout, (int)ab, kin, 1, 1,
            out_planes(ctx->m.env[slot], P, ctx->plan.m_env, idx_plain((long long)a * ldE),
                       idx_split2(a, ldE, 1), 0));
}

// C_E = Lp Rp^T (FP32 accumulation, split-K partials summed in FP64)
// split-K of C_E chosen by the autotuner, per device, plane count and shape
struct SplitKey {
  int dev, planes, m, n;
  long long K;
  bool operator<(const SplitKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (planes != o.planes) return planes < o.planes;
    if (m != o.m) return m < o.m;
    if (n != o.n) return n < o.n;
    return K < o.K;
  }
};
std::map<SplitKey, int> g_split_tuned;
std::mutex g_split_mu;

xtrg_status mixed_ce(xtrg_ctx* ctx, const __nv_bfloat16* Lp, const __nv_bfloat16* Rp, int m, int n,
                     int a2) {
  const int P = ctx->m.P;
  const long long K = (long long)a2 * a2, ld = tc_ld(K);
  const int kb = (int)((K + 63) / 64);
  const int tiles = ((m + 127) / 128) * ((n + 127) / 128);
  // split-K only to fill the persistent CTAs (the kernel's accumulation is
  // unbiased at any chain length): the fewest splits whose work units fill
  // their waves over the SMs to >= 95 %, each split keeping >= 4 K-blocks;
  // the FP32 partials are summed in FP64
  const int sms = ctx->sms;
  int splitk = 1;
  {
    int best = 1;
    double best_eff = 0.0;
    for (int s = 1; s <= SPLITK_MAX && s <= kb / 4; ++s) {
      const long long units = (long long)tiles * s;
      const long long waves = (units + sms - 1) / sms;
      const double eff = (double)units / (double)(waves * sms);
      if (eff > best_eff + 1e-9) {
        best = s;
        best_eff = eff;
      }
      if (eff >= 0.95) break;
    }
    splitk = best;
  }
  ctx->cur_tag = 3;
  TcOperand Al = opnd(Lp, P, m, (int)K, ld, 0, ctx->plan.m_lp, 1);
  TcOperand Br = opnd(Rp, P, n, (int)K, ld, 0, ctx->plan.m_lp, 1);
  TcOutput o;
  memset(&o, 0, sizeof o);
  o.mode = TC_OUT_PARTIAL; o.f32 = ctx->m.part; o.alpha = 1.0;
  // autotuner: the first time a shape is met (outside a graph capture), the
  // heuristic's split and its neighbours are each timed by CUDA events (two
  // launches, the second timed) and the fastest is kept for the shape.  The
  // choice is shared by every context of the process (under a lock, so that
  // concurrent contexts of a batch agree), which keeps the results of equal
  // runs in one process identical.
  int dev = 0;
  CKM(cudaGetDevice(&dev));
  const SplitKey key{dev, P, m, n, K};
  std::unique_lock<std::mutex> lock(g_split_mu);
  const auto hit = g_split_tuned.find(key);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CKM(cudaStreamIsCapturing(ctx->st, &cap));
  if (hit != g_split_tuned.end()) {
    splitk = hit->second;
  } else if (ctx->tune_splits && cap == cudaStreamCaptureStatusNone && kb >= 16) {
    const int lim = SPLITK_MAX < kb / 4 ? SPLITK_MAX : kb / 4;
    const int cand[4] = {splitk, splitk / 2, 2 * splitk, (3 * splitk + 1) / 2};
    cudaEvent_t e0, e1;
    CKM(cudaEventCreate(&e0));
    CKM(cudaEventCreate(&e1));
    int best = splitk;
    float best_ms = 1e30f;
    for (int c = 0; c < 4; ++c) {
      const int sk = cand[c];
      if (sk < 1 || sk > lim || (c > 0 && sk == splitk)) continue;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        CKM(cudaEventRecord(e0, ctx->st));
        CKM(tc_gemm(Al, Br, m, n, (int)K, 1, ctx->m.nprod, sk, o, ctx->m.err, ctx->st));
        CKM(cudaEventRecord(e1, ctx->st));
        CKM(cudaEventSynchronize(e1));
        CKM(cudaEventElapsedTime(&ms, e0, e1));
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = sk;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_split_tuned[key] = best;
    splitk = best;
  }
  lock.unlock();
  TRY(tc(ctx, Al, Br, m, n, (int)K, 1, splitk, o));
  // FP64 C_E (exact fallback, debug scans), its planes in both orientations
  // for the subspace products and ||C_E||^2, in one pass over the partials
  CKM(reduce_partials_planes(ctx->m.part, splitk, m, n, ctx->CE, ctx->m.sb.ce_rm, tc_ld(n),
                             ctx->m.sb.ce_tr, tc_ld(m), ctx->m.sb.ce_ps, ctx->m.sb.ce_ss,
                             ctx->st));
  return XTRG_OK;
}

// Largest orthonormality defect of the subspace truncation's factor that is
// accepted; above it the exact FP64 split runs instead.
constexpr double ORTH_DEFECT_MAX = 1e-4;

// The one host read of a tensor-core product: the bounded-wait flag of the
// GEMMs, the largest discarded weight of the last sweep, the exact-split
// fallbacks and their status.
xtrg_status finish_mixed(xtrg_ctx* ctx) {
  int h = 0;
  double a[4];
  CKM(cudaMemcpyAsync(&h, ctx->m.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CKM(cudaMemcpyAsync(a, ctx->m.acc, sizeof a, cudaMemcpyDeviceToHost, ctx->st));
  CKM(cudaStreamSynchronize(ctx->st));
  if (h) return fail(ctx, XTRG_ETIMEOUT, "a bounded tensor-core pipeline wait expired");
  unsigned long long runs = 0;
  int status = 0;
  memcpy(&runs, &a[1], sizeof runs);
  memcpy(&status, &a[3], sizeof status);
  ctx->fallbacks = (long long)runs;
  if (status == 1) return fail(ctx, XTRG_ETIMEOUT, "exact split: a bounded device barrier expired");
  if (status == 2) return fail(ctx, XTRG_ENUMERIC, "exact split: Jacobi SVD did not converge");
  if (status == 3) return fail(ctx, XTRG_ENUMERIC, "exact split: non-finite singular value");
  ctx->last_trunc = a[0];
  return XTRG_OK;
}

xtrg_status compress_mixed(xtrg_ctx* ctx, DevMpo& C, int dstar, int sweeps) {
  const int L = ctx->L;
  const DevMpo& R = ctx->rho;
  const int kcap = dstar < ctx->cap ? dstar : ctx->cap;
  const bool keep = ctx->cfg.keep_parts != 0;
  double* disc_max = ctx->m.acc;
  const SvdDeviceAcc acc{disc_max, reinterpret_cast<unsigned long long*>(ctx->m.acc + 1),
                         reinterpret_cast<int*>(ctx->m.acc + 3)};
  // every decision of the sweeps is taken on the device: no host read until
  // the end of the product
  CKM(cudaMemsetAsync(ctx->m.err, 0, sizeof(int), ctx->st));
  CKM(cudaMemsetAsync(ctx->m.acc + 3, 0, sizeof(double), ctx->st));
  CKM(subspace_next_seed(ctx->m.sb, ctx->st));
  TRY(mixed_unit_env(ctx, 0));
  TRY(mixed_unit_env(ctx, L));
  for (int j = L - 1; j >= 1; --j) {
    TRY(mixed_right_part(ctx, C, j));
    TRY(mixed_env(ctx, C.site[j], C.dims[j], 4 * C.dims[j + 1], false, ctx->m.rpc[j], R.dims[j], j));
  }
  long long upd = 0;   // updates of this product (the noise seed of its truncation)
  for (int s = 0; s < sweeps; ++s) {
    const bool last = s == sweeps - 1;
    if (last) CKM(cudaMemsetAsync(disc_max, 0, sizeof(double), ctx->st));
    for (int dir = 0; dir < 2; ++dir) {
      for (int step = 0; step < L - 1; ++step, ++upd) {
        const int i = dir == 0 ? step : L - 2 - step;
        // Left-to-right, the left half of bond i is new (environment i was
        // just rebuilt) and the right half is unchanged since it was built
        // from environment i+2; right-to-left the roles swap.  Resident
        // halves are reused; otherwise both are rebuilt.
        if (dir == 0 || !keep) TRY(mixed_left_part(ctx, C, i));
        if (dir == 1 || !keep) TRY(mixed_right_part(ctx, C, i + 1));
        const int m = 4 * C.dims[i], n = 4 * C.dims[i + 2];
        TRY(mixed_ce(ctx, ctx->m.lpc[i], ctx->m.rpc[i + 1], m, n, R.dims[i + 1]));
        TRY(debug_check(ctx, "C_E", ctx->CE, (long long)m * n, i));
        // keep k = min(D*, m, n): the FP32-level C_E has no FP64-exact numerical rank
        int k = kcap < m ? kcap : m;
        k = k < n ? k : n;
        const unsigned long long seed = 0x243F6A8885A308D3ull ^ (unsigned long long)upd;
        cudaEvent_t s0 = nullptr, s1 = nullptr;
        if (ctx->profiling) TRY(ev_pair(ctx, TAG_SPLIT, &s0, &s1));
        const SplitMode mode = dir == 0 ? SPLIT_RIGHT : SPLIT_LEFT;
        const SvdDeviceAcc a{last ? acc.disc_max : nullptr, acc.runs, acc.status};
        if (k > SUBSPACE_MAX_K) {
          // wider than the blocked orthonormalisation handles: exact split
          CKM(svd_split_f64_if(ctx->CE, m, n, k, mode, C.site[i], C.site[i + 1], ctx->svd, ctx->st,
                               ctx->m.acc + 2, 0.0, a));
        } else {
          if (dir == 0)
            CKM(subspace_split(ctx->CE, m, n, k, 1, C.site[i + 1], C.dims[i + 1], C.site[i],
                               C.site[i + 1], seed, ctx->m.sb, ctx->st, a.disc_max, ORTH_DEFECT_MAX));
          else
            CKM(subspace_split(ctx->CE, m, n, k, 0, C.site[i], C.dims[i + 1], C.site[i],
                               C.site[i + 1], seed, ctx->m.sb, ctx->st, a.disc_max, ORTH_DEFECT_MAX));
          // the FP32 orthonormalisation lost orthogonality (steep or rank-
          // deficient spectrum): the exact FP64 Jacobi split replaces it,
          // decided on the device from the defect
          CKM(svd_split_f64_if(ctx->CE, m, n, k, mode, C.site[i], C.site[i + 1], ctx->svd, ctx->st,
                               subspace_defect(ctx->m.sb), ORTH_DEFECT_MAX, a));
        }
        if (s1) CKM(cudaEventRecord(s1, ctx->st));
        C.dims[i + 1] = k;
        TRY(debug_check(ctx, "left factor", C.site[i], (long long)m * k, i));
        TRY(debug_check(ctx, "right factor", C.site[i + 1], (long long)k * n, i));
        ctx->flops_split += 2.0 * m * (double)n * k * 2 + 3.0 * (2.0 * (dir == 0 ? m : n) * k * k);
        if (dir == 0)
          TRY(mixed_env(ctx, C.site[i], k, m, true, ctx->m.lpc[i], R.dims[i + 1], i + 1));
        else
          TRY(mixed_env(ctx, C.site[i + 1], k, n, false, ctx->m.rpc[i + 1], R.dims[i + 1], i + 1));
        ctx->updates++;
      }
    }
  }
  return XTRG_OK;
}

// ------------------------------------------------------------ transfers
// Tr rho, Tr(H rho), Tr(H^2 rho) by left-to-right transfer contractions.
xtrg_status traces(xtrg_ctx* ctx, bool want_h, double out[3]) {
  const int L = ctx->L;
  const DevMpo& R = ctx->rho;
  const DevMpo& H = ctx->H;
  double* v[2] = {ctx->ob[0], ctx->ob[1]};
  // Tr rho: v'[r'] = sum_{r,s} v[r] rho[r][s][s][r']
  CK(dev_fill(v[0], 1.0, 1, ctx->st));
  for (int i = 0; i < L; ++i) {
    const int l = R.dims[i], r = R.dims[i + 1];
    TRY(gemm64(ctx, mk(1, r, 2 * l, 1, v[i & 1], idx_plain(0), idx_split2(2, 1, 0), 0, R.site[i],
                       idx_split2(2, 4LL * r, 3LL * r), idx_plain(1), 0, v[(i + 1) & 1],
                       idx_plain(0), idx_plain(1), 0)));
  }
  CK(cudaMemcpyAsync(&out[0], v[L & 1], sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  out[1] = out[2] = 0.0;
  if (want_h) {
    // Tr(H rho): E'[h'][r'] = sum H[h][s][t][h'] E[h][r] rho[r][t][s][r']
    double* E[2] = {ctx->ob[0], ctx->ob[1]};
    double* T = ctx->ob[2];
    CK(dev_fill(E[0], 1.0, 1, ctx->st));
    for (int i = 0; i < L; ++i) {
      const int l = R.dims[i], r = R.dims[i + 1], hl = H.dims[i], hr = H.dims[i + 1];
      TRY(gemm64(ctx, mk(hl, 4 * r, l, 1, E[i & 1], idx_plain(l), idx_plain(1), 0, R.site[i],
                         idx_plain(4 * r), idx_plain(1), 0, T, idx_plain(4 * r), idx_plain(1), 0)));
      TRY(gemm64(ctx, mk(hr, r, 4 * hl, 1, H.site[i], idx_plain(1), idx_plain(hr), 0, T,
                         idx_split3(2, 2, 4LL * r, r, 2LL * r), idx_plain(1), 0, E[(i + 1) & 1],
                         idx_plain(r), idx_plain(1), 0)));
    }
    CK(cudaMemcpyAsync(&out[1], E[L & 1], sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    // Tr(H H rho): E'[h1'][h2'][r'] = sum E[h1][h2][r] H[h1][s][t][h1'] H[h2][t][v][h2'] rho[r][v][s][r']
    double* T1 = ctx->ob[2];
    double* T2 = ctx->ob[0];
    double* Ea = ctx->ob[1];
    CK(dev_fill(Ea, 1.0, 1, ctx->st));
    for (int i = 0; i < L; ++i) {
      const int l = R.dims[i], r = R.dims[i + 1], hl = H.dims[i], hr = H.dims[i + 1];
      TRY(gemm64(ctx, mk(hl * hl, 4 * r, l, 1, Ea, idx_plain(l), idx_plain(1), 0, R.site[i],
                         idx_plain(4 * r), idx_plain(1), 0, T1, idx_plain(4 * r), idx_plain(1), 0)));
      TRY(gemm64(ctx, mk(hl * 2 * r, 2 * hr, 2 * hl, 1, T1, idx_split3(2, r, 4LL * r, 2LL * r, 1),
                         idx_split2(2, (long long)hl * 4 * r, r), 0, H.site[i],
                         idx_plain(2 * hr), idx_plain(1), 0, T2, idx_plain(2 * hr), idx_plain(1),
                         0)));
      TRY(gemm64(ctx, mk(hr, r, 4 * hl, hr, H.site[i], idx_plain(1), idx_plain(hr), 0, T2,
                         idx_split3(2, 2, 2LL * r * 2 * hr, hr, (long long)r * 2 * hr),
                         idx_plain(2 * hr), 1, Ea, idx_plain(r), idx_plain(1), (long long)hr * r)));
    }
    CK(cudaMemcpyAsync(&out[2], Ea, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  return XTRG_OK;
}

// ||rho||_F^2 = sum rho_{s,t} rho_{s,t} and Tr(rho rho) = sum rho_{s,t} rho_{t,s}
// by left-to-right transfer matrices E[l][m] (FP64).  Both share the first
// contraction of each site, T[m][s][t][x] = sum_l E[l][m] rho[l][s][t][x];
// the second pairs T with rho[m][s][t][y] (Frobenius) or rho[m][t][s][y]
// (the transpose on the physical pair).  Their difference is the
// Hermiticity defect ||rho - rho^T||_F^2 = 2 (||rho||_F^2 - Tr(rho rho))
// of a real rho (Sec. II B: rho^T rho is the positivity-preserving product).
xtrg_status herm_transfers(xtrg_ctx* ctx, double* fro, double* trr) {
  const int L = ctx->L;
  const DevMpo& R = ctx->rho;
  double* T = ctx->ht;
  CK(dev_fill(ctx->hf[0], 1.0, 1, ctx->st));
  CK(dev_fill(ctx->hr[0], 1.0, 1, ctx->st));
  for (int i = 0; i < L; ++i) {
    const int l = R.dims[i], r = R.dims[i + 1];
    double* Ef = ctx->hf[i & 1];
    double* Er = ctx->hr[i & 1];
    for (int which = 0; which < 2; ++which) {
      const double* E = which == 0 ? Ef : Er;
      double* En = which == 0 ? ctx->hf[(i + 1) & 1] : ctx->hr[(i + 1) & 1];
      // T[m][(s,t,x)] = sum_l E[l][m] rho[l][(s,t,x)]
      TRY(gemm64(ctx, mk(l, 4 * r, l, 1, E, idx_plain(1), idx_plain(l), 0, R.site[i],
                         idx_plain(4 * r), idx_plain(1), 0, T, idx_plain(4 * r), idx_plain(1), 0)));
      // E'[x][y] = sum_{(m,s,t)} T[(m,s,t)][x] rho[m][s or t][t or s][y]
      const Idx3 bk = which == 0 ? idx_plain(r) : idx_split3(2, 2, 4LL * r, r, 2LL * r);
      TRY(gemm64(ctx, mk(r, r, 4 * l, 1, T, idx_plain(1), idx_plain(r), 0, R.site[i], bk,
                         idx_plain(1), 0, En, idx_plain(r), idx_plain(1), 0)));
    }
  }
  CK(cudaMemcpyAsync(fro, ctx->hf[L & 1], sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(trr, ctx->hr[L & 1], sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return XTRG_OK;
}

xtrg_status check_mpo(const xtrg_mpo* m, int cap_bond) {
  if (!m || m->L < 2 || m->d != 2 || !m->bond_dims || !m->W) return XTRG_EINVAL;
  if (m->bond_dims[0] != 1 || m->bond_dims[m->L] != 1) return XTRG_EINVAL;
  for (int i = 0; i <= m->L; ++i)
    if (m->bond_dims[i] < 1 || m->bond_dims[i] > cap_bond) return XTRG_EINVAL;
  for (int i = 0; i < m->L; ++i)
    if (!m->W[i]) return XTRG_EINVAL;
  return XTRG_OK;
}

int max_bond(const xtrg_mpo* m) {
  int mx = 1;
  for (int i = 0; i <= m->L; ++i) mx = m->bond_dims[i] > mx ? m->bond_dims[i] : mx;
  return mx;
}

}  // namespace

// ===================================================================== ABI

extern "C" size_t xtrg_workspace_bytes(const xtrg_mpo* H, const xtrg_config* cfg) {
  if (!cfg || check_mpo(H, 1 << 20) != XTRG_OK) return 0;
  Plan p;
  if (!plan_sizes(H->L, max_bond(H), cfg, &p)) return 0;
  return p.total;
}

extern "C" xtrg_status xtrg_create(xtrg_ctx** out, const xtrg_mpo* Hm, const xtrg_config* cfg,
                                   void* dev_workspace, size_t workspace_bytes, void* cuda_stream) {
  if (!out) return XTRG_EINVAL;
  *out = nullptr;
  if (!cfg || check_mpo(Hm, 1 << 20) != XTRG_OK) return XTRG_EINVAL;
  if (!(cfg->tau0 > 0.0) || cfg->order < 1 || cfg->order > 16 || cfg->sweeps < 1 ||
      cfg->init_sweeps < 1 || cfg->dstar < 1 || cfg->dstar > 1024 || !(cfg->svd_rel_tol >= 0.0) ||
      (int)cfg->prec < 0 || (int)cfg->prec > 2 || cfg->orth_block < 0 ||
      cfg->orth_block > SUBSPACE_BLOCK_K || cfg->orth_block % 32)
    return XTRG_EINVAL;
  if (!dev_workspace || ((uintptr_t)dev_workspace % ALIGN) != 0) return XTRG_EINVAL;
  Plan p;
  if (!plan_sizes(Hm->L, max_bond(Hm), cfg, &p)) return XTRG_EINVAL;
  if (workspace_bytes < p.total) return XTRG_ENOMEM;
  xtrg_ctx* ctx = new xtrg_ctx();
  ctx->st = (cudaStream_t)cuda_stream;
  ctx->ws = (char*)dev_workspace;
  ctx->ws_bytes = workspace_bytes;
  ctx->cfg = *cfg;
  ctx->plan = p;
  ctx->L = Hm->L;
  ctx->DH = p.DH;
  ctx->cap = p.cap;
  {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      ctx->sms = n;
  }
  bool ok = carve_mpo(ctx, &ctx->H, p.n_h) && carve_mpo(ctx, &ctx->I, 4) &&
            carve_mpo(ctx, &ctx->rho, p.n_csite) && carve_mpo(ctx, &ctx->C, p.n_csite) &&
            carve_mpo(ctx, &ctx->Y, p.n_site) && carve_mpo(ctx, &ctx->fat, p.n_fat);
  ctx->pp[0] = (double*)carve(ctx, p.n_pp * 8);
  ctx->pp[1] = (double*)carve(ctx, p.n_pp * 8);
  double* envbase = (double*)carve(ctx, (size_t)(ctx->L + 1) * p.n_env * 8);
  ctx->T1 = (double*)carve(ctx, p.n_part * 8);
  ctx->Lp = (double*)carve(ctx, p.n_part * 8);
  ctx->Rp = (double*)carve(ctx, p.n_part * 8);
  ctx->CE = (double*)carve(ctx, p.n_ce * 8);
  ctx->svd.W = (double*)carve(ctx, p.n_svd * 8);
  ctx->svd.V = (double*)carve(ctx, p.n_svd * 8);
  ctx->svd.sig = (double*)carve(ctx, p.n_svd_cols * 8);
  ctx->svd.perm = (int*)carve(ctx, p.n_svd_cols * 4);
  ctx->svd.counter = (int*)carve(ctx, 32);
  ctx->svd.kept = (int*)carve(ctx, 16);
  ctx->svd.stats = (double*)carve(ctx, 64);
  ctx->svd.max_elems = p.n_svd;
  ctx->svd.max_cols = (int)p.n_svd_cols;
  ctx->usbuf = (double*)carve(ctx, p.n_usbuf * 8);
  for (int i = 0; i < 3; ++i) ctx->ob[i] = (double*)carve(ctx, p.n_obs * 8);
  for (int i = 0; i < 2; ++i) {
    ctx->hf[i] = (double*)carve(ctx, p.n_herm * 8);
    ctx->hr[i] = (double*)carve(ctx, p.n_herm * 8);
  }
  ctx->ht = (double*)carve(ctx, 4 * p.n_herm * 8);
  ctx->scal = (double*)carve(ctx, 64 * 8);
  ok = ok && envbase && ctx->pp[0] && ctx->pp[1] && ctx->T1 && ctx->Lp && ctx->Rp && ctx->CE &&
       ctx->svd.W && ctx->svd.V && ctx->svd.sig && ctx->svd.perm && ctx->svd.counter &&
       ctx->svd.kept && ctx->svd.stats && ctx->usbuf && ctx->ob[0] && ctx->ob[1] && ctx->ob[2] &&
       ctx->hf[0] && ctx->hf[1] && ctx->hr[0] && ctx->hr[1] && ctx->ht &&
       ctx->scal;
  if (ok && p.mixed_bytes) {
    const int P = p.planes, L = ctx->L;
    ctx->m.P = P;
    ctx->m.nprod = P == 3 ? 6 : 3;
    for (int k = 0; k < 4 && ok; ++k) {
      __nv_bfloat16* b = (__nv_bfloat16*)carve(ctx, (size_t)L * P * p.m_site[k] * 2);
      ok = b != nullptr;
      for (int i = 0; ok && i < L; ++i) ctx->m.site[k].push_back(b + (size_t)i * P * p.m_site[k]);
    }
    __nv_bfloat16* eb = (__nv_bfloat16*)carve(ctx, (size_t)(L + 1) * P * p.m_env * 2);
    ok = ok && eb;
    for (int i = 0; ok && i <= L; ++i) ctx->m.env.push_back(eb + (size_t)i * P * p.m_env);
    ctx->m.T1 = (__nv_bfloat16*)carve(ctx, P * p.m_t1 * 2);
    ctx->m.T1R = (__nv_bfloat16*)carve(ctx, P * p.m_t1 * 2);
    {
      const size_t np = cfg->keep_parts ? (size_t)L : 1, one = (size_t)P * p.m_lp;
      ctx->m.Lp = (__nv_bfloat16*)carve(ctx, np * one * 2);
      ctx->m.Rp = (__nv_bfloat16*)carve(ctx, np * one * 2);
      for (int i = 0; i < L && ctx->m.Lp && ctx->m.Rp; ++i) {
        const size_t o = cfg->keep_parts ? (size_t)i * one : 0;
        ctx->m.lpc.push_back(ctx->m.Lp + o);
        ctx->m.rpc.push_back(ctx->m.Rp + o);
      }
    }
    ctx->m.Ct = (__nv_bfloat16*)carve(ctx, P * p.m_ct * 2);
    ctx->m.part = (float*)carve(ctx, p.m_part * 4);
    ctx->m.err = (int*)carve(ctx, 16);
    ctx->m.acc = (double*)carve(ctx, 64);
    {
      const size_t c = p.cap, mm = 4 * c;
      float* f = (float*)carve(ctx, subspace_buffer_floats(p.cap) * 4);
      ok = ok && f;
      if (f) {
        const size_t G = (size_t)subspace_orth_ctas(p.cap);
        ctx->m.sb.Q = f; f += mm * c;
        ctx->m.sb.Y = f; f += mm * c;
        ctx->m.sb.out = f; f += mm * mm;
        ctx->m.sb.orth_part = f; f += G * SUBSPACE_BLOCK_K * 32;
        ctx->m.sb.orth_red = f; f += SUBSPACE_BLOCK_K * 32;
        ctx->m.sb.scal = f; f += 64;
        ctx->m.sb.orth_partd = (double*)f; f += 2 * G * 32 * 32;
        ctx->m.sb.orth_redd = (double*)f; f += 2 * 32 * 32;
        ctx->m.sb.orth_max_ctas = (int)G;
      }
      ctx->m.sb.orth_bar = (unsigned*)carve(ctx, 16);
      ok = ok && ctx->m.sb.orth_bar;
      ctx->m.sb.dscal = (double*)carve(ctx, 16);
      ctx->m.sb.pa = (__nv_bfloat16*)carve(ctx, subspace_plane_elems_a(p.cap) * 2);
      ctx->m.sb.pb = (__nv_bfloat16*)carve(ctx, subspace_plane_elems_b(p.cap) * 2);
      ctx->m.sb.psa = (long long)(subspace_plane_elems_a(p.cap) / 3);
      ctx->m.sb.psb = (long long)(subspace_plane_elems_b(p.cap) / 3);
      ctx->m.sb.err = ctx->m.err;
      ctx->m.sb.ce_ps = (long long)(subspace_plane_elems_a(p.cap) / 3);
      ctx->m.sb.ce_rm = (__nv_bfloat16*)carve(ctx, subspace_plane_elems_a(p.cap) * 2);
      ctx->m.sb.ce_tr = (__nv_bfloat16*)carve(ctx, subspace_plane_elems_a(p.cap) * 2);
      ctx->m.sb.ce_ss = (double*)carve(ctx, 16);
      ctx->m.sb.chol_L = (float*)carve(ctx, SUBSPACE_CHOL_FLOATS * 4);
      ctx->m.sb.chol_d = (float*)carve(ctx, SUBSPACE_BLOCK_K * 4);
      ctx->m.sb.chol_li = (float*)carve(ctx, SUBSPACE_BLOCK_K * 4);
      ctx->m.sb.chol_flag = (int*)carve(ctx, 32);
      ctx->m.sb.orth_block = cfg->orth_block ? cfg->orth_block : SUBSPACE_BLOCK_K;
      // C_E's split-K partials are consumed before the split starts
      ctx->m.sb.part = ctx->m.part;
      ctx->m.sb.seed_base = reinterpret_cast<unsigned long long*>(ctx->m.acc + 4);
      ctx->m.sb.part_floats = p.m_part;
      ok = ok && ctx->m.sb.ce_rm && ctx->m.sb.ce_tr && ctx->m.sb.ce_ss && ctx->m.sb.chol_L &&
           ctx->m.sb.chol_d && ctx->m.sb.chol_li && ctx->m.sb.chol_flag;
      ok = ok && ctx->m.sb.dscal && ctx->m.sb.pa && ctx->m.sb.pb;
    }
    ok = ok && ctx->m.T1 && ctx->m.T1R && ctx->m.Lp && ctx->m.Rp && ctx->m.Ct && ctx->m.part &&
         ctx->m.err && ctx->m.acc;
    ctx->mixed_ready = ok;
  }
  if (!ok) {
    delete ctx;
    return XTRG_ENOMEM;
  }
  ctx->env.resize(ctx->L + 1);
  for (int i = 0; i <= ctx->L; ++i) ctx->env[i] = envbase + (size_t)i * p.n_env;
  if (ctx->mixed_ready) {
    const double acc0[8] = {0.0, 0.0, INFINITY, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (cudaMemsetAsync(ctx->m.sb.chol_flag, 0, 32, ctx->st) != cudaSuccess ||
        cudaMemcpyAsync(ctx->m.acc, acc0, sizeof acc0, cudaMemcpyHostToDevice, ctx->st) !=
            cudaSuccess) {
      delete ctx;
      return XTRG_ECUDA;
    }
  }
  // Hamiltonian and identity sites
  for (int i = 0; i <= ctx->L; ++i) ctx->H.dims[i] = Hm->bond_dims[i];
  for (int i = 0; i < ctx->L; ++i) {
    cudaError_t e = cudaMemcpyAsync(ctx->H.site[i], Hm->W[i], sizeof(double) * site_elems(ctx->H, i),
                                    cudaMemcpyHostToDevice, ctx->st);
    if (e == cudaSuccess) e = dev_identity_site(ctx->I.site[i], ctx->st);
    if (e != cudaSuccess) {
      delete ctx;
      return XTRG_ECUDA;
    }
  }
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess) {
    delete ctx;
    return XTRG_ECUDA;
  }
  *out = ctx;
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_init(xtrg_ctx* ctx) {
  if (!ctx) return XTRG_EINVAL;
  const int L = ctx->L;
  ctx->use_mixed = false;  // the series initialisation always runs in FP64
  // Y = I
  for (int i = 0; i <= L; ++i) ctx->Y.dims[i] = 1;
  for (int i = 0; i < L; ++i) CK(dev_identity_site(ctx->Y.site[i], ctx->st));
  for (int k = ctx->cfg.order; k >= 1; --k) {
    bool fat_fits = true;
    for (int i = 0; i <= L; ++i) fat_fits = fat_fits && ctx->Y.dims[i] <= ctx->plan.cap_fat;
    if (fat_fits) {
      // guess: the exact product H^T Y with fused bonds
      for (int i = 0; i <= L; ++i) ctx->fat.dims[i] = ctx->H.dims[i] * ctx->Y.dims[i];
      for (int i = 0; i < L; ++i)
        CK(mpo_exact_product(ctx->H.site[i], ctx->H.dims[i], ctx->H.dims[i + 1], ctx->Y.site[i],
                             ctx->Y.dims[i], ctx->Y.dims[i + 1], ctx->fat.site[i], ctx->st));
      TRY(canonicalize(ctx, ctx->fat.dims, ctx->fat.site, ctx->C));
    } else {
      // the fused bonds would exceed the guess capacity (long-range H such as
      // a 2D snake, with Y near D*): the sweeps start from Y, right-canonical
      TRY(canonicalize(ctx, ctx->Y.dims, ctx->Y.site, ctx->C));
    }
    TRY(compress(ctx, ctx->H, ctx->Y, ctx->C, ctx->cfg.dstar, ctx->cfg.init_sweeps));
    // Y <- I + (-tau0/k) * (H Y)
    const double alpha = -ctx->cfg.tau0 / k;
    std::vector<int> nd(L + 1, 1);
    for (int i = 1; i < L; ++i) nd[i] = ctx->C.dims[i] + 1;
    for (int i = 0; i < L; ++i)
      CK(mpo_direct_sum_site(ctx->C.site[i], ctx->C.dims[i], ctx->C.dims[i + 1], alpha,
                             ctx->I.site[i], 1, 1, i, L, ctx->Y.site[i], ctx->st));
    ctx->Y.dims = nd;
  }
  TRY(canonicalize(ctx, ctx->Y.dims, ctx->Y.site, ctx->C));
  double lns = 0.0;
  TRY(normalize(ctx, ctx->C, &lns));
  std::swap(ctx->rho, ctx->C);
  ctx->lnc = lns;
  ctx->beta = ctx->cfg.tau0;
  ctx->nd = 0;
  ctx->have_rho = true;
  ctx->rho_canonical = true;
  ctx->last_trunc = 0.0;
  return XTRG_OK;
}

namespace {

// Device work of a tensor-core doubling from a right-canonical rho: the guess
// C = rho, rho's operand planes, the sweeps, the normalisation of C.  No
// host read, so it can be captured as one CUDA graph.
xtrg_status mixed_doubling_body(xtrg_ctx* ctx) {
  ctx->C.dims = ctx->rho.dims;
  for (int i = 0; i < ctx->L; ++i)
    CK(cudaMemcpyAsync(ctx->C.site[i], ctx->rho.site[i], sizeof(double) * site_elems(ctx->rho, i),
                       cudaMemcpyDeviceToDevice, ctx->st));
  TRY(mixed_prepare(ctx));
  TRY(compress_mixed(ctx, ctx->C, ctx->cfg.dstar, ctx->cfg.sweeps));
  return normalize_device(ctx, ctx->C);
}

bool graphs_disabled_by_env() {
  static const bool v = []() {
    const char* e = getenv("XTRG_NO_GRAPHS");
    return e && e[0] == '1';
  }();
  return v;
}

// Capture mixed_doubling_body on the context's capture stream.  On any
// failure the capture is abandoned, graphs stay off for this context and the
// caller runs the body directly.
bool capture_doubling(xtrg_ctx* ctx, xtrg_ctx::DoublingGraph* g) {
  if (!ctx->cap_st && cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->cap_st = nullptr;
    return false;
  }
  cudaStream_t user = ctx->st;
  const long long u0 = ctx->updates;
  const unsigned long long l0 = t_xtrg_launches, c0 = t_orth_cluster_calls;
  const double fc0 = ctx->flops_contr, fs0 = ctx->flops_split;
  if (cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ctx->st = ctx->cap_st;
  const xtrg_status body = mixed_doubling_body(ctx);
  ctx->st = user;
  g->out_dims = ctx->C.dims;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(ctx->cap_st, &graph);
  bool ok = body == XTRG_OK && ec == cudaSuccess && graph;
  if (ok && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) ok = false;
  if (graph) cudaGraphDestroy(graph);
  // the host counters advanced while capturing; replays advance them again
  g->d_updates = ctx->updates - u0;
  g->d_launches = t_xtrg_launches - l0;
  g->d_cluster = t_orth_cluster_calls - c0;
  g->d_flops_contr = ctx->flops_contr - fc0;
  g->d_flops_split = ctx->flops_split - fs0;
  ctx->updates = u0;
  ctx->flops_contr = fc0;
  ctx->flops_split = fs0;
  if (!ok) {
    cudaGetLastError();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  return ok;
}

}  // namespace

extern "C" xtrg_status xtrg_double(xtrg_ctx* ctx) {
  if (!ctx) return XTRG_EINVAL;
  if (!ctx->have_rho) return fail(ctx, XTRG_EINVAL, "xtrg_double before xtrg_init");
  ctx->use_mixed = mixed_for_beta(ctx, ctx->beta);
  if (ctx->use_mixed && ctx->rho_canonical) {
    // tensor-core doubling.  Once the bonds are saturated (rho's bonds as at
    // the previous tensor-core doubling, so every launch has the same shape
    // as then), the device work is captured as a CUDA graph per buffer
    // parity and replayed; the host reads the product's results once.
    xtrg_ctx::DoublingGraph* hit = nullptr;
    const bool graphable = !ctx->graphs_off && !ctx->profiling && !debug_on() &&
                           !graphs_disabled_by_env();
    if (graphable) {
      for (auto& g : ctx->graphs)
        if (g.rho0 == ctx->rho.site[0] && g.dims == ctx->rho.dims) hit = &g;
      if (!hit && ctx->rho.dims == ctx->prev_mixed_dims) {
        xtrg_ctx::DoublingGraph g;
        g.rho0 = ctx->rho.site[0];
        g.dims = ctx->rho.dims;
        if (capture_doubling(ctx, &g)) {
          // a stale graph of this parity (other bonds) is replaced
          for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
            if (it->rho0 == g.rho0) {
              cudaGraphExecDestroy(it->exec);
              it = ctx->graphs.erase(it);
            } else {
              ++it;
            }
          }
          ctx->graphs.push_back(g);
          hit = &ctx->graphs.back();
          ctx->graph_captures++;
        } else {
          ctx->graphs_off = true;
        }
      }
    }
    ctx->prev_mixed_dims = ctx->rho.dims;
    if (hit) {
      CK(cudaGraphLaunch(hit->exec, ctx->st));
      ctx->C.dims = hit->out_dims;
      ctx->updates += hit->d_updates;
      ctx->flops_contr += hit->d_flops_contr;
      ctx->flops_split += hit->d_flops_split;
      __atomic_add_fetch(&g_xtrg_launches, hit->d_launches, __ATOMIC_RELAXED);
      __atomic_add_fetch(&g_orth_cluster_calls, hit->d_cluster, __ATOMIC_RELAXED);
      ctx->graph_replays++;
    } else {
      TRY(mixed_doubling_body(ctx));
    }
    TRY(finish_mixed(ctx));
    TRY(resolve_events(ctx));
  } else {
    if (ctx->rho_canonical) {
      // rho from init/double is already right-canonical: right-canonicalising
      // it again changes only the gauge, so the guess is a plain copy
      ctx->C.dims = ctx->rho.dims;
      for (int i = 0; i < ctx->L; ++i)
        CK(cudaMemcpyAsync(ctx->C.site[i], ctx->rho.site[i],
                           sizeof(double) * site_elems(ctx->rho, i), cudaMemcpyDeviceToDevice,
                           ctx->st));
    } else {
      TRY(canonicalize(ctx, ctx->rho.dims, ctx->rho.site, ctx->C));
    }
    if (ctx->use_mixed) {
      TRY(mixed_prepare(ctx));
      TRY(compress_mixed(ctx, ctx->C, ctx->cfg.dstar, ctx->cfg.sweeps));
      TRY(finish_mixed(ctx));
      TRY(resolve_events(ctx));
    } else {
      TRY(compress(ctx, ctx->rho, ctx->rho, ctx->C, ctx->cfg.dstar, ctx->cfg.sweeps));
    }
    TRY(normalize_device(ctx, ctx->C));
  }
  double lns = 0.0;
  TRY(normalize_finish(ctx, &lns));
  std::swap(ctx->rho, ctx->C);
  ctx->lnc = 2.0 * ctx->lnc + lns;
  ctx->beta *= 2.0;
  ctx->nd++;
  ctx->rho_canonical = true;
  return XTRG_OK;
}

// Pointwise-Taylor SETTN step (Sec. II C, Eq. Tay, Fig. SETTNAlg(b)):
// rho(beta + dtau) = sum_{k=0}^{order} (-dtau)^k/k! H^k rho(beta).  Terms
// H^k rho by compressed products H (H^{k-1} rho) (App. D.1; guess: the
// previous term), their sum by the variational MPO sum (App. D.2; guess:
// rho), all in FP64.  The caller's buffer holds the terms k >= 1 and every
// term's overlap environments.
namespace {
size_t settn_sizes(const xtrg_ctx* ctx, int order, size_t* term_slot, size_t* env_slot) {
  const size_t cap = ctx->cap;
  *term_slot = cap * 4 * cap;
  *env_slot = cap * cap;
  return (size_t)order * up((size_t)ctx->L * *term_slot * 8) +
         (size_t)(order + 1) * up((size_t)(ctx->L + 1) * *env_slot * 8);
}
}  // namespace

extern "C" size_t xtrg_settn_workspace_bytes(const xtrg_ctx* ctx, int order) {
  if (!ctx || order < 1 || order > 64) return 0;
  size_t ts, es;
  return settn_sizes(ctx, order, &ts, &es);
}

extern "C" xtrg_status xtrg_settn_step(xtrg_ctx* ctx, double dtau, int order, void* dev_buf,
                                       size_t bytes) {
  if (!ctx) return XTRG_EINVAL;
  if (!ctx->have_rho) return fail(ctx, XTRG_EINVAL, "xtrg_settn_step before xtrg_init");
  if (!(dtau > 0.0) || order < 1 || order > 64)
    return fail(ctx, XTRG_EINVAL, "settn step needs dtau > 0 and 1 <= order <= 64");
  if (!dev_buf || ((uintptr_t)dev_buf % ALIGN) != 0)
    return fail(ctx, XTRG_EINVAL, "settn buffer must be device memory, 256-byte aligned");
  size_t ts = 0, es = 0;
  const size_t need = settn_sizes(ctx, order, &ts, &es);
  if (bytes < need) return fail(ctx, XTRG_ENOMEM, "settn buffer below %zu bytes", need);
  const int L = ctx->L;
  ctx->use_mixed = false;
  char* b = (char*)dev_buf;
  std::vector<DevMpo> T(order);
  for (int k = 0; k < order; ++k) {
    T[k].slot = ts;
    T[k].dims.assign(L + 1, 1);
    T[k].site.resize(L);
    for (int i = 0; i < L; ++i) T[k].site[i] = (double*)b + (size_t)i * ts;
    b += up((size_t)L * ts * 8);
  }
  // terms H^k rho, k = 1..order
  const DevMpo* prev = &ctx->rho;
  for (int k = 0; k < order; ++k) {
    TRY(canonicalize(ctx, prev->dims, prev->site, ctx->C));
    TRY(compress(ctx, ctx->H, *prev, ctx->C, ctx->cfg.dstar, ctx->cfg.sweeps));
    T[k].dims = ctx->C.dims;
    for (int i = 0; i < L; ++i)
      CK(cudaMemcpyAsync(T[k].site[i], ctx->C.site[i], sizeof(double) * site_elems(ctx->C, i),
                         cudaMemcpyDeviceToDevice, ctx->st));
    prev = &T[k];
  }
  std::vector<SumTerm> terms(order + 1);
  double w = 1.0;
  for (int k = 0; k <= order; ++k) {
    if (k > 0) w *= -dtau / k;
    terms[k].T = k == 0 ? &ctx->rho : &T[k - 1];
    terms[k].w = w;
    terms[k].env = (double*)b;
    b += up((size_t)(L + 1) * es * 8);
  }
  // guess: rho itself, right-canonical
  if (ctx->rho_canonical) {
    ctx->C.dims = ctx->rho.dims;
    for (int i = 0; i < L; ++i)
      CK(cudaMemcpyAsync(ctx->C.site[i], ctx->rho.site[i], sizeof(double) * site_elems(ctx->rho, i),
                         cudaMemcpyDeviceToDevice, ctx->st));
  } else {
    TRY(canonicalize(ctx, ctx->rho.dims, ctx->rho.site, ctx->C));
  }
  TRY(compress_sum(ctx, terms, ctx->C, ctx->cfg.dstar, ctx->cfg.sweeps, es));
  double lns = 0.0;
  TRY(normalize(ctx, ctx->C, &lns));
  std::swap(ctx->rho, ctx->C);
  ctx->lnc += lns;
  ctx->beta += dtau;
  ctx->rho_canonical = true;
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_trace(xtrg_ctx* ctx, double* lnZ) {
  if (!ctx || !lnZ) return XTRG_EINVAL;
  if (!ctx->have_rho) return fail(ctx, XTRG_EINVAL, "no state");
  double t[3];
  TRY(traces(ctx, false, t));
  if (!(t[0] > 0.0) || !std::isfinite(t[0]))
    return fail(ctx, XTRG_ENUMERIC, "Tr rho = %g is not positive", t[0]);
  *lnZ = ctx->lnc + std::log(t[0]);
  return XTRG_OK;
}

// <O> = Tr(O rho) / Tr rho for an operator MPO O with bonds <= D* + 1 (e.g.
// the powers of S^z_tot of the Binder ratio, Sec. IV D, Eq. Binder): O is
// copied into the Y slots, and E'[h'][r'] = sum O[h][s][t][h'] E[h][r]
// rho[r][t][s][r'] is carried left to right (FP64).
extern "C" xtrg_status xtrg_expectation(xtrg_ctx* ctx, const xtrg_mpo* O, double* value) {
  if (!ctx || !value) return XTRG_EINVAL;
  if (!ctx->have_rho) return fail(ctx, XTRG_EINVAL, "no state");
  if (check_mpo(O, ctx->cap) != XTRG_OK || O->L != ctx->L)
    return fail(ctx, XTRG_EINVAL, "operator MPO has the wrong length or a bond above %d", ctx->cap);
  const int L = ctx->L;
  DevMpo& Op = ctx->Y;
  for (int i = 0; i <= L; ++i) Op.dims[i] = O->bond_dims[i];
  for (int i = 0; i < L; ++i)
    CK(cudaMemcpyAsync(Op.site[i], O->W[i], sizeof(double) * site_elems(Op, i),
                       cudaMemcpyHostToDevice, ctx->st));
  double t[3];
  TRY(traces(ctx, false, t));   // Tr rho (synchronises, so O's host arrays are free)
  const DevMpo& R = ctx->rho;
  double* E[2] = {ctx->hf[0], ctx->hf[1]};
  double* T = ctx->ht;
  CK(dev_fill(E[0], 1.0, 1, ctx->st));
  for (int i = 0; i < L; ++i) {
    const int l = R.dims[i], r = R.dims[i + 1], hl = Op.dims[i], hr = Op.dims[i + 1];
    TRY(gemm64(ctx, mk(hl, 4 * r, l, 1, E[i & 1], idx_plain(l), idx_plain(1), 0, R.site[i],
                       idx_plain(4 * r), idx_plain(1), 0, T, idx_plain(4 * r), idx_plain(1), 0)));
    TRY(gemm64(ctx, mk(hr, r, 4 * hl, 1, Op.site[i], idx_plain(1), idx_plain(hr), 0, T,
                       idx_split3(2, 2, 4LL * r, r, 2LL * r), idx_plain(1), 0, E[(i + 1) & 1],
                       idx_plain(r), idx_plain(1), 0)));
  }
  double tr_o = 0.0;
  CK(cudaMemcpyAsync(&tr_o, E[L & 1], sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (!(t[0] > 0.0) || !std::isfinite(tr_o))
    return fail(ctx, XTRG_ENUMERIC, "Tr rho = %g, Tr(O rho) = %g", t[0], tr_o);
  *value = tr_o / t[0];
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_observables(xtrg_ctx* ctx, xtrg_obs* o) {
  if (!ctx || !o) return XTRG_EINVAL;
  if (!ctx->have_rho) return fail(ctx, XTRG_EINVAL, "no state");
  double t[3];
  TRY(traces(ctx, true, t));
  if (!(t[0] > 0.0) || !std::isfinite(t[0]) || !std::isfinite(t[1]) || !std::isfinite(t[2]))
    return fail(ctx, XTRG_ENUMERIC, "traces not finite/positive: %g %g %g", t[0], t[1], t[2]);
  const double N = ctx->L, b = ctx->beta;
  const double e1 = t[1] / t[0], e2 = t[2] / t[0];
  memset(o, 0, sizeof *o);
  o->beta = b;
  o->lnZ = ctx->lnc + std::log(t[0]);
  o->f = -o->lnZ / (N * b);
  o->u = e1 / N;
  o->c = b * b * (e2 - e1 * e1) / N;
  // the stored rho is normalised, ||rho||_F = 1, so Z(2 beta) = e^{2 ln c}
  o->lnZ2 = 2.0 * ctx->lnc;
  o->trunc_err = ctx->last_trunc;
  o->herm_defect = NAN;
  if (ctx->herm_check) {
    double fro = 0.0, trr = 0.0;
    TRY(herm_transfers(ctx, &fro, &trr));
    if (!(fro > 0.0) || !std::isfinite(fro) || !std::isfinite(trr))
      return fail(ctx, XTRG_ENUMERIC, "||rho||_F^2 = %g, Tr(rho rho) = %g", fro, trr);
    o->herm_defect = std::sqrt(std::fmax(0.0, 2.0 - 2.0 * trr / fro));
  }
  int mx = 1;
  for (int d : ctx->rho.dims) mx = d > mx ? d : mx;
  o->max_bond = mx;
  o->n_doublings = ctx->nd;
  return XTRG_OK;
}

// MPO entanglement per bond (Sec. IV A, Eq. purif): rho read as a state of
// the doubled local space; its Schmidt values s at each bond give
// p = s^2 / sum s^2 and S_E = -sum p ln p.  A copy of rho brought to
// right-canonical form in FP64 (into C, the scratch MPO of the products) is
// swept left to right: the
// centre site (l s t) x r is split by the FP64 Jacobi SVD, U stays, Lambda V^T
// moves into the next site, and the singular values of each split are the
// Schmidt values of that bond.  Nothing is truncated.
extern "C" xtrg_status xtrg_entanglement(xtrg_ctx* ctx, double* S, int n) {
  if (!ctx || !S) return XTRG_EINVAL;
  if (!ctx->have_rho) return fail(ctx, XTRG_EINVAL, "no state");
  const int L = ctx->L;
  if (n < L - 1) return fail(ctx, XTRG_EINVAL, "S holds %d entries, %d bonds", n, L - 1);
  DevMpo& C = ctx->C;
  // always an FP64 right-canonical form: a state from the tensor-core path is
  // right-orthonormal only to FP32 level, which would bias the Schmidt values
  TRY(canonicalize(ctx, ctx->rho.dims, ctx->rho.site, C));
  std::vector<double> sig;
  for (int i = 0; i + 1 < L; ++i) {
    const int l = C.dims[i], r = C.dims[i + 1], r2 = C.dims[i + 2];
    SvdResult res;
    // keep every nonzero singular value (rel_tol 0): the next site absorbs Lambda V^T
    bool conv = true;
    cudaError_t e = svd_split_f64(C.site[i], 4 * l, r, r, 0.0, SPLIT_RIGHT, ctx->pp[0], ctx->usbuf,
                                  ctx->svd, ctx->st, &res, &conv);
    if (e == cudaErrorLaunchTimeout)
      return fail(ctx, XTRG_ETIMEOUT, "entanglement split: a bounded device barrier expired");
    if (e != cudaSuccess) return fail(ctx, XTRG_ECUDA, "entanglement split: %s", cudaGetErrorString(e));
    if (!conv) return fail(ctx, XTRG_ENUMERIC, "Jacobi SVD at bond %d did not converge", i + 1);
    const int ncols = (4 * l < r) ? 4 * l : r;
    sig.resize(ncols);
    CK(cudaMemcpyAsync(sig.data(), ctx->svd.sig, sizeof(double) * ncols, cudaMemcpyDeviceToHost,
                       ctx->st));
    // site i+1 <- (Lambda V^T) (k x r) times site i+1 (r x 4 r2)
    const int k = res.k;
    TRY(gemm64(ctx, mk(k, 4 * r2, r, 1, ctx->usbuf, idx_plain(r), idx_plain(1), 0, C.site[i + 1],
                       idx_plain(4 * r2), idx_plain(1), 0, ctx->pp[1], idx_plain(4 * r2),
                       idx_plain(1), 0)));
    CK(cudaMemcpyAsync(C.site[i + 1], ctx->pp[1], sizeof(double) * (size_t)k * 4 * r2,
                       cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    C.dims[i + 1] = k;
    double tot = 0.0;
    for (double x : sig) tot += x * x;
    double ent = 0.0;
    if (tot > 0.0)
      for (double x : sig) {
        const double p = x * x / tot;
        if (p > 0.0) ent -= p * std::log(p);
      }
    S[i] = ent;
  }
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_get_state(xtrg_ctx* ctx, int* bond_dims, double* const* W, double* lnc,
                                      double* beta) {
  if (!ctx || !bond_dims) return XTRG_EINVAL;
  if (!ctx->have_rho) return fail(ctx, XTRG_EINVAL, "no state");
  for (int i = 0; i <= ctx->L; ++i) bond_dims[i] = ctx->rho.dims[i];
  if (lnc) *lnc = ctx->lnc;
  if (beta) *beta = ctx->beta;
  if (W) {
    for (int i = 0; i < ctx->L; ++i) {
      if (!W[i]) return fail(ctx, XTRG_EINVAL, "W[%d] is NULL", i);
      CK(cudaMemcpyAsync(W[i], ctx->rho.site[i], sizeof(double) * site_elems(ctx->rho, i),
                         cudaMemcpyDeviceToHost, ctx->st));
    }
    CK(cudaStreamSynchronize(ctx->st));
  }
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_set_state(xtrg_ctx* ctx, const xtrg_mpo* r, double lnc, double beta,
                                      int right_canonical) {
  if (!ctx) return XTRG_EINVAL;
  if (check_mpo(r, ctx->cap) != XTRG_OK || r->L != ctx->L)
    return fail(ctx, XTRG_EINVAL, "state MPO has the wrong length or a bond above %d", ctx->cap);
  if (!(beta > 0.0) || !std::isfinite(lnc)) return fail(ctx, XTRG_EINVAL, "bad beta or lnc");
  for (int i = 0; i <= ctx->L; ++i) ctx->rho.dims[i] = r->bond_dims[i];
  for (int i = 0; i < ctx->L; ++i)
    CK(cudaMemcpyAsync(ctx->rho.site[i], r->W[i], sizeof(double) * site_elems(ctx->rho, i),
                       cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->lnc = lnc;
  ctx->beta = beta;
  ctx->have_rho = true;
  ctx->rho_canonical = right_canonical != 0;
  return XTRG_OK;
}

// ------------------------------------------------------------ checkpoints
// Device checkpoint layout: a 4 KiB header (magic, L, bond dims, ln c, beta,
// doublings, canonical flag) followed by the sites packed back to back.
namespace {
constexpr long long CKPT_MAGIC = 0x58545247434b5054LL;   // "XTRGCKPT"
constexpr size_t CKPT_HEADER = 4096;
struct CkptHeader {
  long long magic;
  int L, nd, canonical, pad;
  double lnc, beta;
  int dims[(CKPT_HEADER - 40) / sizeof(int)];
};
static_assert(sizeof(CkptHeader) <= CKPT_HEADER, "checkpoint header");
}  // namespace

extern "C" size_t xtrg_checkpoint_bytes(const xtrg_ctx* ctx) {
  if (!ctx || ctx->L + 1 > (int)((CKPT_HEADER - 40) / sizeof(int))) return 0;
  return CKPT_HEADER + up((size_t)ctx->L * ctx->cap * 4 * ctx->cap * 8);
}

extern "C" xtrg_status xtrg_checkpoint_save(xtrg_ctx* ctx, void* dev_buf, size_t bytes) {
  if (!ctx || !dev_buf || ((uintptr_t)dev_buf % ALIGN) != 0) return XTRG_EINVAL;
  if (!ctx->have_rho) return fail(ctx, XTRG_EINVAL, "no state to checkpoint");
  const size_t need = xtrg_checkpoint_bytes(ctx);
  if (need == 0 || bytes < need) return fail(ctx, XTRG_ENOMEM, "checkpoint buffer below %zu bytes", need);
  CkptHeader h;
  memset(&h, 0, sizeof h);
  h.magic = CKPT_MAGIC;
  h.L = ctx->L;
  h.nd = ctx->nd;
  h.canonical = ctx->rho_canonical ? 1 : 0;
  h.lnc = ctx->lnc;
  h.beta = ctx->beta;
  for (int i = 0; i <= ctx->L; ++i) h.dims[i] = ctx->rho.dims[i];
  char* d = (char*)dev_buf;
  CK(cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyHostToDevice, ctx->st));
  size_t off = CKPT_HEADER;
  for (int i = 0; i < ctx->L; ++i) {
    const size_t b = sizeof(double) * site_elems(ctx->rho, i);
    CK(cudaMemcpyAsync(d + off, ctx->rho.site[i], b, cudaMemcpyDeviceToDevice, ctx->st));
    off += b;
  }
  // the header is copied from this stack frame: finish before returning
  CK(cudaStreamSynchronize(ctx->st));
  return XTRG_OK;
}

namespace {
// Reads a device checkpoint into dst (bond dims, sites) and returns its
// header values; the sites must fit this context's capacity.
xtrg_status load_checkpoint(xtrg_ctx* ctx, const void* dev_buf, size_t bytes, DevMpo& dst,
                            CkptHeader* hout) {
  if (!dev_buf || ((uintptr_t)dev_buf % ALIGN) != 0) return XTRG_EINVAL;
  if (bytes < CKPT_HEADER) return fail(ctx, XTRG_EINVAL, "checkpoint buffer too small");
  CkptHeader h;
  const char* d = (const char*)dev_buf;
  CK(cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (h.magic != CKPT_MAGIC || h.L != ctx->L)
    return fail(ctx, XTRG_EINVAL, "not a checkpoint of a %d-site context", ctx->L);
  if (h.dims[0] != 1 || h.dims[h.L] != 1)
    return fail(ctx, XTRG_EINVAL, "checkpoint has bad boundary bonds");
  size_t need = CKPT_HEADER;
  for (int i = 0; i < h.L; ++i) {
    if (h.dims[i + 1] < 1 || h.dims[i + 1] > ctx->cap)
      return fail(ctx, XTRG_EINVAL, "checkpoint bond %d = %d exceeds capacity %d", i + 1,
                  h.dims[i + 1], ctx->cap);
    need += sizeof(double) * (size_t)h.dims[i] * 4 * h.dims[i + 1];
  }
  if (bytes < need) return fail(ctx, XTRG_EINVAL, "checkpoint buffer shorter than its sites");
  for (int i = 0; i <= ctx->L; ++i) dst.dims[i] = h.dims[i];
  size_t off = CKPT_HEADER;
  for (int i = 0; i < ctx->L; ++i) {
    const size_t b = sizeof(double) * site_elems(dst, i);
    CK(cudaMemcpyAsync(dst.site[i], d + off, b, cudaMemcpyDeviceToDevice, ctx->st));
    off += b;
  }
  *hout = h;
  return XTRG_OK;
}
}  // namespace

extern "C" xtrg_status xtrg_checkpoint_load(xtrg_ctx* ctx, const void* dev_buf, size_t bytes) {
  if (!ctx || !dev_buf || ((uintptr_t)dev_buf % ALIGN) != 0) return XTRG_EINVAL;
  CkptHeader h;
  TRY(load_checkpoint(ctx, dev_buf, bytes, ctx->rho, &h));
  ctx->lnc = h.lnc;
  ctx->beta = h.beta;
  ctx->nd = h.nd;
  ctx->have_rho = true;
  ctx->rho_canonical = h.canonical != 0;
  return XTRG_OK;
}

// rho_{n,n'} = rho_a rho_b (Sec. II B, after Eq. zshift): intermediate
// inverse temperatures beta_a + beta_b from two saved states, the product
// compressed variationally in FP64 (App. D.1; guess: rho_a).
extern "C" xtrg_status xtrg_cross_product(xtrg_ctx* ctx, const void* ckpt_a, size_t bytes_a,
                                          const void* ckpt_b, size_t bytes_b) {
  if (!ctx || !ckpt_a || !ckpt_b) return XTRG_EINVAL;
  CkptHeader ha, hb;
  TRY(load_checkpoint(ctx, ckpt_a, bytes_a, ctx->rho, &ha));
  ctx->have_rho = false;   // rho now holds factor a only
  TRY(load_checkpoint(ctx, ckpt_b, bytes_b, ctx->Y, &hb));
  ctx->use_mixed = false;
  TRY(canonicalize(ctx, ctx->rho.dims, ctx->rho.site, ctx->C));
  TRY(compress(ctx, ctx->rho, ctx->Y, ctx->C, ctx->cfg.dstar, ctx->cfg.sweeps));
  double lns = 0.0;
  TRY(normalize(ctx, ctx->C, &lns));
  std::swap(ctx->rho, ctx->C);
  ctx->lnc = ha.lnc + hb.lnc + lns;
  ctx->beta = ha.beta + hb.beta;
  ctx->have_rho = true;
  ctx->rho_canonical = true;
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_get_stats(const xtrg_ctx* ctx, xtrg_stats* o) {
  if (!ctx || !o) return XTRG_EINVAL;
  o->contraction_flops = ctx->flops_contr;
  o->split_flops = ctx->flops_split;
  o->tc_flops = ctx->tc_flops;
  o->tc_ms = ctx->tc_ms;
  o->two_site_updates = ctx->updates;
  o->tc_launches = ctx->tc_launches;
  o->kernel_launches = (long long)__atomic_load_n(&g_xtrg_launches, __ATOMIC_RELAXED);
  o->exact_split_fallbacks = ctx->fallbacks;
  o->split_ms = ctx->split_ms;
  o->orth_cluster_calls = (long long)__atomic_load_n(&g_orth_cluster_calls, __ATOMIC_RELAXED);
  o->orth_fallbacks = 0;
  o->orth_full_second_pass = 0;
  o->graph_captures = ctx->graph_captures;
  o->graph_replays = ctx->graph_replays;
  {
    std::lock_guard<std::mutex> lock(g_split_mu);
    o->split_shapes_tuned = (long long)g_split_tuned.size();
  }
  o->orth_deflated_columns = 0;
  if (ctx->mixed_ready && ctx->m.sb.chol_flag) {
    int h[5] = {0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(h, ctx->m.sb.chol_flag, sizeof h, cudaMemcpyDeviceToHost, ctx->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess)
      return XTRG_ECUDA;
    o->orth_fallbacks = h[1];
    o->orth_full_second_pass = h[3];
    o->orth_deflated_columns = h[4];
  }
  o->fp64_update_ms = ctx->tag_ms[TAG_UPDATE64];
  o->fp64_updates_timed = ctx->tag_n[TAG_UPDATE64];
  o->fp64_env_pass_ms = ctx->tag_ms[TAG_ENVPASS64];
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_set_profiling(xtrg_ctx* ctx, int on) {
  if (!ctx) return XTRG_EINVAL;
  ctx->profiling = on != 0;
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_set_herm_check(xtrg_ctx* ctx, int on) {
  if (!ctx) return XTRG_EINVAL;
  ctx->herm_check = on != 0;
  return XTRG_OK;
}

extern "C" xtrg_status xtrg_set_graphs(xtrg_ctx* ctx, int on) {
  if (!ctx) return XTRG_EINVAL;
  ctx->graphs_off = on == 0;
  if (!on) {
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
  }
  return XTRG_OK;
}

// Layout of the scratch of one FP64 tensor-core GEMM call (shared by the
// workspace and the static-scratch entry points): A planes, B planes, split-K
// partials, error flag.
TcGemmScratch tc_gemm_scratch(int M, int N, int K, int batch, int planes, int splitk, bool b_kn) {
  TcGemmScratch w;
  const size_t ld = (size_t)tc_ld(K);
  w.a = up((size_t)planes * batch * M * ld * 2);
  w.b = b_kn ? up((size_t)planes * batch * K * tc_ld(N) * 2)
             : up((size_t)planes * batch * N * ld * 2);
  w.part = up((size_t)splitk * batch * M * N * 4);
  w.total = w.a + w.b + w.part + ALIGN;
  return w;
}

xtrg_status tc_gemm_check_args(const double* A, const double* B, double* C, int M, int N, int K,
                               int batch, int planes, int nprod, int splitk) {
  if (!A || !B || !C) return XTRG_EINVAL;
  if (M < 1 || N < 1 || K < 1 || batch < 1 || planes < 2 || planes > 3 || splitk < 1)
    return XTRG_EINVAL;
  if (!(nprod == 1 || nprod == 3 || (nprod == 6 && planes == 3))) return XTRG_EINVAL;
  return XTRG_OK;
}

xtrg_status tc_gemm_run(const double* A, const double* B, double* C, int M, int N, int K, int batch,
                        int planes, int nprod, int splitk, char* base, cudaStream_t st, bool b_kn) {
  const TcGemmScratch w = tc_gemm_scratch(M, N, K, batch, planes, splitk, b_kn);
  __nv_bfloat16* pa = (__nv_bfloat16*)base;
  __nv_bfloat16* pb = (__nv_bfloat16*)(base + w.a);
  float* part = (float*)(base + w.a + w.b);
  int* err = (int*)(base + w.a + w.b + w.part);
  const long long ld = tc_ld(K);
  const long long ldn = tc_ld(N);
  const long long psA = (long long)batch * M * ld;
  const long long psB = b_kn ? (long long)batch * K * ldn : (long long)batch * N * ld;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return XTRG_ECUDA;
  if (to_planes(A, idx_plain(K), idx_plain(1), (long long)M * K, M, K, batch, pa, ld,
                (long long)M * ld, planes, psA, st) != cudaSuccess)
    return XTRG_ECUDA;
  // B^T rows (K-major), or B's own K x N rows (MN-major operand)
  const cudaError_t eb =
      b_kn ? to_planes(B, idx_plain(N), idx_plain(1), (long long)K * N, K, N, batch, pb, ldn,
                       (long long)K * ldn, planes, psB, st)
           : to_planes(B, idx_plain(K), idx_plain(1), (long long)N * K, N, K, batch, pb, ld,
                       (long long)N * ld, planes, psB, st);
  if (eb != cudaSuccess) return XTRG_ECUDA;
  TcOperand oa{pa, planes, M, K, ld, (long long)M * ld, psA, batch};
  TcOperand ob{pb, planes, N, K, ld, (long long)N * ld, psB, batch};
  if (b_kn) ob = TcOperand{pb, planes, N, K, ldn, (long long)K * ldn, psB, batch, 1};
  TcOutput out;
  memset(&out, 0, sizeof out);
  out.mode = TC_OUT_PARTIAL;
  out.f32 = part;
  out.alpha = 1.0;
  if (tc_gemm(oa, ob, M, N, K, batch, nprod, splitk, out, err, st) != cudaSuccess)
    return XTRG_ECUDA;
  if (reduce_partials(part, splitk, (long long)batch * M * N, C, st) != cudaSuccess)
    return XTRG_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return XTRG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return XTRG_ECUDA;
  return h ? XTRG_ETIMEOUT : XTRG_OK;
}

extern "C" size_t xtrg_tc_gemm_workspace_bytes(int M, int N, int K, int batch, int planes,
                                               int splitk) {
  if (M < 1 || N < 1 || K < 1 || batch < 1 || planes < 1 || planes > 3 || splitk < 1) return 0;
  return tc_gemm_scratch(M, N, K, batch, planes, splitk).total;
}

extern "C" size_t xtrg_tc_gemm_nn_workspace_bytes(int M, int N, int K, int batch, int planes,
                                                  int splitk) {
  if (M < 1 || N < 1 || K < 1 || batch < 1 || planes < 1 || planes > 3 || splitk < 1) return 0;
  return tc_gemm_scratch(M, N, K, batch, planes, splitk, true).total;
}

extern "C" xtrg_status xtrg_tc_gemm_nn(const double* A, const double* B, double* C, int M, int N,
                                       int K, int batch, int planes, int nprod, int splitk,
                                       void* workspace, size_t bytes, void* stream) {
  TRY(tc_gemm_check_args(A, B, C, M, N, K, batch, planes, nprod, splitk));
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0) return XTRG_EINVAL;
  if (bytes < tc_gemm_scratch(M, N, K, batch, planes, splitk, true).total) return XTRG_ENOMEM;
  return tc_gemm_run(A, B, C, M, N, K, batch, planes, nprod, splitk, (char*)workspace,
                     (cudaStream_t)stream, true);
}

extern "C" xtrg_status xtrg_tc_gemm(const double* A, const double* B, double* C, int M, int N,
                                    int K, int batch, int planes, int nprod, int splitk,
                                    void* workspace, size_t bytes, void* stream) {
  TRY(tc_gemm_check_args(A, B, C, M, N, K, batch, planes, nprod, splitk));
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0) return XTRG_EINVAL;
  if (bytes < tc_gemm_scratch(M, N, K, batch, planes, splitk).total) return XTRG_ENOMEM;
  return tc_gemm_run(A, B, C, M, N, K, batch, planes, nprod, splitk, (char*)workspace,
                     (cudaStream_t)stream);
}

const char* xtrg_batch_last_error();   // batch.cu

extern "C" const char* xtrg_last_error(const xtrg_ctx* ctx) {
  return ctx ? ctx->err.c_str() : xtrg_batch_last_error();
}

extern "C" void xtrg_destroy(xtrg_ctx* ctx) {
  if (!ctx) return;
  const char* pt = getenv("XTRG_PROFILE_TAGS");
  if (pt && pt[0] == '1') {
    static const char* names[8] = {"other", "substep1 (env x site)", "substep2 (x site)",
                                   "C_E (split-K)", "env update", "truncation (split)",
                                   "FP64 two-site update", "FP64 right environments"};
    for (int t = 0; t < 8; ++t)
      if (ctx->tag_n[t])
        fprintf(stderr, "xtrg tc %-24s launches %8lld  %10.1f ms  %8.1f TFLOP/s alg\n", names[t],
                ctx->tag_n[t], ctx->tag_ms[t],
                ctx->tag_ms[t] > 0 ? ctx->tag_flops[t] / ctx->tag_ms[t] / 1e9 : 0.0);
  }
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
  delete ctx;
}
