/*
 * xtrg.h -- C ABI of the GB300 XTRG beta-doubling engine.
 *
 * The engine implements the hot path of the exponential thermal tensor
 * renormalization group of arXiv:1801.00142:
 *
 *   rho(tau0) = sum_{k=0}^{Nc} (-tau0)^k H^k / k!           (Eq. RhoTau, Sec. II C)
 *   rho_{n+1} = rho_n^T rho_n,  tau_{n+1} = 2 tau_n          (Eq. rho:scale2, Sec. II B;
 *                                                            positivity-preserving form)
 *
 * where every MPO product is compressed back to bond dimension <= D* by the
 * two-site variational product compression of App. D.1 (cost function
 * Eq. MPO:prod, local solution Eq. LSEProd, environments and splitting of
 * Fig. VMPO), followed by normalisation and the thermodynamic quantities of
 * Eq. ThermalQuan (Sec. III A).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - MPO site tensor i is a dense real array W_i[Dl][d][d][Dr], row-major,
 *   where W_i[l][s][t][r] is the coefficient of |s><t| (row spin s, column
 *   spin t) between left bond l and right bond r.  bond_dims has L+1
 *   entries with bond_dims[0] = bond_dims[L] = 1.  Only d = 2 is supported.
 * - All host pointers passed in are read during the call and never retained:
 *   inputs are copied, the caller keeps ownership of its arrays.
 * - Device memory: the library allocates nothing on the device.  The caller
 *   provides one device workspace of at least xtrg_workspace_bytes() bytes
 *   (256-byte aligned); it is borrowed until xtrg_destroy and never freed by
 *   the library.  The library allocates small host bookkeeping only.
 * - Streams: every device operation is issued on the CUDA stream given to
 *   xtrg_create (a cudaStream_t passed as void*; NULL = legacy default
 *   stream).  Calls that return scalars or bond dimensions to the host
 *   synchronise that stream before returning.
 * - Errors: every call returns an xtrg_status; no exception or abort crosses
 *   the ABI.  After a failure xtrg_last_error(ctx) holds a one-line message.
 *   A context that returned XTRG_ECUDA should be destroyed.
 * - Thread safety: a context must not be used from two threads at once;
 *   different contexts (each with its own workspace and stream) may be driven
 *   from different host threads concurrently, as xtrg_batch_run does.
 */
#ifndef XTRG_H
#define XTRG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  XTRG_OK = 0,
  XTRG_EINVAL = 1,   /* bad argument: shape, size, NULL, unsupported option   */
  XTRG_ENOMEM = 2,   /* workspace too small                                   */
  XTRG_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed           */
  XTRG_ENUMERIC = 4, /* non-finite or non-positive norm/trace, SVD not converged */
  XTRG_ETIMEOUT = 5  /* a bounded device-side wait ran out                    */
} xtrg_status;

/* Arithmetic of the environment and two-site contractions (the O(D^4 d^3)
 * part).  Splitting, canonicalisation, normalisation and traces are FP64 in
 * every mode.  The tensor-core modes store every contraction operand as BF16
 * planes x ~= x0 + x1 (+ x2) and accumulate products of planes in FP32. */
typedef enum {
  XTRG_FP64 = 0,      /* FP64 CUDA-core contractions                           */
  XTRG_BF16X6 = 1,    /* tcgen05, 3 planes, 6 products: ~24 significant bits   */
  XTRG_BF16X3 = 2     /* tcgen05, 2 planes, 3 products: ~16 significant bits   */
} xtrg_precision;

/* An MPO given by host arrays (see conventions above). */
typedef struct {
  int L;                      /* number of sites, >= 2                        */
  int d;                      /* local dimension, must be 2                   */
  const int* bond_dims;       /* L+1 entries, first and last = 1              */
  const double* const* W;     /* L host pointers, W[i] has bond_dims[i]*d*d*bond_dims[i+1] doubles */
} xtrg_mpo;

typedef struct {
  double tau0;          /* initial inverse temperature, > 0                   */
  int order;            /* series order Nc of Eq. RhoTau, 1..16               */
  int dstar;            /* bond dimension cap D*, 1..1024                      */
  int sweeps;           /* full sweeps (L->R then R->L) per doubling, >= 1    */
  int init_sweeps;      /* full sweeps per product in the initialisation      */
  xtrg_precision prec;  /* contraction arithmetic for beta >= beta_switch     */
  double beta_switch;   /* doublings that start below this beta run in FP64   */
  double svd_rel_tol;   /* singular values <= svd_rel_tol * sigma_max are dropped (numerically zero) */
  int keep_parts;       /* tensor-core path: 0 = each two-site update builds both
                           halves of its environment (Fig. VMPO(a)); 1 = the halves
                           of every bond stay resident in device memory, so each
                           update builds one (about 2 L x 4 D*^3 x planes BF16
                           elements more workspace)                            */
  int orth_block;       /* tensor-core path: column-block width of the truncation's
                           orthonormalisation (bonds wider than one block are
                           orthonormalised block by block); 0 = 256, else 32..256
                           in steps of 32                                       */
} xtrg_config;

typedef struct {
  double beta;          /* inverse temperature of the current rho             */
  double lnZ;           /* ln Tr rho(beta)                                    */
  double f;             /* free energy per site, -lnZ / (N beta)              */
  double u;             /* energy per site, Tr(H rho) / (N Tr rho)            */
  double c;             /* specific heat per site, beta^2 (<H^2> - <H>^2) / N */
  double lnZ2;          /* ln Z(2 beta) = ln ||rho(beta)||_F^2 (Sec. II B)    */
  double trunc_err;     /* largest discarded weight of the last sweep          */
  double herm_defect;   /* Hermiticity defect ||rho - rho^T||_F / ||rho||_F of the
                           stored rho (Sec. II B); FP64 transfers, resolved down
                           to ~1.5e-8 (it is a square root of a difference); NaN
                           when switched off (xtrg_set_herm_check)               */
  int max_bond;         /* largest bond dimension of the current rho          */
  int n_doublings;      /* doublings done since xtrg_init                     */
} xtrg_obs;

typedef struct xtrg_ctx xtrg_ctx;

/* Bytes of device workspace a context for (H, cfg) needs; 0 on bad input. */
size_t xtrg_workspace_bytes(const xtrg_mpo* H, const xtrg_config* cfg);

/* Create a context for Hamiltonian MPO H (copied to the workspace).
 * dev_workspace: device pointer, >= xtrg_workspace_bytes(H, cfg) bytes.
 * cuda_stream: cudaStream_t as void*.  On success *out is a new context. */
xtrg_status xtrg_create(xtrg_ctx** out, const xtrg_mpo* H, const xtrg_config* cfg,
                        void* dev_workspace, size_t workspace_bytes, void* cuda_stream);

/* rho <- rho(tau0) by the series of Eq. RhoTau in Horner form, each product
 * H*Y compressed variationally (App. D.1), "+I" an exact direct sum; then
 * normalised.  beta <- tau0. */
xtrg_status xtrg_init(xtrg_ctx* ctx);

/* One doubling: rho <- compress(rho^T rho) with cfg.sweeps full sweeps,
 * normalised; beta <- 2 beta (Eq. rho:scale2).  On the tensor-core path the
 * sweeps take every decision on the device (the exact-split fallback
 * included) and the host reads the product's results once at its end; once
 * the bonds are saturated, the device work of a doubling is captured as a
 * CUDA graph (one per buffer parity) and later doublings replay it
 * (environment XTRG_NO_GRAPHS=1 turns this off; so do profiling and
 * XTRG_DEBUG=1).  A replay computes the same as a direct run. */
xtrg_status xtrg_double(xtrg_ctx* ctx);

/* Pointwise-Taylor SETTN step (Sec. II C, Eq. Tay, Fig. SETTNAlg(b)), the
 * alternative to a doubling with a free step size:
 *   rho(beta + dtau) = sum_{k=0}^{order} (-dtau)^k / k! H^k rho(beta).
 * The terms H^k rho are built by compressed products H (H^{k-1} rho) (App.
 * D.1) and summed by the variational MPO-sum compression (App. D.2, Eq.
 * LSESum), cfg.sweeps sweeps each, bonds <= D*, all in FP64; then normalised;
 * beta <- beta + dtau.  The Taylor remainder is about (dtau ||H||)^{order+1} /
 * (order+1)! relative: the caller chooses order for its dtau.  dev_buf:
 * device memory of at least xtrg_settn_workspace_bytes(ctx, order) bytes,
 * 256-byte aligned, borrowed for the call (the terms k >= 1 and every term's
 * overlap environments).  1 <= order <= 64, dtau > 0. */
size_t xtrg_settn_workspace_bytes(const xtrg_ctx* ctx, int order);
xtrg_status xtrg_settn_step(xtrg_ctx* ctx, double dtau, int order, void* dev_buf, size_t bytes);

/* *lnZ <- ln Tr rho(beta) (a logarithm: Z overflows FP64 for long chains). */
xtrg_status xtrg_trace(xtrg_ctx* ctx, double* lnZ);

/* Thermodynamics of Eq. ThermalQuan at the current beta. */
xtrg_status xtrg_observables(xtrg_ctx* ctx, xtrg_obs* out);

/* <O> = Tr(O rho) / Tr rho of the current state for an operator given as a
 * host MPO (same conventions as xtrg_mpo; L sites, bonds <= D* + 1), e.g. the
 * MPOs of (S^z_tot)^2 and (S^z_tot)^4 whose expectations give the Binder
 * ratio U_4 = <M^2>^2 / <M^4> (Sec. IV D, Eq. Binder).  FP64 transfer
 * contraction; O is copied, the caller keeps its arrays.  Synchronises the
 * stream. */
xtrg_status xtrg_expectation(xtrg_ctx* ctx, const xtrg_mpo* O, double* value);

/* rho_{n,n'} = rho_a rho_b (Sec. II B, after Eq. zshift): the product of two
 * states saved by xtrg_checkpoint_save in this context (or one of the same
 * length and capacity), compressed to D* with cfg.sweeps sweeps in FP64
 * (App. D.1), becomes the current state at beta_a + beta_b with ln c_a +
 * ln c_b + ln s.  For states of the same Hamiltonian (symmetric, commuting)
 * this is rho(beta_a + beta_b): intermediate grid points between doublings. */
xtrg_status xtrg_cross_product(xtrg_ctx* ctx, const void* ckpt_a, size_t bytes_a,
                               const void* ckpt_b, size_t bytes_b);

/* MPO entanglement of the current rho at every bond (Sec. IV A, Eq. purif):
 * rho is read as a state of the doubled local space |s>|t>, normalised in the
 * Frobenius norm; at bond i (between sites i-1 and i, i = 1..L-1) its Schmidt
 * values s_k give p_k = s_k^2 / sum s^2 and S[i-1] = -sum_k p_k ln p_k.
 * S: host array of n >= L-1 doubles.  FP64 throughout (one Jacobi SVD per
 * bond on a copy of rho; rho itself is unchanged).  Synchronises the stream. */
xtrg_status xtrg_entanglement(xtrg_ctx* ctx, double* S, int n);

/* Copy the current normalised rho to host memory.  bond_dims gets L+1 ints;
 * W[i] must hold bond_dims[i]*4*bond_dims[i+1] doubles (query the dims first
 * with W == NULL).  *lnc gets ln c, rho(beta) = e^{lnc} * rho. */
xtrg_status xtrg_get_state(xtrg_ctx* ctx, int* bond_dims, double* const* W, double* lnc,
                           double* beta);

/* Replace the current rho by a host MPO, its log scale lnc and its beta.
 * Bonds must not exceed the context's capacity (D* + 1).  right_canonical:
 * nonzero if sites 1..L-1 are right-orthonormal (as every state returned by
 * xtrg_get_state is), which lets the next doubling skip re-canonicalising;
 * zero for an MPO in any gauge. */
xtrg_status xtrg_set_state(xtrg_ctx* ctx, const xtrg_mpo* rho, double lnc, double beta,
                           int right_canonical);

/* Device-side checkpoint of the current state (rho, ln c, beta, doubling
 * count): xtrg_checkpoint_save copies it into dev_buf, device memory of at
 * least xtrg_checkpoint_bytes(ctx) bytes, 256-byte aligned, owned by the
 * caller; xtrg_checkpoint_load makes a saved state the current one (same
 * chain length, bonds within this context's capacity D* + 1), stream-ordered
 * after the copies, so the next doubling continues from it.  A checkpoint is
 * plain bytes: it may be copied to host memory or to another context of the
 * same length and capacity.  Resuming from a checkpoint is exact (the saved
 * tensors are the FP64 state).  Both calls synchronise the stream (save: its
 * header is staged in host memory; load: the bond dimensions are read back).
 * XTRG_ENOMEM: buffer too small; XTRG_EINVAL: not a checkpoint of this chain. */
size_t xtrg_checkpoint_bytes(const xtrg_ctx* ctx);
xtrg_status xtrg_checkpoint_save(xtrg_ctx* ctx, void* dev_buf, size_t bytes);
xtrg_status xtrg_checkpoint_load(xtrg_ctx* ctx, const void* dev_buf, size_t bytes);

typedef struct {
  double contraction_flops;  /* algorithmic 2*M*N*K of every contraction GEMM       */
  double split_flops;        /* estimated flops of the truncation (split)           */
  double tc_flops;           /* algorithmic flops of the tensor-core GEMM launches   */
  double tc_ms;              /* their summed device time (only while profiling)      */
  long long two_site_updates;
  long long tc_launches;     /* tensor-core GEMM launches (only while profiling)     */
  long long kernel_launches; /* kernels launched by this library, all contexts      */
  long long exact_split_fallbacks; /* tensor-core-path updates that took the exact FP64 split */
  double split_ms;           /* device time of the tensor-core truncations (only while profiling) */
  long long orth_cluster_calls; /* orthonormalisations run as one thread-block cluster, all contexts */
  double fp64_update_ms;     /* device time of the FP64-path two-site updates (only while profiling) */
  long long fp64_updates_timed; /* FP64-path two-site updates timed (only while profiling) */
  double fp64_env_pass_ms;   /* device time of the FP64-path initial right environments (profiling) */
  long long orth_fallbacks;  /* tensor-core truncations whose CholeskyQR2 broke down and were
                                orthonormalised by block Gram-Schmidt instead (this context) */
  long long orth_full_second_pass; /* tensor-core truncations whose first CholeskyQR pass left
                                the basis too far from orthonormal for the first-order second
                                pass, so the full second pass ran (this context) */
  long long orth_deflated_columns; /* columns the first CholeskyQR pass dropped as numerically
                                dependent on the columns before them (this context) */
  long long graph_captures;  /* tensor-core doublings captured as a CUDA graph (this context) */
  long long graph_replays;   /* tensor-core doublings run by replaying a captured graph */
  long long split_shapes_tuned; /* C_E shapes whose split-K the autotuner has chosen by timing
                                the candidates (all contexts of the process share the choice) */
} xtrg_stats;

/* Counters since creation (kernel_launches: since the library was loaded).
 * Synchronises the context's stream (orth_fallbacks, orth_full_second_pass and
 * orth_deflated_columns are counted on the device). */
xtrg_status xtrg_get_stats(const xtrg_ctx* ctx, xtrg_stats* out);

/* on != 0: time every tensor-core GEMM launch, every tensor-core truncation,
 * every FP64-path two-site update and the FP64-path initial environment pass
 * with CUDA events on the context's stream (adds event records; results are
 * resolved at the end of each product, which then synchronises). */
xtrg_status xtrg_set_profiling(xtrg_ctx* ctx, int on);

/* The Hermiticity diagnostic of xtrg_observables: on = 1 (the default)
 * computes herm_defect (FP64 transfer contractions of ||rho||_F^2 and
 * Tr(rho rho), about 16 D^3 flops per site each); 0 leaves it NaN and the
 * thermodynamics (ln Z, f, u, c) unchanged. */
xtrg_status xtrg_set_herm_check(xtrg_ctx* ctx, int on);

/* Graph capture of saturated tensor-core doublings (see xtrg_double): on = 1
 * (the default) allows it, 0 runs every doubling directly and drops the
 * graphs captured so far. */
xtrg_status xtrg_set_graphs(xtrg_ctx* ctx, int on);

/* The tensor-core contraction primitive behind the XTRG_BF16X* modes, exposed
 * on its own: C[b] = A[b] * B[b]^T for row-major FP64 device arrays
 * A (batch x M x K), B (batch x N x K), C (batch x M x N).  A and B are split
 * into `planes` BF16 planes (2 or 3); nprod products of planes are
 * accumulated in FP32 on the tcgen05 tensor cores (1: x0*y0; 3: + x0*y1 +
 * x1*y0; 6: + x0*y2 + x1*y1 + x2*y0); splitk > 1 splits K across CTAs and
 * sums the partials in FP64.  workspace: device memory of at least
 * xtrg_tc_gemm_workspace_bytes() bytes, 256-byte aligned.  Synchronises the
 * stream.  Returns XTRG_ETIMEOUT if a bounded device wait expired. */
size_t xtrg_tc_gemm_workspace_bytes(int M, int N, int K, int batch, int planes, int splitk);
xtrg_status xtrg_tc_gemm(const double* A, const double* B, double* C, int M, int N, int K,
                         int batch, int planes, int nprod, int splitk, void* workspace,
                         size_t workspace_bytes, void* cuda_stream);

/* The same primitive for C[b] = A[b] * B[b] with B given row-major as
 * batch x K x N (FP64, device): B's planes keep that layout and are staged
 * into the tensor cores as an MN-major operand (no transpose pass).  Same
 * precision, splitk and stream behaviour as xtrg_tc_gemm; workspace of at
 * least xtrg_tc_gemm_nn_workspace_bytes() bytes, 256-byte aligned. */
size_t xtrg_tc_gemm_nn_workspace_bytes(int M, int N, int K, int batch, int planes, int splitk);
xtrg_status xtrg_tc_gemm_nn(const double* A, const double* B, double* C, int M, int N, int K,
                            int batch, int planes, int nprod, int splitk, void* workspace,
                            size_t workspace_bytes, void* cuda_stream);

/* xtrg_tc_gemm for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a service of this library.  Same arguments,
 * results and precision as xtrg_tc_gemm, without the workspace: the scratch
 * (operand planes, partial sums, an error flag) lives in one file-scope
 * device array of 16 MiB that every GPU loading this library holds until
 * the process exits.  Sizes must satisfy
 *   r(planes*batch*M*ld*2) + r(planes*batch*N*ld*2) + r(splitk*batch*M*N*4) + 256 <= 16 MiB,
 * with ld = K rounded up to a multiple of 8 and r() rounding up to 256 bytes;
 * larger sizes return XTRG_ENOMEM and do nothing.  The call allocates no
 * device memory.  The first call on a device looks up the array's device
 * address (with that device current), so make it before any stream capture.
 * Every call uses the same array: calls that overlap on the GPU race, so
 * order them (one stream, or events).  Uses the current device and
 * synchronises the given stream. */
xtrg_status xtrg_tc_gemm_static(const double* A, const double* B, double* C, int M, int N, int K,
                                int batch, int planes, int nprod, int splitk, void* cuda_stream);

/* ------------------------------------------------------------------ batch
 * Many independent runs on one GPU: interleaved tau0 grids of one model
 * (Eq. zshift) or different (L, Delta, D*) instances.  The workspace is cut
 * into equal slots of xtrg_batch_plan's slot_bytes (the largest instance's
 * need, rounded up to 256 bytes); min(n, max_concurrent (<= 0: 8), slots
 * that fit) host threads each own one slot and one stream and take instances
 * from a shared queue, largest first.  Instance i runs xtrg_init and
 * n_doublings[i] doublings; its n_doublings[i] + 1 observables rows (beta =
 * tau0 ... 2^n tau0) go to out[off_i ...], off_i = sum_{j<i} (n_doublings[j]
 * + 1).  H, cfg, n_doublings: n host entries, read only; workspace: device
 * memory, 256-byte aligned, borrowed for the call.  The caller's stream is
 * ordered before the first and after the last device work.  On the first
 * failing instance no new instance starts; the call returns that status and
 * xtrg_last_error(NULL) holds its message. */
xtrg_status xtrg_batch_plan(int n, const xtrg_mpo* H, const xtrg_config* cfg,
                            size_t workspace_bytes, int max_concurrent, int* n_slots,
                            size_t* slot_bytes);
xtrg_status xtrg_batch_run(int n, const xtrg_mpo* H, const xtrg_config* cfg,
                           const int* n_doublings, xtrg_obs* out, void* workspace,
                           size_t workspace_bytes, int max_concurrent, void* cuda_stream);

/* Message of the last failure of ctx; with ctx == NULL, of the last batch call. */
const char* xtrg_last_error(const xtrg_ctx* ctx);

/* Free host bookkeeping.  The workspace stays the caller's. */
void xtrg_destroy(xtrg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* XTRG_H */
