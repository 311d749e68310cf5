/*
 * rb.h -- C ABI of librb: the online stage of the velocity-only (solenoidal) reduced-basis
 * method for steady Navier-Stokes flow, on one NVIDIA GB300 (sm_103a).
 *
 * For each parameter query mu = (alpha in degrees, Re) the library
 *   1. evaluates the parameter functions theta(mu) of the affine split (Sec. 2.4,
 *      Eqs. split-a..split-d1),
 *   2. assembles A(mu) = sum_q theta^a_q A_q and f(mu) = sum_q theta^f_q f_q
 *      (Sec. 3.5, reduced affine matrices),
 *   3. runs Newton from u = 0 on the velocity-only reduced equation (Sec. 2.2, Eq. velonly)
 *        R(u; mu) = A(mu) u + sum_q theta^c_q C_q(u, u) - f(mu) = 0,
 *        C_q(u, u)[k] = sum_{j,l} C_q[j][l][k] u_j u_l          (Sec. 3.6, Eq. tensor)
 *      with the tensor Jacobian (Sec. 3.6)
 *        J[k][j] = A(mu)[k][j] + sum_q theta^c_q sum_l (C_q[l][j][k] + C_q[j][l][k]) u_l
 *      and one dense n x n partial-pivot solve per step (Sec. 4.1, Eq. blocksolve-1),
 *      stopping when ||delta||_2 <= tol_update (Sec. 6: update <= 1e-10 in the H1 seminorm,
 *      the Euclidean coefficient norm for an orthonormal POD basis, Sec. 3.2-3.3) and
 *      ||R||_2 <= tol_res * max(1, ||f(mu)||_2),
 *   4. recovers the pressure a posteriori (Sec. 2.2, Eq. sup-vvar; Sec. 4.1, Eq. blocksolve-2)
 *        B(mu) p = fs(mu) - As(mu) u - sum_q theta^c_q Cs_q(u, u).
 *
 * Index convention: C_q[j][l][k] = c_q(u_j, u_l, w_k) -- j advecting, l advected, k test.
 * Matrices are row-major with the test index as the row.
 *
 * Parameter functions (RB_THETA_TRIG): a = alpha * pi / 180, trig_q(a) = cos(q a) for even q
 * and sin(q a) for odd q (trig_0 = 1); theta^a_q = trig_q / Re and
 * theta^c_q = theta^f_q = theta^b_q = trig_q. Polynomial functions (RB_THETA_POLY, the
 * monomials of the truncated rotation series of Sec. 5, Eq. rotsum, in which every pulled-back
 * form is affine): phi = alpha * pi / 180, theta^a_q = phi^q / Re and
 * theta^c_q = theta^f_q = theta^b_q = phi^q. With rb_solve_theta the caller passes theta.
 * theta rows are laid out [theta^a (q_a) | theta^c (q_c) | theta^f (q_f) | theta^b (q_b)].
 *
 * Error behaviour: every function returns an rb_status. A failing call leaves a message for
 * rb_last_error() (per context, per calling thread). A per-query failure (non-convergence,
 * singular Jacobian, non-finite values) is reported in rb_query_info.status and never makes
 * the call fail. All functions are synchronous unless stated otherwise.
 *
 * Threading: one context may be used by one solving thread at a time; the rb_serve_* calls
 * are thread-safe and may be called from any thread while the server runs.
 */
#ifndef RB_H_
#define RB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RB_OK = 0,
  RB_PENDING = 1,       /* rb_serve_poll: result not ready yet */
  RB_ERR_ARG = -1,      /* invalid argument (NULL, size out of range, bad layout) */
  RB_ERR_OOM = -2,      /* device or pinned-host allocation failed / over memory budget */
  RB_ERR_CUDA = -3,     /* a CUDA runtime or driver call failed */
  RB_ERR_STATE = -4,    /* call not valid in the current state (no operators, server off) */
  RB_ERR_TIMEOUT = -5   /* a bounded device-side wait or host wait gave up */
} rb_status;

/* per-query outcome, rb_query_info.status */
enum {
  RB_Q_OK = 0,
  RB_Q_NOT_CONVERGED = 1,  /* iteration cap reached */
  RB_Q_SINGULAR = 2,       /* a pivot of the Jacobian (or of B(mu)) was zero / not finite */
  RB_Q_NONFINITE = 3,      /* NaN or Inf in the residual or update */
  RB_Q_REJECTED = 4        /* query size out of range or cancelled */
};

/* storage type of the convection tensors C and Cs (values are taken as exact): IEEE binary64,
 * binary32, or bfloat16 (the upper 16 bits of a binary32, as uint16_t) */
enum { RB_F64 = 0, RB_F32 = 1, RB_BF16 = 2 };

/* precision of the Newton solve */
enum {
  RB_PREC_FP64 = 0,  /* everything in FP64: contraction, LU, residual */
  RB_PREC_MIXED = 1  /* Jacobian contraction on BF16 tensor cores + FP32 LU (inexact Newton);
                        residual (error-free sliced products on the tensor cores) and
                        convergence test FP64-accurate */
};

/* pressure stage of rb_solve, rb_solve_theta and rb_solve_device */
enum {
  RB_PRESSURE_RECOVER = 0,     /* a-posteriori recovery from the supremizer system
                                  (Sec. 2.2, Eq. sup-vvar; Sec. 4.1, Eq. blocksolve-2) */
  RB_PRESSURE_RECONSTRUCT = 1  /* reconstruction from the velocity coefficients with the
                                  pressure modes of a combined basis (Sec. 4.2):
                                  p = sum_j u_j p^_j, see rb_load_pressure_modes */
};

/* parameter-function family */
enum { RB_THETA_TRIG = 0, RB_THETA_USER = 1, RB_THETA_POLY = 2 };

typedef struct rb_ctx rb_ctx; /* opaque; owns all device memory it allocates */

/* Reduced operators of one n_max set. Host pointers, caller-owned; rb_load_operators copies
 * them (the caller may free them afterwards). Smaller queries use the leading blocks
 * (nested truncation). Pressure operators are optional (B == NULL: no pressure). */
typedef struct {
  int n_max;          /* reduced velocity size, 1..RB_N_MAX */
  int m;              /* pressure / supremizer reduced size, 0..RB_M_MAX (0 if B == NULL) */
  int q_a, q_c, q_f, q_b;  /* affine term counts, q_a, q_c, q_f >= 1 */
  int dtype_c;        /* RB_F64, RB_F32 or RB_BF16: storage of C and Cs (kept on the device in
                         that type; BF16 halves the upload and the device copy of FP32) */
  const double *A;    /* [q_a][n_max][n_max], row = test k, column = trial j */
  const void *C;      /* [q_c][n_max][n_max][n_max], index [j][l][k] */
  const double *f;    /* [q_f][n_max] */
  const double *B;    /* [q_b][m][m] or NULL; row = supremizer test, column = pressure trial */
  const double *As;   /* [q_a][m][n_max] or NULL */
  const void *Cs;     /* [q_c][n_max][n_max][m] or NULL, index [j][l][k'] */
  const double *fs;   /* [q_f][m] or NULL */
} rb_operators;

#define RB_N_MAX 320
#define RB_M_MAX 128
#define RB_Q_MAX 64

typedef struct {
  int precision;      /* RB_PREC_* */
  double tol_update;  /* absolute bound on ||delta||_2 (default 1e-10) */
  double tol_res;     /* bound on ||R||_2 / max(1, ||f(mu)||_2) (default 1e-10) */
  int max_iter;       /* Newton iteration cap (default 50) */
  size_t mem_budget;  /* device bytes the context may allocate (0: 80% of free memory) */
  int use_graph;      /* capture per-iteration launches in CUDA graphs (default 1) */
  int autotune;       /* time kernel variants on first use per shape (default 1; the
                         environment variable RB_AUTOTUNE=0 makes the default 0) */
  int theta_family;   /* RB_THETA_TRIG (default) or RB_THETA_POLY: the functions that mu is
                         mapped through by rb_solve, rb_solve_device and the server
                         (RB_THETA_USER: as RB_THETA_TRIG; theta comes with rb_solve_theta) */
  int serve_slots;    /* serving: queries on the device at once (0: as many as the memory
                         budget admits, at most 4096) */
  int pressure_method;  /* RB_PRESSURE_RECOVER (default) or RB_PRESSURE_RECONSTRUCT: then
                           p_out of the solves is [n_queries][m_r] from the loaded pressure
                           modes, and the server refuses to start */
} rb_config;

typedef struct {
  int status;          /* RB_Q_* */
  int iters;           /* Newton iterations performed */
  int precision_used;  /* RB_PREC_* of the Jacobian in the final iteration */
  int reserved;
  double res_norm;     /* ||R(u_k)||_2 at the last iteration */
  double upd_norm;     /* ||delta_k||_2 at the last iteration */
} rb_query_info;

/* Fill *cfg with the defaults listed above. */
void rb_config_default(rb_config *cfg);

/* Create a context on CUDA device `device`; cfg == NULL means defaults. */
int rb_create(rb_ctx **out, const rb_config *cfg, int device);

/* Destroy a context and free all its device and pinned-host memory (stops the server). */
void rb_destroy(rb_ctx *ctx);

/* Last error message of this context on the calling thread ("" if none). Never NULL.
 * ctx == NULL gives the last error of a context-free call (rb_gepp_solve_static). */
const char *rb_last_error(rb_ctx *ctx);

/* Copy an operator set to the device and build the per-precision layouts (Sec. 3.5-3.6:
 * all reduced operators are precomputed offline; online assembly only weights them).
 * Replaces a previously loaded set. Returns RB_ERR_ARG on bad sizes or NULL arrays,
 * RB_ERR_OOM if the layouts do not fit in the memory budget. */
int rb_load_operators(rb_ctx *ctx, const rb_operators *ops);

/* ---- operator files (the output of the offline stage, Sec. 3.5-3.6) ---------------------
 * A versioned binary file: a 64-byte header (magic "RBOPS\0\0\0", u32 version 1, u32 header
 * size 64, i32 n_max, m, q_a, q_c, q_f, q_b, dtype_c, u32 flags with bit 0 set when pressure
 * operators are present, u64 payload bytes, u64 checksum) and the arrays of rb_operators in
 * field order (A, C, f, then B, As, Cs, fs when present), each C-contiguous in the layout
 * rb_operators documents, C and Cs in their storage type; all little-endian. The checksum is
 * FNV-1a (64-bit) over the payload taken as 8-byte words, a last partial word zero-padded.
 *
 * rb_save_operators writes ops (host arrays, not modified) to path; context-free, errors go
 * to rb_last_error(NULL): RB_ERR_ARG on bad sizes, missing arrays or a failed write.
 * rb_load_operator_file reads path, checks magic, version, sizes, file length and checksum
 * (RB_ERR_ARG naming the failed check; nothing is loaded then) and loads the operators as
 * rb_load_operators does. */
int rb_save_operators(const rb_operators *ops, const char *path);
int rb_load_operator_file(rb_ctx *ctx, const char *path);

/* Solve n_queries queries from host buffers (synchronous).
 *   mu     [n_queries][2] (alpha_deg, Re)
 *   n      [n_queries] reduced sizes 1..n_max, or NULL for n_max
 *   u_out  [n_queries][n_max] velocity coefficients, entries beyond n set to 0
 *   p_out  [n_queries][m] pressure coefficients, or NULL (ignored when no pressure ops)
 *   info   [n_queries] or NULL
 * Queries with n outside 1..n_max get RB_Q_REJECTED. */
int rb_solve(rb_ctx *ctx, const double *mu, int n_queries, const int *n, double *u_out,
             double *p_out, rb_query_info *info);

/* Same with caller-supplied parameter functions theta [n_queries][q_a + q_c + q_f + q_b]. */
int rb_solve_theta(rb_ctx *ctx, const double *theta, int n_queries, const int *n,
                   double *u_out, double *p_out, rb_query_info *info);

/* Solve from device buffers owned by the caller, asynchronously on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). The buffers must stay valid until
 * the stream reaches the end of the work enqueued here. d_n may be NULL (all n_max);
 * d_p and d_info may be NULL. The context's internal scratch is reused by the next call on any
 * stream, so calls on one context must be ordered.
 * The call returns once the solve is enqueued, without waiting for it, except:
 *   - d_n != NULL: the sizes are copied to the host to group the queries by size, which waits
 *     for the work already on cuda_stream (rb_solve_device_sized avoids this);
 *   - the first solve of a new batch shape (batch size, size mix or buffers) sizes its scratch,
 *     runs the autotuner (cfg.autotune) and captures the solve graph, which synchronises;
 *   - with cfg.use_graph == 0 or profiling on, every Newton iteration is checked on the host;
 *   - the FP64 path (RB_PREC_FP64) never waits.
 * A device-side wait of the mixed path that gives up (RB_ERR_TIMEOUT: the results of that solve
 * are invalid) is reported by rb_solve_device_status, by rb_solve, or by the next solve call on
 * the context, once. */
int rb_solve_device(rb_ctx *ctx, const double *d_mu, int n_queries, const int *d_n,
                    double *d_u, double *d_p, rb_query_info *d_info, void *cuda_stream);

/* rb_solve_device with the query sizes also given on the host: h_n [n_queries] (caller-owned,
 * read during the call only) must hold the same values as d_n; then no copy of d_n to the host
 * is needed and a solve of a batch shape seen before only enqueues. h_n == NULL behaves as
 * rb_solve_device; h_n != NULL with d_n == NULL is RB_ERR_ARG. */
int rb_solve_device_sized(rb_ctx *ctx, const double *d_mu, int n_queries, const int *d_n,
                          const int *h_n, double *d_u, double *d_p, rb_query_info *d_info,
                          void *cuda_stream);

/* Outcome of the solves enqueued on this context so far: RB_OK when they have completed without
 * a device-side failure; RB_PENDING when wait == 0 and the last one has not completed yet;
 * RB_ERR_TIMEOUT (once) when a device-side wait of one of them gave up. wait != 0 blocks until
 * the last solve has completed. */
int rb_solve_device_status(rb_ctx *ctx, int wait);

/* ---- pressure reconstruction (Sec. 4.2, combined velocity-pressure basis) -----------------
 * With a combined basis every velocity basis function j carries pressure data p^_j, and the
 * pressure of a solution with velocity coefficients u is p = sum_{j < n} u_j p^_j (the
 * velocity system is unchanged). This assumes that pressure depends linearly on velocity, which
 * the Navier-Stokes equations do not satisfy (Sec. 4.2, remark on linearity): it suits linear
 * models or small parameter ranges; recovery (RB_PRESSURE_RECOVER) has no such restriction.
 *
 * rb_load_pressure_modes copies P_hat [m_r][n_max] (host, row-major, caller-owned): column j
 * holds the coefficients of p^_j in any pressure space of m_r functions (reduced or
 * high-fidelity), 1 <= m_r <= RB_MR_MAX. Queries of size n use the first n columns (nested
 * truncation). Replaces earlier modes; loading new operators drops them. RB_ERR_STATE without
 * operators, RB_ERR_ARG on bad sizes, RB_ERR_OOM over the memory budget. */
#define RB_MR_MAX (1 << 22)
int rb_load_pressure_modes(rb_ctx *ctx, const double *P_hat, int m_r);

/* p_out[b][k] = sum_{j < n_b} P_hat[k][j] u[b][j] in FP64 for b < n_queries, from host buffers:
 * u [n_queries][n_max] (entries from n_b on are not read), n [n_queries] (NULL: n_max),
 * p_out [n_queries][m_r]. A query with n_b outside 1..n_max gets NaN in every entry.
 * RB_ERR_STATE when no modes are loaded. Synchronous. */
int rb_reconstruct_pressure(rb_ctx *ctx, const double *u, int n_queries, const int *n,
                            double *p_out);

/* The same from device buffers, asynchronously on cuda_stream (NULL: the legacy stream). */
int rb_reconstruct_pressure_device(rb_ctx *ctx, const double *d_u, int n_queries,
                                   const int *d_n, double *d_p, void *cuda_stream);

/* Evaluate the residual R(u; mu) (FP64) and, if J_out != NULL, the Jacobian J(u; mu) at
 * caller-given coefficient vectors, for n_queries queries of size n (all equal, <= n_max),
 * from host buffers. precision selects the path (RB_PREC_FP64: FP64 contraction;
 * RB_PREC_MIXED: BF16 tensor-core Jacobian contraction plus A(mu) from FP64, and the residual
 * from the error-free sliced tensor-core product).
 *   u      [n_queries][n]      R_out [n_queries][n]      J_out [n_queries][n][n] (row k)
 * This is the building block of one Newton step (Sec. 3.6), exposed for verification. */
int rb_eval(rb_ctx *ctx, const double *mu, int n_queries, int n, const double *u,
            int precision, double *R_out, double *J_out);

/* Batched Gaussian elimination with partial pivoting (first row of largest magnitude),
 * FP64, on host buffers: solves M_b x_b = rhs_b for b < batch. M [batch][n][n] row-major
 * (not modified), rhs [batch][n], x_out [batch][n], status [batch] (0 ok, RB_Q_SINGULAR).
 * The dense solve of Sec. 4.1 (Eq. blocksolve-1), exposed for verification. */
int rb_gepp_solve(rb_ctx *ctx, int n, int batch, const double *M, const double *rhs,
                  double *x_out, int *status);

/* ---- batched solve without allocation -----------------------------------------------------
 * No counterpart in the paper: this entry point serves callers that cannot allocate device
 * memory when they solve -- processes held to a fixed memory budget, hosts that only lend the
 * library pre-allocated buffers, or runtimes that must not take the allocator's locks on their
 * hot path. It solves
 * M_s x_s = rhs_s for s < batch with the same partial pivoting as rb_gepp_solve, from DEVICE
 * buffers: d_M [batch][n][n] row-major (not modified), d_rhs [batch][n], d_x [batch][n],
 * d_status [batch] (0 or RB_Q_SINGULAR), asynchronously on cuda_stream (NULL: legacy stream).
 * The working copies of the matrices live in one file-scope device array of
 * RB_STATIC_SCRATCH_BYTES, which every GPU that loads this library holds until the process
 * exits; the call makes no cudaMalloc, cudaFree or other allocating call. n outside
 * 1..RB_STATIC_N_MAX or batch < 0 returns RB_ERR_ARG with a message for rb_last_error(NULL).
 * The first call on a device looks up the array's device address with that device current, so
 * make that first call before any stream capture; the address is looked up again when the
 * device's context has changed since (after cudaDeviceReset). Every call uses the same array and it keeps
 * the previous call's contents (each system is copied in before use): calls whose GPU work
 * overlaps (other streams or threads) race on it, so the caller must order them. */
#define RB_STATIC_N_MAX 512
#define RB_STATIC_SCRATCH_BYTES (16u << 20)
int rb_gepp_solve_static(int n, int batch, const double *d_M, const double *d_rhs, double *d_x,
                         int *d_status, void *cuda_stream);

/* ---- offline stage: the reduced operators from high-fidelity data (Sec. 3.2, 3.5, 3.6) -----
 * All synchronous, FP64 on the context's device, from caller-owned host arrays (read only;
 * outputs written in full). Device scratch is allocated within the context's memory budget for
 * the call and freed before it returns. RB_ERR_ARG on bad sizes or indices (message for
 * rb_last_error), RB_ERR_OOM over the budget. */
typedef struct {           /* a sparse high-fidelity matrix in CSR form, rows x cols */
  int rows, cols;
  const int *indptr;       /* [rows + 1], non-decreasing, indptr[0] = 0 */
  const int *indices;      /* [indptr[rows]] column of each entry, 0 <= column < cols */
  const double *values;    /* [indptr[rows]] */
} rb_csr;

typedef struct {           /* one quadrature term of a pointwise trilinear form:           */
  rb_csr P, Q, R;          /*   c(a, v, w) += sum_x weight(x) (P a)(x) (Q v)(x) (R w)(x),    */
  const double *weight;    /*   P, Q, R points x N_h; weight [points] or NULL (all 1)       */
} rb_trilinear_term;

#define RB_POD_K_MAX 128   /* snapshots of one POD */

/* POD by the method of snapshots (Sec. 3.2, Eqs. covmx and spd): the covariance matrix
 * C_ij = phi_i^T Z phi_j of the snapshots S [K][N] (row i = snapshot i) in the inner product Z
 * (N x N, symmetric positive semidefinite, e.g. the H1-seminorm stiffness), its eigenpairs
 * (cyclic Jacobi, FP64) in decreasing order, and the n modes
 * psi_j = lambda_j^(-1/2) sum_i v^j_i phi_i into V_out [n][N] (row j = mode j, orthonormal in Z);
 * lambda_out [K] (or NULL) all K eigenvalues, decreasing. 1 <= n <= K <= RB_POD_K_MAX; lambda_n
 * must exceed K eps lambda_1 (the numerical rank, RB_ERR_ARG otherwise). Eigenvectors, and so
 * modes, are determined up to sign. */
int rb_offline_pod(rb_ctx *ctx, const double *S, int K, int N, const rb_csr *Z, int n,
                   double *V_out, double *lambda_out);

/* Galerkin projection of a high-fidelity matrix (Sec. 3.5, Eq. redorth-final):
 * Mr_out [n][n] = V M V^T for the modes V [n][N] (rows) and M (N x N). 1 <= n <= 128. */
int rb_offline_project(rb_ctx *ctx, const double *V, int n, int N, const rb_csr *M,
                       double *Mr_out);
/* fr_out [n] = V f for f [N]: the reduced right-hand side. 1 <= n <= 128. */
int rb_offline_project_vector(rb_ctx *ctx, const double *V, int n, int N, const double *f,
                              double *fr_out);

/* The third-order tensor of a trilinear form on the modes (Sec. 3.6, Eq. tensor):
 * C_out[j][l][k] = c(psi_j, psi_l, psi_k) = sum_terms sum_x weight(x) (P psi_j)(x) (Q psi_l)(x)
 * (R psi_k)(x), the index order of rb_operators.C (j advecting, l advected, k test), for the
 * modes V [n][N] and n_terms quadrature terms. 1 <= n <= RB_N_MAX. */
int rb_offline_tensor(rb_ctx *ctx, const double *V, int n, int N, const rb_trilinear_term *terms,
                      int n_terms, double *C_out);

/* ---- per-kernel timing ------------------------------------------------------------------
 * While enabled, every kernel the context launches is bracketed by CUDA events on its
 * launching stream; rb_profile_read returns the accumulated device time and launch count of
 * one kernel kind. rb_profile(ctx, 1) resets the counters; timing adds about 1 us per launch. */
enum {
  RB_K_NEWTON_FP64 = 0,  /* fused FP64 Newton (one CTA per query) */
  RB_K_PRESSURE = 1,     /* pressure recovery (FP64 path) / B(mu) p = r solve (mixed) */
  RB_K_BUILD_X = 2,      /* mixed: operand build (theta (x) u, digit slices) */
  RB_K_GEMM_JAC = 3,     /* mixed: tcgen05 Jacobian contraction (BF16 -> FP32) */
  RB_K_GEMM_RES = 4,     /* mixed: tcgen05 sliced residual contraction (-> FP64) */
  RB_K_LU = 5,           /* mixed: FP32 LU, triangular solves, update, stopping test */
  RB_K_INIT = 6,         /* mixed: batch initialisation */
  RB_K_GEMM_PRES = 7,    /* mixed: tcgen05 sliced pressure right-hand side (-> FP64) */
  RB_K_SYSTEM = 8,       /* mixed: Newton system assembly [J | -R] and residual norms */
  RB_K_PREP = 9,         /* mixed: per-query theta, f(mu), A(mu) at the start of a solve */
  RB_K_RECONSTRUCT = 10, /* pressure reconstruction p = P_hat u (either precision) */
  RB_K_NEWTON_SMALL = 11, /* mixed, n_max <= 32: the whole Newton solve, one CTA per query */
  RB_K_OFFLINE_EIG = 12,  /* offline: covariance Gram product and Jacobi eigensolver */
  RB_K_OFFLINE_TENSOR = 13, /* offline: the tensor's triple contraction over the points */
  RB_K_COUNT = 14
};
int rb_profile(rb_ctx *ctx, int enable);
int rb_profile_read(rb_ctx *ctx, int kernel, double *total_ms, long long *launches);
/* Tensor-core work issued while profiling was enabled by the kernels of one kind
 * (RB_K_GEMM_JAC, RB_K_GEMM_RES, RB_K_GEMM_PRES): the multiply-add FLOPs (2 M N K) of every
 * tcgen05.mma the launches executed, padding tiles and every digit or split product included,
 * counted on the device. This is the work the tensor pipe did, as against the method's own
 * contraction count; 0 for the other kinds. Synchronises the device. *flops: host pointer. */
int rb_profile_issued(rb_ctx *ctx, int kernel, double *flops);

/* ---- autotuner (no counterpart in the paper) -----------------------------------------------
 * With cfg.autotune, the first mixed-precision solve of each size bucket and batch-size class
 * (ceil(log2(batch))) times the candidate launch variants on the bucket's shapes and keeps the
 * fastest: the elimination (1 = one warp per query, for n <= 80; 2 = blocked, 32-column panels;
 * 3 = blocked, 16-column panels; 4 = one CTA per query with a row per thread, 32 < n <= 128;
 * RB_ELIMINATION = 1..4 forces one where it applies), the TMA ring depths of the Jacobian and sliced GEMMs and
 * whether each GEMM runs on single CTAs or on CTA pairs (tcgen05 cta_group::2, 256-row tiles).
 * The environment variable RB_GEMM_PAIRS = 0 / 1 restricts the GEMMs to single CTAs / pairs;
 * 2 also forces the 256-column sliced tiles where the bucket allows them (n >= 32).
 * rb_tuning returns the number of tuned buckets; for bucket i < that number it fills
 * out6 = {bucket size, batch class, elimination, Jacobian GEMM stages, sliced GEMM stages,
 *         flags: bit 0 the Jacobian GEMM, bit 1 the sliced GEMM runs on CTA pairs, bit 2 the
 *         sliced GEMM uses 256-column tiles contracted chunk by chunk}
 * and ms3 = the best times (ms) of the elimination, Jacobian GEMM and sliced GEMM. Either
 * pointer may be NULL. */
int rb_tuning(rb_ctx *ctx, int i, int *out6, float *ms3);

/* ---- serving: continuous batching at Newton-iteration granularity --------------------
 * A host thread admits queries into device slots while memory allows and advances every
 * active slot by one Newton iteration per step; converged queries leave and waiting ones
 * join at the next step. Results are the same as rb_solve for the same query. */
int rb_serve_start(rb_ctx *ctx);
/* Stop the server: drain == 1 finishes admitted and queued queries first; drain == 0
 * cancels them (they complete with RB_Q_REJECTED). */
int rb_serve_stop(rb_ctx *ctx, int drain);
/* Enqueue one query (thread-safe). n = 0 means n_max. Returns RB_ERR_ARG for n out of
 * range, RB_ERR_STATE if the server is not running. */
int rb_serve_submit(rb_ctx *ctx, const double mu[2], int n, uint64_t *ticket);
/* Poll a ticket: RB_PENDING until done, then RB_OK with the result copied out
 * (u_out [n_max], p_out [m] or NULL, info or NULL); the ticket is released afterwards
 * and polling it again returns RB_ERR_ARG. */
int rb_serve_poll(rb_ctx *ctx, uint64_t ticket, double *u_out, double *p_out,
                  rb_query_info *info);
/* Latency percentiles (seconds, submit to completion) and throughput since start. */
int rb_serve_stats(rb_ctx *ctx, double *p50_s, double *p99_s, double *solves_per_s);
/* Device slots of the running server: at most this many queries are on the GPU at once;
 * later submissions wait until slots free up (admission by memory). Returns the count or an
 * error code (< 0). */
int rb_serve_slots(rb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RB_H_ */
