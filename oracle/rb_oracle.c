/*
 * rb_oracle.c -- plain, slow, obviously correct FP64 CPU restatement of the online stage of
 * the velocity-only reduced-basis method for steady Navier-Stokes flow.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, calls or includes this
 * file; only the test suite, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * What it follows, step by step:
 *   theta      parameter functions of the affine split (Sec. 2.4, Eqs. split-a..split-d1) in
 *              the synthetic trigonometric family: trig_q(a) = cos(q a) for even q and
 *              sin(q a) for odd q, a = alpha * pi / 180; theta^a_q = trig_q / Re,
 *              theta^c_q = theta^f_q = theta^b_q = trig_q.
 *   assembly   A(mu) = sum_q theta^a_q A_q, f(mu) = sum_q theta^f_q f_q (Sec. 3.5, reduced
 *              affine matrices assembled online by weighted sums).
 *   residual   velocity-only momentum equation (Sec. 2.2, Eq. velonly) in the reduced basis
 *              with the third-order tensor of Sec. 3.6 (Eq. tensor):
 *              R[k] = sum_j A[k][j] u_j + sum_q theta^c_q sum_{j,l} C^q[j][l][k] u_j u_l - f[k]
 *              as a plain triple loop.
 *   Jacobian   Sec. 3.6: J[k][j] = A[k][j] + sum_q theta^c_q sum_l (C^q[l][j][k] + C^q[j][l][k]) u_l,
 *              both index orders written out (not pre-summed).
 *   solve      textbook Gaussian elimination with partial pivoting, pivot = first row of
 *              largest magnitude in the column, then back substitution.
 *   Newton     Sec. 6: iterate u <- u + delta, J delta = -R, from u = 0, stopping when the
 *              update is <= tol_upd in the H1 seminorm, which is the Euclidean norm of the
 *              coefficient vector because the POD basis is orthonormal (Sec. 3.2-3.3);
 *              additionally ||R(u)|| <= tol_res * max(1, ||f(mu)||).
 *   pressure   a posteriori recovery (Sec. 2.2, Eq. sup-vvar; Sec. 4.1, Eq. blocksolve-2):
 *              B(mu) p = fs(mu) - As(mu) u - Cs_mu(u, u), B(mu) = sum_q theta^b_q B_q,
 *              solved by the same elimination. Convection is included (Eq. sup-vvar).
 *   theta (polynomial family) monomials phi^q of the rotation angle from the truncated
 *              rotation series (Sec. 5, Eq. rotsum), theta^a_q = phi^q / Re.
 *   reconstruction  pressure from the velocity coefficients with the pressure data attached
 *              to every velocity basis function of a combined basis (Sec. 4.2):
 *              p = sum_j u_j p^_j, column j of P_hat holding p^_j.
 *
 * Nested truncation: a query of size n <= n_max uses the leading n x n (x n) blocks of every
 * operator, with the full leading dimensions of the stored arrays as strides.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_Q_OK 0
#define ORACLE_Q_NOT_CONVERGED 1
#define ORACLE_Q_SINGULAR 2
#define ORACLE_Q_NONFINITE 3

typedef struct {
  int n_max, m, q_a, q_c, q_f, q_b;
  int c_is_f32;          /* 1: C and Cs stored as float (exact values), 0: double */
  const double *A;       /* [q_a][n_max][n_max] */
  const void *C;         /* [q_c][n_max][n_max][n_max], index [j][l][k] */
  const double *f;       /* [q_f][n_max] */
  const double *B;       /* [q_b][m][m] or NULL */
  const double *As;      /* [q_a][m][n_max] or NULL */
  const void *Cs;        /* [q_c][n_max][n_max][m] or NULL, index [j][l][k'] */
  const double *fs;      /* [q_f][m] or NULL */
  int theta_family;      /* 0: trigonometric family, 2: polynomial family (below) */
} oracle_ops;

typedef struct {
  int status, iters;
  double res_norm, upd_norm;
} oracle_info;

static double c_at(const oracle_ops *o, int q, int j, int l, int k) {
  size_t nm = (size_t)o->n_max;
  size_t idx = (((size_t)q * nm + (size_t)j) * nm + (size_t)l) * nm + (size_t)k;
  return o->c_is_f32 ? (double)((const float *)o->C)[idx] : ((const double *)o->C)[idx];
}

static double cs_at(const oracle_ops *o, int q, int j, int l, int k) {
  size_t nm = (size_t)o->n_max, m = (size_t)o->m;
  size_t idx = (((size_t)q * nm + (size_t)j) * nm + (size_t)l) * m + (size_t)k;
  return o->c_is_f32 ? (double)((const float *)o->Cs)[idx] : ((const double *)o->Cs)[idx];
}

/* trig_q(a): cos(q a) for even q, sin(q a) for odd q (trig_0 = 1). */
static double trig(int q, double a) {
  return (q % 2 == 0) ? cos((double)q * a) : sin((double)q * a);
}

/* Polynomial family: the truncated rotation series R(a) = sum_i phi^i R_i (Sec. 5, Eq. rotsum)
   makes every pulled-back form affine in the monomials phi^i of the rotation angle
   phi = alpha * pi / 180 (the forms a, b, c of Sec. 5.2 expand in phi^(i+j), phi^(i+j+1),
   phi^(i+j+2)); the viscous form carries 1/Re (u_inf = 1). Term q is phi^q. */
static double mono(int q, double phi) {
  double v = 1.0;
  for (int i = 0; i < q; ++i) v *= phi;
  return v;
}

/* theta laid out as [theta^a (q_a) | theta^c (q_c) | theta^f (q_f) | theta^b (q_b)]. */
void oracle_theta(const oracle_ops *o, double alpha_deg, double re, double *theta) {
  const double pi = 3.14159265358979323846;
  double a = alpha_deg * pi / 180.0;
  int p = 0;
  if (o->theta_family == 2) {
    for (int q = 0; q < o->q_a; ++q) theta[p++] = mono(q, a) / re;
    for (int q = 0; q < o->q_c; ++q) theta[p++] = mono(q, a);
    for (int q = 0; q < o->q_f; ++q) theta[p++] = mono(q, a);
    for (int q = 0; q < o->q_b; ++q) theta[p++] = mono(q, a);
    return;
  }
  for (int q = 0; q < o->q_a; ++q) theta[p++] = trig(q, a) / re;
  for (int q = 0; q < o->q_c; ++q) theta[p++] = trig(q, a);
  for (int q = 0; q < o->q_f; ++q) theta[p++] = trig(q, a);
  for (int q = 0; q < o->q_b; ++q) theta[p++] = trig(q, a);
}

/* A(mu) (n x n, dense, row = test k) and f(mu) (n). */
void oracle_assemble(const oracle_ops *o, int n, const double *theta, double *A, double *f) {
  const double *ta = theta, *tf = theta + o->q_a + o->q_c;
  size_t nm = (size_t)o->n_max;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int q = 0; q < o->q_a; ++q) s += ta[q] * o->A[((size_t)q * nm + k) * nm + j];
      A[(size_t)k * n + j] = s;
    }
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int q = 0; q < o->q_f; ++q) s += tf[q] * o->f[(size_t)q * nm + k];
    f[k] = s;
  }
}

/* Convection term Cmu(u, u)[k] = sum_q theta^c_q sum_{j,l} C^q[j][l][k] u_j u_l. */
void oracle_convection(const oracle_ops *o, int n, const double *theta, const double *u,
                       double *out) {
  const double *tc = theta + o->q_a;
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int q = 0; q < o->q_c; ++q) {
      double sq = 0.0;
      for (int j = 0; j < n; ++j)
        for (int l = 0; l < n; ++l) sq += c_at(o, q, j, l, k) * u[j] * u[l];
      s += tc[q] * sq;
    }
    out[k] = s;
  }
}

/* R(u; mu) = A(mu) u + Cmu(u, u) - f(mu). */
void oracle_residual(const oracle_ops *o, int n, const double *theta, const double *u,
                     double *R) {
  double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
  double *f = (double *)malloc(sizeof(double) * (size_t)n);
  double *cv = (double *)malloc(sizeof(double) * (size_t)n);
  oracle_assemble(o, n, theta, A, f);
  oracle_convection(o, n, theta, u, cv);
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += A[(size_t)k * n + j] * u[j];
    R[k] = s + cv[k] - f[k];
  }
  free(A); free(f); free(cv);
}

/* J[k][j] = A(mu)[k][j] + sum_q theta^c_q sum_l (C^q[l][j][k] + C^q[j][l][k]) u_l. */
void oracle_jacobian(const oracle_ops *o, int n, const double *theta, const double *u,
                     double *J) {
  const double *tc = theta + o->q_a;
  double *f = (double *)malloc(sizeof(double) * (size_t)n);
  oracle_assemble(o, n, theta, J, f);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int q = 0; q < o->q_c; ++q) {
        double sq = 0.0;
        for (int l = 0; l < n; ++l)
          sq += (c_at(o, q, l, j, k) + c_at(o, q, j, l, k)) * u[l];
        s += tc[q] * sq;
      }
      J[(size_t)k * n + j] += s;
    }
  free(f);
}

/* Gaussian elimination with partial pivoting on M (n x n, row-major, overwritten) and the
 * right-hand side b (overwritten by the solution). Pivot: first row of largest |.|.
 * Returns 0, or 1 when a pivot is exactly zero or not finite. */
int oracle_gepp_solve(int n, double *M, double *b) {
  for (int p = 0; p < n; ++p) {
    int r = p;
    double best = fabs(M[(size_t)p * n + p]);
    for (int i = p + 1; i < n; ++i) {
      double v = fabs(M[(size_t)i * n + p]);
      if (v > best) { best = v; r = i; }
    }
    if (!(best > 0.0) || !isfinite(best)) return 1;
    if (r != p) {
      for (int j = 0; j < n; ++j) {
        double t = M[(size_t)p * n + j];
        M[(size_t)p * n + j] = M[(size_t)r * n + j];
        M[(size_t)r * n + j] = t;
      }
      double t = b[p]; b[p] = b[r]; b[r] = t;
    }
    double piv = M[(size_t)p * n + p];
    for (int i = p + 1; i < n; ++i) {
      double lip = M[(size_t)i * n + p] / piv;
      M[(size_t)i * n + p] = lip;
      for (int j = p + 1; j < n; ++j) M[(size_t)i * n + j] -= lip * M[(size_t)p * n + j];
      b[i] -= lip * b[p];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= M[(size_t)i * n + j] * b[j];
    b[i] = s / M[(size_t)i * n + i];
  }
  return 0;
}

static double norm2(int n, const double *v) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += v[i] * v[i];
  return sqrt(s);
}

static int all_finite(int n, const double *v) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(v[i])) return 0;
  return 1;
}

/* Newton from u = 0 (Sec. 3.6 Jacobian, Sec. 6 stopping rule). u has n entries.
 * Iteration it: R = R(u), J = J(u), solve J delta = -R, u += delta; converged when
 * ||delta|| <= tol_upd and ||R|| <= tol_res * max(1, ||f(mu)||). trace_res / trace_upd
 * (max_iter entries, may be NULL) receive ||R|| and ||delta|| per iteration. */
void oracle_newton_theta(const oracle_ops *o, int n, const double *theta, double tol_upd,
                         double tol_res, int max_iter, double *u, oracle_info *info,
                         double *trace_res, double *trace_upd) {
  double *R = (double *)malloc(sizeof(double) * (size_t)n);
  double *J = (double *)malloc(sizeof(double) * (size_t)n * n);
  double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
  double *f = (double *)malloc(sizeof(double) * (size_t)n);
  oracle_assemble(o, n, theta, A, f);
  double fscale = norm2(n, f);
  if (fscale < 1.0) fscale = 1.0;
  for (int i = 0; i < n; ++i) u[i] = 0.0;
  info->status = ORACLE_Q_NOT_CONVERGED;
  info->iters = 0;
  info->res_norm = info->upd_norm = 0.0;
  for (int it = 0; it < max_iter; ++it) {
    oracle_residual(o, n, theta, u, R);
    oracle_jacobian(o, n, theta, u, J);
    double rn = norm2(n, R);
    for (int i = 0; i < n; ++i) R[i] = -R[i];
    info->iters = it + 1;
    info->res_norm = rn;
    if (!all_finite(n, R)) { info->status = ORACLE_Q_NONFINITE; break; }
    if (oracle_gepp_solve(n, J, R)) { info->status = ORACLE_Q_SINGULAR; break; }
    if (!all_finite(n, R)) { info->status = ORACLE_Q_NONFINITE; break; }
    for (int i = 0; i < n; ++i) u[i] += R[i];
    double dn = norm2(n, R);
    info->upd_norm = dn;
    if (trace_res) trace_res[it] = rn;
    if (trace_upd) trace_upd[it] = dn;
    if (dn <= tol_upd && rn <= tol_res * fscale) { info->status = ORACLE_Q_OK; break; }
  }
  free(R); free(J); free(A); free(f);
}

/* Pressure recovery: B(mu) p = fs(mu) - As(mu) u - Cs_mu(u, u). Returns 0 or 1 (singular). */
int oracle_pressure_theta(const oracle_ops *o, int n, const double *theta, const double *u,
                          double *p) {
  int m = o->m;
  const double *ta = theta, *tc = theta + o->q_a, *tf = theta + o->q_a + o->q_c;
  const double *tb = theta + o->q_a + o->q_c + o->q_f;
  size_t nm = (size_t)o->n_max;
  double *Bm = (double *)malloc(sizeof(double) * (size_t)m * m);
  for (int k = 0; k < m; ++k) {
    double s = 0.0;
    for (int q = 0; q < o->q_f; ++q) s += tf[q] * o->fs[(size_t)q * m + k];
    for (int q = 0; q < o->q_a; ++q) {
      double sq = 0.0;
      for (int j = 0; j < n; ++j) sq += o->As[((size_t)q * m + k) * nm + j] * u[j];
      s -= ta[q] * sq;
    }
    for (int q = 0; q < o->q_c; ++q) {
      double sq = 0.0;
      for (int j = 0; j < n; ++j)
        for (int l = 0; l < n; ++l) sq += cs_at(o, q, j, l, k) * u[j] * u[l];
      s -= tc[q] * sq;
    }
    p[k] = s;
    for (int i = 0; i < m; ++i) {
      double b = 0.0;
      for (int q = 0; q < o->q_b; ++q) b += tb[q] * o->B[((size_t)q * m + k) * m + i];
      Bm[(size_t)k * m + i] = b;
    }
  }
  int rc = oracle_gepp_solve(m, Bm, p);
  free(Bm);
  return rc;
}

static void solve_one(const oracle_ops *o, int n, const double *theta, double tol_upd,
                      double tol_res, int max_iter, double *u_row, double *p_row,
                      oracle_info *inf) {
  oracle_newton_theta(o, n, theta, tol_upd, tol_res, max_iter, u_row, inf, NULL, NULL);
  if (p_row && o->m > 0 && o->B) {
    if (inf->status == ORACLE_Q_OK) {
      if (oracle_pressure_theta(o, n, theta, u_row, p_row)) inf->status = ORACLE_Q_SINGULAR;
    } else {
      for (int i = 0; i < o->m; ++i) p_row[i] = 0.0;
    }
  }
}

/* Batch of queries mu[b] = (alpha_deg, Re), sizes nsz[b] (NULL: n_max). u_out is
 * [nq][n_max] (entries beyond n set to 0), p_out [nq][m] or NULL, info [nq].
 * OpenMP over queries with nthreads threads (<= 0: runtime default). */
void oracle_solve_batch(const oracle_ops *o, int nq, const double *mu, const int *nsz,
                        double tol_upd, double tol_res, int max_iter, double *u_out,
                        double *p_out, oracle_info *info, int nthreads) {
  int nt = o->q_a + o->q_c + o->q_f + o->q_b;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < nq; ++b) {
    double theta[512];
    int n = nsz ? nsz[b] : o->n_max;
    double *u_row = u_out + (size_t)b * o->n_max;
    for (int i = 0; i < o->n_max; ++i) u_row[i] = 0.0;
    if (nt > 512) { info[b].status = ORACLE_Q_NONFINITE; continue; }
    oracle_theta(o, mu[2 * b], mu[2 * b + 1], theta);
    solve_one(o, n, theta, tol_upd, tol_res, max_iter, u_row,
              p_out ? p_out + (size_t)b * o->m : NULL, &info[b]);
  }
}

/* Same with caller-supplied parameter functions theta[b][q_a + q_c + q_f + q_b]. */
void oracle_solve_theta_batch(const oracle_ops *o, int nq, const double *theta,
                              const int *nsz, double tol_upd, double tol_res, int max_iter,
                              double *u_out, double *p_out, oracle_info *info, int nthreads) {
  int nt = o->q_a + o->q_c + o->q_f + o->q_b;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < nq; ++b) {
    int n = nsz ? nsz[b] : o->n_max;
    double *u_row = u_out + (size_t)b * o->n_max;
    for (int i = 0; i < o->n_max; ++i) u_row[i] = 0.0;
    solve_one(o, n, theta + (size_t)b * nt, tol_upd, tol_res, max_iter, u_row,
              p_out ? p_out + (size_t)b * o->m : NULL, &info[b]);
  }
}

/* Pressure reconstruction (Sec. 4.2): p[k] = sum_{j < n} P_hat[k][j] u[j] for P_hat [m_r][n_max]
   (column j = the pressure data of velocity basis function j), j ascending. */
void oracle_reconstruct(const double *P_hat, int m_r, int n_max, int n, const double *u,
                        double *p) {
  for (int k = 0; k < m_r; ++k) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += P_hat[(size_t)k * n_max + j] * u[j];
    p[k] = s;
  }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
