// rb_kernels.cuh -- launch parameters and host launchers of the librb kernels (internal).
#pragma once
#include "rb_internal.cuh"

namespace rb {

struct NewtonParams {
  DevOps o;
  const double *mu;     // [nq][2] or nullptr when theta is given
  const double *theta;  // [nq][n_theta] or nullptr
  const int *nsz;       // [nq] or nullptr (n_max)
  int nq, max_iter, grid, j_in_smem;
  double tol_upd, tol_res;
  double *u_out;        // [nq][n_max]
  rb_query_info *info;  // [nq] or nullptr
  double *jscratch;     // [grid][n_max^2] when the Jacobian does not fit in shared memory
  // escalation of the mixed path: only the queries it handed over (status kQEscalate) are
  // solved (again from u = 0: the exact Newton of the FP64 path), and only if *run_if != 0
  // (nullptr: a plain FP64 solve); their iteration counts add to the mixed ones
  const int *run_if;
  int resume;
};

// internal per-query status of the mixed path: its chord steps stalled even with a fresh
// Jacobian, so the FP64 Newton solves the query (never returned)
constexpr int kQEscalate = 16;

struct PressureParams {
  DevOps o;
  const double *mu, *theta;
  const int *nsz;
  int nq;
  const double *u;      // [nq][n_max]
  double *p_out;        // [nq][m]
  rb_query_info *info;  // [nq] or nullptr
};

struct EvalParams {
  DevOps o;
  const double *mu;
  int nq, n;
  const double *u;      // [nq][n]
  double *R_out;        // [nq][n]
  double *J_out;        // [nq][n][n]
};

size_t fp64_smem_bytes(const DevOps &o, bool j_in_smem);
size_t pressure_smem_bytes(const DevOps &o);

cudaError_t launch_newton_fp64(const NewtonParams &p, int sms, cudaStream_t st);
cudaError_t launch_pressure(const PressureParams &p, int sms, cudaStream_t st);
cudaError_t launch_eval_fp64(const EvalParams &p, int sms, cudaStream_t st);
cudaError_t launch_gepp_fp64(double *M, double *rhs, int n, int batch, int *status, int sms,
                             cudaStream_t st);
cudaError_t launch_build_dt(const void *C, int dtype, double *Dt, int nm, int qc, int sms,
                            cudaStream_t st);
cudaError_t launch_convert(const void *src, int dtype, double *dst, size_t count, int sms,
                           cudaStream_t st);

}  // namespace rb
