// rb_small.cuh -- the single-launch Newton solve of small systems (internal).
#pragma once
#include "rb_internal.cuh"

namespace rb {

constexpr int kSmallMaxN = 32;  // one warp eliminates the n x n system (a row per lane)

struct SmallParams {
  DevOps o;
  const double *mu;     // [nq][2], or nullptr when theta is given
  const double *theta;  // [nq][n_theta], or nullptr
  const int *nsz;       // [nq] sizes, or nullptr (n_max)
  int nq, nb, max_iter; // nb: the launch's size (n_max of the layouts below), <= kSmallMaxN
  double tol_upd, tol_res;
  const float2 *Dt2;    // [q_c][nb(l)][nb(k)][nb(j)] D~ as double-float
  const float2 *A2;     // [q_a][nb][nb] A_q as double-float
  double *u;            // [nq][n_max] out
  rb_query_info *info;  // [nq] out, or nullptr
};

size_t small_smem_bytes(const DevOps &o, int nb);
cudaError_t launch_newton_small(const SmallParams &p, int sms, cudaStream_t st);

}  // namespace rb
