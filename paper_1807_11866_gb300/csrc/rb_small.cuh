// rb_small.cuh -- the single-launch Newton solve of small systems (internal).
#pragma once
#include "rb_internal.cuh"

namespace rb {

constexpr int kSmallMaxN = 32;  // one warp eliminates the n x n system (a row per lane)
constexpr int kSmallStages = 3;  // shared-memory ring of the D~ stream (bulk copies)

// Rows (q, l) of D~ per bulk copy for launch size nb: an even count (16-byte aligned copies for
// any nb), about 20 KB per copy; the D~ copy is padded to a whole number of such chunks.
__host__ __device__ inline int small_chunk_rows(int nb) {
  const int rb = 8 * nb * nb;
  const int c = (20480 / rb) & ~1;
  return c < 2 ? 2 : c;
}
__host__ __device__ inline int small_dt_rows(int q_c, int nb) {
  const int ch = small_chunk_rows(nb);
  return (q_c * nb + ch - 1) / ch * ch;
}

struct SmallParams {
  DevOps o;
  const double *mu;     // [nq][2], or nullptr when theta is given
  const double *theta;  // [nq][n_theta], or nullptr
  const int *nsz;       // [nq] sizes, or nullptr (n_max)
  int nq, nb, max_iter; // nb: the launch's size (n_max of the layouts below), <= kSmallMaxN
  double tol_upd, tol_res;
  const float2 *Dt2;    // [small_dt_rows][nb(k)][nb(j)]: rows (q, l) of D~ as double-float,
                        // zero rows past q_c nb
  const float2 *A2;     // [q_a][nb][nb] A_q as double-float
  double *u;            // [nq][n_max] out
  rb_query_info *info;  // [nq] out, or nullptr
  int *err;             // sticky error word: a bounded wait of the D~ stream gave up
};

size_t small_smem_bytes(const DevOps &o, int nb);
cudaError_t launch_newton_small(const SmallParams &p, int sms, cudaStream_t st);

}  // namespace rb
