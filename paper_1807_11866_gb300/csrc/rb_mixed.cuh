// rb_mixed.cuh -- internal interface of the mixed-precision (tensor-core) path.
#pragma once
#include <cuda.h>

#include "rb_internal.cuh"

namespace rb {

enum { kPlain = 0, kSliced = 1 };
constexpr int kTcBN = 128;     // output tile width (columns (k, j))
constexpr int kDigitBits = 7;  // signed digits |d| <= 127 of the sliced product

struct TcGemmParams {
  int m_tiles, n_tiles;  // 128-row (query) and kTcBN-column tiles
  int kb;                // K blocks of 64
  int S;                 // digit slices (sliced mode)
  int b_pad, n_pad;      // rows between consecutive slices of X and of W
  int nq;                // valid query rows
  int nb;                // Jacobian size of the layout (columns valid: nb * nb)
  int wexp;              // exponent of the W fixed-point grid
  int ldj;               // row stride of Jc
  float *Jc;             // plain: [b_pad][n_pad] FP32
  const int *xexp;       // sliced: per-row exponent of X
  const float2 *uf;      // sliced: u_b[j] as (hi, lo) floats, [b_pad][nb]
  double *Rc;            // sliced: [b_pad][nb], accumulated with atomics
  int *err;              // device error word (bounded waits)
};

cudaError_t launch_tc_gemm(int mode, const CUtensorMap &tmX, const CUtensorMap &tmW,
                           const TcGemmParams &p, int sms, cudaStream_t st);

}  // namespace rb
