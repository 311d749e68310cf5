// rb_mixed.cuh -- internal interface of the mixed-precision (tensor-core) path.
#pragma once
#include <cuda.h>

#include "rb_internal.cuh"

namespace rb {

// kSliced: per-column double-float sums in TMEM, contracted with u at the end of a tile;
// kSlicedWide: 256-column tiles, every chunk contracted with u at once (needs nj >= 32).
enum { kPlain = 0, kSliced = 1, kSlicedWide = 2 };
constexpr int kTcBN = 128;     // output tile width (columns (k, j))
constexpr int kDigitBits = 7;  // base-128 balanced digits (|d| <= 64) of the sliced product

// One tcgen05 GEMM launch. Columns c = k * nj + j (k < nk, j < nj) of W; rows b = queries.
// K is split in up to two segments with their own fixed-point grids (sliced mode):
// segment 0 = convection (q, l), segment 1 = linear affine term (q).
struct TcGemmParams {
  int m_tiles, n_tiles;  // 128-row (query) and kTcBN-column tiles
  int group_m;           // row tiles per group of the tile order (set by launch_tc_gemm)
  int lsplit, full_tiles;  // sliced: tiles past full_tiles run as lsplit level parts each
                           // (set by launch_tc_gemm)
  int kb[2];             // K blocks of 64 per segment (kb[1] = 0: no second segment)
  int S[2];              // digit slices per segment (sliced mode)
  int nsplit;            // plain mode: 1 (BF16) or 3 (split BF16: hi*hi + hi*lo + lo*hi)
  int b_pad, n_pad;      // rows between consecutive slices of X and of W
  int nq;                // valid query rows
  int nk, nj;            // output rows per query and contraction length (columns = nk * nj)
  int wexp[2];           // exponent of the W fixed-point grid per segment
  int ldj;               // row stride of Jc
  float *Jc;             // plain: [b_pad][n_pad] FP32
  const int *xexp;       // sliced: per-row exponent of X, [2][b_pad]
  const float2 *ufT;     // sliced: u_b[j] as (hi, lo) floats, transposed [nj][b_pad]
  double *out;           // sliced: [b_pad][nk], accumulated with atomics
  int *err;              // device error word (bounded waits)
  const int *lmax;       // sliced, one segment: if set, the highest digit level L = i + j of
                         // the launch, read on the device (levels 2..*lmax, at most S[0] + 1)
  const int *run_if;     // if set, the launch does nothing unless *run_if != 0 (read on the
                         // device: a Jacobian that only some chord steps ask for)
  unsigned tx_extra;     // single-CTA variants, tests of the bounded waits only: bytes the first
                         // stage of CTA 0 expects beyond what its copies bring (0 normally), so
                         // that its consumer's wait runs out and raises the error word
  unsigned long long *issued;  // if set (profiling): += the FLOPs (2 M N K) of the MMAs issued
};

cudaError_t launch_tc_gemm(int mode, const CUtensorMap &tmX, const CUtensorMap &tmW,
                           const TcGemmParams &p, int sms, cudaStream_t st, int stages = 0,
                           bool pair = false);

}  // namespace rb
