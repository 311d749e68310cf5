// rb_mixed.cu -- mixed-precision batched Newton (inexact Newton, Sec. 3.6 Jacobian on tensor cores).
//
// Once per query at its start: theta(mu_b), f(mu_b) (k_prep_theta) and A(mu_b), B(mu_b) in
// double-float (k_affine_sum). Per Newton iteration, for every active query b of the batch:
//   1. k_build_x: X_b = theta^c(mu_b) (x) u_b as split BF16 (hi, lo) for the Jacobian GEMM; the
//      base-128 digit slices of theta^c (x) u_b / 2 for the sliced GEMM; u_b as (hi, lo) floats
//      (transposed); R^c_b = 0.
//   2. k_tc_gemm<kPlain>:  J^c = X W^T on tcgen05 (split BF16, FP32 accumulate) -> Jc (FP32).
//   3. k_tc_gemm<kSliced>: R^c_b[k] = sum_j u_b[j] (X'_b W^T)[(k,j)] = C_mu(u_b, u_b)[k] from
//      exact digit products, contracted in double-float -> FP64.
//   4. k_newton_system: [J | -R] with J = fl32(A(mu)) + J^c and R = A(mu) u (double-float)
//      + C_mu(u, u) - f(mu); residual norms.
//   5. k_lu_mixed_warp (warp per query, n <= 80), k_lu_cta (CTA per query, row per thread,
//      n <= 128) or k_lu_blocked (CTA per query, blocked right-looking elimination), as the
//      autotuner picks: FP32 GEPP on [J | -R]; u += delta in FP64; stopping rule (Sec. 6) on the
//      FP64 norms. Iteration 2 keeps its factors; from iteration 3 on (chord steps) steps 1-2
//      skip the Jacobian, step 4 assembles only -R and step 5 solves with the kept factors.
// The Jacobian is inexact (BF16 convection part, FP32 elimination); the residual and the test
// are FP64-accurate, so the iteration converges to the FP64 solution at the linear rate
// ||J~^-1 (J~ - J)||. After the last iteration the pressure right-hand side
// fs(mu) - As(mu) u - Cs_mu(u, u) (Eq. sup-vvar) takes Cs_mu(u, u) from the same sliced GEMM with
// W = 2 Cs and As(mu) u in double-float (k_as_u); B(mu) p = r is solved by FP32 LU with
// double-float iterative refinement (Eq. blocksolve-2). The whole solve is one CUDA graph with a
// device-side loop over the FP64-residual iterations.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "rb_ctx.h"
#include "rb_mixed.cuh"
#include "rb_small.cuh"

namespace rb {

struct SlicedW {  // one sliced weight operand [S][Npad][Kpad]
  __nv_bfloat16 *d = nullptr;
  int Npad = 0, nk = 0, wexp[2] = {0, 0};
  CUtensorMap tm, tm64;  // 128-row boxes (single-CTA tiles), 64-row boxes (CTA pairs)
};

// Mixed-path state of one size bucket: operator layouts truncated to nb (the reduced bases are
// nested, so a size-n query is the leading n-block of any bucket nb >= n) and the batch
// scratch of the queries solved at that size. The root bucket (nb = n_max) also owns what all
// buckets share: the device words, the gather scratch of a bucketed batch and the solve graph.
struct MixedState {
  MixedState *root = nullptr;   // the n_max bucket (itself for the root)
  // operator layouts for the Jacobian size nb
  int nb = 0, Kpad0 = 0, kb0 = 0, kb1 = 0, Kpad = 0, Npad = 0, S0 = 0, S1 = 0, Smax = 0;
  __nv_bfloat16 *Wj = nullptr;  // [2][Npad][Kpad0] split BF16 D~ (hi, lo)
  CUtensorMap tmWj;
  SlicedW WR, WP;               // residual [D~ | A], pressure [2 Cs | As]
  float2 *A2 = nullptr;         // [q_a][nb][nb] A_q as double-float (hi, lo)
  float2 *As2 = nullptr;        // [q_a][m][nb] As_q as double-float
  float2 *B2 = nullptr;         // [q_b][m][m] B_q as double-float
  float2 *Dt2 = nullptr;        // root, n_max <= kSmallMaxN: D~ as double-float [q_c][l][k][j]
  // batch scratch
  int bcap = 0;
  __nv_bfloat16 *Xj = nullptr, *Xd = nullptr;  // Xj: [3][bcap][Kpad0] (hi, hi, lo)
  int *xexp = nullptr;          // [2][bcap]
  float2 *ufT = nullptr;        // [nb][bcap]
  float2 *u2 = nullptr;         // [bcap][nb] u as double-float (hi, lo), for the assembly
  float *Jc = nullptr;          // [bcap][Npad]
  double *Rc = nullptr;         // [bcap][nb]
  double *Rp = nullptr;         // [bcap][m]
  double *Th = nullptr;         // [bcap][n_theta] theta rows
  double *Fm = nullptr;         // [bcap][nb] f(mu)
  float2 *Amu = nullptr;        // [bcap][nb * nb] A(mu) as double-float
  double *Asu = nullptr;        // [bcap][m] As(mu) u
  float2 *Bmu = nullptr;        // [bcap][m][m] B(mu) as double-float
  float *Jaug = nullptr;        // [bcap][nb][aug_ld(nb)] augmented Newton matrices (or factors)
  int *Piv = nullptr;           // [bcap][nb] pivot rows of the factors kept for chord steps
  double *dU = nullptr;         // [bcap][nb] each query's last update (chord steps' residual)
  int *refresh = nullptr;       // raised by a chord step that contracts too slowly
  double2 *Rn = nullptr;        // [bcap] (unused, max(1, ||f(mu)||)) of the queries
  double *Rg = nullptr;         // [bcap][(nb + 7) / 8] row-group sums of R^2 (in Rn's block)
  CUtensorMap tmXj, tmXd;
  // autotuned launch variants of this bucket (0 = not tuned: defaults), per batch-size class
  struct Tune {
    int klass = -1;      // ceil(log2(batch)) the choice was made for
    int lu = 0;          // 1 warp per query, 2 blocked with 32-column panels, 3 blocked 16
    int st_plain = 0, st_sliced = 0;  // TMA ring depths of the two GEMMs
    int pair_plain = 0;   // 1: CTA pairs (tcgen05 cta_group::2)
    int pair_sliced = 0;  // 0 single CTAs, 1 CTA pairs, 2 CTA pairs on 256-column tiles
    float ms[4] = {0, 0, 0, 0};       // best times: elimination, plain GEMM, sliced GEMM
  } tune;
  // shared, owned by the root
  int *dev_words = nullptr;     // [0] active count, [1] error word, [2] iterations,
                                // [5] sticky error word of graph solves, [8..] scratch
  int *h_words = nullptr;       // pinned mirror; [12..15] copy of words [4..7] after a graph solve
  // asynchronous graph solves: the last one's completion event and whether its words are unread
  cudaEvent_t done_ev = nullptr;
  bool pending = false;
  cudaStream_t pending_st = nullptr;
  int *h_perm = nullptr;        // pinned bucket order of the last solve (capacity h_perm_cap)
  int h_perm_cap = 0;
  cudaEvent_t perm_ev = nullptr;  // its upload has completed
  rb_query_info *info_own = nullptr;
  int info_cap = 0;
  std::map<int, MixedState *> buckets;  // nb < n_max
  // gather scratch of a bucketed batch (query order sorted by bucket)
  int gcap = 0;
  int serve_cap = 0;  // root only: slots of the running server (0: not serving)
  int *perm = nullptr, *n_g = nullptr;
  double *mu_g = nullptr, *theta_g = nullptr, *u_g = nullptr, *p_g = nullptr;
  rb_query_info *info_g = nullptr;
  // whole-solve CUDA graph (prologue, two ladder iterations, a device-side while loop over
  // FP64-residual iterations, pressure), keyed by the solve's buffers, buckets and scratch epoch
  uint64_t epoch = 1;
  cudaStream_t cap[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec = nullptr;
  struct {
    const double *mu, *theta, *p; const int *n; double *u; rb_query_info *info; int nq;
    uint64_t epoch;
    std::vector<int> parts;
  } gkey{};
};

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2D BF16 tensor [rows][cols] (cols contiguous), box 64 x box_rows, 128-byte swizzle.
static bool make_map(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// ---------------------------------------------------------------------------------------
// Balanced base-128 digits of the fixed-point magnitude F < 2^(7S - 1): d_S .. d_2 in [-64, 63]
// (a digit of 64 or more borrows from the next one), d_1 in [0, 64]; every |d| <= 64, so the
// product of two digits is at most 2^12 and 4096 of them add exactly in FP32. Written with the
// sign of v to slices 0 .. S-1.
__device__ __forceinline__ void balanced_digits(long long F, float sg, int S, __nv_bfloat16 *out,
                                                size_t slice_stride) {
  for (int i = S; i >= 2; --i) {
    int r = (int)(F & 127);
    F >>= kDigitBits;
    if (r >= 64) {
      r -= 128;
      F += 1;
    }
    out[(size_t)(i - 1) * slice_stride] = __float2bfloat16_rn(sg * (float)r);
  }
  out[0] = __float2bfloat16_rn(sg * (float)F);
}

// digits of v on the grid 2^(e - 7 i), i = 1..S, with one binade of headroom (|v| < 2^(e-1)),
// the magnitude truncated toward 0 on the finest grid
__device__ __forceinline__ void digits7(double v, double scale /* 2^(7S - e) */, int S,
                                        __nv_bfloat16 *out, size_t slice_stride) {
  const long long F = __double2ll_rz(fabs(v) * scale);
  balanced_digits(F, v < 0 ? -1.f : 1.f, S, out, slice_stride);
}

// Same digits from the FP64 bit pattern with integer operations only (GB300's FP64 pipe is
// narrow and its conversions slow). e is the grid exponent.
__device__ __forceinline__ long long fixed_bits(double v, int e, int S) {
  const unsigned long long mag = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  const int E = (int)(mag >> 52);
  if (E == 0) return 0;  // zero or subnormal: below every grid used here
  const unsigned long long M = (mag & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int sh = 1075 + e - kDigitBits * S - E;  // |v| 2^(7S - e) = M 2^-sh
  if (sh >= 64) return 0;
  return (long long)(sh >= 0 ? (M >> sh) : (M << (-sh)));
}

__device__ __forceinline__ void digits7_int(double v, int e, int S, __nv_bfloat16 *out,
                                            size_t slice_stride) {
  balanced_digits(fixed_bits(v, e, S), v < 0 ? -1.f : 1.f, S, out, slice_stride);
}

// exponent e with |v| < 2^e from the bit pattern of a nonnegative maximum (frexp convention)
__device__ __forceinline__ int exp_of_bits(unsigned long long mag) {
  return mag == 0 ? 0 : (int)(mag >> 52) - 1022;
}

__global__ void k_absmax(const double *x, size_t count, unsigned long long *out) {
  double m = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_split_f2(const double *x, float2 *y, size_t count) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const float h = (float)x[e];
    y[e] = make_float2(h, (float)(x[e] - (double)h));
  }
}

// y[q][r][c] = (hi, lo) of x[(q * src_rows + r) * ldx + c] for r < rows, c < cols: the
// double-float copy of the leading rows x cols block of q_count matrices (a bucket's
// truncation of an operator).
__global__ void k_split_trunc(const double *x, float2 *y, int q_count, int rows, int src_rows,
                              int ldx, int cols) {
  const size_t total = (size_t)q_count * rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t qr = e / cols;
    const int c = (int)(e - qr * cols);
    const size_t q = qr / rows, r = qr - q * rows;
    const double v = x[(q * src_rows + r) * ldx + c];
    const float h = (float)v;
    y[e] = make_float2(h, (float)(v - (double)h));
  }
}

// Rows of a bucketed batch in bucket order: dst[i] = src[perm[i]].
__global__ void k_gather(int nq, const int *perm, const double *mu, const double *theta,
                         int n_theta, const int *n, double *mu_g, double *theta_g, int *n_g) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
    const int s = perm[i];
    if (mu) {
      mu_g[2 * i] = mu[2 * s];
      mu_g[2 * i + 1] = mu[2 * s + 1];
    }
    if (theta)
      for (int t = 0; t < n_theta; ++t) theta_g[(size_t)i * n_theta + t] = theta[(size_t)s * n_theta + t];
    n_g[i] = n[s];
  }
}

// Serving slots into a size-bucketed batch: mu, n, u and info of slot perm[i] to row i (one
// warp per query).
__global__ void k_gather_slots(int nq, const int *perm, int nm, const double *mu, const int *n,
                               const double *u, const rb_query_info *info, double *mu_g, int *n_g,
                               double *u_g, rb_query_info *info_g) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nq; i += nw) {
    const int s = perm[i];
    for (int j = lane; j < nm; j += 32) u_g[(size_t)i * nm + j] = u[(size_t)s * nm + j];
    if (lane == 0) {
      mu_g[2 * i] = mu[2 * s];
      mu_g[2 * i + 1] = mu[2 * s + 1];
      n_g[i] = n[s];
      info_g[i] = info[s];
    }
  }
}

// Results back to the caller's order: dst[perm[i]] = src[i] (one warp per query).
__global__ void k_scatter(int nq, const int *perm, int nm, int m, const double *u_g,
                          const double *p_g, const rb_query_info *info_g, double *u, double *p,
                          rb_query_info *info) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nq; i += nw) {
    const int d = perm[i];
    for (int j = lane; j < nm; j += 32) u[(size_t)d * nm + j] = u_g[(size_t)i * nm + j];
    if (p)
      for (int j = lane; j < m; j += 32) p[(size_t)d * m + j] = p_g[(size_t)i * m + j];
    if (lane == 0) info[d] = info_g[i];
  }
}

// Sliced weight operand W[c][kappa], c = k * nb + j (k < nk, j < nb):
//   kind 0 (residual): kappa = q * nb + l < Kpad0 -> D~_q[k][j][l] (Dt [q][l][k][j]);
//                      kappa = Kpad0 + q          -> A_q[k][j]
//   kind 1 (pressure): kappa = q * nb + l         -> 2 Cs_q[j][l][k] (Cs [q][j][l][m]);
//                      kappa = Kpad0 + q          -> As_q[k][j]
// plus, for kind 0, the split BF16 copy of the convection part (Wj [2][Npad][Kpad0]).
struct BuildWParams {
  DevOps o;
  int kind, nb, nk, Kpad0, Kpad, Npad, S0, S1, wexp0, wexp1;
  __nv_bfloat16 *Wd, *Wj;
};

__global__ void k_build_w(BuildWParams p) {
  const DevOps &o = p.o;
  const size_t total = (size_t)p.Npad * p.Kpad;
  const size_t nm = (size_t)o.n_max;
  const double sc0 = ldexp(1.0, kDigitBits * p.S0 - p.wexp0);
  const double sc1 = ldexp(1.0, kDigitBits * p.S1 - p.wexp1);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int kap = (int)(e % p.Kpad);
    const int c = (int)(e / p.Kpad);
    double v = 0.0;
    const bool seg1 = kap >= p.Kpad0;
    if (c < p.nk * p.nb) {
      const int k = c / p.nb, j = c % p.nb;
      if (!seg1) {
        if (kap < o.q_c * p.nb) {
          const int q = kap / p.nb, l = kap % p.nb;
          v = p.kind == 0 ? o.Dt[(((size_t)q * nm + l) * nm + k) * nm + j]
                          : 2.0 * o.Cs[(((size_t)q * nm + j) * nm + l) * o.m + k];
        }
      } else {
        const int q = kap - p.Kpad0;
        if (q < o.q_a)
          v = p.kind == 0 ? o.A[((size_t)q * nm + k) * nm + j] : o.As[((size_t)q * o.m + k) * nm + j];
      }
    }
    if (p.Wj && !seg1) {  // split BF16 copy of the convection part: [w_hi ; w_lo]
      const float vf = (float)v;
      const __nv_bfloat16 hi = __float2bfloat16_rn(vf);
      p.Wj[(size_t)c * p.Kpad0 + kap] = hi;
      p.Wj[(size_t)p.Npad * p.Kpad0 + (size_t)c * p.Kpad0 + kap] =
          __float2bfloat16_rn(vf - __bfloat162float(hi));
    }
    digits7(v, seg1 ? sc1 : sc0, seg1 ? p.S1 : p.S0, p.Wd + e, total);
  }
}

// Start of a batch: status NOT_CONVERGED (active) or REJECTED, u = 0 (if u is given).
__global__ void k_mixed_init(int nq, int nm, const int *nsz, double *u, rb_query_info *info) {
  for (int b = blockIdx.x; b < nq; b += gridDim.x) {
    const int n = nsz ? nsz[b] : nm;
    if (u)
      for (int i = threadIdx.x; i < nm; i += blockDim.x) u[(size_t)b * nm + i] = 0.0;
    if (threadIdx.x == 0) {
      rb_query_info q = {(n >= 1 && n <= nm) ? RB_Q_NOT_CONVERGED : RB_Q_REJECTED, 0,
                         RB_PREC_MIXED, 0, 0.0, 0.0};
      info[b] = q;
    }
  }
}

struct BuildXParams {
  DevOps o;
  const double *theta;  // [nq][n_theta] per-query theta rows
  const int *nsz;
  int nq, nb, Kpad0, Kpad, S0, S1, b_pad, max_iter, mode;  // mode 0: active, 1: converged
  int digits;       // 1: also write the digit slices, exponents and u pairs (sliced GEMM)
  int split;        // 1: write the split BF16 operand of the Jacobian GEMM (mode 0)
  const double *u;  // [nq][n_max]
  const rb_query_info *info;
  __nv_bfloat16 *Xj, *Xd;
  int *xexp;        // [2][b_pad]
  float2 *ufT;      // [nb][b_pad]
  float2 *u2;       // [b_pad][nb] u as double-float (mode 0), read by the assembly
  double *out;      // [b_pad][nout], zeroed for each built query (not in increment mode)
  int nout;
  // increment mode (chord steps): the operand of C(u, u) - C(u - d, u - d) = J^c(d) (u - d / 2)
  // instead of C(u, u): X = theta^c (x) d on its own grid, the contraction vector u - d / 2,
  // the output accumulated onto the previous C(u - d, u - d); the digit level the launch needs
  // is raised into *lmax (see k_build_x)
  int incr;
  const double *dU;  // [nq][nb] the last update d of each query
  int *lmax;
};

__device__ __forceinline__ bool is_active(const rb_query_info &q, int max_iter) {
  return q.status == RB_Q_NOT_CONVERGED && q.iters < max_iter;
}

__device__ __forceinline__ int exp_of_max(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

// Balanced digits of two neighbouring elements, stored as BF16 pairs (4-byte stores).
__device__ __forceinline__ void digits_pair(double v0, double v1, int e, int S, __nv_bfloat16 *out,
                                            size_t slice_stride) {
  long long F0 = fixed_bits(v0, e, S), F1 = fixed_bits(v1, e, S);
  const float s0 = __double_as_longlong(v0) < 0 ? -1.f : 1.f;  // sign bits (no FP64 compare)
  const float s1 = __double_as_longlong(v1) < 0 ? -1.f : 1.f;
  for (int i = S; i >= 1; --i) {
    int r0 = (int)F0, r1 = (int)F1;
    if (i > 1) {
      r0 = (int)(F0 & 127);
      r1 = (int)(F1 & 127);
      F0 >>= kDigitBits;
      F1 >>= kDigitBits;
      if (r0 >= 64) { r0 -= 128; F0 += 1; }
      if (r1 >= 64) { r1 -= 128; F1 += 1; }
    }
    *reinterpret_cast<__nv_bfloat162 *>(out + (size_t)(i - 1) * slice_stride) =
        __floats2bfloat162_rn(s0 * (float)r0, s1 * (float)r1);
  }
}

// X operands of one Newton iteration, one warp per query (lanes over pairs of K columns):
// the split BF16 rows of theta^c (x) u for the Jacobian GEMM and, with `digits`, the digit
// slices of theta^c (x) u / 2 and theta^a on their grids, the row exponents, u as float pairs
// (transposed) and a zeroed output row for the sliced GEMM. theta comes from the per-query rows.
__global__ void __launch_bounds__(kThreads) k_build_x(BuildXParams p) {
  const DevOps &o = p.o;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  __shared__ float thh_s[kWarps][RB_Q_MAX];  // theta^c rounded to FP32, per warp
  float *thh = thh_s[threadIdx.x >> 5];
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < p.nq; b += nw) {
    const rb_query_info qi = p.info[b];
    const bool want = p.mode == 0 ? is_active(qi, p.max_iter) : qi.status == RB_Q_OK;
    if (!want) continue;
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    const double *ta = p.theta + (size_t)b * o.n_theta, *tc = ta + o.q_a;
    const double *ub = p.u + (size_t)b * o.n_max;
    const bool jsplit = p.mode == 0 && p.split;
    float2 *u2b = p.u2 + (size_t)b * p.nb;
    if (p.mode == 0) {
      // u as double-float for the system assembly (and the Jacobian operand below), theta^c
      // rounded to FP32: no FP64 conversion in the loops that follow
      for (int j = lane; j < p.nb; j += 32) {
        float h = 0.f, lo = 0.f;
        if (j < n) df_split(ub[j], h, lo);
        u2b[j] = make_float2(h, lo);
      }
      if (jsplit)
        for (int q = lane; q < o.q_c; q += 32) {
          float h, lo;
          df_split(tc[q], h, lo);
          thh[q] = h;
        }
      __syncwarp();
    }
    // the vector in the operand: u, or the last update d in increment mode
    const double *vb = p.incr ? p.dU + (size_t)b * p.nb : ub;
    // (theta^c (x) v)[kap] at kap = q nb + l, zero past the query's size
    auto xval = [&](int q, int l) -> double {
      return (q < o.q_c && l < n) ? tc[q] * vb[l] : 0.0;
    };
    // grid exponents from the integer bit patterns (|x| orders like its bits). The largest
    // |theta^c_q u_l| is the rounded product of the largest factors (rounding is monotone),
    // so the maximum over the row needs only the maxima of theta^c and u.
    const unsigned long long absmask = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long m0 = 0, m1 = 0, mu = 0, mt = 0;
    if (p.digits) {
      unsigned long long mv = 0;
      for (int q = lane; q < o.q_c; q += 32) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(tc[q]) & absmask;
        mt = v > mt ? v : mt;
      }
      for (int l = lane; l < n; l += 32) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(ub[l]) & absmask;
        mu = v > mu ? v : mu;
        const unsigned long long w = (unsigned long long)__double_as_longlong(vb[l]) & absmask;
        mv = w > mv ? w : mv;
      }
      for (int q = lane; q < o.q_a; q += 32) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(ta[q]) & absmask;
        m1 = v > m1 ? v : m1;
      }
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, mt, off);
        const unsigned long long c = __shfl_xor_sync(0xffffffffu, mu, off);
        const unsigned long long d = __shfl_xor_sync(0xffffffffu, m1, off);
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, mv, off);
        mt = a > mt ? a : mt;
        mu = c > mu ? c : mu;
        m1 = d > m1 ? d : m1;
        mv = w > mv ? w : mv;
      }
      m0 = (unsigned long long)__double_as_longlong(__longlong_as_double((long long)mt) *
                                                    __longlong_as_double((long long)mv)) & absmask;
    }
    // digits on the grid with one binade of headroom (balanced digits); the operand of C(u, u)
    // holds x / 2: the same digits recorded one binade lower (increment mode: x itself)
    const int ex0 = exp_of_bits(m0) + 1, e0 = p.incr ? ex0 : ex0 - 1, e1 = exp_of_bits(m1) + 1;
    if (p.incr && lane == 0) {
      // Digit levels the increment needs: its truncation (pairs i + j > L dropped, on the grid of
      // d) must stay below that of the full product on the grid of u (pairs i + j > S + 1). Every
      // 7 binary digits by which d lies below u saves one level.
      const unsigned long long mtu = (unsigned long long)__double_as_longlong(
          __longlong_as_double((long long)mt) * __longlong_as_double((long long)mu)) & absmask;
      const int e0u = exp_of_bits(mtu);  // the grid exponent of the full product's x / 2
      int need = 2;
      if (m0 != 0) {
        const int below = e0u - ex0;
        need = p.S0 + 1 - (below > 0 ? below / kDigitBits : 0);
        need = max(2, min(p.S0 + 1, need));
      }
      atomicMax(p.lmax, need);
    }
    const size_t sstride = (size_t)p.b_pad * p.Kpad;
    const size_t jstride = (size_t)p.b_pad * p.Kpad0;
    // Kpad0 and Kpad are multiples of 64: a pair never straddles the segment boundary. The
    // lane's (q, l) of kap = 2 lane + 64 i advance without a division per step.
    int q = (2 * lane) / p.nb, l = 2 * lane - q * p.nb;
    // the linear segment (theta^a digits) serves the pressure GEMM only (mode 1)
    const int kend = p.mode == 0 ? p.Kpad0 : p.Kpad;
#pragma unroll 2
    for (int kap = 2 * lane; kap < kend; kap += 64) {
      const size_t off = (size_t)b * p.Kpad + kap;
      if (kap < p.Kpad0) {
        const int q1 = l + 1 < p.nb ? q : q + 1, l1 = l + 1 < p.nb ? l + 1 : 0;
        if (jsplit) {
          // split BF16 operand of the Jacobian GEMM: [x_hi | x_hi | x_lo], always from u, from
          // the FP32 product of the rounded factors (within 2 FP32 ulps of theta^c_q u_l: far
          // below the 16 bits that the split keeps)
          const float f0 = (q < o.q_c && l < n) ? thh[q] * u2b[l].x : 0.f;
          const float f1 = (q1 < o.q_c && l1 < n) ? thh[q1] * u2b[l1].x : 0.f;
          const __nv_bfloat162 hi = __floats2bfloat162_rn(f0, f1);
          const __nv_bfloat162 lo =
              __floats2bfloat162_rn(f0 - __low2float(hi), f1 - __high2float(hi));
          __nv_bfloat162 *xj = reinterpret_cast<__nv_bfloat162 *>(p.Xj + (size_t)b * p.Kpad0 + kap);
          xj[0] = hi;
          xj[jstride / 2] = hi;
          xj[jstride] = lo;
        }
        if (p.digits) digits_pair(xval(q, l), xval(q1, l1), ex0, p.S0, p.Xd + off, sstride);
      } else if (p.digits) {
        const int qa = kap - p.Kpad0;
        digits_pair(qa < o.q_a ? ta[qa] : 0.0, qa + 1 < o.q_a ? ta[qa + 1] : 0.0, e1, p.S1,
                    p.Xd + off, sstride);
      }
      l += 64;
      while (l >= p.nb) {
        l -= p.nb;
        ++q;
      }
    }
    if (!p.digits) continue;
    // the contraction vector: u, or u - d / 2 in increment mode
    for (int j = lane; j < p.nb; j += 32) {
      const double v = j < n ? (p.incr ? ub[j] - 0.5 * vb[j] : ub[j]) : 0.0;
      float hi, lo;
      df_split(v, hi, lo);
      p.ufT[(size_t)j * p.b_pad + b] = make_float2(hi, lo);
    }
    if (!p.incr)
      for (int k = lane; k < p.nout; k += 32) p.out[(size_t)b * p.nout + k] = 0.0;
    if (lane == 0) {
      p.xexp[b] = e0;
      p.xexp[p.b_pad + b] = e1;
    }
  }
}

// ---- per-query data computed once, when a query starts (iteration count 0) --------------
// theta row (FP64), f(mu) (FP64) and A(mu) = sum_q theta^a_q A_q (double-float, Sec. 2.4 affine
// split) are fixed for the whole Newton solve of a query: every later kernel reads them instead
// of evaluating the parameter functions and re-assembling the affine sums.
struct PrepParams {
  DevOps o;
  const double *mu, *theta_in;  // theta_in: [nq][n_theta] caller rows, or null: from mu
  int nq, nb, max_iter;
  const rb_query_info *info;
  double *Th;                   // [nq][n_theta]
  double *Fm;                   // [nq][nb]
  const int *nsz;               // [nq] sizes, or null: all nb
  double2 *Rn;                  // [nq]: (0, max(1, ||f(mu)||)) of the starting queries
  int all;                      // 1: every active query, not only the starting ones
};

__device__ __forceinline__ bool starts(const rb_query_info &q, int max_iter) {
  return is_active(q, max_iter) && q.iters == 0;
}
// queries whose per-query data (theta, f, A(mu), B(mu)) is built: those that start, or every
// active one (all: the serving path rebuilds it in each step's size-bucketed batch)
__device__ __forceinline__ bool prepares(const rb_query_info &q, int max_iter, int all) {
  return is_active(q, max_iter) && (all || q.iters == 0);
}

// theta and f(mu) of the starting queries, one warp per query.
// A block takes 8 queries at a time. The FP64 pipe of this GPU issues about two operations per
// clock per SM, a cost paid per warp instruction whatever the number of active lanes, so every
// distinct parameter-function value (term q < the largest term count) of the 8 queries is
// evaluated by its own thread first (all lanes busy), then each warp assembles one query's theta
// row from them, f(mu) and max(1, ||f(mu)||); the values are theta_eval_strided's, bit for bit.
constexpr int kPrepQ = 8;
__global__ void __launch_bounds__(256) k_prep_theta(PrepParams p) {
  const DevOps &o = p.o;
  __shared__ double tv[kPrepQ][RB_Q_MAX];
  __shared__ double inv_re[kPrepQ];
  __shared__ int flag[kPrepQ];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int qmax = max(max(o.q_a, o.q_c), max(o.q_f, o.q_b));
  for (int b0 = blockIdx.x * kPrepQ; b0 < p.nq; b0 += gridDim.x * kPrepQ) {
    if (threadIdx.x < kPrepQ) {
      const int b = b0 + threadIdx.x;
      const bool f = b < p.nq && prepares(p.info[b], p.max_iter, p.all);
      flag[threadIdx.x] = f;
      if (f && !p.theta_in) inv_re[threadIdx.x] = 1.0 / p.mu[2 * b + 1];
    }
    __syncthreads();
    if (!p.theta_in)
      for (int t = threadIdx.x; t < kPrepQ * qmax; t += blockDim.x) {
        const int qi = t / qmax, q = t - qi * qmax;
        if (!flag[qi]) continue;
        const double a = p.mu[2 * (b0 + qi)] * 0.017453292519943295769;  // pi / 180
        double v;
        if (o.theta_family == RB_THETA_POLY) {
          v = 1.0;
          for (int k = 0; k < q; ++k) v *= a;
        } else {
          v = trig_q(q, a);
        }
        tv[qi][q] = v;
      }
    __syncthreads();
    const int b = b0 + w;
    if (w < kPrepQ && flag[w]) {
      double *th = p.Th + (size_t)b * o.n_theta;
      if (p.theta_in) {
        for (int i = lane; i < o.n_theta; i += 32) th[i] = p.theta_in[(size_t)b * o.n_theta + i];
      } else {
        for (int i = lane; i < o.n_theta; i += 32) {
          int q = i;
          double scale = 1.0;
          if (q < o.q_a) {
            scale = inv_re[w];
          } else {
            q -= o.q_a;
            if (q >= o.q_c) {
              q -= o.q_c;
              if (q >= o.q_f) q -= o.q_f;
            }
          }
          th[i] = tv[w][q] * scale;
        }
      }
      __syncwarp();
      const double *tf = th + o.q_a + o.q_c;
      const int n = p.nsz ? p.nsz[b] : p.nb;
      double ff = 0.0;
      for (int k = lane; k < p.nb; k += 32) {
        double s = 0.0;
        for (int q = 0; q < o.q_f; ++q) s = fma(tf[q], o.f[(size_t)q * o.n_max + k], s);
        p.Fm[(size_t)b * p.nb + k] = s;
        if (k < n) ff += s * s;
      }
      ff = warp_sum(ff);
      if (lane == 0) p.Rn[b] = make_double2(0.0, fmax(1.0, sqrt(ff)));  // scale of the residual test
    }
    __syncthreads();  // tv and flag are reused by the next 8 queries
  }
}

// Affine sums of the starting queries: out_b = sum_q theta_{off+q}(b) Q_q in double-float, for
// A(mu) (A_q, theta^a) and B(mu) (B_q, theta^b). A block holds kAsmQ queries' coefficients and
// each thread one element, so every Q_q element read serves kAsmQ queries.
constexpr int kAsmQ = 8;

struct AffineParams {
  int nq, max_iter, all, n_theta, th_off, qn;
  size_t nn;                  // elements per matrix
  const rb_query_info *info;
  const double *Th;           // [nq][n_theta]
  const float2 *Q2;           // [qn][nn] double-float terms
  float2 *out;                // [nq][nn]
};

__global__ void __launch_bounds__(256) k_affine_sum(AffineParams p) {
  extern __shared__ float2 ta_s[];  // [kAsmQ][qn]
  __shared__ int flag[kAsmQ];
  const int qa = p.qn;
  const size_t nn = p.nn;
  for (int g = blockIdx.y; g * kAsmQ < p.nq; g += gridDim.y) {
    const int b0 = g * kAsmQ;
    __syncthreads();
    if (threadIdx.x < kAsmQ) {
      const int b = b0 + threadIdx.x;
      flag[threadIdx.x] = b < p.nq && prepares(p.info[b], p.max_iter, p.all);
    }
    __syncthreads();
    int any = 0;
#pragma unroll
    for (int r = 0; r < kAsmQ; ++r) any |= flag[r];
    if (!any) continue;
    for (int i = threadIdx.x; i < kAsmQ * qa; i += blockDim.x) {
      const int r = i / qa, q = i - r * qa;
      float h = 0.f, l = 0.f;
      if (flag[r]) df_split(p.Th[(size_t)(b0 + r) * p.n_theta + p.th_off + q], h, l);
      ta_s[i] = make_float2(h, l);
    }
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn;
         e += (size_t)gridDim.x * blockDim.x) {
      float ah[kAsmQ], al[kAsmQ];
#pragma unroll
      for (int r = 0; r < kAsmQ; ++r) ah[r] = al[r] = 0.f;
#pragma unroll 2
      for (int q = 0; q < qa; ++q) {
        const float2 a2 = __ldg(p.Q2 + (size_t)q * nn + e);
#pragma unroll
        for (int r = 0; r < kAsmQ; ++r) {
          const float2 t = ta_s[r * qa + q];
          df_fma(ah[r], al[r], t.x, t.y, a2.x, a2.y);
        }
      }
#pragma unroll
      for (int r = 0; r < kAsmQ; ++r)
        if (flag[r]) p.out[(size_t)(b0 + r) * nn + e] = make_float2(ah[r], al[r]);
    }
  }
}

struct LuParams {
  DevOps o;
  const int *nsz;
  int nq, nb, ldj, max_iter;
  double tol_upd, tol_res;
  const float2 *Amu;     // [nq][nb * nb] A(mu) as double-float (k_affine_sum)
  const double *Fm;      // [nq][nb] f(mu)
  float *Jaug;           // [nq][nb][lda] augmented Newton matrices [J | -R] (warp path)
  double2 *Rn;           // [nq]: (unused, max(1, ||f||)), set when the query starts
  double *Rg;            // [nq][(nb + 7) / 8]: sums of R[k]^2 over the system's row groups
  int lda;
  const float *Jc;       // [b_pad][ldj]
  const double *Rc;      // [b_pad][nb]: C_mu(u, u)
  double *u;             // [nq][n_max], updated in place
  const float2 *u2;      // [nq][nb] u as double-float, written by k_build_x this iteration
  rb_query_info *info;   // [nq]
  int *active;           // count of queries still active after this iteration
  int eval_only;         // 1: write R and J (FP64) to R_out / J_out instead of solving
  double *R_out, *J_out;
  int rmode;             // residual source: kResZero, kResLow, kResExact, or -1: per query
                         // from its iteration count (0 -> zero, 1 -> low, >= 2 -> exact)
  int chord;             // 1: the Jacobian factored at iteration 2 serves the later iterations
  int rung_all;          // -1, or the rung every active query of the launch is on (0 zero,
                         // 1 low, 2 FP64-accurate, 3 FP64-accurate chord step)
  int *Piv;              // [nq][nb]: pivot rows of the kept factorisation (chord)
  double *dU;            // [nq][nb]: the update of each query's last iteration, or null
  int *refresh;          // chord steps: raised when a query's chord step contracts too slowly
                         // (that query factors a fresh Jacobian at its next iteration), or null
  int *escalate;         // raised when a query is handed to the FP64 Newton (kQEscalate)
  const int *run_if;     // k_newton_system<., 4>: runs only if *run_if != 0
};

// Residual source of one Newton iteration (the precision ladder of the inexact Newton):
//   kResZero  u = 0: R = -f(mu) exactly and J = A(mu) (no contraction needed),
//   kResLow   R = (A(mu) + J~^c / 2) u - f(mu) from the FP32/BF16 Jacobian (Euler identity);
//             only used to approach the root, never to declare convergence,
//   kResExact R = A(mu) u + [C_mu(u, u)]_sliced - f(mu), FP64-accurate.
enum { kResZero = 0, kResLow = 1, kResExact = 2, kResLadder = -1 };

__device__ __forceinline__ int rung_of(int rmode, int iters) {
  return rmode >= 0 ? rmode : (iters == 0 ? kResZero : (iters == 1 ? kResLow : kResExact));
}

// Chord steps (Jacobian reuse): from the second FP64-residual iteration on (iteration count
// >= 3), a query reuses the factorisation of its first one (count 2), kept in its [J | -R]
// block with the pivot rows in Piv and marked by Rn[b].x = 1 (0 from the query's start); only
// the residual is new.
// Per-query escalation. Rn[b].x holds the query's state: 0 no factors yet, 1 factors kept at
// iteration 2, 2 a fresh Jacobian requested, 3 factors kept from such a refresh. A chord step
// that shrinks the update by less than kChordSlow (a Jacobian that has drifted from the
// iterate) requests a refresh: the next iteration factors the Jacobian at the current iterate.
// If a chord step with the refreshed factors is slow again, the low-precision Jacobian itself
// is too inexact for this query (kappa 2^-16 not small): the query leaves the mixed loop with
// status kQEscalate and the FP64 Newton (the exact Newton of the plain path) solves it from
// u = 0, as the oracle does: a stalled iterate may lie where Newton converges poorly.
__device__ __forceinline__ bool chord_step(const LuParams &p, int b, int iters) {
  const double s = p.Rn[b].x;
  return p.chord && p.rmode < 0 && iters >= 3 && (s == 1.0 || s == 3.0);
}
__device__ __forceinline__ bool chord_keep(const LuParams &p, int b, int iters) {
  return p.chord && p.rmode < 0 && (iters == 2 || (iters >= 3 && p.Rn[b].x == 2.0));
}
constexpr double kChordSlow = 0.25;
// after a chord step of query b (one thread): dn = ||delta_k||, prev = ||delta_{k-1}||; returns
// the query's new status (kQEscalate when handed to the FP64 Newton)
__device__ __forceinline__ int chord_watch(const LuParams &p, int b, bool chord, int status,
                                           double dn, double prev) {
  if (!chord || status != RB_Q_NOT_CONVERGED || !p.refresh || !(dn > kChordSlow * prev))
    return status;
  if (p.Rn[b].x == 3.0 && p.escalate) {
    atomicOr(p.escalate, 1);
    return kQEscalate;
  }
  p.Rn[b].x = 2.0;
  atomicOr(p.refresh, 1);
  return status;
}
// the state after keeping factors: 1 at iteration 2, 3 after a refresh
__device__ __forceinline__ double kept_state(const LuParams &p, int b) {
  return p.Rn[b].x == 2.0 ? 3.0 : 1.0;
}


constexpr int kWarpLuMaxN = 80;  // warp-per-query elimination up to this size

// Row stride of the augmented Newton matrix [J | -R] of the warp kernel: >= nb + 1, a multiple
// of 4 with an odd number of float4 chunks (bank-conflict-free float4 rows, see gepp_aug_warp).
__host__ __device__ inline int aug_ld(int nb) {
  int ld = (nb + 1 + 3) & ~3;
  if (((ld >> 2) & 1) == 0) ld += 4;
  return ld;
}

// Rows k0 .. k0 + 7 of query b's Newton system, by one warp (lanes over column pairs):
// J[k][:] = fl32(A(mu)[k][:]) + J^c[k][:] and R[k] = A(mu)[k][:] u (double-float) + convection
// part - f[k] (residual source RM). The 8 rows' loads of a column block are issued before their
// arithmetic, and the row sums are reduce-scattered over the warp (df_warp_reduce8). Rows
// k >= n are skipped. Returns sum_k R[k]^2 of the group in lane 0 (not EVAL).
// J: the destination of rows k0 .. k0 + 7 of [J | -R] (row stride p.lda; global memory or the
// elimination's shared slab), unused with EVAL.
template <int RM, bool EVAL, bool JAC>
__device__ __forceinline__ double newton_rows8(const LuParams &p, int b, int n, int k0, float *J) {
  const int lane = threadIdx.x & 31;
  const int nb = p.nb;
  const bool vec = (nb & 1) == 0;  // even rows: 16-byte A(mu) and 8-byte J^c pairs are aligned
  const float2 *am = p.Amu + ((size_t)b * nb + k0) * nb;
  const float *jc = p.Jc + (size_t)b * p.ldj + (size_t)k0 * nb;
  const float2 *u2 = p.u2 + (size_t)b * nb;
  const int rows = min(8, n - k0);
  float rh[8], rl[8], ch[8], cl[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) rh[r] = rl[r] = ch[r] = cl[r] = 0.f;
  for (int j = 2 * lane; j < n; j += 64) {
    const bool two = j + 1 < n;
    float4 a[8];
    float2 c[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      a[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      c[r] = make_float2(0.f, 0.f);
      if (r < rows) {
        const float2 *ar = am + (size_t)r * nb + j;
        const float *cr = jc + (size_t)r * nb + j;
        if (two && vec) {
          a[r] = __ldg(reinterpret_cast<const float4 *>(ar));
          if (RM != kResZero && (JAC || RM == kResLow)) c[r] = __ldg(reinterpret_cast<const float2 *>(cr));
        } else {
          const float2 a0 = __ldg(ar), a1 = two ? __ldg(ar + 1) : make_float2(0.f, 0.f);
          a[r] = make_float4(a0.x, a0.y, a1.x, a1.y);
          if (RM != kResZero && (JAC || RM == kResLow))
            c[r] = make_float2(__ldg(cr), two ? __ldg(cr + 1) : 0.f);
        }
      }
    }
    float uh0 = 0.f, ul0 = 0.f, uh1 = 0.f, ul1 = 0.f;
    if (RM != kResZero) {
      if (two && vec) {
        const float4 uu = __ldg(reinterpret_cast<const float4 *>(u2 + j));
        uh0 = uu.x, ul0 = uu.y, uh1 = uu.z, ul1 = uu.w;
      } else {
        const float2 u0 = __ldg(u2 + j);
        uh0 = u0.x, ul0 = u0.y;
        if (two) {
          const float2 u1 = __ldg(u2 + j + 1);
          uh1 = u1.x, ul1 = u1.y;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (r < rows) {
        const float v0 = (a[r].x + a[r].y) + c[r].x, v1 = (a[r].z + a[r].w) + c[r].y;
        if (RM != kResZero) {
          df_fma(rh[r], rl[r], a[r].x, a[r].y, uh0, ul0);
          df_fma(rh[r], rl[r], a[r].z, a[r].w, uh1, ul1);
        }
        if (RM == kResLow) ch[r] = fmaf(0.5f * c[r].y, uh1, fmaf(0.5f * c[r].x, uh0, ch[r]));
        if (EVAL) {
          double *jo = p.J_out + ((size_t)b * n + k0 + r) * n + j;
          jo[0] = (double)v0;
          if (two) jo[1] = (double)v1;
        } else if (JAC) {  // a chord step keeps the factors stored in J's place
          float *jr = J + (size_t)r * p.lda + j;
          if (two) *reinterpret_cast<float2 *>(jr) = make_float2(v0, v1);
          else jr[0] = v0;
        }
      }
    }
  }
  if (RM != kResZero) df_warp_reduce8(rh, rl);
  if (RM == kResLow) df_warp_reduce8(ch, cl);
  const int r = lane >> 2, k = k0 + r;
  if (EVAL) {  // R in FP64 for the caller
    if ((lane & 3) == 0 && r < rows) {
      const double rlin = RM != kResZero ? (double)rh[0] + (double)rl[0] : 0.0;
      const double conv = RM == kResExact ? p.Rc[(size_t)b * nb + k]
                                          : (RM == kResLow ? (double)ch[0] + (double)cl[0] : 0.0);
      p.R_out[(size_t)b * n + k] = rlin + conv - p.Fm[(size_t)b * nb + k];
    }
    return 0.0;
  }
  // R = A(mu) u + C_mu(u, u) - f(mu) in double-float (no FP64 instruction per row: each would
  // occupy the narrow FP64 pipe for the whole warp); -R rounded to FP32 into column n
  float Rs = 0.f;
  if ((lane & 3) == 0 && r < rows) {
    float Rh = 0.f, Rl = 0.f;
    if (RM != kResZero) Rh = rh[0], Rl = rl[0];
    if (RM == kResExact) {
      float a, c;
      df_split(p.Rc[(size_t)b * nb + k], a, c);
      df_add(Rh, Rl, a, c);
    } else if (RM == kResLow) {
      df_add(Rh, Rl, ch[0], cl[0]);
    }
    float fh, fl;
    df_split(p.Fm[(size_t)b * nb + k], fh, fl);
    df_add(Rh, Rl, -fh, -fl);
    float e;
    two_sum(Rh, Rl, Rs, e);
    float *row = J + (size_t)r * p.lda;
    row[n] = -Rs;
    const int c_pad = ((n >> 2) << 2) + 4;  // columns n + 1 .. c_pad - 1 pad the last chunk
    for (int c = n + 1; c < c_pad; ++c) row[c] = 0.f;
  }
  // the group's sum of R[k]^2 in FP32 (the stopping test needs a few digits of the norm), unless
  // some |R[k]| lies outside [2^-60, 2^60], where squares could leave the FP32 range
  const float a = fabsf(Rs);
  if (__any_sync(0xffffffffu, a > 0x1p60f || (a > 0.f && a < 0x1p-60f)))
    return warp_sum((double)Rs * (double)Rs);
  return f32_to_f64(warp_sum(Rs * Rs));
}

// Newton systems of the active queries: one warp per (query, group of 8 rows), so the work
// splits evenly over the resident warps whatever the batch size. Writes the augmented matrix
// [J | -R] (FP32, row stride lda, the right-hand side in column n, zero padding up to the next
// multiple of 4) and the group's sum of R[k]^2 to Rg[b][g] (the elimination adds the groups in
// order: deterministic). With EVAL, J and R go to J_out / R_out in FP64 instead.
// FIXED >= 0: every active query of the launch is on rung FIXED (LuParams::rung_all), so the
// kernel holds one variant only (fewer registers, more resident warps); -1: per query.
constexpr int system_blocks(int fixed) { return fixed == 0 || fixed == 3 ? 3 : 2; }
template <bool EVAL, int FIXED>
__global__ void __launch_bounds__(kThreads, system_blocks(FIXED)) k_newton_system(LuParams p) {
  if (FIXED == 4 && *(volatile const int *)p.run_if == 0) return;  // no query refreshes
  const int lane = threadIdx.x & 31;
  const int G = (p.nb + 7) >> 3;
  const long long units = (long long)p.nq * G;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < units; t += nw) {
    const int b = (int)(t / G), g = (int)(t - (long long)b * G);
    const rb_query_info qi = p.info[b];
    if (!is_active(qi, p.max_iter)) continue;
    const int n = p.nsz ? p.nsz[b] : p.nb;
    const int k0 = 8 * g;
    if (k0 >= n) continue;
    float *Jg = EVAL ? nullptr : p.Jaug + ((size_t)b * p.nb + k0) * p.lda;
    double r2;
    if (FIXED == 0) {
      r2 = newton_rows8<kResZero, EVAL, true>(p, b, n, k0, Jg);
    } else if (FIXED == 1) {
      r2 = newton_rows8<kResLow, EVAL, true>(p, b, n, k0, Jg);
    } else if (FIXED == 2) {
      r2 = newton_rows8<kResExact, EVAL, true>(p, b, n, k0, Jg);
    } else if (FIXED == 3) {  // chord steps; a query refreshing its Jacobian is left to FIXED 4
      if (!chord_step(p, b, qi.iters)) continue;
      r2 = newton_rows8<kResExact, EVAL, false>(p, b, n, k0, Jg);
    } else if (FIXED == 4) {  // the queries of a chord launch that refresh their Jacobian
      if (chord_step(p, b, qi.iters)) continue;
      r2 = newton_rows8<kResExact, EVAL, true>(p, b, n, k0, Jg);
    } else {
      const int rm = rung_of(p.rmode, qi.iters);
      r2 = rm == kResZero  ? newton_rows8<kResZero, EVAL, true>(p, b, n, k0, Jg)
           : rm == kResLow ? newton_rows8<kResLow, EVAL, true>(p, b, n, k0, Jg)
           : (!EVAL && chord_step(p, b, qi.iters)) ? newton_rows8<kResExact, EVAL, false>(p, b, n, k0, Jg)
                                                   : newton_rows8<kResExact, EVAL, true>(p, b, n, k0, Jg);
    }
    if (!EVAL && lane == 0) p.Rg[(size_t)b * G + g] = r2;
  }
}

// ||R|| from the sums of squares of a query's gn row groups (every lane of the calling warps,
// all 32 present): the lanes take the groups, rounded to FP32 by integer operations, and add them
// in FP32 (the stopping test needs a few digits of the norm); sums outside [2^-100, 2^100] are
// added in FP64 instead, in group order.
__device__ __forceinline__ double norm_of_groups(const double *rg, int gn) {
  float s = 0.f;
  bool wide = false;
  for (int g = threadIdx.x & 31; g < gn; g += 32) {
    float h, l;
    df_split(rg[g], h, l);
    s += h;
    wide |= !(h == 0.f || (h >= 0x1p-100f && h < 0x1p100f));
  }
  if (!__any_sync(0xffffffffu, wide)) return f32_to_f64(sqrtf(warp_sum(s)));
  double t = 0.0;
  for (int g = 0; g < gn; ++g) t += rg[g];
  return sqrt(t);
}
__device__ __forceinline__ double residual_norm(const LuParams &p, int b, int n) {
  return norm_of_groups(p.Rg + (size_t)b * ((p.nb + 7) >> 3), (n + 7) >> 3);
}

// Warp-per-query elimination of the systems k_newton_system assembled: copy the query's
// augmented matrix into the warp's shared slab, solve, update u, apply the stopping rule.
struct WarpLuSmem {
  int pseq, stp, J, per_warp;  // byte offsets within a warp's slab
  __host__ __device__ WarpLuSmem(int nb, int lda) {
    int p = 0;
    pseq = p; p += 4 * ((nb + 3) & ~3);
    stp = p; p += 4 * ((nb + 3) & ~3);
    p = (p + 15) & ~15;
    J = p; p += 4 * nb * lda;
    per_warp = (p + 15) & ~15;
  }
};

// R lane slots of rows (n <= 32 R). Blocks of at most kLuWarpBlock threads; with two slots the
// kernel stays within 96 registers, so that 20 warps (5 per scheduler) can be resident.
constexpr int kLuWarpBlock = 128;
template <int R>
__global__ void __launch_bounds__(kLuWarpBlock, R == 2 ? 5 : 2) k_lu_mixed_warp(LuParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const WarpLuSmem L(p.nb, p.lda);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  uint8_t *slab = smb + (size_t)w * L.per_warp;
  float *J = reinterpret_cast<float *>(slab + L.J);
  int *pseq = reinterpret_cast<int *>(slab + L.pseq);
  int *stp = reinterpret_cast<int *>(slab + L.stp);
  const int ld = p.lda;
  int my_active = 0;
  for (int b = blockIdx.x * wpc + w; b < p.nq; b += gridDim.x * wpc) {
    rb_query_info qi = p.info[b];
    if (!is_active(qi, p.max_iter)) continue;
    const int n = p.nsz ? p.nsz[b] : p.nb;
    double *ub = p.u + (size_t)b * p.o.n_max;
    const int rm = rung_of(p.rmode, qi.iters);
    const bool chord = chord_step(p, b, qi.iters), keep = chord_keep(p, b, qi.iters);
    const double rn = residual_norm(p, b, n), fscale = p.Rn[b].y;
    float4 *gJ = reinterpret_cast<float4 *>(p.Jaug + (size_t)b * p.nb * ld);
    const int n4 = n * ld / 4;
    {
      float4 *dst = reinterpret_cast<float4 *>(J);
      for (int i = lane; i < n4; i += 32) cp_async16(dst + i, gJ + i);
      if (chord)
        for (int i = lane; i < n; i += 32) pseq[i] = p.Piv[(size_t)b * p.nb + i];
      cp_async_wait_all();
    }
    __syncwarp();
    qi.iters += 1;
    qi.res_norm = rn;
    qi.precision_used = RB_PREC_MIXED;
    float x[R];
    if (!isfinite(rn)) {
      qi.status = RB_Q_NONFINITE;
    } else if (chord ? chord_solve_warp<R>(J, ld, n, pseq, stp, x) : gepp_aug_warp<R>(J, ld, n, x, pseq)) {
      qi.status = RB_Q_SINGULAR;
    } else {
      if (keep) {  // the factors (L in the eliminated places, U) and pivots for the chord steps
        __syncwarp();
        const float4 *src = reinterpret_cast<const float4 *>(J);
        for (int i = lane; i < n4; i += 32) gJ[i] = src[i];
        for (int i = lane; i < n; i += 32) p.Piv[(size_t)b * p.nb + i] = pseq[i];
        if (lane == 0) p.Rn[b].x = kept_state(p, b);
      }
      // u += delta in FP64; ||delta|| in FP32 unless some |delta_k| exceeds 2^60
      float dl = 0.f;
      bool wide = false;
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const int k = lane + 32 * s;
        if (k < n) {
          const double d = f32_to_f64(x[s]);
          dl = fmaf(x[s], x[s], dl);
          wide |= !(fabsf(x[s]) <= 0x1p60f);
          ub[k] += d;
          if (p.dU) p.dU[(size_t)b * p.nb + k] = d;
        }
      }
      double dn;
      if (!__any_sync(0xffffffffu, wide)) {
        dn = f32_to_f64(sqrtf(warp_sum(dl)));
      } else {
        double dd = 0.0;
#pragma unroll
        for (int s = 0; s < R; ++s)
          if (lane + 32 * s < n) dd += (double)x[s] * (double)x[s];
        dn = sqrt(warp_sum(dd));
      }
      const double prev = qi.upd_norm;
      qi.upd_norm = dn;
      if (!isfinite(dn)) qi.status = RB_Q_NONFINITE;
      else if (rm != kResLow && dn <= p.tol_upd && rn <= p.tol_res * fscale) qi.status = RB_Q_OK;
      if (lane == 0) qi.status = chord_watch(p, b, chord, qi.status, dn, prev);
    }
    if (lane == 0) {
      p.info[b] = qi;
      if (is_active(qi, p.max_iter)) ++my_active;
    }
    __syncwarp();
  }
  if (lane == 0 && my_active) atomicAdd(p.active, my_active);
}

// ---- CTA-per-query elimination in shared memory (32 < n <= 128) --------------------------
// One CTA of ceil(nb / 32) warps per query, one row per thread (gepp_aug_cta): the augmented
// matrix copied into shared memory, FP32 elimination by panels of 4 columns with one barrier
// per pivot step; update and stopping rule as in the warp kernel.
constexpr int kCtaLuMaxN = 128;
struct CtaLuSmem {
  int J, pseq, keys, lmp, stepv, dinvv, xs, red, total;  // byte offsets
  __host__ __device__ CtaLuSmem(int nb, int lda) {
    const int n4 = (nb + 3) & ~3;
    int p = 0;
    J = p; p += 4 * nb * lda;
    pseq = p; p += 4 * n4;
    keys = p; p += 4 * 8;
    lmp = p; p += 4 * 16;
    stepv = p; p += 4 * n4;
    dinvv = p; p += 4 * n4;
    xs = p; p += 4 * n4;
    p = (p + 7) & ~7;
    red = p; p += 8 * 4;
    total = (p + 15) & ~15;
  }
};

// Chord step of the CTA kernel: warp 0 solves with the factors kept in shared memory (forward
// substitution in pivot order, back substitution on U; chord_solve_warp with ceil(n / 32) row
// slots), the solution goes to xs; returns, uniformly over the CTA, whether a pivot was unusable.
__device__ __forceinline__ bool chord_solve_cta(const float *J, int ld, int n, const int *pseq,
                                                int *stp, unsigned *flag, float *xs) {
  const int lane = threadIdx.x & 31;
  if ((threadIdx.x >> 5) == 0) {
    bool bad;
    if (n <= 64) {
      float x[2];
      bad = chord_solve_warp<2>(J, ld, n, pseq, stp, x);
      if (!bad)
#pragma unroll
        for (int s = 0; s < 2; ++s)
          if (lane + 32 * s < n) xs[lane + 32 * s] = x[s];
    } else if (n <= 96) {
      float x[3];
      bad = chord_solve_warp<3>(J, ld, n, pseq, stp, x);
      if (!bad)
#pragma unroll
        for (int s = 0; s < 3; ++s)
          if (lane + 32 * s < n) xs[lane + 32 * s] = x[s];
    } else {
      float x[4];
      bad = chord_solve_warp<4>(J, ld, n, pseq, stp, x);
      if (!bad)
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (lane + 32 * s < n) xs[lane + 32 * s] = x[s];
    }
    if (lane == 0) flag[0] = bad ? 1u : 0u;
  }
  __syncthreads();
  const bool bad = flag[0] != 0u;
  __syncthreads();  // flag and xs are read before the next query reuses them
  return bad;
}

__global__ void __launch_bounds__(kCtaLuMaxN) k_lu_cta(LuParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const CtaLuSmem L(p.nb, p.lda);
  float *J = reinterpret_cast<float *>(smb + L.J);
  int *pseq = reinterpret_cast<int *>(smb + L.pseq);
  unsigned *keys = reinterpret_cast<unsigned *>(smb + L.keys);
  float *lmp = reinterpret_cast<float *>(smb + L.lmp);
  int *stepv = reinterpret_cast<int *>(smb + L.stepv);
  float *dinvv = reinterpret_cast<float *>(smb + L.dinvv);
  float *xs = reinterpret_cast<float *>(smb + L.xs);
  double *red = reinterpret_cast<double *>(smb + L.red);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ld = p.lda;
  int my_active = 0;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    rb_query_info qi = p.info[b];
    if (!is_active(qi, p.max_iter)) continue;  // uniform over the CTA
    const int n = p.nsz ? p.nsz[b] : p.nb;
    double *ub = p.u + (size_t)b * p.o.n_max;
    const int rm = rung_of(p.rmode, qi.iters);
    const bool chord = chord_step(p, b, qi.iters), keep = chord_keep(p, b, qi.iters);
    const double rn = residual_norm(p, b, n), fscale = p.Rn[b].y;
    float4 *gJ = reinterpret_cast<float4 *>(p.Jaug + (size_t)b * p.nb * ld);
    const int n4 = n * ld / 4;
    {
      float4 *dst = reinterpret_cast<float4 *>(J);
      for (int i = tid; i < n4; i += blockDim.x) cp_async16(dst + i, gJ + i);
      if (chord)
        for (int i = tid; i < n; i += blockDim.x) pseq[i] = p.Piv[(size_t)b * p.nb + i];
      cp_async_wait_all();
    }
    __syncthreads();
    qi.iters += 1;
    qi.res_norm = rn;
    qi.precision_used = RB_PREC_MIXED;
    if (!isfinite(rn)) {
      qi.status = RB_Q_NONFINITE;
    } else if (chord ? chord_solve_cta(J, ld, n, pseq, stepv, keys, xs)
                     : gepp_aug_cta(J, ld, n, pseq, keys, lmp, stepv, dinvv, xs)) {
      qi.status = RB_Q_SINGULAR;
    } else {
      if (keep) {  // the factors (L in the eliminated places, U) and pivots for the chord steps
        const float4 *src = reinterpret_cast<const float4 *>(J);
        for (int i = tid; i < n4; i += blockDim.x) gJ[i] = src[i];
        for (int i = tid; i < n; i += blockDim.x) p.Piv[(size_t)b * p.nb + i] = pseq[i];
        if (tid == 0) p.Rn[b].x = kept_state(p, b);
      }
      double dl = 0.0;
      if (tid < n) {
        const double d = (double)xs[tid];
        dl = d * d;
        ub[tid] += d;
        if (p.dU) p.dU[(size_t)b * p.nb + tid] = d;
      }
      dl = warp_sum(dl);
      if (lane == 0) red[w] = dl;
      __syncthreads();
      double tot = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
      const double dn = sqrt(tot);
      const double prev = qi.upd_norm;
      qi.upd_norm = dn;
      if (!isfinite(dn)) qi.status = RB_Q_NONFINITE;
      else if (rm != kResLow && dn <= p.tol_upd && rn <= p.tol_res * fscale) qi.status = RB_Q_OK;
      if (tid == 0) qi.status = chord_watch(p, b, chord, qi.status, dn, prev);
    }
    if (tid == 0) {
      p.info[b] = qi;
      if (is_active(qi, p.max_iter)) ++my_active;
    }
    __syncthreads();  // shared memory is reused by the next query
  }
  if (tid == 0 && my_active) atomicAdd(p.active, my_active);
}

// ---- blocked elimination for large systems (n_max > 80), one CTA per query --------------
// Right-looking blocked Gaussian elimination with partial pivoting on the query's augmented
// matrix [J | -R] (global, row stride lda, the right-hand side in column n): for each panel of
// kPB columns, (a) the tall panel is factored in shared memory with partial pivoting,
// (b) its row interchanges are applied to the columns right of it, (c) the panel's row block
// becomes U12 = L11^-1 A12, (d) the trailing matrix takes the rank-kPB update
// A22 -= L21 U12 in 4 x 4 register tiles. The right-hand side is eliminated along, so back
// substitution on U (blocks of 32 rows from the bottom) ends the solve.
// Panel width PB (32 or 16, picked by the autotuner); panel row stride PB + 1 in shared memory
// (odd: conflict-free column reads).
template <int PB>
struct BlkLuSmem {
  static constexpr int kPLd = PB + 1;
  int P, U, perm, rmap, tl, red, x, dred, total;  // byte offsets
  __host__ __device__ BlkLuSmem(int nb, int lda) {
    int p = 0;
    P = p; p += 4 * nb * kPLd;
    p = (p + 15) & ~15;
    U = p; p += 4 * PB * lda;
    perm = p; p += 4 * PB;
    rmap = p; p += 4 * nb;     // a panel's row interchanges as one permutation
    tl = p; p += 4 * (PB + 1); // rows at or past the panel's height that it moves, and their count
    red = p; p += 4 * kWarps;
    x = p; p += 4 * ((nb + 3) & ~3);
    p = (p + 7) & ~7;
    dred = p; p += 8 * 4 * kWarps;
    total = (p + 15) & ~15;
  }
};

// pivot key for panel rows r < 512: leading 14 mantissa bits of |v|, then the lower row
__device__ __forceinline__ unsigned pivot_key9(float v, int r) {
  return (__float_as_uint(fabsf(v)) & 0xFFFFFE00u) | (unsigned)(511 - r);
}

template <int PB>
__global__ void __launch_bounds__(kThreads, 2) k_lu_blocked(LuParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  constexpr int kPB = PB, kPLd = PB + 1;
  const int nb = p.nb, lda = p.lda;
  const BlkLuSmem<PB> L(nb, lda);
  float *P = reinterpret_cast<float *>(smb + L.P);
  float *U = reinterpret_cast<float *>(smb + L.U);
  int *perm = reinterpret_cast<int *>(smb + L.perm);
  int *rmap = reinterpret_cast<int *>(smb + L.rmap);
  int *tl = reinterpret_cast<int *>(smb + L.tl);
  unsigned *red = reinterpret_cast<unsigned *>(smb + L.red);
  float *xs = reinterpret_cast<float *>(smb + L.x);
  double *dred = reinterpret_cast<double *>(smb + L.dred);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int my_active = 0;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    rb_query_info qi = p.info[b];
    if (!is_active(qi, p.max_iter)) continue;
    const int n = p.nsz ? p.nsz[b] : nb;
    double *ub = p.u + (size_t)b * p.o.n_max;
    const int rm = rung_of(p.rmode, qi.iters);
    const bool chord = chord_step(p, b, qi.iters), keep = chord_keep(p, b, qi.iters);
    const double rn = residual_norm(p, b, n), fscale = p.Rn[b].y;
    float *M = p.Jaug + (size_t)b * nb * lda;
    bool sing = !isfinite(rn);
    if (chord && !sing) {
      // forward substitution with the kept factors, panel by panel as they were made: the
      // panel's row interchanges on b, L11 (unit lower) by warp 0, then b -= L21 b_panel with a
      // thread per row below
      for (int i = tid; i < n; i += blockDim.x) xs[i] = M[(size_t)i * lda + n];
      __syncthreads();
      for (int k0 = 0; k0 < n; k0 += kPB) {
        const int kb = min(kPB, n - k0);
        if (tid == 0)
          for (int j = 0; j < kb; ++j) {
            const int pr = p.Piv[(size_t)b * nb + k0 + j];
            if (pr != k0 + j) {
              const float t = xs[k0 + j];
              xs[k0 + j] = xs[pr];
              xs[pr] = t;
            }
          }
        __syncthreads();
        if (w == 0) {
          const bool own = lane < kb;
          float mrow[kPB];
#pragma unroll
          for (int jj = 0; jj < kPB; ++jj)
            mrow[jj] = (own && jj < lane) ? M[(size_t)(k0 + lane) * lda + k0 + jj] : 0.f;
          float y = own ? xs[k0 + lane] : 0.f;
#pragma unroll
          for (int jj = 0; jj < kPB; ++jj) {
            if (jj >= kb) break;
            const float xj = __shfl_sync(0xffffffffu, y, jj);
            if (own && lane > jj) y = fmaf(-mrow[jj], xj, y);
          }
          if (own) xs[k0 + lane] = y;
        }
        __syncthreads();
        for (int r = k0 + kb + tid; r < n; r += blockDim.x) {
          const float *row = M + (size_t)r * lda + k0;
          float s = xs[r];
          for (int j = 0; j < kb; ++j) s = fmaf(-row[j], xs[k0 + j], s);
          xs[r] = s;
        }
        __syncthreads();
      }
    }
    for (int k0 = 0; k0 < n && !sing && !chord; k0 += kPB) {
      const int kb = min(kPB, n - k0), rows = n - k0;
      // (a) load and factor the panel: rows k0 .. n-1, columns k0 .. k0+kb-1
      for (int e = tid; e < rows * kPB; e += blockDim.x) {
        const int r = e / kPB, c = e - r * kPB;
        P[r * kPLd + c] = c < kb ? M[(size_t)(k0 + r) * lda + k0 + c] : 0.f;
      }
      __syncthreads();
      // pivot keys of column 0, per warp into red; each step below then needs two barriers:
      // after the interchange, and after the update, which also finds the next column's keys
      // (the threads update the same rows j + 1 + tid, ... that the next search covers)
      {
        unsigned key = 0;
        for (int r = tid; r < rows; r += blockDim.x) {
          const unsigned k = pivot_key9(P[r * kPLd], r);
          key = k > key ? k : key;
        }
        key = __reduce_max_sync(0xffffffffu, key);
        if (lane == 0) red[w] = key;
        __syncthreads();
      }
      for (int j = 0; j < kb; ++j) {
        unsigned key = red[0];
#pragma unroll
        for (int i = 1; i < kWarps; ++i) key = red[i] > key ? red[i] : key;
        const int pr = 511 - (int)(key & 511u);
        const float pv = P[pr * kPLd + j];
        if (!(fabsf(pv) > 0.f) || !isfinite(pv)) {  // the same in every thread
          sing = true;
          break;
        }
        if (pr != j && tid < kPB) {
          const float t = P[j * kPLd + tid];
          P[j * kPLd + tid] = P[pr * kPLd + tid];
          P[pr * kPLd + tid] = t;
        }
        if (tid == 0) perm[j] = pr;
        __syncthreads();  // the interchange done and red read by every thread
        const float rinv = __frcp_rn(pv);
        unsigned nkey = 0;
        for (int r = j + 1 + tid; r < rows; r += blockDim.x) {
          float *Pr = P + r * kPLd;
          const float l = Pr[j] * rinv;
          Pr[j] = l;
          for (int c = j + 1; c < kb; ++c) Pr[c] = fmaf(-l, P[j * kPLd + c], Pr[c]);
          if (j + 1 < kb) {
            const unsigned k = pivot_key9(Pr[j + 1], r);
            nkey = k > nkey ? k : nkey;
          }
        }
        if (j + 1 < kb) {
          nkey = __reduce_max_sync(0xffffffffu, nkey);
          if (lane == 0) red[w] = nkey;
        }
        __syncthreads();
      }
      if (sing) break;
      // U11 (the panel's top rows, L11 in their strict lower part) back to the matrix for the
      // back substitution; when the factors are kept, L21 and the panel's pivots as well
      const int kept_rows = keep ? rows : kb;
      for (int e = tid; e < kept_rows * kb; e += blockDim.x) {
        const int r = e / kb, c = e - r * kb;
        M[(size_t)(k0 + r) * lda + k0 + c] = P[r * kPLd + c];
      }
      if (keep && tid < kb) p.Piv[(size_t)b * nb + k0 + tid] = k0 + perm[tid];
      // (b) the panel's row interchanges on the columns right of it, as one permutation: row r
      // of the panel's rows takes the old row rmap[r]; tl lists the rows r >= kb it changes
      for (int r = tid; r < rows; r += blockDim.x) rmap[r] = r;
      __syncthreads();
      if (tid == 0) {
        for (int j = 0; j < kb; ++j) {
          const int pr = perm[j], t = rmap[j];
          rmap[j] = rmap[pr];
          rmap[pr] = t;
        }
        int cnt = 0;
        for (int j = 0; j < kb; ++j) {
          const int pr = perm[j];
          if (pr < kb || rmap[pr] == pr) continue;
          bool dup = false;
          for (int t = 0; t < cnt; ++t) dup = dup || tl[t] == pr;
          if (!dup) tl[cnt++] = pr;
        }
        tl[kPB] = cnt;
      }
      __syncthreads();
      // (c) U12 = L11^-1 A12, one thread per column, the column's kb entries in registers: all
      // its loads issued at once, the solve a chain of FMAs on registers. A row at or past kb that
      // the interchanges move receives a row above kb (each swap hands the pivot position's
      // current row, by induction one of the rows above kb, to the pivot row's place), so those
      // rows are copied before the rows above kb are overwritten, and after every pivot row has
      // been read into v.
      const int c_lo = k0 + kb, nt = tl[kPB];
      for (int c = c_lo + tid; c <= n; c += blockDim.x) {
        float v[kPB];
#pragma unroll
        for (int j = 0; j < kPB; ++j) v[j] = j < kb ? M[(size_t)(k0 + rmap[j]) * lda + c] : 0.f;
        for (int t = 0; t < nt; ++t)
          M[(size_t)(k0 + tl[t]) * lda + c] = M[(size_t)(k0 + rmap[tl[t]]) * lda + c];
#pragma unroll
        for (int j = 1; j < kPB; ++j) {
          if (j < kb) {  // P holds the panel's rows only (kb <= rows <= nb)
            float s = v[j];
#pragma unroll
            for (int i = 0; i < j; ++i) s = fmaf(-P[j * kPLd + i], v[i], s);
            v[j] = s;
          }
        }
#pragma unroll
        for (int j = 0; j < kPB; ++j)
          if (j < kb) {
            U[j * lda + c] = v[j];
            M[(size_t)(k0 + j) * lda + c] = v[j];
          }
      }
      __syncthreads();
      // (d) trailing update of rows k0+kb .. n-1, columns c_lo .. n, in tiles of 4 rows x 4 columns
      const int r_lo = kb, nrow = rows - kb;
      if (nrow > 0) {
        const int cc_lo = c_lo >> 2, cc_hi = n >> 2;  // float4 chunks covering columns c_lo .. n
        const int nch = cc_hi - cc_lo + 1, nrb = (nrow + 3) >> 2;
        // store the 4 x 4 tile acc of rows r0.. and chunk cc (only columns c_lo .. n)
        auto store_tile = [&](int r0, int cc, const float4 (&acc)[4]) {
          const int c4 = 4 * cc;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (r0 + i >= rows) break;
            float *row = M + (size_t)(k0 + r0 + i) * lda + c4;
            if (c4 >= c_lo && c4 + 3 <= n) {
              reinterpret_cast<float4 *>(row)[0] = acc[i];
            } else {  // first or last chunk: only columns c_lo .. n
              if (c4 + 0 >= c_lo && c4 + 0 <= n) row[0] = acc[i].x;
              if (c4 + 1 >= c_lo && c4 + 1 <= n) row[1] = acc[i].y;
              if (c4 + 2 >= c_lo && c4 + 2 <= n) row[2] = acc[i].z;
              if (c4 + 3 >= c_lo && c4 + 3 <= n) row[3] = acc[i].w;
            }
          }
        };
        if (PB <= 16 && nrb <= (int)blockDim.x) {
          // a thread keeps one row block's multipliers in registers and walks a strided set of
          // column chunks: one shared-memory load of U per 16 multiply-adds
          const int G = blockDim.x / nrb;  // threads per row block
          if (tid < G * nrb) {
            const int rb4 = tid % nrb, g = tid / nrb;
            const int r0 = r_lo + 4 * rb4;
            float l[4][PB <= 16 ? PB : 1];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < (PB <= 16 ? PB : 1); ++j)
                l[i][j] = (j < kb && r0 + i < rows) ? P[(r0 + i) * kPLd + j] : 0.f;
            for (int cc = cc_lo + g; cc <= cc_hi; cc += G) {
              float4 acc[4];
#pragma unroll
              for (int i = 0; i < 4; ++i)
                acc[i] = r0 + i < rows ? reinterpret_cast<const float4 *>(M + (size_t)(k0 + r0 + i) * lda)[cc]
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int j = 0; j < (PB <= 16 ? PB : 1); ++j) {
                if (j >= kb) break;
                const float4 u = reinterpret_cast<const float4 *>(U + j * lda)[cc];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  acc[i].x = fmaf(-l[i][j], u.x, acc[i].x);
                  acc[i].y = fmaf(-l[i][j], u.y, acc[i].y);
                  acc[i].z = fmaf(-l[i][j], u.z, acc[i].z);
                  acc[i].w = fmaf(-l[i][j], u.w, acc[i].w);
                }
              }
              store_tile(r0, cc, acc);
            }
          }
        } else {
          for (int t = tid; t < nch * nrb; t += blockDim.x) {
            const int rb4 = t / nch, cc = cc_lo + (t - rb4 * nch);
            const int r0 = r_lo + 4 * rb4;
            float4 acc[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              acc[i] = r0 + i < rows ? reinterpret_cast<const float4 *>(M + (size_t)(k0 + r0 + i) * lda)[cc]
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int j = 0; j < kb; ++j) {
              const float4 u = reinterpret_cast<const float4 *>(U + j * lda)[cc];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const float l = r0 + i < rows ? P[(r0 + i) * kPLd + j] : 0.f;
                acc[i].x = fmaf(-l, u.x, acc[i].x);
                acc[i].y = fmaf(-l, u.y, acc[i].y);
                acc[i].z = fmaf(-l, u.z, acc[i].z);
                acc[i].w = fmaf(-l, u.w, acc[i].w);
              }
            }
            store_tile(r0, cc, acc);
          }
        }
      }
      __syncthreads();
    }
    qi.iters += 1;
    qi.res_norm = rn;
    qi.precision_used = RB_PREC_MIXED;
    if (!isfinite(rn)) {
      qi.status = RB_Q_NONFINITE;
    } else if (sing) {
      qi.status = RB_Q_SINGULAR;
    } else {
      if (keep && tid == 0) p.Rn[b].x = kept_state(p, b);  // factors and pivots kept for chords
      // back substitution, blocks of 32 rows from the bottom: warp 0 solves the diagonal block,
      // then every thread updates the right-hand side of one row above it (a chord step has
      // its forward-substituted right-hand side in xs already)
      if (!chord)
        for (int i = tid; i < n; i += blockDim.x) xs[i] = M[(size_t)i * lda + n];
      __syncthreads();
      for (int i1 = n; i1 > 0; i1 -= 32) {
        const int i0 = max(0, i1 - 32);
        if (w == 0) {
          const int r = i0 + lane;
          const bool own = r < i1;
          float mrow[32];  // the lane's row of the diagonal block, loaded before the chain
#pragma unroll
          for (int jj = 0; jj < 32; ++jj)
            mrow[jj] = (own && i0 + jj < i1) ? M[(size_t)r * lda + i0 + jj] : 0.f;
          float y = own ? xs[r] : 0.f;
          const float d = own ? __frcp_rn(M[(size_t)r * lda + r]) : 0.f;
#pragma unroll
          for (int jj = 31; jj >= 0; --jj) {
            if (i0 + jj >= i1) continue;
            const float xj = __shfl_sync(0xffffffffu, y * d, jj);
            if (own && lane < jj) y = fmaf(-mrow[jj], xj, y);
          }
          if (own) xs[r] = y * d;
        }
        __syncthreads();
        for (int r = tid; r < i0; r += blockDim.x) {
          const float *row = M + (size_t)r * lda;
          float s = xs[r];
          for (int j = i0; j < i1; ++j) s = fmaf(-row[j], xs[j], s);
          xs[r] = s;
        }
        __syncthreads();
      }
      double dl = 0.0;
      for (int i = tid; i < n; i += blockDim.x) {
        const double d = (double)xs[i];
        dl += d * d;
        ub[i] += d;
        if (p.dU) p.dU[(size_t)b * p.nb + i] = d;
      }
      const double dn = sqrt(block_sum(dl, dred));
      const double prev = qi.upd_norm;
      qi.upd_norm = dn;
      if (!isfinite(dn)) qi.status = RB_Q_NONFINITE;
      else if (rm != kResLow && dn <= p.tol_upd && rn <= p.tol_res * fscale) qi.status = RB_Q_OK;
      if (tid == 0) qi.status = chord_watch(p, b, chord, qi.status, dn, prev);
    }
    if (tid == 0) {
      p.info[b] = qi;
      if (is_active(qi, p.max_iter)) ++my_active;
    }
    __syncthreads();
  }
  if (tid == 0 && my_active) atomicAdd(p.active, my_active);
}

// ---- pressure (Eq. sup-vvar, Eq. blocksolve-2) ----------------------------------------------
// As(mu) u for the converged queries, double-float on the CUDA cores:
//   out[b][k] = sum_q theta^a_q(b) sum_j As_q[k][j] u_b[j].
// A block holds kAsQ queries' u and kAsR rows of one As_q at a time in shared memory; thread
// (b, k) accumulates the dot product of its pair for each q.
constexpr int kAsQ = 16, kAsR = 16;

struct AsuParams {
  DevOps o;
  const double *theta;  // [nq][n_theta]
  const int *nsz;
  int nq, nb;           // nb: the bucket size (columns of As2)
  const double *u;      // [nq][n_max]
  const rb_query_info *info;
  const float2 *As2;    // [q_a][m][nb] double-float
  double *out;          // [b_pad][m]
};

__host__ __device__ inline int odd_ld(int n) { return n | 1; }

__global__ void __launch_bounds__(256) k_as_u(AsuParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  __shared__ float2 ts[kAsQ * RB_Q_MAX];
  __shared__ int flag[kAsQ];
  const DevOps &o = p.o;
  const int nm = p.nb, ldr = odd_ld(nm), m = o.m, qa = o.q_a;
  float2 *us = (float2 *)smb;        // [kAsQ][ldr]
  float2 *as = us + kAsQ * ldr;      // [kAsR][ldr]
  const int tid = threadIdx.x, bi = tid >> 4, ki = tid & 15;
  const int k = blockIdx.x * kAsR + ki;
  for (int g = blockIdx.y; g * kAsQ < p.nq; g += gridDim.y) {
    const int b0 = g * kAsQ;
    __syncthreads();
    if (tid < kAsQ) flag[tid] = b0 + tid < p.nq && p.info[b0 + tid].status == RB_Q_OK;
    __syncthreads();
    int any = 0;
#pragma unroll
    for (int r = 0; r < kAsQ; ++r) any |= flag[r];
    if (!any) continue;
    for (int i = tid; i < kAsQ * nm; i += blockDim.x) {
      const int r = i / nm, j = i - r * nm, b = b0 + r;
      float h = 0.f, l = 0.f;
      if (flag[r] && j < (p.nsz ? p.nsz[b] : nm)) df_split(p.u[(size_t)b * o.n_max + j], h, l);
      us[r * ldr + j] = make_float2(h, l);
    }
    for (int i = tid; i < kAsQ * qa; i += blockDim.x) {
      const int r = i / qa, q = i - r * qa;
      float h = 0.f, l = 0.f;
      if (flag[r]) df_split(p.theta[(size_t)(b0 + r) * o.n_theta + q], h, l);
      ts[i] = make_float2(h, l);
    }
    float ah = 0.f, al = 0.f;
    for (int q = 0; q < qa; ++q) {
      __syncthreads();
      for (int i = tid; i < kAsR * nm; i += blockDim.x) {
        const int r = i / nm, j = i - r * nm, kk = blockIdx.x * kAsR + r;
        as[r * ldr + j] = kk < m ? __ldg(p.As2 + ((size_t)q * m + kk) * nm + j) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      float dh = 0.f, dl = 0.f;
      const float2 *ur = us + bi * ldr, *ar = as + ki * ldr;
#pragma unroll 4
      for (int j = 0; j < nm; ++j) {
        const float2 uu = ur[j], aa = ar[j];
        df_fma(dh, dl, uu.x, uu.y, aa.x, aa.y);
      }
      const float2 t = ts[bi * qa + q];
      df_fma(ah, al, t.x, t.y, dh, dl);
    }
    if (flag[bi] && k < m) p.out[(size_t)(b0 + bi) * m + k] = (double)ah + (double)al;
  }
}

// Pressure solve per converged query: r = fs(mu) - As(mu) u - Cs_mu(u, u) in FP64, B(mu) in
// double-float, B(mu) p = r by FP32 LU plus two steps of iterative refinement with the residual
// r - B(mu) p in double-float (B(mu) is well conditioned, so each step gains the FP32 digits).
struct PresSolveParams {
  DevOps o;
  const double *theta;  // [nq][n_theta]
  int nq;
  const float2 *Bmu;    // [nq][m][m] B(mu) double-float (k_affine_sum)
  const double *Rp;     // [b_pad][m]: Cs_mu(u, u), + As(mu) u when Asu is null (sliced GEMM)
  const double *Asu;    // [b_pad][m]: As(mu) u (k_as_u), or null when Rp includes it
  double *p_out;        // [nq][m]
  rb_query_info *info;
};

constexpr int kPresRefine = 2;

// shared-memory slab of one warp's pressure solve (bytes): B(mu) in double-float (for the
// refinement residuals) and [B | r] in FP32 (row stride aug_ld(m)), factored in place.
struct PresSmem {
  int th, r, pv, pf, Bd, Ba, pseq, stp, total, ldd, lda;
  __host__ __device__ PresSmem(const DevOps &o) {
    const int m = o.m, m4 = (m + 3) & ~3;
    ldd = odd_ld(m);
    lda = aug_ld(m);
    int p = 0;
    th = p; p += 8 * ((o.n_theta + 1) & ~1);
    r = p; p += 8 * m;
    pv = p; p += 8 * m;
    pf = p; p += 8 * m;
    Bd = p; p += 8 * m * ldd;
    p = (p + 15) & ~15;
    Ba = p; p += 4 * m * lda;
    pseq = p; p += 4 * m4;
    stp = p; p += 4 * m4;
    total = (p + 15) & ~15;
  }
};

// B(mu) p = r per converged query, one warp: [fl32(B) | fl32(r)] eliminated by the panel-4 warp
// routine (gepp_aug_warp), which leaves its factors in place; each of the kPresRefine
// refinement steps puts the residual r - B(mu) p (double-float) in the right-hand-side column
// and solves with those factors (chord_solve_warp). R lane slots: m <= 32 R.
template <int R>
__global__ void __launch_bounds__(kThreads) k_pressure_solve_warp(PresSolveParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const DevOps &o = p.o;
  const int m = o.m, mm = m * m;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const PresSmem L(o);
  uint8_t *slab = smb + (size_t)w * L.total;
  double *th = (double *)(slab + L.th), *r = (double *)(slab + L.r), *pv = (double *)(slab + L.pv);
  float2 *pf = (float2 *)(slab + L.pf), *Bd = (float2 *)(slab + L.Bd);
  float *Ba = (float *)(slab + L.Ba);
  int *pseq = (int *)(slab + L.pseq), *stp = (int *)(slab + L.stp);
  const int ldd = L.ldd, lda = L.lda;
  const int c_pad = ((m >> 2) << 2) + 4;  // right-hand side in column m, zero padding to c_pad
  for (int b = blockIdx.x * wpc + w; b < p.nq; b += gridDim.x * wpc) {
    double *prow = p.p_out + (size_t)b * m;
    if (p.info[b].status != RB_Q_OK) {
      for (int i = lane; i < m; i += 32) prow[i] = 0.0;
      continue;
    }
    for (int i = lane; i < o.n_theta; i += 32) th[i] = p.theta[(size_t)b * o.n_theta + i];
    __syncwarp();
    const double *tf = th + o.q_a + o.q_c;
    for (int k = lane; k < m; k += 32) {
      double sf = 0.0;
      for (int q = 0; q < o.q_f; ++q) sf = fma(tf[q], o.fs[(size_t)q * m + k], sf);
      r[k] = sf - p.Rp[(size_t)b * m + k] - (p.Asu ? p.Asu[(size_t)b * m + k] : 0.0);
      float *row = Ba + k * lda;
      row[m] = (float)r[k];
      for (int c = m + 1; c < c_pad; ++c) row[c] = 0.f;
    }
    // B(mu) (double-float, built at the query's start) and its FP32 rounding for the elimination
    {
      const float2 *bq = p.Bmu + (size_t)b * mm;
      for (int e = lane; e < mm; e += 32) {
        const float2 v = __ldg(bq + e);
        const int k = e / m, j = e - k * m;
        Bd[k * ldd + j] = v;
        Ba[k * lda + j] = v.x + v.y;
      }
    }
    __syncwarp();
    float x[R];
    if (gepp_aug_warp<R>(Ba, lda, m, x, pseq)) {
      for (int i = lane; i < m; i += 32) prow[i] = 0.0;
      if (lane == 0) p.info[b].status = RB_Q_SINGULAR;
      __syncwarp();
      continue;
    }
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (lane + 32 * s < m) pv[lane + 32 * s] = (double)x[s];
    __syncwarp();
    bool bad = false;
    for (int it = 0; it < kPresRefine && !bad; ++it) {
      // residual r - B(mu) p, rows owned by lanes, p as double-float pairs
      for (int j = lane; j < m; j += 32) {
        float ph, pl;
        df_split(pv[j], ph, pl);
        pf[j] = make_float2(ph, pl);
      }
      __syncwarp();
      for (int k = lane; k < m; k += 32) {
        float h = 0.f, l = 0.f;
        const float2 *bk = Bd + k * ldd;
        for (int j = 0; j < m; ++j) df_fma(h, l, bk[j].x, bk[j].y, pf[j].x, pf[j].y);
        Ba[k * lda + m] = (float)(r[k] - ((double)h + (double)l));
      }
      __syncwarp();
      bad = chord_solve_warp<R>(Ba, lda, m, pseq, stp, x);
#pragma unroll
      for (int s = 0; s < R; ++s)
        if (!bad && lane + 32 * s < m) pv[lane + 32 * s] += (double)x[s];
      __syncwarp();
    }
    for (int i = lane; i < m; i += 32) prow[i] = pv[i];
    __syncwarp();
  }
}

// Block variant for large m: B(mu) in FP64 and block-cooperative FP64 elimination.
struct PresBlockSmem {
  int th, r, red, Bm, total;
  __host__ __device__ PresBlockSmem(const DevOps &o) {
    int p = 0;
    th = p; p += 8 * ((o.n_theta + 1) & ~1);
    r = p; p += 8 * o.m;
    red = p; p += 8 * 4 * kWarps;
    Bm = p; p += 8 * o.m * o.m;
    total = (p + 15) & ~15;
  }
};

__global__ void __launch_bounds__(kThreads) k_pressure_solve(PresSolveParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const DevOps &o = p.o;
  const int m = o.m;
  const PresBlockSmem L(o);
  double *th = (double *)(smb + L.th), *r = (double *)(smb + L.r);
  double *red = (double *)(smb + L.red), *Bm = (double *)(smb + L.Bm);
  const int tid = threadIdx.x;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    double *prow = p.p_out + (size_t)b * m;
    if (p.info[b].status != RB_Q_OK) {
      for (int i = tid; i < m; i += blockDim.x) prow[i] = 0.0;
      continue;
    }
    for (int i = tid; i < o.n_theta; i += blockDim.x) th[i] = p.theta[(size_t)b * o.n_theta + i];
    __syncthreads();
    const double *tf = th + o.q_a + o.q_c, *tb = tf + o.q_f;
    for (int e = tid; e < m * m; e += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < o.q_b; ++q) s = fma(tb[q], __ldg(o.B + (size_t)q * m * m + e), s);
      Bm[e] = s;
    }
    for (int k = tid; k < m; k += blockDim.x) {
      double sf = 0.0;
      for (int q = 0; q < o.q_f; ++q) sf = fma(tf[q], o.fs[(size_t)q * m + k], sf);
      r[k] = sf - p.Rp[(size_t)b * m + k] - (p.Asu ? p.Asu[(size_t)b * m + k] : 0.0);
    }
    __syncthreads();
    const bool sing = gepp_solve_block<double>(Bm, m, m, r, red);
    for (int i = tid; i < m; i += blockDim.x) prow[i] = sing ? 0.0 : r[i];
    if (sing && tid == 0) p.info[b].status = RB_Q_SINGULAR;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// host side
static void release_state(rb_ctx *ctx, MixedState *M) {
  for (void *q : {(void *)M->Wj, (void *)M->WR.d, (void *)M->WP.d, (void *)M->A2, (void *)M->As2,
                  (void *)M->B2, (void *)M->Dt2, (void *)M->Xj, (void *)M->Xd, (void *)M->xexp, (void *)M->ufT,
                  (void *)M->u2, (void *)M->Jc, (void *)M->Rc, (void *)M->Rp, (void *)M->Th, (void *)M->Fm,
                  (void *)M->Amu, (void *)M->Asu, (void *)M->Bmu, (void *)M->Jaug, (void *)M->Rn,
                  (void *)M->Piv, (void *)M->dU, (void *)M->refresh})
    ctx_free(ctx, q);
  if (M->root == M) {
    for (auto &kv : M->buckets) {
      release_state(ctx, kv.second);
      delete kv.second;
    }
    for (void *q : {(void *)M->dev_words, (void *)M->info_own, (void *)M->perm, (void *)M->n_g,
                    (void *)M->mu_g, (void *)M->theta_g, (void *)M->u_g, (void *)M->p_g,
                    (void *)M->info_g})
      ctx_free(ctx, q);
    if (M->h_words) cudaFreeHost(M->h_words);
    if (M->h_perm) cudaFreeHost(M->h_perm);
    if (M->done_ev) cudaEventDestroy(M->done_ev);
    if (M->perm_ev) cudaEventDestroy(M->perm_ev);
    if (M->gexec) cudaGraphExecDestroy(M->gexec);
    for (cudaStream_t c : M->cap)
      if (c) cudaStreamDestroy(c);
  }
}

void mixed_release(rb_ctx *ctx) {
  MixedState *M = ctx->mixed;
  if (!M) return;
  release_state(ctx, M);
  delete M;
  ctx->mixed = nullptr;
}

// digits of the convection segment (RB_DIGITS) and of the linear segment (RB_DIGITS_LINEAR)
static int sliced_digits(const char *var, int dflt) {
  const char *e = getenv(var);
  const int s = e ? atoi(e) : dflt;
  return std::min(8, std::max(2, s));
}

// Elimination variant forced by RB_ELIMINATION (1 warp per query, 2 / 3 blocked with 32- / 16-
// column panels, 4 CTA per query with a row per thread), where it applies to size nb; 0: none.
static int elim_policy(int nb) {
  const char *e = getenv("RB_ELIMINATION");
  const int k = (e && *e) ? atoi(e) : 0;
  if (k == 1 && nb <= kWarpLuMaxN) return 1;
  if (k == 2 || k == 3) return k;
  if (k == 4 && nb > 32 && nb <= kCtaLuMaxN) return 4;
  return 0;
}

// CTA-pair policy of the tcgen05 GEMMs (RB_GEMM_PAIRS): -1 unset (the autotuner decides; single
// CTAs untuned), 0 single CTAs only, 1 CTA pairs only, 2 CTA pairs with the wide sliced variant
// wherever it applies (nb >= 32).
static int pair_policy() {
  const char *e = getenv("RB_GEMM_PAIRS");
  if (!e || !*e) return -1;
  const int v = atoi(e);
  return v <= 0 ? 0 : (v == 1 ? 1 : 2);
}
constexpr int kWideMinN = 32;  // the wide sliced variant needs nj >= 32 (two row changes per part)
// Untuned defaults (the serving path, RB_AUTOTUNE=0): what the tuner picks on the benchmark
// workloads — CTA pairs for the Jacobian GEMM from n = 40, the wide sliced tiles from n = 32.
static bool use_pairs_plain(const MixedState *M) {
  if (M->tune.klass >= 0) return M->tune.pair_plain != 0;
  const int pol = pair_policy();
  return pol >= 0 ? pol >= 1 : M->nb >= 40;
}
// sliced GEMM variant: 0 single CTAs, 1 CTA pairs, 2 CTA pairs with 256-column tiles
static int sliced_variant(const MixedState *M) {
  if (M->tune.klass >= 0) return M->tune.pair_sliced;
  const int pol = pair_policy();
  if (pol < 0) return M->nb >= kWideMinN ? 2 : 0;
  return pol == 2 ? (M->nb >= kWideMinN ? 2 : 1) : (pol == 1 ? 1 : 0);
}
static cudaError_t launch_sliced(const MixedState *M, const SlicedW &W, const TcGemmParams &g,
                                 int sms, cudaStream_t st, int stages, int variant) {
  if (variant == 2) return launch_tc_gemm(kSlicedWide, M->tmXd, W.tm, g, sms, st, stages, true);
  return launch_tc_gemm(kSliced, M->tmXd, variant == 1 ? W.tm64 : W.tm, g, sms, st, stages, variant == 1);
}

static int absmax_exp(rb_ctx *ctx, MixedState *M, const double *x, size_t count, int *e_out,
                      cudaStream_t st) {
  unsigned long long *mx = (unsigned long long *)(M->root->dev_words + 8);
  cudaMemsetAsync(mx, 0, 8, st);
  k_absmax<<<ctx->sms * 4, 256, 0, st>>>(x, count, mx);
  unsigned long long hm = 0;
  cudaError_t e = cudaMemcpyAsync(&hm, mx, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "operator exponent");
  double dmax;
  memcpy(&dmax, &hm, 8);
  int ex = 0;
  if (dmax > 0) frexp(dmax, &ex);
  *e_out = ex + 1;  // one binade of headroom for the balanced digits
  return RB_OK;
}

// One sliced weight operand at the bucket's size. The grid exponent comes from the whole
// operator (an upper bound for every truncation), so all buckets share one fixed-point grid.
static int build_sliced(rb_ctx *ctx, MixedState *M, SlicedW &W, int kind, int nk,
                        __nv_bfloat16 *Wj, cudaStream_t st) {
  const DevOps &o = ctx->ops;
  W.nk = nk;
  W.Npad = round_up(nk * M->nb, kTcBN);
  void *p;
  int rc = ctx_alloc(ctx, &p, 2 * (size_t)M->Smax * W.Npad * M->Kpad, "W digit slices");
  if (rc != RB_OK) return rc;
  W.d = (__nv_bfloat16 *)p;
  const size_t nm = o.n_max;
  if (kind == 0) {
    if ((rc = absmax_exp(ctx, M, o.Dt, (size_t)o.q_c * nm * nm * nm, &W.wexp[0], st)) != RB_OK) return rc;
    if (M->kb1 && (rc = absmax_exp(ctx, M, o.A, (size_t)o.q_a * nm * nm, &W.wexp[1], st)) != RB_OK) return rc;
  } else {
    if ((rc = absmax_exp(ctx, M, o.Cs, (size_t)o.q_c * nm * nm * o.m, &W.wexp[0], st)) != RB_OK) return rc;
    W.wexp[0] += 1;  // the operand holds 2 Cs
    if (M->kb1 && (rc = absmax_exp(ctx, M, o.As, (size_t)o.q_a * o.m * nm, &W.wexp[1], st)) != RB_OK) return rc;
  }
  BuildWParams bw{o, kind, M->nb, nk, M->Kpad0, M->Kpad, W.Npad, M->S0, M->S1, W.wexp[0], W.wexp[1], W.d, Wj};
  k_build_w<<<ctx->sms * 8, 256, 0, st>>>(bw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_build_w");
  if (!make_map(&W.tm, W.d, (uint64_t)M->Smax * W.Npad, M->Kpad, kTcBN) ||
      !make_map(&W.tm64, W.d, (uint64_t)M->Smax * W.Npad, M->Kpad, kTcBN / 2))
    return set_error(ctx, RB_ERR_CUDA, "tensor map encode (W)");
  return RB_OK;
}

// The root state (nb = n_max) with the shared words; its layouts are built on first use.
static int mixed_root(rb_ctx *ctx, cudaStream_t st) {
  if (ctx->mixed) return RB_OK;
  if (!encode_fn()) return set_error(ctx, RB_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if (ctx->cc_major != 10) return set_error(ctx, RB_ERR_ARG, "tensor-core path needs an sm_10x GPU");
  MixedState *M = new MixedState();
  M->root = M;
  M->nb = ctx->ops.n_max;
  ctx->mixed = M;
  void *p;
  int rc;
  if ((rc = ctx_alloc(ctx, &p, 64, "mixed words")) != RB_OK) return rc;
  M->dev_words = (int *)p;
  cudaMemsetAsync(M->dev_words, 0, 64, st);
  if (cudaMallocHost(&M->h_words, 64) != cudaSuccess) return set_error(ctx, RB_ERR_OOM, "pinned words");
  memset(M->h_words, 0, 64);
  if (cudaEventCreateWithFlags(&M->done_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&M->perm_ev, cudaEventDisableTiming) != cudaSuccess)
    return set_error(ctx, RB_ERR_CUDA, "solve events");
  return RB_OK;
}

// Build the operator layouts of one bucket (once per operator set and bucket size).
static int mixed_layouts(rb_ctx *ctx, MixedState *M, cudaStream_t st) {
  if (M->Wj) return RB_OK;
  const DevOps &o = ctx->ops;
  M->Kpad0 = round_up(o.q_c * M->nb, 64);
  M->kb0 = M->Kpad0 / 64;
  M->S0 = sliced_digits("RB_DIGITS", 5);
  M->S1 = sliced_digits("RB_DIGITS_LINEAR", 7);
  // K segment 1 (theta^a (x) the linear operator, one block of 64: Q_a <= RB_Q_MAX) serves the
  // pressure right-hand side only: there the sliced GEMM gives Cs_mu(u, u) + As(mu) u in one
  // launch, where the CUDA cores would take Q_a m n double-float multiply-adds per query
  // (about 6 us per unit of Q_a at n = 50, m = 30, 4096 queries) and the GEMM pays one tile
  // contraction per digit level of the segment (about 12 us each): taken when Q_a > 2 S1. The
  // residual's linear term A(mu) u stays in double-float on the CUDA cores (its launches use
  // segment 0 only): a chord step's increment would need that segment contracted with d and all
  // of its digit pairs at every step.
  M->kb1 = (o.m > 0 && o.B && o.As && o.q_a > 2 * M->S1) ? 1 : 0;
  M->Kpad = M->Kpad0 + 64 * M->kb1;
  M->Npad = round_up(M->nb * M->nb, kTcBN);
  M->Smax = M->kb1 ? std::max(M->S0, M->S1) : M->S0;
  int rc;
  void *p;
  const int nm = o.n_max, nb = M->nb;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)o.q_a * nb * nb, "A (double-float)")) != RB_OK) return rc;
  M->A2 = (float2 *)p;
  k_split_trunc<<<ctx->sms * 4, 256, 0, st>>>(o.A, M->A2, o.q_a, nb, nm, nm, nb);
  if (o.m > 0 && o.B) {
    if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)o.q_a * o.m * nb, "As (double-float)")) != RB_OK) return rc;
    M->As2 = (float2 *)p;
    k_split_trunc<<<ctx->sms * 4, 256, 0, st>>>(o.As, M->As2, o.q_a, o.m, o.m, nm, nb);
    if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)o.q_b * o.m * o.m, "B (double-float)")) != RB_OK) return rc;
    M->B2 = (float2 *)p;
    k_split_f2<<<ctx->sms * 4, 256, 0, st>>>(o.B, M->B2, (size_t)o.q_b * o.m * o.m);
  }
  if ((rc = ctx_alloc(ctx, &p, 2 * 2 * (size_t)M->Npad * M->Kpad0, "W (split BF16)")) != RB_OK) return rc;
  M->Wj = (__nv_bfloat16 *)p;
  if ((rc = build_sliced(ctx, M, M->WR, 0, M->nb, M->Wj, st)) != RB_OK) return rc;
  if (o.m > 0 && o.B && (rc = build_sliced(ctx, M, M->WP, 1, o.m, nullptr, st)) != RB_OK) return rc;
  if (!make_map(&M->tmWj, M->Wj, 2 * (uint64_t)M->Npad, M->Kpad0, kTcBN))
    return set_error(ctx, RB_ERR_CUDA, "tensor map encode (Wj)");
  M->root->epoch += 1;
  return RB_OK;
}

// Bucket size of a query of size n: n rounded up to 8 (n <= 64), 16 (n <= 128) or 32, at most
// n_max. The bucket's layouts are built on its first use.
static int bucket_size(int n, int n_max) {
  const int g = n <= 64 ? 8 : (n <= 128 ? 16 : 32);
  return std::min((n + g - 1) / g * g, n_max);
}

static MixedState *bucket(rb_ctx *ctx, int nb) {
  MixedState *R = ctx->mixed;
  if (nb >= R->nb) return R;
  auto it = R->buckets.find(nb);
  if (it != R->buckets.end()) return it->second;
  MixedState *M = new MixedState();
  M->root = R;
  M->nb = nb;
  M->dev_words = R->dev_words;
  M->h_words = R->h_words;
  R->buckets[nb] = M;
  return M;
}

static int mixed_batch_scratch(rb_ctx *ctx, MixedState *M, int nq) {
  const int b_pad = round_up(std::max(nq, 1), 256);  // whole 256-row tiles of a CTA pair
  if (b_pad <= M->bcap) return RB_OK;
  for (void *q : {(void *)M->Xj, (void *)M->Xd, (void *)M->xexp, (void *)M->ufT, (void *)M->u2, (void *)M->Jc,
                  (void *)M->Rc, (void *)M->Rp, (void *)M->Th, (void *)M->Fm, (void *)M->Amu,
                  (void *)M->Asu, (void *)M->Bmu, (void *)M->Jaug, (void *)M->Rn, (void *)M->Piv,
                  (void *)M->dU, (void *)M->refresh})
    ctx_free(ctx, q);
  M->Jaug = nullptr;
  M->Piv = nullptr;
  M->dU = nullptr;
  M->refresh = nullptr;
  M->Bmu = nullptr;
  M->Rn = nullptr;
  M->Rg = nullptr;
  M->Xj = M->Xd = nullptr; M->xexp = nullptr; M->ufT = nullptr; M->u2 = nullptr; M->Jc = nullptr;
  M->Rc = M->Rp = M->Th = M->Fm = M->Asu = nullptr;
  M->Amu = nullptr;
  M->bcap = 0;
  int rc;
  void *p;
  const int m = std::max(ctx->ops.m, 1);
  const size_t xs0 = (size_t)b_pad * M->Kpad0, xs = (size_t)b_pad * M->Kpad;
  if ((rc = ctx_alloc(ctx, &p, 2 * 3 * xs0, "X (split BF16)")) != RB_OK) return rc;
  M->Xj = (__nv_bfloat16 *)p;
  if ((rc = ctx_alloc(ctx, &p, 2 * xs * M->Smax, "X digit slices")) != RB_OK) return rc;
  M->Xd = (__nv_bfloat16 *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad, "X exponents")) != RB_OK) return rc;
  M->xexp = (int *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb, "u (float pairs)")) != RB_OK) return rc;
  M->ufT = (float2 *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb, "u (double-float)")) != RB_OK) return rc;
  M->u2 = (float2 *)p;
  if ((rc = ctx_alloc(ctx, &p, 4 * (size_t)b_pad * M->Npad, "J^c (FP32)")) != RB_OK) return rc;
  M->Jc = (float *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb, "R (FP64)")) != RB_OK) return rc;
  M->Rc = (double *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * m, "pressure rhs (FP64)")) != RB_OK) return rc;
  M->Rp = (double *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * ctx->ops.n_theta, "theta rows")) != RB_OK) return rc;
  M->Th = (double *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb, "f(mu)")) != RB_OK) return rc;
  M->Fm = (double *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb * M->nb, "A(mu) (double-float)")) != RB_OK) return rc;
  M->Amu = (float2 *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * m, "As(mu) u")) != RB_OK) return rc;
  M->Asu = (double *)p;
  if (ctx->ops.m > 0 && ctx->ops.B) {
    if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * ctx->ops.m * ctx->ops.m, "B(mu) (double-float)")) != RB_OK)
      return rc;
    M->Bmu = (float2 *)p;
  }
  if ((rc = ctx_alloc(ctx, &p, 4 * (size_t)b_pad * M->nb, "pivot rows")) != RB_OK) return rc;
  M->Piv = (int *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb, "last updates")) != RB_OK) return rc;
  M->dU = (double *)p;
  if ((rc = ctx_alloc(ctx, &p, 16, "refresh word")) != RB_OK) return rc;
  M->refresh = (int *)p;
  cudaMemsetAsync(M->refresh, 0, 16, ctx->stream);
  if ((rc = ctx_alloc(ctx, &p, 4 * (size_t)b_pad * M->nb * aug_ld(M->nb), "Newton systems")) != RB_OK) return rc;
  M->Jaug = (float *)p;
  const size_t groups = (size_t)(M->nb + 7) / 8;
  if ((rc = ctx_alloc(ctx, &p, 16 * (size_t)b_pad + 8 * (size_t)b_pad * groups, "residual norms")) != RB_OK)
    return rc;
  M->Rn = (double2 *)p;
  M->Rg = (double *)(M->Rn + b_pad);
  // zero once so that padded rows never hold NaN bit patterns
  cudaMemsetAsync(M->Xj, 0, 2 * 3 * xs0, ctx->stream);
  cudaMemsetAsync(M->Xd, 0, 2 * xs * M->Smax, ctx->stream);
  cudaMemsetAsync(M->xexp, 0, 8 * (size_t)b_pad, ctx->stream);
  cudaMemsetAsync(M->ufT, 0, 8 * (size_t)b_pad * M->nb, ctx->stream);
  cudaMemsetAsync(M->u2, 0, 8 * (size_t)b_pad * M->nb, ctx->stream);
  if (!make_map(&M->tmXj, M->Xj, 3 * (uint64_t)b_pad, M->Kpad0, 128) ||
      !make_map(&M->tmXd, M->Xd, (uint64_t)M->Smax * b_pad, M->Kpad, 128))
    return set_error(ctx, RB_ERR_CUDA, "tensor map encode (X)");
  M->bcap = b_pad;
  M->root->epoch += 1;
  return RB_OK;
}

static int launch_build_x(rb_ctx *ctx, MixedState *M, int nq, const int *d_n, const double *d_u,
                          const rb_query_info *d_info, int mode, int digits, double *out, int nout,
                          cudaStream_t st, int split = 1, int incr = 0) {
  BuildXParams bx{};
  bx.split = split;
  bx.incr = incr;
  bx.dU = M->dU;
  bx.lmax = M->root->dev_words + 6;
  bx.o = ctx->ops;
  bx.theta = M->Th;
  bx.nsz = d_n;
  bx.nq = nq;
  bx.nb = M->nb;
  bx.Kpad0 = M->Kpad0;
  bx.Kpad = M->Kpad;
  bx.S0 = M->S0;
  bx.S1 = M->S1;
  bx.b_pad = M->bcap;
  bx.max_iter = ctx->cfg.max_iter;
  bx.mode = mode;
  bx.digits = digits;
  bx.u = d_u;
  bx.info = d_info;
  bx.Xj = M->Xj;
  bx.Xd = M->Xd;
  bx.xexp = M->xexp;
  bx.ufT = M->ufT;
  bx.u2 = M->u2;
  bx.out = out;
  bx.nout = nout;
  const int mk = prof_begin(ctx, RB_K_BUILD_X, st);
  k_build_x<<<std::max(1, std::min((nq + kWarps - 1) / kWarps, ctx->sms * 8)), kThreads, 0, st>>>(bx);
  prof_end(ctx, mk, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_build_x");
  return RB_OK;
}

static TcGemmParams gemm_params(MixedState *M, int nq) {
  TcGemmParams g{};
  g.m_tiles = round_up(nq, 128) / 128;
  g.S[0] = M->S0;
  g.S[1] = M->S1;
  g.b_pad = M->bcap;
  g.nq = nq;
  g.nj = M->nb;
  g.xexp = M->xexp;
  g.ufT = M->ufT;
  g.err = M->root->dev_words + 1;
  return g;
}

// theta rows, f(mu) and A(mu) of the queries that start (active, iteration count 0).
static int launch_prep(rb_ctx *ctx, MixedState *M, const double *d_mu, const double *d_theta,
                       int nq, const int *nsz, const rb_query_info *info, cudaStream_t st,
                       int all = 0) {
  const DevOps &o = ctx->ops;
  PrepParams pp{};
  pp.o = o;
  pp.mu = d_mu;
  pp.theta_in = d_theta;
  pp.nq = nq;
  pp.nb = M->nb;
  pp.max_iter = ctx->cfg.max_iter;
  pp.info = info;
  pp.Th = M->Th;
  pp.Fm = M->Fm;
  pp.nsz = nsz;
  pp.Rn = M->Rn;
  pp.all = all;
  const int mk = prof_begin(ctx, RB_K_PREP, st);
  k_prep_theta<<<std::max(1, std::min((nq + kPrepQ - 1) / kPrepQ, ctx->sms * 16)), 256, 0, st>>>(pp);
  auto affine = [&](const float2 *Q2, int qn, int th_off, size_t nn, float2 *out) {
    AffineParams ap{nq, ctx->cfg.max_iter, all, o.n_theta, th_off, qn, nn, info, M->Th, Q2, out};
    dim3 grid((unsigned)std::min<size_t>((nn + 255) / 256, 1024),
              (unsigned)std::max(1, std::min((nq + kAsmQ - 1) / kAsmQ, 65535)));
    k_affine_sum<<<grid, 256, sizeof(float2) * kAsmQ * qn, st>>>(ap);
  };
  affine(M->A2, o.q_a, 0, (size_t)M->nb * M->nb, M->Amu);  // A(mu), theta^a
  if (M->B2 && M->Bmu)                                      // B(mu), theta^b
    affine(M->B2, o.q_b, o.q_a + o.q_c + o.q_f, (size_t)o.m * o.m, M->Bmu);
  prof_end(ctx, mk, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_affine_sum");
  return RB_OK;
}

// One Newton step's contraction work for the whole batch: X build + both GEMMs.
// The contractions one Newton iteration needs: the Jacobian GEMM (jac) and the FP64-accurate
// residual's sliced GEMM (exact).
// The Jacobian and sliced GEMMs cover the first nq_jac / nq_exact rows of the batch (all nq by
// default): the server orders a group's queries by iteration count, so only the rows that need
// a contraction get one (rows past them may take overhanging tile rows, which their rung never
// reads).
// incr (chord steps, no Jacobian): the residual's convection part is updated by the increment
// C(u, u) = C(u - d, u - d) + J^c(d) (u - d / 2) from the previous iteration's one (exact in
// exact arithmetic: C is quadratic), with as many digit levels as d's size needs.
static int mixed_contract(rb_ctx *ctx, MixedState *M, int nq, const int *d_n, const double *d_u,
                          const rb_query_info *d_info, bool jac, bool exact, cudaStream_t st,
                          int nq_jac = -1, int nq_exact = -1, bool incr = false) {
  if (!jac && !exact) return RB_OK;
  if (incr) {
    cudaError_t e0 = cudaMemsetAsync(M->root->dev_words + 6, 0, 4, st);
    if (e0 != cudaSuccess) return cuda_fail(ctx, e0, "words");
  }
  // a chord step (incr, no Jacobian) still contracts the Jacobian when one of its queries asked
  // for a fresh one (the bucket's refresh word, read on the device)
  const bool cond_jac = incr && !jac && M->refresh;
  int rc = launch_build_x(ctx, M, nq, d_n, d_u, d_info, 0, exact ? 1 : 0, M->Rc, M->nb, st,
                          (jac || cond_jac) ? 1 : 0, incr && exact && !jac ? 1 : 0);
  if (rc != RB_OK) return rc;
  TcGemmParams g = gemm_params(M, nq_jac >= 0 ? nq_jac : nq);
  g.n_tiles = M->Npad / kTcBN;
  g.kb[0] = M->kb0;
  g.kb[1] = 0;
  g.n_pad = M->Npad;
  g.nk = M->nb;
  g.ldj = M->Npad;
  g.Jc = M->Jc;
  g.nsplit = 3;
  int mk;
  cudaError_t e;
  if (cond_jac) g.run_if = M->refresh;
  if (jac || cond_jac) {
    // RB_TEST_WAIT_DEFICIT=1 (tests of the failure path only): the single-CTA Jacobian GEMM's
    // first stage waits for 16 bytes that never come, so the bounded wait gives up
    const char *td = getenv("RB_TEST_WAIT_DEFICIT");
    g.tx_extra = (td && atoi(td) == 1 && !use_pairs_plain(M)) ? 16u : 0u;
    g.issued = prof_issued(ctx, RB_K_GEMM_JAC);
    mk = prof_begin(ctx, RB_K_GEMM_JAC, st);
    e = launch_tc_gemm(kPlain, M->tmXj, M->tmWj, g, ctx->sms, st, M->tune.st_plain, use_pairs_plain(M));
    prof_end(ctx, mk, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_tc_gemm (Jacobian)");
  }
  if (!exact) return RB_OK;
  if (nq_exact >= 0) {
    const TcGemmParams ge = gemm_params(M, nq_exact);
    g.m_tiles = ge.m_tiles;
    g.nq = ge.nq;
  } else {
    const TcGemmParams ge = gemm_params(M, nq);
    g.m_tiles = ge.m_tiles;
    g.nq = ge.nq;
  }
  g.tx_extra = 0;
  g.run_if = nullptr;
  g.kb[1] = 0;  // convection only: A(mu) u is added in the assembly
  g.n_tiles = M->WR.Npad / kTcBN;
  g.n_pad = M->WR.Npad;
  g.wexp[0] = M->WR.wexp[0];
  g.wexp[1] = M->WR.wexp[1];
  g.out = M->Rc;
  if (incr && !jac) g.lmax = M->root->dev_words + 6;
  g.issued = prof_issued(ctx, RB_K_GEMM_RES);
  mk = prof_begin(ctx, RB_K_GEMM_RES, st);
  e = launch_sliced(M, M->WR, g, ctx->sms, st, M->tune.st_sliced, sliced_variant(M));
  prof_end(ctx, mk, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_tc_gemm (residual)");
  return RB_OK;
}

static int launch_elimination(rb_ctx *ctx, MixedState *M, LuParams &lp, int nq, cudaStream_t st,
                              int kind);

// Elimination variant of a bucket: the tuned one, else the forced one, else the default (warp
// per query up to n = 80, CTA per query up to 128, blocked above).
static int elim_kind(const MixedState *M) {
  if (M->tune.lu) return M->tune.lu;
  const int epol = elim_policy(M->nb);
  return epol ? epol : (M->nb <= kWarpLuMaxN ? 1 : (M->nb <= kCtaLuMaxN ? 4 : 2));
}
// Chord steps (Jacobian reuse from the second FP64-residual iteration on): every elimination
// kernel keeps its factors and pivots when asked (warp, CTA per query, blocked); RB_CHORD=0
// turns them off.
// Chord steps take the residual's convection part as an increment on the previous one
// (RB_INCREMENT=0: the full product at every step).
static bool incr_residual() {
  const char *e = getenv("RB_INCREMENT");
  return !(e && *e && atoi(e) == 0);
}

static bool bucket_chord(const MixedState *M) {
  const char *e = getenv("RB_CHORD");
  if (e && *e && atoi(e) == 0) return false;
  const int k = elim_kind(M);
  return (k == 1 && M->nb <= kWarpLuMaxN) || (k == 4 && M->nb <= kCtaLuMaxN) || k == 2 || k == 3;
}

// Newton step of the batch: k_newton_system assembles [J | -R] per query, then one warp
// (nb <= 80) or one CTA (blocked elimination) per query solves it, as the autotuner chose.
static int launch_lu(rb_ctx *ctx, MixedState *M, LuParams &lp, int nq, cudaStream_t st) {
  lp.Amu = M->Amu;
  lp.Fm = M->Fm;
  lp.Jaug = M->Jaug;
  lp.Rn = M->Rn;
  lp.Rg = M->Rg;
  lp.lda = aug_ld(M->nb);
  {
    // one warp per (query, 8-row group), two blocks of 8 warps per SM, grid-stride
    const long long units = (long long)nq * ((M->nb + 7) / 8);
    const int grid = (int)std::max(1LL, std::min((units + kWarps - 1) / kWarps, 2LL * ctx->sms));
    const int mk = prof_begin(ctx, RB_K_SYSTEM, st);
    const int fixed = lp.eval_only ? -1 : lp.rung_all;
    const long long per_sm = system_blocks(fixed);
    const int grid2 = (int)std::max(1LL, std::min((units + kWarps - 1) / kWarps, per_sm * ctx->sms));
    if (lp.eval_only) k_newton_system<true, -1><<<grid, kThreads, 0, st>>>(lp);
    else if (fixed == 0) k_newton_system<false, 0><<<grid2, kThreads, 0, st>>>(lp);
    else if (fixed == 1) k_newton_system<false, 1><<<grid2, kThreads, 0, st>>>(lp);
    else if (fixed == 2) k_newton_system<false, 2><<<grid2, kThreads, 0, st>>>(lp);
    else if (fixed == 3) k_newton_system<false, 3><<<grid2, kThreads, 0, st>>>(lp);
    else k_newton_system<false, -1><<<grid, kThreads, 0, st>>>(lp);
    if (fixed == 3 && lp.refresh) {
      // the queries whose last chord step asked for a fresh Jacobian; then the word is cleared
      // for the chord steps of this iteration to raise again
      LuParams lr = lp;
      lr.run_if = lp.refresh;
      k_newton_system<false, 4><<<grid, kThreads, 0, st>>>(lr);
      cudaMemsetAsync(lp.refresh, 0, 4, st);
    }
    prof_end(ctx, mk, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_newton_system");
  }
  if (lp.eval_only) return RB_OK;
  return launch_elimination(ctx, M, lp, nq, st, elim_kind(M));
}

template <int PB>
static cudaError_t launch_blocked(const rb_ctx *ctx, const LuParams &lp, int nq, cudaStream_t st) {
  const size_t smem = BlkLuSmem<PB>(lp.nb, lp.lda).total;
  cudaError_t e = cudaFuncSetAttribute(k_lu_blocked<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_blocked<PB>, kThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(nq, std::max(1, per_sm) * ctx->sms));
  k_lu_blocked<PB><<<grid, kThreads, smem, st>>>(lp);
  return cudaGetLastError();
}

// Elimination variant `kind`: 1 warp per query (nb <= 80), 2 blocked (32-column panels),
// 3 blocked (16-column panels).
static int launch_elimination(rb_ctx *ctx, MixedState *M, LuParams &lp, int nq, cudaStream_t st,
                              int kind) {
  if (kind == 4 && M->nb <= kCtaLuMaxN) {
    const size_t smem = CtaLuSmem(M->nb, lp.lda).total;
    const int threads = 32 * ((M->nb + 31) / 32);
    cudaError_t e = cudaFuncSetAttribute(k_lu_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lu_cta, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_cta, threads, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_cta attr");
    const int grid = std::max(1, std::min(nq, std::max(1, per_sm) * ctx->sms));
    const int mk = prof_begin(ctx, RB_K_LU, st);
    k_lu_cta<<<grid, threads, smem, st>>>(lp);
    prof_end(ctx, mk, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_cta");
    return RB_OK;
  }
  if (kind >= 2 || M->nb > kWarpLuMaxN) {
    const int mk = prof_begin(ctx, RB_K_LU, st);
    const cudaError_t e = kind == 3 ? launch_blocked<16>(ctx, lp, nq, st) : launch_blocked<32>(ctx, lp, nq, st);
    prof_end(ctx, mk, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_blocked");
    return RB_OK;
  }
  // warps per block: the most resident warps per SM (shared memory and registers)
  const int per_warp = WarpLuSmem(M->nb, lp.lda).per_warp;
  const bool two = M->nb <= 64;
  const void *kern = two ? (const void *)k_lu_mixed_warp<2> : (const void *)k_lu_mixed_warp<3>;
  int wpc = 1, best = 0, best_blocks = 1;
  for (int c = 1; c <= kLuWarpBlock / 32; ++c) {
    const size_t sm = (size_t)c * per_warp;
    if (sm > (size_t)ctx->max_smem) break;
    int blocks = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * c, sm) != cudaSuccess)
      return cuda_fail(ctx, cudaGetLastError(), "k_lu_mixed_warp occupancy");
    if (blocks * c > best) {
      best = blocks * c;
      best_blocks = std::max(1, blocks);
      wpc = c;
    }
  }
  const size_t smem = (size_t)wpc * per_warp;
  const int grid = std::max(1, std::min((nq + wpc - 1) / wpc, best_blocks * ctx->sms));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_mixed_warp attr");
  const int mk = prof_begin(ctx, RB_K_LU, st);
  if (two) k_lu_mixed_warp<2><<<grid, 32 * wpc, smem, st>>>(lp);
  else k_lu_mixed_warp<3><<<grid, 32 * wpc, smem, st>>>(lp);
  prof_end(ctx, mk, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_mixed_warp");
  return RB_OK;
}

static rb_query_info *own_info(rb_ctx *ctx, int nq) {
  MixedState *M = ctx->mixed;
  if (M->info_cap < nq) {
    ctx_free(ctx, M->info_own);
    M->info_own = nullptr;
    M->info_cap = 0;
    void *p;
    if (ctx_alloc(ctx, &p, sizeof(rb_query_info) * (size_t)nq, "info") != RB_OK) return nullptr;
    M->info_own = (rb_query_info *)p;
    M->info_cap = nq;
  }
  return M->info_own;
}

static int check_words(rb_ctx *ctx, cudaStream_t st, const char *what) {
  MixedState *M = ctx->mixed;
  cudaError_t e = cudaMemcpyAsync(M->h_words, M->dev_words, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  if (M->h_words[1])
    return set_error(ctx, RB_ERR_TIMEOUT, "%s: tensor-core pipeline wait gave up (code %d)", what,
                     M->h_words[1]);
  return RB_OK;
}

static int mixed_pressure(rb_ctx *ctx, MixedState *M, int nq, const int *d_n, const double *d_u,
                          double *d_p, rb_query_info *info, cudaStream_t st) {
  const DevOps &o = ctx->ops;
  int rc = launch_build_x(ctx, M, nq, d_n, d_u, info, 1, 1, M->Rp, o.m, st);
  if (rc != RB_OK) return rc;
  TcGemmParams g = gemm_params(M, nq);
  g.kb[0] = M->kb0;
  g.kb[1] = M->kb1;
  g.n_tiles = M->WP.Npad / kTcBN;
  g.n_pad = M->WP.Npad;
  g.nk = o.m;
  g.wexp[0] = M->WP.wexp[0];
  g.wexp[1] = M->WP.wexp[1];
  g.out = M->Rp;
  g.issued = prof_issued(ctx, RB_K_GEMM_PRES);
  int mk = prof_begin(ctx, RB_K_GEMM_PRES, st);
  cudaError_t e = launch_sliced(M, M->WP, g, ctx->sms, st, M->tune.st_sliced, sliced_variant(M));
  prof_end(ctx, mk, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_tc_gemm (pressure)");
  mk = prof_begin(ctx, RB_K_PRESSURE, st);
  if (!M->kb1) {  // As(mu) u not in the GEMM's output: in double-float on the CUDA cores
    AsuParams ap{o, M->Th, d_n, nq, M->nb, d_u, info, M->As2, M->Asu};
    const size_t asmem = sizeof(float2) * (size_t)(kAsQ + kAsR) * odd_ld(M->nb);
    e = cudaFuncSetAttribute(k_as_u, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asmem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_as_u attr");
    dim3 agrid((unsigned)((o.m + kAsR - 1) / kAsR), (unsigned)std::max(1, std::min((nq + kAsQ - 1) / kAsQ, 65535)));
    k_as_u<<<agrid, 256, asmem, st>>>(ap);
  }
  PresSolveParams pp{o, M->Th, nq, M->Bmu, M->Rp, M->kb1 ? nullptr : M->Asu, d_p, info};
  const size_t per_warp = PresSmem(o).total;
  if (o.m <= 32 * kWarpRows && per_warp <= 24 * 1024) {
    const int wpc = std::max(1, std::min(8, (int)((192 * 1024) / per_warp)));
    const size_t smem = wpc * per_warp;
    auto kern = o.m <= 32 ? k_pressure_solve_warp<1> : (o.m <= 64 ? k_pressure_solve_warp<2> : k_pressure_solve_warp<3>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_pressure_solve_warp attr");
    kern<<<std::max(1, std::min((nq + wpc - 1) / wpc, ctx->sms * 8)), 32 * wpc, smem, st>>>(pp);
  } else {
    const size_t smem = PresBlockSmem(o).total;
    e = cudaFuncSetAttribute(k_pressure_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_pressure_solve attr");
    k_pressure_solve<<<std::max(1, std::min(nq, ctx->sms * 8)), kThreads, smem, st>>>(pp);
  }
  prof_end(ctx, mk, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_pressure_solve");
  return RB_OK;
}

// ---- one batch solve ----------------------------------------------------------------------
// The batch is split into size buckets (contiguous ranges of a bucket-sorted copy, or the
// caller's buffers themselves when every query uses the n_max layouts); the pieces below are run
// by the stream path with a host check per iteration and captured once by the graph path.
struct SolveArgs {
  const double *mu, *theta;
  int nq;
  const int *n;
  double *u, *p;
  rb_query_info *info;
};

struct Part {
  MixedState *M;
  SolveArgs a;
};

static LuParams solve_lu_params(rb_ctx *ctx, MixedState *M, const SolveArgs &a) {
  LuParams lp{};
  lp.o = ctx->ops;
  lp.nsz = a.n;
  lp.nq = a.nq;
  lp.nb = M->nb;
  lp.ldj = M->Npad;
  lp.max_iter = ctx->cfg.max_iter;
  lp.tol_upd = ctx->cfg.tol_update;
  lp.tol_res = ctx->cfg.tol_res;
  lp.Jc = M->Jc;
  lp.Rc = M->Rc;
  lp.u = a.u;
  lp.u2 = M->u2;
  lp.info = a.info;
  lp.active = M->root->dev_words;  // one active count over all buckets
  lp.rmode = kResLadder;  // every query climbs zero -> low -> exact with its own iterations
  lp.chord = bucket_chord(M) ? 1 : 0;
  lp.Piv = M->Piv;
  lp.dU = lp.chord && incr_residual() ? M->dU : nullptr;
  lp.refresh = lp.chord && incr_residual() ? M->refresh : nullptr;
  lp.escalate = lp.refresh ? M->refresh + 1 : nullptr;
  lp.rung_all = -1;
  return lp;
}

// words[0] active count of the last iteration, [1] error word, [2] iterations done
static int solve_prologue(rb_ctx *ctx, const std::vector<Part> &parts, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ctx->mixed->dev_words, 0, 16, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "words");
  for (const Part &pt : parts) {
    const SolveArgs &a = pt.a;
    const int mk = prof_begin(ctx, RB_K_INIT, st);
    k_mixed_init<<<std::max(1, std::min(a.nq, ctx->sms * 8)), 128, 0, st>>>(a.nq, ctx->ops.n_max, a.n, a.u, a.info);
    prof_end(ctx, mk, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_mixed_init");
    const int rc = launch_prep(ctx, pt.M, a.mu, a.theta, a.nq, a.n, a.info, st);
    if (rc != RB_OK) return rc;
    if (pt.M->refresh && (e = cudaMemsetAsync(pt.M->refresh, 0, 8, st)) != cudaSuccess)
      return cuda_fail(ctx, e, "refresh word");
  }
  return RB_OK;
}

// Newton iteration `it` of every bucket (0: u = 0, 1: low-precision residual, 2: FP64-accurate
// residual, 3: the same, a chord step where the bucket keeps its factors; the kernels pick each
// query's rung from its own iteration count).
static int solve_iteration(rb_ctx *ctx, const std::vector<Part> &parts, int it, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ctx->mixed->dev_words, 0, 4, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "words");
  int rc;
  for (const Part &pt : parts) {
    const bool chord = it >= 3 && bucket_chord(pt.M);
    const bool jac = it >= 1 && !chord;
    if ((rc = mixed_contract(ctx, pt.M, pt.a.nq, pt.a.n, pt.a.u, pt.a.info, jac, it >= 2, st, -1, -1,
                             chord && incr_residual())) != RB_OK)
      return rc;
    LuParams lp = solve_lu_params(ctx, pt.M, pt.a);
    // every active query of a batch solve is on iteration `it`
    lp.rung_all = it == 0 ? 0 : (it == 1 ? 1 : (it >= 3 && lp.chord ? 3 : 2));
    if ((rc = launch_lu(ctx, pt.M, lp, pt.a.nq, st)) != RB_OK) return rc;
  }
  return RB_OK;
}

// The queries whose chord steps stalled even with a refreshed Jacobian (status kQEscalate) are
// solved by the FP64 Newton, one CTA per query; a bucket where no query was handed over returns
// at once (its escalation word is 0).
static int escalation_grid(const rb_ctx *ctx, int nq) { return std::max(1, std::min(nq, ctx->sms)); }

// the FP64 Jacobians of the escalation's CTAs, when they do not fit in shared memory: sized for
// the largest grid once, so that a captured graph's pointer stays valid
static int escalation_scratch(rb_ctx *ctx) {
  const DevOps &o = ctx->ops;
  if (fp64_smem_bytes(o, true) <= (size_t)ctx->max_smem) return RB_OK;
  void *before = ctx->jscratch.ptr;
  const int rc = ctx->jscratch.reserve(ctx, sizeof(double) * (size_t)ctx->sms * o.n_max * o.n_max,
                                       "FP64 Jacobian scratch");
  if (rc == RB_OK && ctx->jscratch.ptr != before) ctx->mixed->epoch += 1;
  return rc;
}

static int solve_escalated(rb_ctx *ctx, const std::vector<Part> &parts, cudaStream_t st) {
  const DevOps &o = ctx->ops;
  for (const Part &pt : parts) {
    if (!pt.M->refresh || !bucket_chord(pt.M) || !incr_residual()) continue;
    NewtonParams np{};
    np.o = o;
    np.mu = pt.a.theta ? nullptr : pt.a.mu;
    np.theta = pt.a.theta;
    np.nsz = pt.a.n;
    np.nq = pt.a.nq;
    np.max_iter = ctx->cfg.max_iter;
    np.tol_upd = ctx->cfg.tol_update;
    np.tol_res = ctx->cfg.tol_res;
    np.u_out = pt.a.u;
    np.info = pt.a.info;
    np.j_in_smem = fp64_smem_bytes(o, true) <= (size_t)ctx->max_smem ? 1 : 0;
    if (!np.j_in_smem) {
      if (ctx->jscratch.cap < sizeof(double) * (size_t)escalation_grid(ctx, pt.a.nq) * o.n_max * o.n_max)
        return set_error(ctx, RB_ERR_STATE, "escalation scratch not reserved");
      np.jscratch = (double *)ctx->jscratch.ptr;
    }
    np.grid = escalation_grid(ctx, pt.a.nq);
    np.run_if = pt.M->refresh + 1;
    np.resume = 1;
    const cudaError_t e = launch_newton_fp64(np, ctx->sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_newton_fp64 (escalation)");
  }
  return RB_OK;
}

static int solve_pressure(rb_ctx *ctx, const std::vector<Part> &parts, cudaStream_t st) {
  for (const Part &pt : parts) {
    const int rc = mixed_pressure(ctx, pt.M, pt.a.nq, pt.a.n, pt.a.u, pt.a.p, pt.a.info, st);
    if (rc != RB_OK) return rc;
  }
  return RB_OK;
}

// words[2] += 1; keep looping while queries are active and the iteration cap is not reached
__global__ void k_loop_cond(cudaGraphConditionalHandle h, int *words, int max_iter) {
  const int it = ++words[2];
  cudaGraphSetConditional(h, (words[0] > 0 && it < max_iter) ? 1u : 0u);
}

// End of a graph solve: the error word of this solve into the sticky word 5, which only the host
// clears once it has reported it (a solve that gave up is reported by a later call).
__global__ void k_latch_error(int *words) { words[5] |= words[1]; }

// ---- autotuner ------------------------------------------------------------------------------
// Synthetic, well-conditioned systems of the bucket's shape for timing the elimination variants:
// [J | -R] = [4 I + noise | 1], unit norms, every query active on the FP64-residual rung.
__global__ void k_tune_fill(int nq, int nb, int lda, float *Jaug, double2 *Rn, double *Rg,
                            rb_query_info *info, double *u, int ldu, int max_iter) {
  const size_t total = (size_t)nq * nb * lda;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % lda), r = (int)((e / lda) % nb);
    uint32_t h = (uint32_t)e * 2654435761u;
    h ^= h >> 15;
    const float v = ((float)(h & 0xFFFF) / 65536.f - 0.5f) * 0.1f;
    Jaug[e] = c < nb ? (c == r ? 4.f + v : v) : (c == nb ? 1.f : 0.f);
  }
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nq; b += gridDim.x * blockDim.x) {
    Rn[b] = make_double2(0.0, 1.0);
    const int G = (nb + 7) / 8;
    for (int g = 0; g < G; ++g) Rg[(size_t)b * G + g] = g == 0 ? 1.0 : 0.0;
    rb_query_info q = {RB_Q_NOT_CONVERGED, 2, RB_PREC_MIXED, 0, 0.0, 0.0};
    (void)max_iter;
    info[b] = q;
    for (int j = 0; j < ldu; ++j) u[(size_t)b * ldu + j] = 0.0;
  }
}

static int ceil_log2(int v) {
  int k = 0;
  while ((1 << k) < v) ++k;
  return k;
}

// Time the candidate launch variants of one bucket on `cnt` queries (once per batch-size class)
// and keep the fastest: elimination (warp per query if nb <= 80, blocked with 32- or 16-column
// panels) and the TMA ring depths of the two GEMMs. Run before the solve graph is captured.
static int autotune(rb_ctx *ctx, MixedState *M, int cnt, cudaStream_t st) {
  const int klass = ceil_log2(std::max(cnt, 1));
  if (M->tune.klass == klass) return RB_OK;
  const DevOps &o = ctx->ops;
  void *pu = nullptr, *pi = nullptr;
  int rc = ctx_alloc(ctx, &pu, 8 * (size_t)cnt * o.n_max, "tuning u");
  if (rc != RB_OK) return rc;
  if ((rc = ctx_alloc(ctx, &pi, sizeof(rb_query_info) * (size_t)cnt, "tuning info")) != RB_OK) {
    ctx_free(ctx, pu);
    return rc;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](auto &&launch) -> float {  // best of two, ms
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, st);
      if (launch() != RB_OK) return -1.f;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return best;
  };
  MixedState::Tune t;
  t.klass = klass;
  // elimination
  LuParams lp{};
  lp.o = o;
  lp.nq = cnt;
  lp.nb = M->nb;
  lp.ldj = M->Npad;
  lp.max_iter = 1 << 20;
  lp.u = (double *)pu;
  lp.info = (rb_query_info *)pi;
  lp.active = M->root->dev_words + 8;
  lp.rmode = kResExact;
  lp.Jaug = M->Jaug;
  lp.Rn = M->Rn;
  lp.Rg = M->Rg;
  lp.lda = aug_ld(M->nb);
  float best = 1e30f;
  const int epol = elim_policy(M->nb);
  for (int kind = (M->nb <= kWarpLuMaxN ? 1 : 2); kind <= 4; ++kind) {
    if (kind == 4 && (M->nb <= 32 || M->nb > kCtaLuMaxN)) continue;
    if (epol && kind != epol) continue;
    const float ms = timed([&]() {
      k_tune_fill<<<ctx->sms * 4, 256, 0, st>>>(cnt, M->nb, lp.lda, M->Jaug, M->Rn, M->Rg, lp.info, lp.u, o.n_max, 0);
      cudaEventRecord(e0, st);  // time the elimination only
      return launch_elimination(ctx, M, lp, cnt, st, kind);
    });
    if (ms < 0.f) { rc = set_error(ctx, RB_ERR_CUDA, "autotune (elimination)"); break; }
    if (ms < best) { best = ms; t.lu = kind; t.ms[0] = ms; }
  }
  // GEMMs on the bucket's operands (their outputs are rebuilt before every use)
  TcGemmParams g = gemm_params(M, cnt);
  g.n_tiles = M->Npad / kTcBN;
  g.kb[0] = M->kb0;
  g.n_pad = M->Npad;
  g.nk = M->nb;
  g.ldj = M->Npad;
  g.Jc = M->Jc;
  g.nsplit = 3;
  best = 1e30f;
  const int policy = pair_policy();
  for (int v = 0; v < 6; ++v) {  // stages 4, 6, 7; single CTAs, then CTA pairs
    const int stg = v % 3 == 0 ? 4 : (v % 3 == 1 ? 6 : 7);
    const bool pair = v >= 3;
    if (policy >= 0 && pair != (policy >= 1)) continue;
    if (rc != RB_OK) break;
    const float ms = timed([&]() {
      const cudaError_t e = launch_tc_gemm(kPlain, M->tmXj, M->tmWj, g, ctx->sms, st, stg, pair);
      return e == cudaSuccess ? RB_OK : RB_ERR_CUDA;
    });
    if (ms < 0.f) { rc = set_error(ctx, RB_ERR_CUDA, "autotune (Jacobian GEMM)"); break; }
    if (ms < best) { best = ms; t.st_plain = stg; t.pair_plain = pair; t.ms[1] = ms; }
  }
  g.n_tiles = M->WR.Npad / kTcBN;
  g.n_pad = M->WR.Npad;
  g.wexp[0] = M->WR.wexp[0];
  g.wexp[1] = M->WR.wexp[1];
  g.out = M->Rc;
  best = 1e30f;
  for (int v = 0; v < 9; ++v) {  // single CTAs, CTA pairs, CTA pairs with 256-column tiles
    const int stg = v % 3 == 0 ? 4 : (v % 3 == 1 ? 6 : 7);
    const int variant = v / 3;
    if (variant == 2 && M->nb < kWideMinN) continue;
    if (policy == 0 && variant != 0) continue;
    if (policy == 1 && variant == 0) continue;
    if (policy == 2 && variant != (M->nb >= kWideMinN ? 2 : 1)) continue;
    if (rc != RB_OK) break;
    const float ms = timed([&]() {
      const cudaError_t e = launch_sliced(M, M->WR, g, ctx->sms, st, stg, variant);
      return e == cudaSuccess ? RB_OK : RB_ERR_CUDA;
    });
    if (ms < 0.f) { rc = set_error(ctx, RB_ERR_CUDA, "autotune (sliced GEMM)"); break; }
    if (ms < best) { best = ms; t.st_sliced = stg; t.pair_sliced = variant; t.ms[2] = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  ctx_free(ctx, pu);
  ctx_free(ctx, pi);
  if (rc != RB_OK) return rc;
  M->tune = t;
  M->root->epoch += 1;  // the solve graph holds the previous variants
  return check_words(ctx, st, "autotune");
}

int mixed_tuning(rb_ctx *ctx, int i, int *out6, float *ms3) {
  MixedState *R = ctx->mixed;
  if (!R) return 0;
  std::vector<MixedState *> tuned;
  for (auto &kv : R->buckets)
    if (kv.second->tune.klass >= 0) tuned.push_back(kv.second);
  if (R->tune.klass >= 0) tuned.push_back(R);
  if (i >= 0 && i < (int)tuned.size()) {
    const MixedState *M = tuned[i];
    if (out6) {
      const int v[6] = {M->nb, M->tune.klass, M->tune.lu, M->tune.st_plain, M->tune.st_sliced,
                        M->tune.pair_plain | (M->tune.pair_sliced >= 1 ? 2 : 0) |
                            (M->tune.pair_sliced == 2 ? 4 : 0)};
      for (int k = 0; k < 6; ++k) out6[k] = v[k];
    }
    if (ms3)
      for (int k = 0; k < 3; ++k) ms3[k] = M->tune.ms[k];
  }
  return (int)tuned.size();
}

// The whole solve: gather (bucketed batches), prologue, rungs 0 and 1, a while-loop node over
// FP64-residual iterations, pressure, scatter.
struct SolvePlan {
  SolveArgs caller;                // the caller's buffers
  std::vector<Part> parts;
  bool gathered = false;           // parts work on the bucket-sorted copy
  bool pres = false;
};

static int plan_edges(rb_ctx *ctx, const SolvePlan &pl, bool first, cudaStream_t st) {
  MixedState *R = ctx->mixed;
  const DevOps &o = ctx->ops;
  const SolveArgs &c = pl.caller;
  if (first) {
    if (!pl.gathered) return RB_OK;
    k_gather<<<std::max(1, std::min((c.nq + 255) / 256, ctx->sms * 4)), 256, 0, st>>>(
        c.nq, R->perm, c.theta ? nullptr : c.mu, c.theta, o.n_theta, c.n, R->mu_g, R->theta_g, R->n_g);
  } else {
    if (!pl.gathered) return RB_OK;
    k_scatter<<<std::max(1, std::min((c.nq + 7) / 8, ctx->sms * 8)), 256, 0, st>>>(
        c.nq, R->perm, o.n_max, std::max(o.m, 1), R->u_g, pl.pres ? R->p_g : nullptr, R->info_g,
        c.u, pl.pres ? c.p : nullptr, c.info);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RB_OK : cuda_fail(ctx, e, first ? "k_gather" : "k_scatter");
}

static int build_solve_graph(rb_ctx *ctx, const SolvePlan &pl, const std::vector<int> &key_parts) {
  MixedState *M = ctx->mixed;
  for (cudaStream_t &c : M->cap)
    if (!c && cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess)
      return set_error(ctx, RB_ERR_CUDA, "capture stream");
  cudaStream_t cs = M->cap[0], cb = M->cap[1];
  if (M->gexec) {
    cudaGraphExecDestroy(M->gexec);
    M->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(ctx, e, "graph capture begin");
  }
  int rc = RB_OK;
  bool body_open = false;
  do {
    if ((rc = plan_edges(ctx, pl, true, cs)) != RB_OK) break;
    if ((rc = solve_prologue(ctx, pl.parts, cs)) != RB_OK) break;
    for (int r = 0; r < 3 && rc == RB_OK; ++r) {
      if ((rc = solve_iteration(ctx, pl.parts, r, cs)) != RB_OK) break;
      k_loop_cond<<<1, 1, 0, cs>>>(h, M->dev_words, ctx->cfg.max_iter);
    }
    if (rc != RB_OK) break;
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd)) != cudaSuccess) break;
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cn;
    if ((e = cudaGraphAddNode(&cn, g, dv.data(), nullptr, dv.size(), &np)) != cudaSuccess) break;
    if ((e = cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess) break;
    if ((e = cudaStreamBeginCaptureToGraph(cb, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed)) != cudaSuccess) break;
    body_open = true;
    if ((rc = solve_iteration(ctx, pl.parts, 3, cb)) != RB_OK) break;
    k_loop_cond<<<1, 1, 0, cb>>>(h, M->dev_words, ctx->cfg.max_iter);
    cudaGraph_t bg;
    body_open = false;
    if ((e = cudaStreamEndCapture(cb, &bg)) != cudaSuccess) break;
    if ((rc = solve_escalated(ctx, pl.parts, cs)) != RB_OK) break;
    if (pl.pres && (rc = solve_pressure(ctx, pl.parts, cs)) != RB_OK) break;
    if ((rc = plan_edges(ctx, pl, false, cs)) != RB_OK) break;
    k_latch_error<<<1, 1, 0, cs>>>(M->dev_words);
  } while (false);
  if (body_open) {
    cudaGraph_t bg;
    cudaStreamEndCapture(cb, &bg);
  }
  cudaGraph_t gout = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &gout);
  if (rc == RB_OK && e == cudaSuccess && e2 == cudaSuccess) {
    e = cudaGraphInstantiate(&M->gexec, g, 0);
    if (e != cudaSuccess) M->gexec = nullptr;
  }
  cudaGraphDestroy(g);
  if (rc != RB_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "solve graph");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "solve graph capture");
  const SolveArgs &c = pl.caller;
  M->gkey.mu = c.mu;
  M->gkey.theta = c.theta;
  M->gkey.p = c.p;
  M->gkey.n = c.n;
  M->gkey.u = c.u;
  M->gkey.info = c.info;
  M->gkey.nq = c.nq;
  M->gkey.epoch = M->epoch;
  M->gkey.parts = key_parts;
  return RB_OK;
}

// Gather scratch of a bucketed batch (grow-only).
static int gather_scratch(rb_ctx *ctx, int nq, bool theta) {
  MixedState *R = ctx->mixed;
  const DevOps &o = ctx->ops;
  const int need = std::max(nq, 1);
  if (need <= R->gcap && (!theta || R->theta_g)) return RB_OK;
  for (void *q : {(void *)R->perm, (void *)R->n_g, (void *)R->mu_g, (void *)R->theta_g,
                  (void *)R->u_g, (void *)R->p_g, (void *)R->info_g})
    ctx_free(ctx, q);
  R->perm = R->n_g = nullptr;
  R->mu_g = R->theta_g = R->u_g = R->p_g = nullptr;
  R->info_g = nullptr;
  R->gcap = 0;
  const int cap = std::max(need, R->gcap);
  void *p;
  int rc;
  if ((rc = ctx_alloc(ctx, &p, 4 * (size_t)cap, "bucket order")) != RB_OK) return rc;
  R->perm = (int *)p;
  if ((rc = ctx_alloc(ctx, &p, 4 * (size_t)cap, "bucket sizes")) != RB_OK) return rc;
  R->n_g = (int *)p;
  if ((rc = ctx_alloc(ctx, &p, 16 * (size_t)cap, "bucket mu")) != RB_OK) return rc;
  R->mu_g = (double *)p;
  if (theta) {
    if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)cap * o.n_theta, "bucket theta")) != RB_OK) return rc;
    R->theta_g = (double *)p;
  }
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)cap * o.n_max, "bucket u")) != RB_OK) return rc;
  R->u_g = (double *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)cap * std::max(o.m, 1), "bucket p")) != RB_OK) return rc;
  R->p_g = (double *)p;
  if ((rc = ctx_alloc(ctx, &p, sizeof(rb_query_info) * (size_t)cap, "bucket info")) != RB_OK) return rc;
  R->info_g = (rb_query_info *)p;
  R->gcap = cap;
  R->epoch += 1;
  return RB_OK;
}

// Outcome of the graph solves enqueued so far: RB_OK, RB_PENDING (wait == 0 and the last one
// has not completed) or RB_ERR_TIMEOUT (a device-side wait of one of them gave up; reported once).
int mixed_solve_status(rb_ctx *ctx, int wait) {
  MixedState *R = ctx->mixed;
  if (!R || !R->pending) return RB_OK;
  cudaError_t e = wait ? cudaEventSynchronize(R->done_ev) : cudaEventQuery(R->done_ev);
  if (e == cudaErrorNotReady) return RB_PENDING;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "solve completion");
  R->pending = false;
  const int w = R->h_words[13];
  if (w) {
    R->h_words[13] = 0;
    e = cudaMemsetAsync(R->dev_words + 5, 0, 4, R->pending_st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "words");
    return set_error(ctx, RB_ERR_TIMEOUT,
                     "mixed solve: tensor-core pipeline wait gave up (code %d); the results of "
                     "that solve are not valid", w);
  }
  return RB_OK;
}

// Small operator sets (n_max <= kSmallMaxN) and batches of at most a few queries per SM: the
// whole Newton solve of each query in one launch (k_newton_small, one CTA per query) instead of
// the tensor-core pipeline, whose per-iteration launches dominate there; pressure by the FP64
// recovery kernel. RB_SMALL = 0 / 1 turns the choice off / forces it for any small set.
static bool use_small_path(const rb_ctx *ctx, int nq) {
  if (ctx->ops.n_max > kSmallMaxN) return false;
  const char *e = getenv("RB_SMALL");
  if (e && *e) return atoi(e) != 0;
  return nq <= 2 * ctx->sms;
}

static int solve_small(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                       const int *d_n, double *d_u, double *d_p, rb_query_info *info,
                       cudaStream_t st) {
  MixedState *R = ctx->mixed;
  const DevOps &o = ctx->ops;
  int rc;
  if ((rc = mixed_layouts(ctx, R, st)) != RB_OK) return rc;
  const int nb = o.n_max;
  if (!R->Dt2) {  // D~ as double-float, [q_c][l][k][j] with the n_max strides
    void *p;
    const size_t nn = (size_t)nb * nb;
    if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)o.q_c * nb * nn, "D~ (double-float)")) != RB_OK) return rc;
    R->Dt2 = (float2 *)p;
    k_split_f2<<<ctx->sms * 4, 256, 0, st>>>(o.Dt, R->Dt2, (size_t)o.q_c * nb * nn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "D~ (double-float)");
  }
  SmallParams sp{};
  sp.o = o;
  sp.mu = d_theta ? nullptr : d_mu;
  sp.theta = d_theta;
  sp.nsz = d_n;
  sp.nq = nq;
  sp.nb = nb;
  sp.max_iter = ctx->cfg.max_iter;
  sp.tol_upd = ctx->cfg.tol_update;
  sp.tol_res = ctx->cfg.tol_res;
  sp.Dt2 = R->Dt2;
  sp.A2 = R->A2;
  sp.u = d_u;
  sp.info = info;
  const int mk = prof_begin(ctx, RB_K_NEWTON_SMALL, st);
  cudaError_t e = launch_newton_small(sp, ctx->sms, st);
  prof_end(ctx, mk, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_newton_small");
  if (d_p && o.m > 0 && o.B)  // the FP64 recovery of Eq. sup-vvar for the converged queries
    if ((rc = solve_pressure(ctx, d_mu, d_theta, nq, d_n, d_u, d_p, info, st)) != RB_OK) return rc;
  // as for a graph solve: the error words come back behind the solve, read by
  // mixed_solve_status without a synchronisation here
  e = cudaMemcpyAsync(R->h_words + 12, R->dev_words + 4, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(R->done_ev, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "solve completion");
  R->pending = true;
  R->pending_st = st;
  return RB_OK;
}

int solve_mixed(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq, const int *d_n,
                const int *h_n, double *d_u, double *d_p, rb_query_info *d_info, cudaStream_t st) {
  int rc = mixed_root(ctx, st);
  if (rc != RB_OK) return rc;
  // an earlier asynchronous solve that has completed and failed is reported now
  if ((rc = mixed_solve_status(ctx, 0)) != RB_OK && rc != RB_PENDING) return rc;
  MixedState *R = ctx->mixed;
  const DevOps &o = ctx->ops;
  rb_query_info *info = d_info ? d_info : own_info(ctx, nq);
  if (!info) return set_error(ctx, RB_ERR_OOM, "info scratch");
  if (use_small_path(ctx, nq)) return solve_small(ctx, d_mu, d_theta, nq, d_n, d_u, d_p, info, st);
  SolvePlan pl;
  pl.caller = {d_mu, d_theta, nq, d_n, d_u, d_p, info};
  pl.pres = d_p && o.m > 0 && o.B;
  // size buckets from the host copy of the sizes
  std::vector<int> hn;
  if (d_n) {
    hn.resize(nq);
    if (h_n) {
      std::copy(h_n, h_n + nq, hn.begin());
    } else {
      cudaError_t e = cudaMemcpyAsync(hn.data(), d_n, 4 * (size_t)nq, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "query sizes");
    }
  }
  std::map<int, std::vector<int>> groups;  // bucket size -> query indices
  for (int i = 0; i < nq && d_n; ++i) {
    const int n = hn[i];
    groups[(n >= 1 && n <= o.n_max) ? bucket_size(n, o.n_max) : o.n_max].push_back(i);
  }
  std::vector<int> key_parts;
  if (groups.size() <= 1 && (groups.empty() || groups.begin()->first == o.n_max)) {
    if ((rc = mixed_layouts(ctx, R, st)) != RB_OK) return rc;
    if ((rc = mixed_batch_scratch(ctx, R, nq)) != RB_OK) return rc;
    pl.parts.push_back({R, pl.caller});
    key_parts = {R->nb, 0, nq};
  } else {
    if ((rc = gather_scratch(ctx, nq, d_theta != nullptr)) != RB_OK) return rc;
    std::vector<int> perm;
    perm.reserve(nq);
    std::vector<std::pair<MixedState *, std::pair<int, int>>> ranges;
    for (auto &kv : groups) {
      MixedState *M = bucket(ctx, kv.first);
      if ((rc = mixed_layouts(ctx, M, st)) != RB_OK) return rc;
      if ((rc = mixed_batch_scratch(ctx, M, (int)kv.second.size())) != RB_OK) return rc;
      ranges.push_back({M, {(int)perm.size(), (int)kv.second.size()}});
      perm.insert(perm.end(), kv.second.begin(), kv.second.end());
    }
    // the order goes up from pinned memory without a synchronisation; the previous solve's
    // upload from the same buffer has completed before it is overwritten
    cudaError_t e = cudaEventSynchronize(R->perm_ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bucket order");
    if (R->h_perm_cap < nq) {
      if (R->h_perm) cudaFreeHost(R->h_perm);
      R->h_perm = nullptr;
      R->h_perm_cap = 0;
      if (cudaMallocHost(&R->h_perm, 4 * (size_t)nq) != cudaSuccess)
        return set_error(ctx, RB_ERR_OOM, "pinned bucket order");
      R->h_perm_cap = nq;
    }
    std::copy(perm.begin(), perm.end(), R->h_perm);
    e = cudaMemcpyAsync(R->perm, R->h_perm, 4 * (size_t)nq, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(R->perm_ev, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bucket order");
    const int mm = std::max(o.m, 1);
    for (auto &r : ranges) {
      const int off = r.second.first, cnt = r.second.second;
      SolveArgs a{d_theta ? nullptr : R->mu_g + 2 * (size_t)off,
                  d_theta ? R->theta_g + (size_t)off * o.n_theta : nullptr, cnt, R->n_g + off,
                  R->u_g + (size_t)off * o.n_max, pl.pres ? R->p_g + (size_t)off * mm : nullptr,
                  R->info_g + off};
      pl.parts.push_back({r.first, a});
      key_parts.insert(key_parts.end(), {r.first->nb, off, cnt});
    }
    pl.gathered = true;
  }
  if (ctx->cfg.autotune)
    for (const Part &pt : pl.parts)
      if ((rc = autotune(ctx, pt.M, pt.a.nq, st)) != RB_OK) return rc;
  if ((rc = escalation_scratch(ctx)) != RB_OK) return rc;  // before any capture
  if (ctx->cfg.use_graph && !ctx->prof) {
    const auto &k = R->gkey;
    if (!R->gexec || k.mu != d_mu || k.theta != d_theta || k.p != d_p || k.n != d_n || k.u != d_u ||
        k.info != info || k.nq != nq || k.epoch != R->epoch || k.parts != key_parts) {
      if ((rc = build_solve_graph(ctx, pl, key_parts)) != RB_OK) return rc;
    }
    cudaError_t e = cudaGraphLaunch(R->gexec, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve graph launch");
    // no synchronisation: the error words come back to pinned memory behind the solve and are
    // read by mixed_solve_status (rb_solve_device_status, rb_solve, or the next solve)
    e = cudaMemcpyAsync(R->h_words + 12, R->dev_words + 4, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(R->done_ev, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve completion");
    R->pending = true;
    R->pending_st = st;
    return RB_OK;
  }
  if ((rc = plan_edges(ctx, pl, true, st)) != RB_OK) return rc;
  if ((rc = solve_prologue(ctx, pl.parts, st)) != RB_OK) return rc;
  for (int it = 0; it < ctx->cfg.max_iter; ++it) {
    if ((rc = solve_iteration(ctx, pl.parts, std::min(it, 3), st)) != RB_OK) return rc;
    if ((rc = check_words(ctx, st, "mixed Newton step")) != RB_OK) return rc;
    if (R->h_words[0] == 0) break;
  }
  if ((rc = solve_escalated(ctx, pl.parts, st)) != RB_OK) return rc;
  if (pl.pres && (rc = solve_pressure(ctx, pl.parts, st)) != RB_OK) return rc;
  if ((rc = plan_edges(ctx, pl, false, st)) != RB_OK) return rc;
  if ((rc = check_words(ctx, st, "mixed solve")) != RB_OK) return rc;
  if (ctx->prof) prof_collect(ctx);
  return RB_OK;
}

// ---- pieces used by the continuous-batching server (the n_max layouts) --------------------
int mixed_prepare(rb_ctx *ctx, int capacity, cudaStream_t st) {
  int rc = mixed_root(ctx, st);
  if (rc != RB_OK) return rc;
  if ((rc = mixed_layouts(ctx, ctx->mixed, st)) != RB_OK) return rc;
  if ((rc = mixed_batch_scratch(ctx, ctx->mixed, capacity)) != RB_OK) return rc;
  // the server's gather buffers at full capacity, so that no step reallocates them
  ctx->mixed->serve_cap = capacity;
  if ((rc = gather_scratch(ctx, capacity, false)) != RB_OK) return rc;
  return own_info(ctx, 1) ? RB_OK : set_error(ctx, RB_ERR_OOM, "info scratch");
}

// Device bytes one more slot of batch state costs (X operands, Jacobian, residual, LU).
size_t mixed_slot_bytes(const rb_ctx *ctx) {
  const DevOps &o = ctx->ops;
  const size_t nb = o.n_max, Kpad0 = (size_t)round_up(o.q_c * o.n_max, 64);
  const size_t Npad = (size_t)round_up(o.n_max * o.n_max, kTcBN);
  const int S = 8;
  return 2 * 3 * Kpad0 + 2 * S * Kpad0 + 8 + 8 * nb + 4 * Npad + 8 * nb + 8 * (size_t)(o.m + 1) +
         8 * nb + 64 + 8 * (size_t)o.n_theta + 8 * nb + 8 * nb * nb + 8 * (size_t)(o.m + 1) +
         4 * nb * (size_t)aug_ld((int)nb) + 16 + 8 * ((nb + 7) / 8) + 8 * (size_t)o.m * o.m;
}

// One serving step, size-bucketed: the live slots (host lists of slot, size and iteration count)
// are grouped by bucket size, adjacent buckets merged from the largest down until each group
// holds at least kServeGroupMin queries (a group runs at its largest size: few live queries make
// one batch, as many launches as a batch solve; many make one per size range), and gathered into
// the groups' batches; each group rebuilds the
// per-query data of its queries (theta, f, A(mu), B(mu); slots change places between steps, so
// nothing per query is kept across steps and the Jacobian is refactored each iteration), runs
// one Newton iteration with the contractions its queries' rungs need, recovers the pressure of
// the queries that converge, and the slots get u, p and the status back.
constexpr int kServeGroupMin = 512;
int mixed_serve_step(rb_ctx *ctx, const double *d_mu, const int *d_n, double *d_u, double *d_p,
                     rb_query_info *d_info, const std::vector<int> &slots,
                     const std::vector<int> &slot_n, const std::vector<int> &slot_iters,
                     std::vector<int> &perm, cudaStream_t st) {
  MixedState *R = ctx->mixed;
  const DevOps &o = ctx->ops;
  const int nm = o.n_max, mm = std::max(o.m, 1);
  struct Group { MixedState *M; int off, cnt; bool jac, exact; int c1, c2; };
  std::map<int, std::vector<int>> by;
  for (size_t i = 0; i < slots.size(); ++i) {
    const int n = slot_n[i];
    if (n < 1 || n > nm) continue;  // rejected at admission: nothing to compute
    by[bucket_size(n, nm)].push_back((int)i);
  }
  // merge adjacent buckets, largest first, into groups of at least kServeGroupMin queries
  std::vector<std::pair<int, std::vector<int>>> merged;  // (group size nb, members)
  for (auto it = by.rbegin(); it != by.rend(); ++it) {
    if (merged.empty() || (int)merged.back().second.size() >= kServeGroupMin)
      merged.push_back({it->first, {}});
    auto &mem = merged.back().second;
    mem.insert(mem.end(), it->second.begin(), it->second.end());
  }
  perm.clear();
  std::vector<Group> groups;
  int rc;
  for (auto &kv : merged) {
    MixedState *M = kv.first == nm ? R : bucket(ctx, kv.first);
    if ((rc = mixed_layouts(ctx, M, st)) != RB_OK) return rc;
    // a bucket's batch scratch is sized for all of the server's slots when it first has to
    // grow, so that the changing group sizes of a busy server do not reallocate it again (each
    // reallocation synchronises the device); where that does not fit, exactly what is needed
    const int cnt = (int)kv.second.size();
    const int want = cnt <= M->bcap ? cnt : std::max(cnt, R->serve_cap);
    rc = mixed_batch_scratch(ctx, M, want);
    if (rc == RB_ERR_OOM && want > cnt) rc = mixed_batch_scratch(ctx, M, cnt);
    if (rc != RB_OK) return rc;
    // members by iteration count, highest first: the rows that need the sliced residual
    // (count >= 2) lead, then those that need the Jacobian (count >= 1)
    std::stable_sort(kv.second.begin(), kv.second.end(),
                     [&](int x, int y) { return slot_iters[x] > slot_iters[y]; });
    Group g{M, (int)perm.size(), (int)kv.second.size(), false, false, 0, 0};
    for (int i : kv.second) {
      perm.push_back(slots[i]);
      g.c1 += slot_iters[i] >= 1;
      g.c2 += slot_iters[i] >= 2;
    }
    g.jac = g.c1 > 0;
    g.exact = g.c2 > 0;
    groups.push_back(g);
  }
  const int total = (int)perm.size();
  if (total == 0) return RB_OK;
  if ((rc = gather_scratch(ctx, total, false)) != RB_OK) return rc;
  // perm stays alive until the caller synchronises the stream at the end of the step
  cudaError_t e = cudaMemcpyAsync(R->perm, perm.data(), 4 * (size_t)total, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "serve bucket order");
  k_gather_slots<<<std::max(1, std::min((total + 7) / 8, ctx->sms * 8)), 256, 0, st>>>(
      total, R->perm, nm, d_mu, d_n, d_u, d_info, R->mu_g, R->n_g, R->u_g, R->info_g);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "k_gather_slots");
  const bool pres = d_p && o.m > 0 && o.B;
  for (const Group &g : groups) {
    const SolveArgs a{R->mu_g + 2 * (size_t)g.off, nullptr, g.cnt, R->n_g + g.off,
                      R->u_g + (size_t)g.off * nm, pres ? R->p_g + (size_t)g.off * mm : nullptr,
                      R->info_g + g.off};
    cudaMemsetAsync(R->dev_words, 0, 4, st);
    if ((rc = launch_prep(ctx, g.M, a.mu, nullptr, g.cnt, a.n, a.info, st, 1)) != RB_OK) return rc;
    if ((rc = mixed_contract(ctx, g.M, g.cnt, a.n, a.u, a.info, g.jac, g.exact, st, g.c1, g.c2)) != RB_OK)
      return rc;
    LuParams lp = solve_lu_params(ctx, g.M, a);
    lp.chord = 0;
    if ((rc = launch_lu(ctx, g.M, lp, g.cnt, st)) != RB_OK) return rc;
    // only rows with an FP64-accurate residual (the first c2) can have converged
    if (pres && g.exact && (rc = mixed_pressure(ctx, g.M, g.c2, a.n, a.u, a.p, a.info, st)) != RB_OK)
      return rc;
  }
  k_scatter<<<std::max(1, std::min((total + 7) / 8, ctx->sms * 8)), 256, 0, st>>>(
      total, R->perm, nm, mm, R->u_g, pres ? R->p_g : nullptr, R->info_g, d_u, pres ? d_p : nullptr,
      d_info);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "k_scatter");
  return RB_OK;
}

int mixed_error_word(rb_ctx *ctx, cudaStream_t st) {
  return check_words(ctx, st, "serving step");
}

int eval_mixed(rb_ctx *ctx, const double *d_mu, int nq, int n, const double *d_u, int precision,
               double *d_R, double *d_J, cudaStream_t st) {
  if (precision != RB_PREC_MIXED) return set_error(ctx, RB_ERR_ARG, "unknown precision %d", precision);
  int rc = mixed_root(ctx, st);
  if (rc != RB_OK) return rc;
  MixedState *M = ctx->mixed;
  if ((rc = mixed_layouts(ctx, M, st)) != RB_OK) return rc;
  if ((rc = mixed_batch_scratch(ctx, M, nq)) != RB_OK) return rc;
  const DevOps &o = ctx->ops;
  // the layouts use n_max-length rows: widen u and pass sizes
  if ((rc = ctx->jscratch.reserve(ctx, 8 * (size_t)nq * o.n_max + 4 * (size_t)nq + 256, "eval staging")) != RB_OK)
    return rc;
  double *uw = (double *)ctx->jscratch.ptr;
  int *nsz = (int *)(uw + (size_t)nq * o.n_max);
  rb_query_info *info = own_info(ctx, nq);
  if (!info) return set_error(ctx, RB_ERR_OOM, "info scratch");
  cudaMemsetAsync(uw, 0, 8 * (size_t)nq * o.n_max, st);
  cudaMemcpy2DAsync(uw, 8 * o.n_max, d_u, 8 * n, 8 * n, nq, cudaMemcpyDeviceToDevice, st);
  std::vector<int> hn(nq, n);
  cudaMemcpyAsync(nsz, hn.data(), 4 * (size_t)nq, cudaMemcpyHostToDevice, st);
  k_mixed_init<<<std::min(nq, ctx->sms * 8), 128, 0, st>>>(nq, o.n_max, nsz, nullptr, info);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_mixed_init");
  cudaMemsetAsync(M->dev_words, 0, 8, st);
  if ((rc = launch_prep(ctx, M, d_mu, nullptr, nq, nsz, info, st)) != RB_OK) return rc;
  if ((rc = mixed_contract(ctx, M, nq, nsz, uw, info, true, true, st)) != RB_OK) return rc;
  const SolveArgs a{d_mu, nullptr, nq, nsz, uw, nullptr, info};
  LuParams lp = solve_lu_params(ctx, M, a);
  lp.rmode = kResExact;
  lp.eval_only = 1;
  lp.R_out = d_R;
  lp.J_out = d_J;
  if ((rc = launch_lu(ctx, M, lp, nq, st)) != RB_OK) return rc;
  rc = check_words(ctx, st, "rb_eval (mixed)");
  cudaStreamSynchronize(st);  // hn is a host vector read by the copy above
  return rc;
}

}  // namespace rb
