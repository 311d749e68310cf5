// rb_mixed.cu -- mixed-precision batched Newton (inexact Newton, Sec. 3.6 Jacobian on tensor cores).
//
// Per iteration, for every active query b of the batch:
//   1. k_build_x: X_b = theta^c(mu_b) (x) u_b as split BF16 (hi, lo) for the Jacobian GEMM; the
//      7-bit digit slices of theta^c (x) u_b / 2 for the sliced GEMM; u_b as (hi, lo) floats
//      (transposed); R^c_b = 0.
//   2. k_tc_gemm<kPlain>:  J^c = X W^T on tcgen05 (split BF16, FP32 accumulate) -> Jc (FP32).
//   3. k_tc_gemm<kSliced>: R^c_b[k] = sum_j u_b[j] (X'_b W^T)[(k,j)] = C_mu(u_b, u_b)[k] from
//      exact digit products, contracted in double-float -> FP64.
//   4. k_lu_mixed(_warp): A(mu) and A(mu) u in double-float on the CUDA cores;
//      R = A(mu) u + C_mu(u, u) - f(mu); J = fl32(A(mu)) + J^c; GEPP in FP32 on J delta = -R;
//      u += delta in FP64; stopping rule (Sec. 6) on the FP64 norms.
// The Jacobian is inexact (BF16 convection part, FP32 elimination); the residual and the test
// are FP64-accurate, so the iteration converges to the FP64 solution at the linear rate
// ||J~^-1 (J~ - J)||. After the last iteration the pressure right-hand side
// fs(mu) - As(mu) u - Cs_mu(u, u) (Eq. sup-vvar) takes Cs_mu(u, u) from the same sliced GEMM with
// W = 2 Cs and As(mu) u in double-float, and B(mu) p = r is solved in FP64 (Eq. blocksolve-2).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rb_ctx.h"
#include "rb_mixed.cuh"

namespace rb {

struct SlicedW {  // one sliced weight operand [S][Npad][Kpad]
  __nv_bfloat16 *d = nullptr;
  int Npad = 0, nk = 0, wexp[2] = {0, 0};
  CUtensorMap tm;
};

struct MixedState {
  // operator layouts for the Jacobian size nb (= n_max)
  int nb = 0, Kpad0 = 0, kb0 = 0, kb1 = 0, Kpad = 0, Npad = 0, S0 = 0, S1 = 0, Smax = 0;
  __nv_bfloat16 *Wj = nullptr;  // [2][Npad][Kpad0] split BF16 D~ (hi, lo)
  CUtensorMap tmWj;
  SlicedW WR, WP;               // residual [D~ | A], pressure [2 Cs | As]
  float2 *A2 = nullptr;         // [q_a][n_max][n_max] A_q as double-float (hi, lo)
  float2 *As2 = nullptr;        // [q_a][m][n_max] As_q as double-float
  // batch scratch
  int bcap = 0;
  __nv_bfloat16 *Xj = nullptr, *Xd = nullptr;  // Xj: [3][bcap][Kpad0] (hi, hi, lo)
  int *xexp = nullptr;          // [2][bcap]
  float2 *ufT = nullptr;        // [nb][bcap]
  float *Jc = nullptr;          // [bcap][Npad]
  double *Rc = nullptr;         // [bcap][nb]
  double *Rp = nullptr;         // [bcap][m]
  CUtensorMap tmXj, tmXd;
  float *lu_scratch = nullptr;
  int lu_grid = 0;
  int *dev_words = nullptr;     // [0] active count, [1] error word, [8..] scratch
  int *h_words = nullptr;       // pinned mirror
  rb_query_info *info_own = nullptr;
  int info_cap = 0;
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
// signed 7-bit digits of v on the grid 2^(e - 7 i), i = 1..S (|v| < 2^e), truncated toward 0
__device__ __forceinline__ void digits7(double v, double scale /* 2^(7S - e) */, int S,
                                        __nv_bfloat16 *out, size_t slice_stride) {
  const long long F = __double2ll_rz(fabs(v) * scale);
  const float sg = v < 0 ? -1.f : 1.f;
  for (int i = 1; i <= S; ++i) {
    const int d = (int)((F >> (kDigitBits * (S - i))) & 127);
    out[(size_t)(i - 1) * slice_stride] = __float2bfloat16_rn(sg * (float)d);
  }
}

// Same digits from the FP64 bit pattern with integer operations only (GB300's FP64 pipe is
// narrow and its conversions slow). e is the grid exponent (|v| < 2^e).
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
  const long long F = fixed_bits(v, e, S);
  const float sg = v < 0 ? -1.f : 1.f;
  for (int i = 1; i <= S; ++i) {
    const int d = (int)((F >> (kDigitBits * (S - i))) & 127);
    out[(size_t)(i - 1) * slice_stride] = __float2bfloat16_rn(sg * (float)d);
  }
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
  const double *mu, *theta;
  const int *nsz;
  int nq, nb, Kpad0, Kpad, S0, S1, b_pad, max_iter, mode;  // mode 0: active, 1: converged
  int digits;       // 1: also write the digit slices, exponents and u pairs (sliced GEMM)
  const double *u;  // [nq][n_max]
  const rb_query_info *info;
  __nv_bfloat16 *Xj, *Xd;
  int *xexp;        // [2][b_pad]
  float2 *ufT;      // [nb][b_pad]
  double *out;      // [b_pad][nout], zeroed for each built query
  int nout;
};

__device__ __forceinline__ bool is_active(const rb_query_info &q, int max_iter) {
  return q.status == RB_Q_NOT_CONVERGED && q.iters < max_iter;
}

__device__ __forceinline__ int exp_of_max(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

__global__ void __launch_bounds__(kThreads) k_build_x(BuildXParams p) {
  __shared__ double th[4 * RB_Q_MAX];
  __shared__ double red[2 * kWarps];
  const DevOps &o = p.o;
  const int tid = threadIdx.x;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    const rb_query_info qi = p.info[b];
    const bool want = p.mode == 0 ? is_active(qi, p.max_iter) : qi.status == RB_Q_OK;
    if (!want) continue;
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    if (p.theta) {
      for (int i = tid; i < o.n_theta; i += blockDim.x) th[i] = p.theta[(size_t)b * o.n_theta + i];
    } else {
      theta_eval(o, p.mu[2 * b], p.mu[2 * b + 1], th);
    }
    __syncthreads();
    const double *ta = th, *tc = th + o.q_a;
    const double *ub = p.u + (size_t)b * o.n_max;
    // grid exponents from the integer bit patterns (|x| orders like its bits)
    unsigned long long m0 = 0, m1 = 0;
    const unsigned long long absmask = 0x7FFFFFFFFFFFFFFFull;
    for (int kap = tid; kap < o.q_c * p.nb; kap += blockDim.x) {
      const int q = kap / p.nb, l = kap % p.nb;
      if (l < n) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(tc[q] * ub[l]) & absmask;
        m0 = v > m0 ? v : m0;
      }
    }
    for (int q = tid; q < o.q_a; q += blockDim.x) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(ta[q]) & absmask;
      m1 = v > m1 ? v : m1;
    }
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long a = __shfl_xor_sync(0xffffffffu, m0, off);
      const unsigned long long c = __shfl_xor_sync(0xffffffffu, m1, off);
      m0 = a > m0 ? a : m0;
      m1 = c > m1 ? c : m1;
    }
    unsigned long long *ured = reinterpret_cast<unsigned long long *>(red);
    if ((tid & 31) == 0) {
      ured[tid >> 5] = m0;
      ured[kWarps + (tid >> 5)] = m1;
    }
    __syncthreads();
    unsigned long long mx0 = 0, mx1 = 0;
    for (int i = 0; i < kWarps; ++i) {
      mx0 = ured[i] > mx0 ? ured[i] : mx0;
      mx1 = ured[kWarps + i] > mx1 ? ured[kWarps + i] : mx1;
    }
    // the sliced operand holds x / 2: same digits as x on the grid one binade higher
    const int ex0 = exp_of_bits(mx0), e0 = ex0 - 1, e1 = exp_of_bits(mx1);
    const size_t sstride = (size_t)p.b_pad * p.Kpad;
    const size_t jstride = (size_t)p.b_pad * p.Kpad0;
    for (int kap = tid; kap < p.Kpad; kap += blockDim.x) {
      const size_t off = (size_t)b * p.Kpad + kap;
      if (kap < p.Kpad0) {
        double x = 0.0;
        if (kap < o.q_c * p.nb) {
          const int q = kap / p.nb, l = kap % p.nb;
          if (l < n) x = tc[q] * ub[l];
        }
        if (p.mode == 0) {
          // split BF16 operand of the Jacobian GEMM: [x_hi | x_hi | x_lo]
          const float xf = (float)x;
          const __nv_bfloat16 hi = __float2bfloat16_rn(xf);
          const __nv_bfloat16 lo = __float2bfloat16_rn(xf - __bfloat162float(hi));
          __nv_bfloat16 *xj = p.Xj + (size_t)b * p.Kpad0 + kap;
          xj[0] = hi;
          xj[jstride] = hi;
          xj[2 * jstride] = lo;
        }
        if (p.digits) digits7_int(x, ex0, p.S0, p.Xd + off, sstride);
      } else if (p.digits) {
        const int q = kap - p.Kpad0;
        digits7_int(q < o.q_a ? ta[q] : 0.0, e1, p.S1, p.Xd + off, sstride);
      }
    }
    if (!p.digits) {
      __syncthreads();
      continue;
    }
    for (int j = tid; j < p.nb; j += blockDim.x) {
      const double v = j < n ? ub[j] : 0.0;
      const float hi = (float)v;
      p.ufT[(size_t)j * p.b_pad + b] = make_float2(hi, (float)(v - (double)hi));
    }
    for (int k = tid; k < p.nout; k += blockDim.x) p.out[(size_t)b * p.nout + k] = 0.0;
    if (tid == 0) {
      p.xexp[b] = e0;
      p.xexp[p.b_pad + b] = e1;
    }
    __syncthreads();
  }
}

struct LuParams {
  DevOps o;
  const double *mu, *theta;
  const int *nsz;
  int nq, nb, ldj, max_iter, j_in_smem;
  double tol_upd, tol_res;
  const float2 *A2;      // [q_a][n_max][n_max] A_q as double-float (hi, lo)
  const float *Jc;       // [b_pad][ldj]
  const double *Rc;      // [b_pad][nb]: A(mu) u + C_mu(u, u)
  double *u;             // [nq][n_max], updated in place
  rb_query_info *info;   // [nq]
  float *scratch;        // [grid][nb * nb] when J is not in shared memory
  int *active;           // count of queries still active after this iteration
  int eval_only;         // 1: write R and J (FP64) to R_out / J_out instead of solving
  double *R_out, *J_out;
  int rmode;             // residual source: kResZero, kResLow, kResExact, or -1: per query
                         // from its iteration count (0 -> zero, 1 -> low, >= 2 -> exact)
};

// Residual source of one Newton iteration (the precision ladder of the inexact Newton):
//   kResZero  u = 0: R = -f(mu) exactly and J = A(mu) (no contraction needed),
//   kResLow   R = (A(mu) + J~^c / 2) u - f(mu) from the FP32/BF16 Jacobian (Euler identity);
//             only used to approach the root, never to declare convergence,
//   kResExact R = [A(mu) u + C_mu(u, u)]_sliced - f(mu), FP64-accurate.
enum { kResZero = 0, kResLow = 1, kResExact = 2, kResLadder = -1 };

__device__ __forceinline__ int rung_of(int rmode, int iters) {
  return rmode >= 0 ? rmode : (iters == 0 ? kResZero : (iters == 1 ? kResLow : kResExact));
}

struct LuSmem {
  int th, R, fm, red, tah, uh, rhs, J, total;  // offsets in bytes
  __host__ __device__ LuSmem(const DevOps &o, int nb, bool j_in_smem) {
    int p = 0;
    th = p; p += 8 * ((o.n_theta + 1) & ~1);
    R = p; p += 8 * nb;
    fm = p; p += 8 * nb;
    red = p; p += 8 * 4 * kWarps;
    tah = p; p += 8 * o.q_a;           // theta^a as (hi, lo) floats
    uh = p; p += 8 * nb;               // u as (hi, lo) floats
    rhs = p; p += 4 * ((nb + 3) & ~3);
    p = (p + 15) & ~15;
    J = p;
    if (j_in_smem) p += 4 * nb * nb;
    total = p;
  }
};

// Rows k0 .. k0 + R - 1 of the Newton system, by one warp: J[k][:] = fl32(A(mu)[k][:]) + J^c[k][:]
// and R[k] = A(mu)[k][:] u (double-float) + convection part - f[k]. R rows at once keep R
// independent A loads in flight per lane.
template <int RR>
__device__ __forceinline__ void lu_rows(const LuParams &p, int rm, int b, int n, int k0,
                                        const float2 *ta, const float2 *u2, const double *fm,
                                        float *J, int ld, double *R) {
  const int lane = threadIdx.x & 31;
  const size_t nm = (size_t)p.o.n_max;
  const float *jc = p.Jc + (size_t)b * p.ldj;
  const bool with_jc = rm != kResZero;
  float rh[RR], rl[RR], clow[RR];
#pragma unroll
  for (int r = 0; r < RR; ++r) rh[r] = rl[r] = clow[r] = 0.f;
  for (int j = lane; j < n; j += 32) {
    const float2 uj = u2[j];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const int k = k0 + r;
      if (k < n) {
        float ah = 0.f, al = 0.f;
        for (int q = 0; q < p.o.q_a; ++q) {
          const float2 a2 = __ldg(p.A2 + ((size_t)q * nm + k) * nm + j);
          df_fma(ah, al, ta[q].x, ta[q].y, a2.x, a2.y);
        }
        const float c = with_jc ? jc[(size_t)k * p.nb + j] : 0.f;
        const float v = (ah + al) + c;
        df_fma(rh[r], rl[r], ah, al, uj.x, uj.y);
        if (rm == kResLow) clow[r] = fmaf(0.5f * c, uj.x, clow[r]);
        if (p.eval_only)
          p.J_out[((size_t)b * n + k) * n + j] = (double)v;
        else
          J[(size_t)k * ld + j] = v;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    const int k = k0 + r;
    const double rlin = df_warp_sum(rh[r], rl[r]);
    const float cl = rm == kResLow ? warp_sum(clow[r]) : 0.f;
    if (lane == 0 && k < n) {
      const double conv = rm == kResExact ? p.Rc[(size_t)b * p.nb + k] : (double)cl;
      R[k] = rlin + conv - fm[k];
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_lu_mixed(LuParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const DevOps &o = p.o;
  const LuSmem L(o, p.nb, p.j_in_smem != 0);
  double *th = (double *)(smb + L.th), *R = (double *)(smb + L.R);
  double *fm = (double *)(smb + L.fm), *red = (double *)(smb + L.red);
  float2 *ta = (float2 *)(smb + L.tah), *u2 = (float2 *)(smb + L.uh);
  float *rhs = (float *)(smb + L.rhs);
  float *J = p.j_in_smem ? (float *)(smb + L.J) : p.scratch + (size_t)blockIdx.x * p.nb * p.nb;
  const int tid = threadIdx.x, w = tid >> 5;
  const size_t nm = (size_t)o.n_max;
  int my_active = 0;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    rb_query_info qi = p.info[b];
    if (!is_active(qi, p.max_iter)) continue;
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    if (p.theta) {
      for (int i = tid; i < o.n_theta; i += blockDim.x) th[i] = p.theta[(size_t)b * o.n_theta + i];
    } else {
      theta_eval(o, p.mu[2 * b], p.mu[2 * b + 1], th);
    }
    __syncthreads();
    const double *tf = th + o.q_a + o.q_c;
    double *ub = p.u + (size_t)b * nm;
    for (int k = tid; k < n; k += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < o.q_f; ++q) s = fma(tf[q], o.f[(size_t)q * nm + k], s);
      fm[k] = s;
      float h, l;
      df_split(ub[k], h, l);
      u2[k] = make_float2(h, l);
    }
    for (int q = tid; q < o.q_a; q += blockDim.x) {
      float h, l;
      df_split(th[q], h, l);
      ta[q] = make_float2(h, l);
    }
    __syncthreads();
    const int rm = rung_of(p.rmode, qi.iters);
    for (int k0 = 4 * w; k0 < n; k0 += 4 * kWarps) lu_rows<4>(p, rm, b, n, k0, ta, u2, fm, J, n, R);
    __syncthreads();
    if (p.eval_only) {
      for (int k = tid; k < n; k += blockDim.x) p.R_out[(size_t)b * n + k] = R[k];
      __syncthreads();
      continue;
    }
    double rl = 0.0, fl = 0.0;
    for (int i = tid; i < n; i += blockDim.x) {
      rl += R[i] * R[i];
      fl += fm[i] * fm[i];
      rhs[i] = (float)(-R[i]);
    }
    const double rn = sqrt(block_sum(rl, red));
    const double fscale = fmax(1.0, sqrt(block_sum(fl, red)));
    qi.iters += 1;
    qi.res_norm = rn;
    qi.precision_used = RB_PREC_MIXED;
    if (!isfinite(rn)) {
      qi.status = RB_Q_NONFINITE;
    } else if (gepp_solve_block<float>(J, n, n, rhs, red)) {
      qi.status = RB_Q_SINGULAR;
    } else {
      double dl = 0.0;
      for (int i = tid; i < n; i += blockDim.x) {
        const double d = (double)rhs[i];
        dl += d * d;
        ub[i] += d;
      }
      const double dn = sqrt(block_sum(dl, red));
      qi.upd_norm = dn;
      if (!isfinite(dn)) qi.status = RB_Q_NONFINITE;
      else if (rm != kResLow && dn <= p.tol_upd && rn <= p.tol_res * fscale) qi.status = RB_Q_OK;
    }
    if (tid == 0) {
      p.info[b] = qi;
      if (is_active(qi, p.max_iter)) ++my_active;
    }
    __syncthreads();
  }
  if (tid == 0 && my_active) atomicAdd(p.active, my_active);
}

// Warp-per-query variant of k_lu_mixed for small Jacobians (no block barriers): each warp
// owns one query at a time and its own shared-memory slab.
struct WarpLuSmem {
  int th, R, fm, tah, uh, rhs, J, per_warp;  // byte offsets within a warp's slab
  __host__ __device__ WarpLuSmem(const DevOps &o, int nb) {
    int p = 0;
    th = p; p += 8 * ((o.n_theta + 1) & ~1);
    R = p; p += 8 * nb;
    fm = p; p += 8 * nb;
    tah = p; p += 8 * o.q_a;
    uh = p; p += 8 * nb;
    rhs = p; p += 4 * ((nb + 3) & ~3);
    p = (p + 15) & ~15;
    J = p; p += 4 * nb * (nb + 1);
    per_warp = (p + 15) & ~15;
  }
};

__global__ void __launch_bounds__(kThreads) k_lu_mixed_warp(LuParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const DevOps &o = p.o;
  const WarpLuSmem L(o, p.nb);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  uint8_t *slab = smb + (size_t)w * L.per_warp;
  double *th = (double *)(slab + L.th), *R = (double *)(slab + L.R), *fm = (double *)(slab + L.fm);
  float2 *ta = (float2 *)(slab + L.tah), *u2 = (float2 *)(slab + L.uh);
  float *rhs = (float *)(slab + L.rhs), *J = (float *)(slab + L.J);
  const int ld = p.nb + 1;
  const size_t nm = (size_t)o.n_max;
  int my_active = 0;
  for (int b = blockIdx.x * wpc + w; b < p.nq; b += gridDim.x * wpc) {
    rb_query_info qi = p.info[b];
    if (!is_active(qi, p.max_iter)) continue;
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    if (p.theta) {
      for (int i = lane; i < o.n_theta; i += 32) th[i] = p.theta[(size_t)b * o.n_theta + i];
    } else {
      theta_eval_strided(o, p.mu[2 * b], p.mu[2 * b + 1], th, lane, 32);
    }
    __syncwarp();
    const double *tf = th + o.q_a + o.q_c;
    double *ub = p.u + (size_t)b * nm;
    for (int k = lane; k < n; k += 32) {
      double sf = 0.0;
      for (int q = 0; q < o.q_f; ++q) sf = fma(tf[q], o.f[(size_t)q * nm + k], sf);
      fm[k] = sf;
      float h, l;
      df_split(ub[k], h, l);
      u2[k] = make_float2(h, l);
    }
    for (int q = lane; q < o.q_a; q += 32) {
      float h, l;
      df_split(th[q], h, l);
      ta[q] = make_float2(h, l);
    }
    __syncwarp();
    const int rm = rung_of(p.rmode, qi.iters);
    for (int k0 = 0; k0 < n; k0 += 8) lu_rows<8>(p, rm, b, n, k0, ta, u2, fm, J, ld, R);
    __syncwarp();
    if (p.eval_only) {
      for (int k = lane; k < n; k += 32) p.R_out[(size_t)b * n + k] = R[k];
      __syncwarp();
      continue;
    }
    double rl = 0.0, fl = 0.0;
    for (int i = lane; i < n; i += 32) {
      rl += R[i] * R[i];
      fl += fm[i] * fm[i];
      rhs[i] = (float)(-R[i]);
    }
    const double rn = sqrt(warp_sum(rl));
    const double fscale = fmax(1.0, sqrt(warp_sum(fl)));
    __syncwarp();
    qi.iters += 1;
    qi.res_norm = rn;
    qi.precision_used = RB_PREC_MIXED;
    if (!isfinite(rn)) {
      qi.status = RB_Q_NONFINITE;
    } else if (gepp_solve_warp<float>(J, ld, n, rhs)) {
      qi.status = RB_Q_SINGULAR;
    } else {
      double dl = 0.0;
      for (int i = lane; i < n; i += 32) {
        const double d = (double)rhs[i];
        dl += d * d;
        ub[i] += d;
      }
      const double dn = sqrt(warp_sum(dl));
      qi.upd_norm = dn;
      if (!isfinite(dn)) qi.status = RB_Q_NONFINITE;
      else if (rm != kResLow && dn <= p.tol_upd && rn <= p.tol_res * fscale) qi.status = RB_Q_OK;
    }
    if (lane == 0) {
      p.info[b] = qi;
      if (is_active(qi, p.max_iter)) ++my_active;
    }
    __syncwarp();
  }
  if (lane == 0 && my_active) atomicAdd(p.active, my_active);
}

// Pressure: r = fs(mu) - (As(mu) u + Cs_mu(u, u)), B(mu) p = r in FP64 (Eq. blocksolve-2).
struct PresSolveParams {
  DevOps o;
  const double *mu, *theta;
  const int *nsz;
  int nq;
  const double *u;    // [nq][n_max]
  const float2 *As2;  // [q_a][m][n_max] double-float
  const double *Rp;   // [b_pad][m]: Cs_mu(u, u) (sliced GEMM)
  double *p_out;     // [nq][m]
  rb_query_info *info;
};

// (As(mu) u)[k] for rows k0 .. k0 + RR - 1 by one warp in double-float:
// sum_j sum_q theta^a_q As_q[k][j] u_j, with theta^a (ta) and u (u2) pre-split.
template <int RR>
__device__ __forceinline__ void as_u_rows(const PresSolveParams &p, int n, int k0, int m,
                                          const float2 *ta, const float2 *u2, double *out) {
  const int lane = threadIdx.x & 31;
  const size_t nm = (size_t)p.o.n_max;
  float rh[RR], rl[RR];
#pragma unroll
  for (int r = 0; r < RR; ++r) rh[r] = rl[r] = 0.f;
  for (int j = lane; j < n; j += 32) {
    const float2 uj = u2[j];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const int k = k0 + r;
      if (k < m) {
        float ah = 0.f, al = 0.f;
        for (int q = 0; q < p.o.q_a; ++q) {
          const float2 a2 = __ldg(p.As2 + ((size_t)q * p.o.m + k) * nm + j);
          df_fma(ah, al, ta[q].x, ta[q].y, a2.x, a2.y);
        }
        df_fma(rh[r], rl[r], ah, al, uj.x, uj.y);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    const double v = df_warp_sum(rh[r], rl[r]);
    if (lane == 0 && k0 + r < m) out[k0 + r] = v;
  }
}

// shared-memory slab of one pressure solve (bytes)
struct PresSmem {
  int th, r, asu, ta, u2, red, Bm, total;
  __host__ __device__ PresSmem(const DevOps &o, bool with_red) {
    int p = 0;
    th = p; p += 8 * ((o.n_theta + 1) & ~1);
    r = p; p += 8 * o.m;
    asu = p; p += 8 * o.m;
    ta = p; p += 8 * o.q_a;
    u2 = p; p += 8 * o.n_max;
    red = p; p += with_red ? 8 * 4 * kWarps : 0;
    Bm = p; p += 8 * o.m * (o.m + 1);
    total = (p + 15) & ~15;
  }
};

__device__ __forceinline__ void pressure_rhs_prep(const PresSolveParams &p, int b, int n,
                                                  const double *th, float2 *ta, float2 *u2,
                                                  int t0, int stride) {
  const double *ub = p.u + (size_t)b * p.o.n_max;
  for (int j = t0; j < n; j += stride) {
    float h, l;
    df_split(ub[j], h, l);
    u2[j] = make_float2(h, l);
  }
  for (int q = t0; q < p.o.q_a; q += stride) {
    float h, l;
    df_split(th[q], h, l);
    ta[q] = make_float2(h, l);
  }
}

__global__ void __launch_bounds__(kThreads) k_pressure_solve(PresSolveParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const DevOps &o = p.o;
  const int m = o.m;
  const PresSmem L(o, true);
  double *th = (double *)(smb + L.th), *r = (double *)(smb + L.r), *asu = (double *)(smb + L.asu);
  float2 *ta = (float2 *)(smb + L.ta), *u2 = (float2 *)(smb + L.u2);
  double *red = (double *)(smb + L.red), *Bm = (double *)(smb + L.Bm);
  const int tid = threadIdx.x, w = tid >> 5;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    double *prow = p.p_out + (size_t)b * m;
    if (p.info[b].status != RB_Q_OK) {
      for (int i = tid; i < m; i += blockDim.x) prow[i] = 0.0;
      continue;
    }
    if (p.theta) {
      for (int i = tid; i < o.n_theta; i += blockDim.x) th[i] = p.theta[(size_t)b * o.n_theta + i];
    } else {
      theta_eval(o, p.mu[2 * b], p.mu[2 * b + 1], th);
    }
    __syncthreads();
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    pressure_rhs_prep(p, b, n, th, ta, u2, tid, blockDim.x);
    __syncthreads();
    for (int k0 = 4 * w; k0 < m; k0 += 4 * kWarps) as_u_rows<4>(p, n, k0, m, ta, u2, asu);
    const double *tf = th + o.q_a + o.q_c, *tb = tf + o.q_f;
    for (int e = tid; e < m * m; e += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < o.q_b; ++q) s = fma(tb[q], __ldg(o.B + (size_t)q * m * m + e), s);
      Bm[e] = s;
    }
    __syncthreads();
    for (int k = tid; k < m; k += blockDim.x) {
      double sf = 0.0;
      for (int q = 0; q < o.q_f; ++q) sf = fma(tf[q], o.fs[(size_t)q * m + k], sf);
      r[k] = sf - p.Rp[(size_t)b * m + k] - asu[k];
    }
    __syncthreads();
    const bool sing = gepp_solve_block<double>(Bm, m, m, r, red);
    for (int i = tid; i < m; i += blockDim.x) prow[i] = sing ? 0.0 : r[i];
    if (sing && tid == 0) p.info[b].status = RB_Q_SINGULAR;
    __syncthreads();
  }
}

// Warp-per-query variant of k_pressure_solve for small m.
__global__ void __launch_bounds__(kThreads) k_pressure_solve_warp(PresSolveParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const DevOps &o = p.o;
  const int m = o.m;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const PresSmem L(o, false);
  uint8_t *slab = smb + (size_t)w * L.total;
  double *th = (double *)(slab + L.th), *r = (double *)(slab + L.r), *asu = (double *)(slab + L.asu);
  float2 *ta = (float2 *)(slab + L.ta), *u2 = (float2 *)(slab + L.u2);
  double *Bm = (double *)(slab + L.Bm);
  const int ld = m + 1;
  for (int b = blockIdx.x * wpc + w; b < p.nq; b += gridDim.x * wpc) {
    double *prow = p.p_out + (size_t)b * m;
    if (p.info[b].status != RB_Q_OK) {
      for (int i = lane; i < m; i += 32) prow[i] = 0.0;
      continue;
    }
    if (p.theta) {
      for (int i = lane; i < o.n_theta; i += 32) th[i] = p.theta[(size_t)b * o.n_theta + i];
    } else {
      theta_eval_strided(o, p.mu[2 * b], p.mu[2 * b + 1], th, lane, 32);
    }
    __syncwarp();
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    pressure_rhs_prep(p, b, n, th, ta, u2, lane, 32);
    __syncwarp();
    for (int k0 = 0; k0 < m; k0 += 8) as_u_rows<8>(p, n, k0, m, ta, u2, asu);
    const double *tf = th + o.q_a + o.q_c, *tb = tf + o.q_f;
    for (int k = 0; k < m; ++k)
      for (int i = lane; i < m; i += 32) {
        double sb = 0.0;
        for (int q = 0; q < o.q_b; ++q) sb = fma(tb[q], __ldg(o.B + ((size_t)q * m + k) * m + i), sb);
        Bm[k * ld + i] = sb;
      }
    __syncwarp();
    for (int k = lane; k < m; k += 32) {
      double sf = 0.0;
      for (int q = 0; q < o.q_f; ++q) sf = fma(tf[q], o.fs[(size_t)q * m + k], sf);
      r[k] = sf - p.Rp[(size_t)b * m + k] - asu[k];
    }
    __syncwarp();
    const bool sing = gepp_solve_warp<double>(Bm, ld, m, r);
    for (int i = lane; i < m; i += 32) prow[i] = sing ? 0.0 : r[i];
    if (sing && lane == 0) p.info[b].status = RB_Q_SINGULAR;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------
// host side
void mixed_release(rb_ctx *ctx) {
  MixedState *M = ctx->mixed;
  if (!M) return;
  for (void *q : {(void *)M->Wj, (void *)M->WR.d, (void *)M->WP.d, (void *)M->A2, (void *)M->As2, (void *)M->Xj,
                  (void *)M->Xd, (void *)M->xexp, (void *)M->ufT, (void *)M->Jc, (void *)M->Rc,
                  (void *)M->Rp, (void *)M->lu_scratch, (void *)M->dev_words, (void *)M->info_own})
    ctx_free(ctx, q);
  if (M->h_words) cudaFreeHost(M->h_words);
  delete M;
  ctx->mixed = nullptr;
}

// digits of the convection segment (RB_DIGITS) and of the linear segment (RB_DIGITS_LINEAR)
static int sliced_digits(const char *var, int dflt) {
  const char *e = getenv(var);
  const int s = e ? atoi(e) : dflt;
  return std::min(8, std::max(2, s));
}

static int absmax_exp(rb_ctx *ctx, const double *x, size_t count, int *e_out, cudaStream_t st) {
  MixedState *M = ctx->mixed;
  unsigned long long *mx = (unsigned long long *)(M->dev_words + 8);
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
  *e_out = ex;
  return RB_OK;
}

static int build_sliced(rb_ctx *ctx, SlicedW &W, int kind, int nk, __nv_bfloat16 *Wj,
                        cudaStream_t st) {
  MixedState *M = ctx->mixed;
  const DevOps &o = ctx->ops;
  W.nk = nk;
  W.Npad = round_up(nk * M->nb, kTcBN);
  void *p;
  int rc = ctx_alloc(ctx, &p, 2 * (size_t)M->Smax * W.Npad * M->Kpad, "W digit slices");
  if (rc != RB_OK) return rc;
  W.d = (__nv_bfloat16 *)p;
  const size_t nm = o.n_max;
  if (kind == 0) {
    if ((rc = absmax_exp(ctx, o.Dt, (size_t)o.q_c * nm * nm * nm, &W.wexp[0], st)) != RB_OK) return rc;
    if (M->kb1 && (rc = absmax_exp(ctx, o.A, (size_t)o.q_a * nm * nm, &W.wexp[1], st)) != RB_OK) return rc;
  } else {
    if ((rc = absmax_exp(ctx, o.Cs, (size_t)o.q_c * nm * nm * o.m, &W.wexp[0], st)) != RB_OK) return rc;
    W.wexp[0] += 1;  // the operand holds 2 Cs
    if (M->kb1 && (rc = absmax_exp(ctx, o.As, (size_t)o.q_a * o.m * nm, &W.wexp[1], st)) != RB_OK) return rc;
  }
  BuildWParams bw{o, kind, M->nb, nk, M->Kpad0, M->Kpad, W.Npad, M->S0, M->S1, W.wexp[0], W.wexp[1], W.d, Wj};
  k_build_w<<<ctx->sms * 8, 256, 0, st>>>(bw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_build_w");
  if (!make_map(&W.tm, W.d, (uint64_t)M->Smax * W.Npad, M->Kpad, kTcBN))
    return set_error(ctx, RB_ERR_CUDA, "tensor map encode (W)");
  return RB_OK;
}

// Build the operator layouts of the mixed path (once per operator set).
static int mixed_layouts(rb_ctx *ctx, cudaStream_t st) {
  if (ctx->mixed && ctx->mixed->Wj) return RB_OK;
  if (!encode_fn()) return set_error(ctx, RB_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if (ctx->cc_major != 10) return set_error(ctx, RB_ERR_ARG, "tensor-core path needs an sm_10x GPU");
  if (!ctx->mixed) ctx->mixed = new MixedState();
  MixedState *M = ctx->mixed;
  const DevOps &o = ctx->ops;
  M->nb = o.n_max;
  M->Kpad0 = round_up(o.q_c * M->nb, 64);
  M->kb0 = M->Kpad0 / 64;
  // the linear affine term A(mu) u is evaluated in double-float on the CUDA cores, so the
  // sliced GEMM carries the convection segment only (the kernel also supports a second one)
  M->kb1 = 0;
  M->Kpad = M->Kpad0 + 64 * M->kb1;
  M->Npad = round_up(M->nb * M->nb, kTcBN);
  M->S0 = sliced_digits("RB_DIGITS", 6);
  M->S1 = sliced_digits("RB_DIGITS_LINEAR", 7);
  M->Smax = M->kb1 ? std::max(M->S0, M->S1) : M->S0;
  int rc;
  void *p;
  if ((rc = ctx_alloc(ctx, &p, 64, "mixed words")) != RB_OK) return rc;
  M->dev_words = (int *)p;
  cudaMemsetAsync(M->dev_words, 0, 64, st);
  if (cudaMallocHost(&M->h_words, 64) != cudaSuccess) return set_error(ctx, RB_ERR_OOM, "pinned words");
  const size_t nm = o.n_max;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)o.q_a * nm * nm, "A (double-float)")) != RB_OK) return rc;
  M->A2 = (float2 *)p;
  k_split_f2<<<ctx->sms * 4, 256, 0, st>>>(o.A, M->A2, (size_t)o.q_a * nm * nm);
  if (o.m > 0 && o.B) {
    if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)o.q_a * o.m * nm, "As (double-float)")) != RB_OK) return rc;
    M->As2 = (float2 *)p;
    k_split_f2<<<ctx->sms * 4, 256, 0, st>>>(o.As, M->As2, (size_t)o.q_a * o.m * nm);
  }
  if ((rc = ctx_alloc(ctx, &p, 2 * 2 * (size_t)M->Npad * M->Kpad0, "W (split BF16)")) != RB_OK) return rc;
  M->Wj = (__nv_bfloat16 *)p;
  if ((rc = build_sliced(ctx, M->WR, 0, M->nb, M->Wj, st)) != RB_OK) return rc;
  if (o.m > 0 && o.B && (rc = build_sliced(ctx, M->WP, 1, o.m, nullptr, st)) != RB_OK) return rc;
  if (!make_map(&M->tmWj, M->Wj, 2 * (uint64_t)M->Npad, M->Kpad0, kTcBN))
    return set_error(ctx, RB_ERR_CUDA, "tensor map encode (Wj)");
  return RB_OK;
}

static int mixed_batch_scratch(rb_ctx *ctx, int nq) {
  MixedState *M = ctx->mixed;
  const int b_pad = round_up(std::max(nq, 1), 128);
  if (b_pad <= M->bcap) return RB_OK;
  for (void *q : {(void *)M->Xj, (void *)M->Xd, (void *)M->xexp, (void *)M->ufT, (void *)M->Jc,
                  (void *)M->Rc, (void *)M->Rp})
    ctx_free(ctx, q);
  M->Xj = M->Xd = nullptr; M->xexp = nullptr; M->ufT = nullptr; M->Jc = nullptr;
  M->Rc = M->Rp = nullptr;
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
  if ((rc = ctx_alloc(ctx, &p, 4 * (size_t)b_pad * M->Npad, "J^c (FP32)")) != RB_OK) return rc;
  M->Jc = (float *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb, "R (FP64)")) != RB_OK) return rc;
  M->Rc = (double *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * m, "pressure rhs (FP64)")) != RB_OK) return rc;
  M->Rp = (double *)p;
  // zero once so that padded rows never hold NaN bit patterns
  cudaMemsetAsync(M->Xj, 0, 2 * 3 * xs0, ctx->stream);
  cudaMemsetAsync(M->Xd, 0, 2 * xs * M->Smax, ctx->stream);
  cudaMemsetAsync(M->xexp, 0, 8 * (size_t)b_pad, ctx->stream);
  cudaMemsetAsync(M->ufT, 0, 8 * (size_t)b_pad * M->nb, ctx->stream);
  if (!make_map(&M->tmXj, M->Xj, 3 * (uint64_t)b_pad, M->Kpad0, 128) ||
      !make_map(&M->tmXd, M->Xd, (uint64_t)M->Smax * b_pad, M->Kpad, 128))
    return set_error(ctx, RB_ERR_CUDA, "tensor map encode (X)");
  M->bcap = b_pad;
  return RB_OK;
}

static int launch_build_x(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                          const int *d_n, const double *d_u, const rb_query_info *d_info,
                          int mode, int digits, double *out, int nout, cudaStream_t st) {
  MixedState *M = ctx->mixed;
  BuildXParams bx{};
  bx.o = ctx->ops;
  bx.mu = d_mu;
  bx.theta = d_theta;
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
  bx.out = out;
  bx.nout = nout;
  const int mk = prof_begin(ctx, RB_K_BUILD_X, st);
  k_build_x<<<std::min(nq, ctx->sms * 8), kThreads, 0, st>>>(bx);
  prof_end(ctx, mk, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_build_x");
  return RB_OK;
}

static TcGemmParams gemm_params(rb_ctx *ctx, int nq) {
  MixedState *M = ctx->mixed;
  TcGemmParams g{};
  g.m_tiles = round_up(nq, 128) / 128;
  g.S[0] = M->S0;
  g.S[1] = M->S1;
  g.b_pad = M->bcap;
  g.nq = nq;
  g.nj = M->nb;
  g.xexp = M->xexp;
  g.ufT = M->ufT;
  g.err = M->dev_words + 1;
  return g;
}

// One Newton step's contraction work for the whole batch: X build + both GEMMs.
static int mixed_contract(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                          const int *d_n, const double *d_u, const rb_query_info *d_info,
                          bool exact, cudaStream_t st) {
  MixedState *M = ctx->mixed;
  int rc = launch_build_x(ctx, d_mu, d_theta, nq, d_n, d_u, d_info, 0, exact ? 1 : 0, M->Rc, M->nb, st);
  if (rc != RB_OK) return rc;
  TcGemmParams g = gemm_params(ctx, nq);
  g.n_tiles = M->Npad / kTcBN;
  g.kb[0] = M->kb0;
  g.kb[1] = 0;
  g.n_pad = M->Npad;
  g.nk = M->nb;
  g.ldj = M->Npad;
  g.Jc = M->Jc;
  g.nsplit = 3;
  int mk = prof_begin(ctx, RB_K_GEMM_JAC, st);
  cudaError_t e = launch_tc_gemm(kPlain, M->tmXj, M->tmWj, g, ctx->sms, st);
  prof_end(ctx, mk, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_tc_gemm (Jacobian)");
  if (!exact) return RB_OK;
  g.kb[1] = M->kb1;
  g.n_tiles = M->WR.Npad / kTcBN;
  g.n_pad = M->WR.Npad;
  g.wexp[0] = M->WR.wexp[0];
  g.wexp[1] = M->WR.wexp[1];
  g.out = M->Rc;
  mk = prof_begin(ctx, RB_K_GEMM_RES, st);
  e = launch_tc_gemm(kSliced, M->tmXd, M->WR.tm, g, ctx->sms, st);
  prof_end(ctx, mk, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_tc_gemm (residual)");
  return RB_OK;
}

constexpr int kWarpLuMaxN = 80;  // warp-per-query elimination up to this size

static int launch_lu(rb_ctx *ctx, LuParams &lp, int nq, cudaStream_t st) {
  MixedState *M = ctx->mixed;
  if (M->nb <= kWarpLuMaxN) {
    const int per_warp = WarpLuSmem(ctx->ops, M->nb).per_warp;
    const int wpc = std::max(1, std::min(8, (200 * 1024) / per_warp));
    const size_t smem = (size_t)wpc * per_warp;
    const int per_sm = std::max(1, std::min(64 / wpc, (int)((size_t)ctx->smem_per_sm / (smem + 1024))));
    const int grid = std::max(1, std::min((nq + wpc - 1) / wpc, per_sm * ctx->sms));
    cudaError_t e = cudaFuncSetAttribute(k_lu_mixed_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_mixed_warp attr");
    const int mk = prof_begin(ctx, RB_K_LU, st);
    k_lu_mixed_warp<<<grid, 32 * wpc, smem, st>>>(lp);
    prof_end(ctx, mk, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_mixed_warp");
    return RB_OK;
  }
  const size_t smem_in = LuSmem(ctx->ops, M->nb, true).total;
  lp.j_in_smem = smem_in <= (size_t)ctx->max_smem ? 1 : 0;
  const size_t smem = LuSmem(ctx->ops, M->nb, lp.j_in_smem != 0).total;
  const int per_sm = std::max(1, std::min(2048 / kThreads, (int)((size_t)ctx->smem_per_sm / (smem + 1024))));
  const int grid = std::max(1, std::min(nq, per_sm * ctx->sms));
  if (!lp.j_in_smem) {
    if (M->lu_grid < grid) {
      ctx_free(ctx, M->lu_scratch);
      M->lu_scratch = nullptr;
      M->lu_grid = 0;
      void *p;
      int rc = ctx_alloc(ctx, &p, 4 * (size_t)grid * M->nb * M->nb, "LU scratch");
      if (rc != RB_OK) return rc;
      M->lu_scratch = (float *)p;
      M->lu_grid = grid;
    }
    lp.scratch = M->lu_scratch;
  }
  cudaError_t e = cudaFuncSetAttribute(k_lu_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_mixed attr");
  const int mk = prof_begin(ctx, RB_K_LU, st);
  k_lu_mixed<<<grid, kThreads, smem, st>>>(lp);
  prof_end(ctx, mk, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_mixed");
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

static int mixed_pressure(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                          const int *d_n, const double *d_u, double *d_p, rb_query_info *info,
                          cudaStream_t st) {
  MixedState *M = ctx->mixed;
  const DevOps &o = ctx->ops;
  int rc = launch_build_x(ctx, d_mu, d_theta, nq, d_n, d_u, info, 1, 1, M->Rp, o.m, st);
  if (rc != RB_OK) return rc;
  TcGemmParams g = gemm_params(ctx, nq);
  g.kb[0] = M->kb0;
  g.kb[1] = M->kb1;
  g.n_tiles = M->WP.Npad / kTcBN;
  g.n_pad = M->WP.Npad;
  g.nk = o.m;
  g.wexp[0] = M->WP.wexp[0];
  g.wexp[1] = M->WP.wexp[1];
  g.out = M->Rp;
  int mk = prof_begin(ctx, RB_K_GEMM_PRES, st);
  cudaError_t e = launch_tc_gemm(kSliced, M->tmXd, M->WP.tm, g, ctx->sms, st);
  prof_end(ctx, mk, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_tc_gemm (pressure)");
  PresSolveParams pp{o, d_mu, d_theta, d_n, nq, d_u, M->As2, M->Rp, d_p, info};
  const size_t per_warp = PresSmem(o, false).total;
  if (per_warp <= 24 * 1024) {
    const int wpc = std::max(1, std::min(8, (int)((192 * 1024) / per_warp)));
    const size_t smem = wpc * per_warp;
    e = cudaFuncSetAttribute(k_pressure_solve_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_pressure_solve_warp attr");
    mk = prof_begin(ctx, RB_K_PRESSURE, st);
    k_pressure_solve_warp<<<std::min((nq + wpc - 1) / wpc, ctx->sms * 8), 32 * wpc, smem, st>>>(pp);
    prof_end(ctx, mk, st);
  } else {
    const size_t smem = PresSmem(o, true).total;
    e = cudaFuncSetAttribute(k_pressure_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_pressure_solve attr");
    mk = prof_begin(ctx, RB_K_PRESSURE, st);
    k_pressure_solve<<<std::min(nq, ctx->sms * 8), kThreads, smem, st>>>(pp);
    prof_end(ctx, mk, st);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_pressure_solve");
  return RB_OK;
}

int solve_mixed(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq, const int *d_n,
                double *d_u, double *d_p, rb_query_info *d_info, cudaStream_t st) {
  int rc = mixed_layouts(ctx, st);
  if (rc != RB_OK) return rc;
  if ((rc = mixed_batch_scratch(ctx, nq)) != RB_OK) return rc;
  MixedState *M = ctx->mixed;
  rb_query_info *info = d_info ? d_info : own_info(ctx, nq);
  if (!info) return set_error(ctx, RB_ERR_OOM, "info scratch");
  const DevOps &o = ctx->ops;
  int mk = prof_begin(ctx, RB_K_INIT, st);
  k_mixed_init<<<std::min(nq, ctx->sms * 8), 128, 0, st>>>(nq, o.n_max, d_n, d_u, info);
  prof_end(ctx, mk, st);
  cudaMemsetAsync(M->dev_words, 0, 8, st);
  LuParams lp{};
  lp.o = o;
  lp.mu = d_mu;
  lp.theta = d_theta;
  lp.nsz = d_n;
  lp.nq = nq;
  lp.nb = M->nb;
  lp.ldj = M->Npad;
  lp.max_iter = ctx->cfg.max_iter;
  lp.tol_upd = ctx->cfg.tol_update;
  lp.tol_res = ctx->cfg.tol_res;
  lp.A2 = M->A2;
  lp.Jc = M->Jc;
  lp.Rc = M->Rc;
  lp.u = d_u;
  lp.info = info;
  lp.active = M->dev_words;
  lp.rmode = kResLadder;  // every query climbs zero -> low -> exact with its own iterations
  for (int it = 0; it < ctx->cfg.max_iter; ++it) {
    cudaMemsetAsync(M->dev_words, 0, 4, st);
    if (it >= 1 && (rc = mixed_contract(ctx, d_mu, d_theta, nq, d_n, d_u, info, it >= 2, st)) != RB_OK)
      return rc;
    if ((rc = launch_lu(ctx, lp, nq, st)) != RB_OK) return rc;
    if ((rc = check_words(ctx, st, "mixed Newton step")) != RB_OK) return rc;
    if (M->h_words[0] == 0) break;
  }
  if (d_p && o.m > 0 && o.B) {
    if ((rc = mixed_pressure(ctx, d_mu, d_theta, nq, d_n, d_u, d_p, info, st)) != RB_OK) return rc;
    if ((rc = check_words(ctx, st, "pressure recovery")) != RB_OK) return rc;
  }
  if (ctx->prof) prof_collect(ctx);
  return RB_OK;
}

// ---- pieces used by the continuous-batching server ----------------------------------------
int mixed_prepare(rb_ctx *ctx, int capacity, cudaStream_t st) {
  int rc = mixed_layouts(ctx, st);
  if (rc != RB_OK) return rc;
  if ((rc = mixed_batch_scratch(ctx, capacity)) != RB_OK) return rc;
  return own_info(ctx, 1) ? RB_OK : set_error(ctx, RB_ERR_OOM, "info scratch");
}

// Device bytes one more slot of batch state costs (X operands, Jacobian, residual, LU).
size_t mixed_slot_bytes(const rb_ctx *ctx) {
  const DevOps &o = ctx->ops;
  const size_t nb = o.n_max, Kpad0 = (size_t)round_up(o.q_c * o.n_max, 64);
  const size_t Npad = (size_t)round_up(o.n_max * o.n_max, kTcBN);
  const int S = 8;
  return 2 * 3 * Kpad0 + 2 * S * Kpad0 + 8 + 8 * nb + 4 * Npad + 8 * nb + 8 * (size_t)(o.m + 1) +
         8 * nb + 64;
}

// One Newton iteration for every live slot: the contraction work the slots' ladder rungs need,
// then elimination and update (no host synchronisation).
int mixed_iteration(rb_ctx *ctx, const double *d_mu, int nq, const int *d_n, double *d_u,
                    rb_query_info *info, bool need_jacobian, bool need_exact, cudaStream_t st) {
  MixedState *M = ctx->mixed;
  int rc;
  cudaMemsetAsync(M->dev_words, 0, 4, st);
  if (need_jacobian &&
      (rc = mixed_contract(ctx, d_mu, nullptr, nq, d_n, d_u, info, need_exact, st)) != RB_OK)
    return rc;
  LuParams lp{};
  lp.o = ctx->ops;
  lp.mu = d_mu;
  lp.nsz = d_n;
  lp.nq = nq;
  lp.nb = M->nb;
  lp.ldj = M->Npad;
  lp.max_iter = ctx->cfg.max_iter;
  lp.tol_upd = ctx->cfg.tol_update;
  lp.tol_res = ctx->cfg.tol_res;
  lp.A2 = M->A2;
  lp.Jc = M->Jc;
  lp.Rc = M->Rc;
  lp.u = d_u;
  lp.info = info;
  lp.active = M->dev_words;
  lp.rmode = kResLadder;
  return launch_lu(ctx, lp, nq, st);
}

// Pressure for every slot whose status is RB_Q_OK.
int mixed_pressure_ok(rb_ctx *ctx, const double *d_mu, int nq, const int *d_n, const double *d_u,
                      double *d_p, rb_query_info *info, cudaStream_t st) {
  if (!(ctx->ops.m > 0 && ctx->ops.B && d_p)) return RB_OK;
  return mixed_pressure(ctx, d_mu, nullptr, nq, d_n, d_u, d_p, info, st);
}

int mixed_error_word(rb_ctx *ctx, cudaStream_t st) {
  return check_words(ctx, st, "serving step");
}

int eval_mixed(rb_ctx *ctx, const double *d_mu, int nq, int n, const double *d_u, int precision,
               double *d_R, double *d_J, cudaStream_t st) {
  if (precision != RB_PREC_MIXED) return set_error(ctx, RB_ERR_ARG, "unknown precision %d", precision);
  int rc = mixed_layouts(ctx, st);
  if (rc != RB_OK) return rc;
  if ((rc = mixed_batch_scratch(ctx, nq)) != RB_OK) return rc;
  MixedState *M = ctx->mixed;
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
  if ((rc = mixed_contract(ctx, d_mu, nullptr, nq, nsz, uw, info, true, st)) != RB_OK) return rc;
  LuParams lp{};
  lp.rmode = kResExact;
  lp.o = o;
  lp.mu = d_mu;
  lp.nsz = nsz;
  lp.nq = nq;
  lp.nb = M->nb;
  lp.ldj = M->Npad;
  lp.max_iter = ctx->cfg.max_iter;
  lp.A2 = M->A2;
  lp.Jc = M->Jc;
  lp.Rc = M->Rc;
  lp.u = uw;
  lp.info = info;
  lp.active = M->dev_words;
  lp.eval_only = 1;
  lp.R_out = d_R;
  lp.J_out = d_J;
  if ((rc = launch_lu(ctx, lp, nq, st)) != RB_OK) return rc;
  return check_words(ctx, st, "rb_eval (mixed)");
}

}  // namespace rb
