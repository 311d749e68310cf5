// rb_mixed.cu -- mixed-precision batched Newton (inexact Newton, Sec. 3.6 Jacobian on tensor cores).
//
// Per iteration, for every active query b of the batch:
//   1. k_build_x: X_b = theta^c(mu_b) (x) u_b (BF16) for the Jacobian GEMM, and the 7-bit digit
//      slices of X'_b = X_b / 2 for the sliced residual GEMM; u_b as (hi, lo) floats; R^c_b = 0.
//   2. k_tc_gemm<kPlain>:  J^c = X W^T on tcgen05 (BF16 in, FP32 accumulate) -> Jc (FP32).
//   3. k_tc_gemm<kSliced>: R^c_b[k] = sum_j u_b[j] (X'_b W^T)[(k,j)], exact digit products,
//      double-float contraction -> FP64 (the convection term C_mu(u_b, u_b), Eq. velonly).
//   4. k_lu_mixed: R = A(mu) u - f(mu) + R^c in FP64; J = fl32(A(mu)) + J^c; GEPP in FP32 on
//      J delta = -R; u += delta in FP64; stopping rule (Sec. 6) on the FP64 norms.
// The Jacobian is inexact (BF16 convection part), the residual and the test are FP64-accurate,
// so the iteration converges to the FP64 solution (linearly at rate ~ ||J^-1 (J~ - J)||).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "rb_ctx.h"
#include "rb_mixed.cuh"

namespace rb {

struct MixedState {
  // operator layouts for the Jacobian size nb (= n_max)
  int nb = 0, K = 0, Kpad = 0, kb = 0, Npad = 0, S = 0, wexp = 0;
  __nv_bfloat16 *Wj = nullptr;  // [Npad][Kpad]
  __nv_bfloat16 *Wd = nullptr;  // [S][Npad][Kpad]
  CUtensorMap tmWj, tmWd;
  // batch scratch
  int bcap = 0;
  __nv_bfloat16 *Xj = nullptr, *Xd = nullptr;
  int *xexp = nullptr;
  float2 *uf = nullptr;
  float *Jc = nullptr;
  double *Rc = nullptr;
  CUtensorMap tmXj, tmXd;
  float *lu_scratch = nullptr;
  int lu_grid = 0;
  int *dev_words = nullptr;  // [0] active count, [1] error word
  int *h_words = nullptr;    // pinned mirror
  rb_query_info *info_own = nullptr;
  int info_cap = 0;
  int last_launches = 0;
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
  const double a = fabs(v) * scale;
  const long long F = __double2ll_rz(a);
  const float sg = v < 0 ? -1.f : 1.f;
  for (int i = 1; i <= S; ++i) {
    const int d = (int)((F >> (kDigitBits * (S - i))) & 127);
    out[(size_t)(i - 1) * slice_stride] = __float2bfloat16_rn(sg * (float)d);
  }
}

__global__ void k_absmax(const double *x, size_t count, unsigned long long *out) {
  double m = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// W[(k,j)][(q,l)] = D~_q[k][j][l] from Dt [q][l][k][j] (n_max strides): BF16 copy and S digit
// slices on the grid 2^(wexp - 7 i).
__global__ void k_build_w(const double *Dt, int nm, int qc, int nb, int Kpad, int Npad, int S,
                          int wexp, __nv_bfloat16 *Wj, __nv_bfloat16 *Wd) {
  const size_t total = (size_t)Npad * Kpad;
  const double scale = ldexp(1.0, kDigitBits * S - wexp);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int kap = (int)(e % Kpad);
    const int c = (int)(e / Kpad);
    double v = 0.0;
    if (c < nb * nb && kap < qc * nb) {
      const int k = c / nb, j = c % nb, q = kap / nb, l = kap % nb;
      v = Dt[(((size_t)q * nm + l) * nm + k) * nm + j];
    }
    Wj[e] = __float2bfloat16_rn((float)v);
    digits7(v, scale, S, Wd + e, total);
  }
}

// Start of a batch: status NOT_CONVERGED (active) or REJECTED, u = 0.
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
  int nq, nb, Kpad, S, b_pad, max_iter;
  const double *u;  // [nq][n_max]
  const rb_query_info *info;
  __nv_bfloat16 *Xj, *Xd;
  int *xexp;
  float2 *uf;
  double *Rc;
};

__device__ __forceinline__ bool is_active(const rb_query_info &q, int max_iter) {
  return q.status == RB_Q_NOT_CONVERGED && q.iters < max_iter;
}

__global__ void __launch_bounds__(kThreads) k_build_x(BuildXParams p) {
  __shared__ double th[4 * RB_Q_MAX];
  __shared__ double red[4 * kWarps];
  const DevOps &o = p.o;
  const int tid = threadIdx.x;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    if (!is_active(p.info[b], p.max_iter)) continue;
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    if (p.theta) {
      for (int i = tid; i < o.n_theta; i += blockDim.x) th[i] = p.theta[(size_t)b * o.n_theta + i];
    } else {
      theta_eval(o, p.mu[2 * b], p.mu[2 * b + 1], th);
    }
    __syncthreads();
    const double *tc = th + o.q_a;
    const double *ub = p.u + (size_t)b * o.n_max;
    double m = 0.0;
    for (int kap = tid; kap < o.q_c * p.nb; kap += blockDim.x) {
      const int q = kap / p.nb, l = kap % p.nb;
      if (l < n) m = fmax(m, fabs(0.5 * tc[q] * ub[l]));
    }
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    double mx = 0.0;
    for (int i = 0; i < kWarps; ++i) mx = fmax(mx, red[i]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    const double scale = ldexp(1.0, kDigitBits * p.S - e);
    const size_t sstride = (size_t)p.b_pad * p.Kpad;
    for (int kap = tid; kap < p.Kpad; kap += blockDim.x) {
      double x = 0.0;
      if (kap < o.q_c * p.nb) {
        const int q = kap / p.nb, l = kap % p.nb;
        if (l < n) x = tc[q] * ub[l];
      }
      const size_t off = (size_t)b * p.Kpad + kap;
      p.Xj[off] = __float2bfloat16_rn((float)x);
      digits7(0.5 * x, scale, p.S, p.Xd + off, sstride);
    }
    for (int j = tid; j < p.nb; j += blockDim.x) {
      const double v = j < n ? ub[j] : 0.0;
      const float hi = (float)v;
      p.uf[(size_t)b * p.nb + j] = make_float2(hi, (float)(v - (double)hi));
      p.Rc[(size_t)b * p.nb + j] = 0.0;
    }
    if (tid == 0) p.xexp[b] = e;
    __syncthreads();
  }
}

struct LuParams {
  DevOps o;
  const double *mu, *theta;
  const int *nsz;
  int nq, nb, ldj, max_iter, j_in_smem;
  double tol_upd, tol_res;
  const float *Jc;
  const double *Rc;
  double *u;             // [nq][n_max], updated in place
  rb_query_info *info;   // [nq]
  float *scratch;        // [grid][nb * nb] when J is not in shared memory
  int *active;           // count of queries still active after this iteration
  int eval_only;         // 1: write R and J (FP64) to R_out / J_out instead of solving
  double *R_out, *J_out;
};

struct LuSmem {
  int th, u, R, fm, red, rhs, J, total;  // offsets in bytes
  __host__ __device__ LuSmem(const DevOps &o, int nb, bool j_in_smem) {
    int p = 0;
    th = p; p += 8 * ((o.n_theta + 1) & ~1);
    u = p; p += 8 * nb;
    R = p; p += 8 * nb;
    fm = p; p += 8 * nb;
    red = p; p += 8 * 4 * kWarps;
    rhs = p; p += 4 * ((nb + 3) & ~3);
    p = (p + 15) & ~15;
    J = p;
    if (j_in_smem) p += 4 * nb * nb;
    total = p;
  }
};

__global__ void __launch_bounds__(kThreads) k_lu_mixed(LuParams p) {
  extern __shared__ __align__(16) uint8_t smb[];
  const DevOps &o = p.o;
  const LuSmem L(o, p.nb, p.j_in_smem != 0);
  double *th = (double *)(smb + L.th), *u = (double *)(smb + L.u), *R = (double *)(smb + L.R);
  double *fm = (double *)(smb + L.fm), *red = (double *)(smb + L.red);
  float *rhs = (float *)(smb + L.rhs);
  float *J = p.j_in_smem ? (float *)(smb + L.J) : p.scratch + (size_t)blockIdx.x * p.nb * p.nb;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
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
    double *ub = p.u + (size_t)b * nm;
    for (int i = tid; i < n; i += blockDim.x) u[i] = ub[i];
    __syncthreads();
    const double *tf = th + o.q_a + o.q_c;
    for (int k = tid; k < n; k += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < o.q_f; ++q) s = fma(tf[q], o.f[(size_t)q * nm + k], s);
      fm[k] = s;
    }
    __syncthreads();
    // A(mu) in FP64: J = fl32(A(mu)) + J^c, R = A(mu) u - f + R^c; one warp per row
    const float *jc = p.Jc + (size_t)b * p.ldj;
    for (int k = w; k < n; k += kWarps) {
      double r = 0.0;
      for (int j = lane; j < n; j += 32) {
        double a = 0.0;
        for (int q = 0; q < o.q_a; ++q) a = fma(th[q], __ldg(o.A + ((size_t)q * nm + k) * nm + j), a);
        r = fma(a, u[j], r);
        if (p.eval_only)
          p.J_out[((size_t)b * n + k) * n + j] = a + (double)jc[k * p.nb + j];
        else
          J[(size_t)k * n + j] = (float)a + jc[k * p.nb + j];
      }
      r = warp_sum(r);
      if (lane == 0) R[k] = r - fm[k] + p.Rc[(size_t)b * p.nb + k];
    }
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
        ub[i] = u[i] + d;
      }
      const double dn = sqrt(block_sum(dl, red));
      qi.upd_norm = dn;
      if (!isfinite(dn)) qi.status = RB_Q_NONFINITE;
      else if (dn <= p.tol_upd && rn <= p.tol_res * fscale) qi.status = RB_Q_OK;
    }
    if (tid == 0) {
      p.info[b] = qi;
      if (is_active(qi, p.max_iter)) ++my_active;
    }
    __syncthreads();
  }
  if (tid == 0 && my_active) atomicAdd(p.active, my_active);
}

// ---------------------------------------------------------------------------------------
// host side
void mixed_release(rb_ctx *ctx) {
  MixedState *M = ctx->mixed;
  if (!M) return;
  ctx_free(ctx, M->Wj);
  ctx_free(ctx, M->Wd);
  ctx_free(ctx, M->Xj);
  ctx_free(ctx, M->Xd);
  ctx_free(ctx, M->xexp);
  ctx_free(ctx, M->uf);
  ctx_free(ctx, M->Jc);
  ctx_free(ctx, M->Rc);
  ctx_free(ctx, M->lu_scratch);
  ctx_free(ctx, M->dev_words);
  ctx_free(ctx, M->info_own);
  if (M->h_words) cudaFreeHost(M->h_words);
  delete M;
  ctx->mixed = nullptr;
}

static int sliced_digits() {
  const char *e = getenv("RB_DIGITS");
  int s = e ? atoi(e) : 6;
  return std::min(8, std::max(2, s));
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
  M->K = o.q_c * M->nb;
  M->Kpad = round_up(M->K, 64);
  M->kb = M->Kpad / 64;
  M->Npad = round_up(M->nb * M->nb, kTcBN);
  M->S = sliced_digits();
  int rc;
  void *p;
  const size_t wsz = (size_t)M->Npad * M->Kpad;
  if ((rc = ctx_alloc(ctx, &p, 2 * wsz, "W (BF16)")) != RB_OK) return rc;
  M->Wj = (__nv_bfloat16 *)p;
  if ((rc = ctx_alloc(ctx, &p, 2 * wsz * M->S, "W digit slices")) != RB_OK) return rc;
  M->Wd = (__nv_bfloat16 *)p;
  if ((rc = ctx_alloc(ctx, &p, 64, "mixed words")) != RB_OK) return rc;
  M->dev_words = (int *)p;
  if (cudaMallocHost(&M->h_words, 64) != cudaSuccess) return set_error(ctx, RB_ERR_OOM, "pinned words");
  // global exponent of the W grid
  cudaMemsetAsync(M->dev_words, 0, 64, st);
  unsigned long long *mx = (unsigned long long *)(M->dev_words + 8);
  const size_t dcount = (size_t)o.q_c * o.n_max * o.n_max * o.n_max;
  k_absmax<<<ctx->sms * 4, 256, 0, st>>>(o.Dt, dcount, mx);
  unsigned long long hm = 0;
  cudaError_t e = cudaMemcpyAsync(&hm, mx, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "W exponent");
  double dmax;
  memcpy(&dmax, &hm, 8);
  int we = 0;
  if (dmax > 0) frexp(dmax, &we);
  M->wexp = we;
  k_build_w<<<ctx->sms * 8, 256, 0, st>>>(o.Dt, o.n_max, o.q_c, M->nb, M->Kpad, M->Npad, M->S,
                                          M->wexp, M->Wj, M->Wd);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_build_w");
  if (!make_map(&M->tmWj, M->Wj, M->Npad, M->Kpad, kTcBN) ||
      !make_map(&M->tmWd, M->Wd, (uint64_t)M->S * M->Npad, M->Kpad, kTcBN))
    return set_error(ctx, RB_ERR_CUDA, "tensor map encode (W)");
  return RB_OK;
}

static int mixed_batch_scratch(rb_ctx *ctx, int nq) {
  MixedState *M = ctx->mixed;
  const int b_pad = round_up(std::max(nq, 1), 128);
  if (b_pad <= M->bcap) return RB_OK;
  ctx_free(ctx, M->Xj); ctx_free(ctx, M->Xd); ctx_free(ctx, M->xexp); ctx_free(ctx, M->uf);
  ctx_free(ctx, M->Jc); ctx_free(ctx, M->Rc);
  M->Xj = M->Xd = nullptr; M->xexp = nullptr; M->uf = nullptr; M->Jc = nullptr; M->Rc = nullptr;
  M->bcap = 0;
  int rc;
  void *p;
  const size_t xs = (size_t)b_pad * M->Kpad;
  if ((rc = ctx_alloc(ctx, &p, 2 * xs, "X (BF16)")) != RB_OK) return rc;
  M->Xj = (__nv_bfloat16 *)p;
  if ((rc = ctx_alloc(ctx, &p, 2 * xs * M->S, "X digit slices")) != RB_OK) return rc;
  M->Xd = (__nv_bfloat16 *)p;
  if ((rc = ctx_alloc(ctx, &p, 4 * (size_t)b_pad, "X exponents")) != RB_OK) return rc;
  M->xexp = (int *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb, "u (float pairs)")) != RB_OK) return rc;
  M->uf = (float2 *)p;
  if ((rc = ctx_alloc(ctx, &p, 4 * (size_t)b_pad * M->Npad, "J^c (FP32)")) != RB_OK) return rc;
  M->Jc = (float *)p;
  if ((rc = ctx_alloc(ctx, &p, 8 * (size_t)b_pad * M->nb, "R^c (FP64)")) != RB_OK) return rc;
  M->Rc = (double *)p;
  // zero once so that padded rows never hold NaN bit patterns
  cudaMemsetAsync(M->Xj, 0, 2 * xs, ctx->stream);
  cudaMemsetAsync(M->Xd, 0, 2 * xs * M->S, ctx->stream);
  cudaMemsetAsync(M->xexp, 0, 4 * (size_t)b_pad, ctx->stream);
  cudaMemsetAsync(M->uf, 0, 8 * (size_t)b_pad * M->nb, ctx->stream);
  if (!make_map(&M->tmXj, M->Xj, b_pad, M->Kpad, 128) ||
      !make_map(&M->tmXd, M->Xd, (uint64_t)M->S * b_pad, M->Kpad, 128))
    return set_error(ctx, RB_ERR_CUDA, "tensor map encode (X)");
  M->bcap = b_pad;
  return RB_OK;
}

// One Newton step's contraction work for the whole batch: X build + both GEMMs.
static int mixed_contract(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                          const int *d_n, const double *d_u, const rb_query_info *d_info,
                          cudaStream_t st) {
  MixedState *M = ctx->mixed;
  const DevOps &o = ctx->ops;
  BuildXParams bx{};
  bx.o = o;
  bx.mu = d_mu;
  bx.theta = d_theta;
  bx.nsz = d_n;
  bx.nq = nq;
  bx.nb = M->nb;
  bx.Kpad = M->Kpad;
  bx.S = M->S;
  bx.b_pad = M->bcap;
  bx.max_iter = ctx->cfg.max_iter;
  bx.u = d_u;
  bx.info = d_info;
  bx.Xj = M->Xj;
  bx.Xd = M->Xd;
  bx.xexp = M->xexp;
  bx.uf = M->uf;
  bx.Rc = M->Rc;
  k_build_x<<<std::min(nq, ctx->sms * 8), kThreads, 0, st>>>(bx);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_build_x");
  TcGemmParams g{};
  g.m_tiles = round_up(nq, 128) / 128;
  g.n_tiles = M->Npad / kTcBN;
  g.kb = M->kb;
  g.S = M->S;
  g.b_pad = M->bcap;
  g.n_pad = M->Npad;
  g.nq = nq;
  g.nb = M->nb;
  g.wexp = M->wexp;
  g.ldj = M->Npad;
  g.Jc = M->Jc;
  g.xexp = M->xexp;
  g.uf = M->uf;
  g.Rc = M->Rc;
  g.err = M->dev_words + 1;
  e = launch_tc_gemm(kPlain, M->tmXj, M->tmWj, g, ctx->sms, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_tc_gemm (Jacobian)");
  e = launch_tc_gemm(kSliced, M->tmXd, M->tmWd, g, ctx->sms, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_tc_gemm (residual)");
  return RB_OK;
}

static int launch_lu(rb_ctx *ctx, LuParams &lp, int nq, cudaStream_t st) {
  MixedState *M = ctx->mixed;
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
  k_lu_mixed<<<grid, kThreads, smem, st>>>(lp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_lu_mixed");
  return RB_OK;
}

static rb_query_info *own_info(rb_ctx *ctx, int nq) {
  MixedState *M = ctx->mixed;
  if (M->info_cap < nq) {
    ctx_free(ctx, M->info_own);
    void *p;
    if (ctx_alloc(ctx, &p, sizeof(rb_query_info) * (size_t)nq, "info") != RB_OK) return nullptr;
    M->info_own = (rb_query_info *)p;
    M->info_cap = nq;
  }
  return M->info_own;
}

int solve_mixed(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq, const int *d_n,
                double *d_u, double *, rb_query_info *d_info, cudaStream_t st) {
  int rc = mixed_layouts(ctx, st);
  if (rc != RB_OK) return rc;
  if ((rc = mixed_batch_scratch(ctx, nq)) != RB_OK) return rc;
  MixedState *M = ctx->mixed;
  rb_query_info *info = d_info ? d_info : own_info(ctx, nq);
  if (!info) return set_error(ctx, RB_ERR_OOM, "info scratch");
  const DevOps &o = ctx->ops;
  k_mixed_init<<<std::min(nq, ctx->sms * 8), 128, 0, st>>>(nq, o.n_max, d_n, d_u, info);
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
  lp.Jc = M->Jc;
  lp.Rc = M->Rc;
  lp.u = d_u;
  lp.info = info;
  lp.active = M->dev_words;
  int launches = 1;
  for (int it = 0; it < ctx->cfg.max_iter; ++it) {
    cudaMemsetAsync(M->dev_words, 0, 4, st);
    if ((rc = mixed_contract(ctx, d_mu, d_theta, nq, d_n, d_u, info, st)) != RB_OK) return rc;
    if ((rc = launch_lu(ctx, lp, nq, st)) != RB_OK) return rc;
    launches += 4;
    cudaError_t e = cudaMemcpyAsync(M->h_words, M->dev_words, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mixed Newton step");
    if (M->h_words[1]) return set_error(ctx, RB_ERR_TIMEOUT, "tensor-core pipeline wait gave up (code %d)", M->h_words[1]);
    if (M->h_words[0] == 0) break;
  }
  M->last_launches = launches;
  return RB_OK;
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
  void *p;
  if ((rc = ctx->jscratch.reserve(ctx, 8 * (size_t)nq * o.n_max + 4 * (size_t)nq + 256, "eval staging")) != RB_OK) return rc;
  p = ctx->jscratch.ptr;
  double *uw = (double *)p;
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
  if ((rc = mixed_contract(ctx, d_mu, nullptr, nq, nsz, uw, info, st)) != RB_OK) return rc;
  LuParams lp{};
  lp.o = o;
  lp.mu = d_mu;
  lp.nsz = nsz;
  lp.nq = nq;
  lp.nb = M->nb;
  lp.ldj = M->Npad;
  lp.max_iter = ctx->cfg.max_iter;
  lp.Jc = M->Jc;
  lp.Rc = M->Rc;
  lp.u = uw;
  lp.info = info;
  lp.active = M->dev_words;
  lp.eval_only = 1;
  lp.R_out = d_R;
  lp.J_out = d_J;
  if ((rc = launch_lu(ctx, lp, nq, st)) != RB_OK) return rc;
  e = cudaMemcpyAsync(M->h_words, M->dev_words, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_eval (mixed)");
  if (M->h_words[1]) return set_error(ctx, RB_ERR_TIMEOUT, "tensor-core pipeline wait gave up (code %d)", M->h_words[1]);
  return RB_OK;
}

}  // namespace rb

extern "C" int rb_debug_last_launches(rb_ctx *ctx) {
  return (ctx && ctx->mixed) ? ctx->mixed->last_launches : 0;
}
