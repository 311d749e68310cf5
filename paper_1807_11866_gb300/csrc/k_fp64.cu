// k_fp64.cu -- FP64 kernels of the online stage: one CTA per query, every step in FP64.
//
//  * k_newton_fp64: theta (Sec. 2.4) -> tensor Jacobian of the convection term (Sec. 3.6)
//    -> A(mu) assembly (Sec. 3.5) and residual of Eq. velonly (Sec. 2.2) -> GEPP solve
//    (Sec. 4.1, Eq. blocksolve-1) -> update and stopping rule (Sec. 6), looped in-kernel.
//    The residual uses the Euler identity of the quadratic convection term,
//    J^c(u) u = 2 C_mu(u, u), so R = (A(mu) + J^c / 2) u - f(mu) costs O(n^2) once J^c is
//    formed: the FP64 work per iteration is one contraction (Q_c n^3 multiply-adds).
//  * k_pressure: a posteriori pressure recovery (Sec. 2.2, Eq. sup-vvar; Eq. blocksolve-2).
//  * k_eval_fp64, k_gepp_fp64: single steps exposed through rb_eval / rb_gepp_solve.
//  * k_build_dt, k_convert: load-time layout builders.
#include <cuda_bf16.h>

#include "rb_kernels.cuh"

namespace rb {

// ---------------------------------------------------------------------------------------
// J^c[k][j] = sum_{q,l} xs[q*n + l] * D~_q[k][j][l] into J (ld = n), xs = theta^c_q u_l.
// Streams D~ from L2/HBM: for fixed (q, l) the n x n block is read row by row, so
// consecutive threads read consecutive j (coalesced); no reuse, FP64-ALU bound.
// A thread takes P elements (base + i kThreads + tid), P a compile-time count matched to the
// elements left: FP64 instructions occupy the pipe whether or not their predicate is on, so
// a fixed unrolled count with a run-time guard would issue every slot (16 of them where a
// single small query needs 2).
constexpr int kP = 16;
template <int P>
__device__ __forceinline__ void contract_fp64_part(const DevOps &o, int n, const double *xs,
                                                   double *J, int base) {
  const int tid = threadIdx.x;
  const int nn = n * n;
  const size_t nm = (size_t)o.n_max, nm2 = nm * nm;
  int off[P];
  double acc[P];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const int e = base + i * kThreads + tid;
    const int k = e / n, j = e - (e / n) * n;
    off[i] = (e < nn) ? (int)(k * nm + j) : 0;
    acc[i] = 0.0;
  }
  for (int q = 0; q < o.q_c; ++q) {
    const double *Dq = o.Dt + (size_t)q * nm * nm2;
    const double *xq = xs + q * n;
#pragma unroll 8  // loads of 8 rows in flight: the stream is L2-latency bound at small n
    for (int l = 0; l < n; ++l) {
      const double x = xq[l];
      const double *row = Dq + (size_t)l * nm2;
#pragma unroll
      for (int i = 0; i < P; ++i) acc[i] = fma(x, __ldg(row + off[i]), acc[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const int e = base + i * kThreads + tid;
    if (e < nn) J[e] = acc[i];
  }
}

__device__ void contract_fp64(const DevOps &o, int n, const double *xs, double *J) {
  const int nn = n * n;
  for (int base = 0; base < nn; base += kThreads * kP) {
    switch (min(kP, (nn - base + kThreads - 1) / kThreads)) {  // uniform over the block
      case 1: contract_fp64_part<1>(o, n, xs, J, base); break;
      case 2: contract_fp64_part<2>(o, n, xs, J, base); break;
      case 3: contract_fp64_part<3>(o, n, xs, J, base); break;
      case 4: contract_fp64_part<4>(o, n, xs, J, base); break;
      case 5: contract_fp64_part<5>(o, n, xs, J, base); break;
      case 6: contract_fp64_part<6>(o, n, xs, J, base); break;
      case 7: contract_fp64_part<7>(o, n, xs, J, base); break;
      case 8: contract_fp64_part<8>(o, n, xs, J, base); break;
      case 9: contract_fp64_part<9>(o, n, xs, J, base); break;
      case 10: contract_fp64_part<10>(o, n, xs, J, base); break;
      case 11: contract_fp64_part<11>(o, n, xs, J, base); break;
      case 12: contract_fp64_part<12>(o, n, xs, J, base); break;
      case 13: contract_fp64_part<13>(o, n, xs, J, base); break;
      case 14: contract_fp64_part<14>(o, n, xs, J, base); break;
      case 15: contract_fp64_part<15>(o, n, xs, J, base); break;
      default: contract_fp64_part<16>(o, n, xs, J, base); break;
    }
  }
}

// A(mu)[k][j] = sum_q theta^a_q A_q[k][j] (row stride n).
__device__ void assemble_a(const DevOps &o, int n, const double *th, double *Am) {
  const size_t nm = (size_t)o.n_max;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int k = e / n, j = e - k * n;
    double a = 0.0;
    for (int q = 0; q < o.q_a; ++q) a = fma(th[q], __ldg(o.A + ((size_t)q * nm + k) * nm + j), a);
    Am[e] = a;
  }
}

// J <- A(mu) + J^c and R = (A(mu) + J^c / 2) u - f(mu); one warp per row k. Am: A(mu) built
// once per query (shared memory), or null: summed here from the A_q.
__device__ void row_pass_fp64(const DevOps &o, int n, const double *th, const double *u,
                              const double *fm, double *J, double *R, const double *Am) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t nm = (size_t)o.n_max;
  for (int k = w; k < n; k += kWarps) {
    double r = 0.0;
    for (int j = lane; j < n; j += 32) {
      double a = 0.0;
      if (Am) a = Am[k * n + j];
      else
        for (int q = 0; q < o.q_a; ++q) a = fma(th[q], __ldg(o.A + ((size_t)q * nm + k) * nm + j), a);
      const double jc = J[(size_t)k * n + j];
      r = fma(a + 0.5 * jc, u[j], r);
      J[(size_t)k * n + j] = a + jc;
    }
    r = warp_sum(r);
    if (lane == 0) R[k] = r - fm[k];
  }
}

// f(mu)[k] = sum_q theta^f_q f_q[k]
__device__ void assemble_f(const DevOps &o, int n, const double *th, double *fm) {
  const double *tf = th + o.q_a + o.q_c;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < o.q_f; ++q) s = fma(tf[q], o.f[(size_t)q * o.n_max + k], s);
    fm[k] = s;
  }
}

__device__ void load_theta(const DevOps &o, const double *mu, const double *theta, int b,
                           double *th) {
  if (theta) {
    for (int i = threadIdx.x; i < o.n_theta; i += blockDim.x) th[i] = theta[(size_t)b * o.n_theta + i];
  } else {
    theta_eval(o, mu[2 * b], mu[2 * b + 1], th);
  }
}

// shared-memory carve-up of the per-query FP64 kernels (in doubles); A(mu) is kept in shared
// memory for small sets (n_max <= kFp64SmallN), where the per-iteration latency dominates
constexpr int kFp64SmallN = 32;
struct Fp64Smem {
  int th, u, R, fm, xs, red, piv, J, Am, total;
  __host__ __device__ Fp64Smem(const DevOps &o, bool j_in_smem) {
    int p = 0;
    th = p; p += (o.n_theta + 1) & ~1;
    u = p; p += o.n_max;
    R = p; p += o.n_max;
    fm = p; p += o.n_max;
    xs = p; p += o.q_c * o.n_max;
    red = p; p += 4 * kWarps;
    piv = p; p += (o.n_max + 1) / 2;  // ints
    p = (p + 1) & ~1;
    J = p;
    if (j_in_smem) p += o.n_max * o.n_max;
    Am = p;
    if (j_in_smem && o.n_max <= kFp64SmallN) p += o.n_max * o.n_max;
    total = p;
  }
};

size_t fp64_smem_bytes(const DevOps &o, bool j_in_smem) {
  return sizeof(double) * (size_t)Fp64Smem(o, j_in_smem).total;
}

__global__ void __launch_bounds__(kThreads) k_newton_fp64(NewtonParams p) {
  extern __shared__ double sm[];
  const DevOps &o = p.o;
  const Fp64Smem L(o, p.j_in_smem != 0);
  double *th = sm + L.th, *u = sm + L.u, *R = sm + L.R, *fm = sm + L.fm, *xs = sm + L.xs;
  double *red = sm + L.red;
  int *piv = reinterpret_cast<int *>(sm + L.piv);
  double *J = p.j_in_smem ? sm + L.J : p.jscratch + (size_t)blockIdx.x * o.n_max * o.n_max;
  double *Am = (p.j_in_smem && o.n_max <= kFp64SmallN) ? sm + L.Am : nullptr;
  const int tid = threadIdx.x;
  if (p.run_if && *(volatile const int *)p.run_if == 0) return;  // nothing handed over

  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    int it0 = 0;
    if (p.resume) {  // only the queries the mixed path handed over, solved again from u = 0
      const rb_query_info qe = p.info[b];
      if (qe.status != kQEscalate) continue;  // uniform over the CTA
      it0 = qe.iters;
    }
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    double *urow = p.u_out + (size_t)b * o.n_max;
    if (n < 1 || n > o.n_max) {
      for (int i = tid; i < o.n_max; i += blockDim.x) urow[i] = 0.0;
      if (tid == 0 && p.info) {
        rb_query_info q = {RB_Q_REJECTED, 0, RB_PREC_FP64, 0, 0.0, 0.0};
        p.info[b] = q;
      }
      continue;
    }
    load_theta(o, p.mu, p.theta, b, th);
    for (int i = tid; i < n; i += blockDim.x) u[i] = 0.0;
    __syncthreads();
    assemble_f(o, n, th, fm);
    if (Am) assemble_a(o, n, th, Am);
    __syncthreads();
    double fl = 0.0;
    for (int i = tid; i < n; i += blockDim.x) fl += fm[i] * fm[i];
    const double fscale = fmax(1.0, sqrt(block_sum(fl, red)));

    int status = RB_Q_NOT_CONVERGED, iters = 0;
    double rn = 0.0, dn = 0.0;
    for (int it = 0; it < p.max_iter; ++it) {
      const double *tc = th + o.q_a;
      for (int i = tid; i < o.q_c * n; i += blockDim.x) xs[i] = tc[i / n] * u[i % n];
      __syncthreads();
      contract_fp64(o, n, xs, J);
      __syncthreads();
      row_pass_fp64(o, n, th, u, fm, J, R, Am);
      __syncthreads();
      double rl = 0.0;
      for (int i = tid; i < n; i += blockDim.x) rl += R[i] * R[i];
      rn = sqrt(block_sum(rl, red));
      iters = it + 1;
      if (!isfinite(rn)) { status = RB_Q_NONFINITE; break; }
      for (int i = tid; i < n; i += blockDim.x) R[i] = -R[i];
      __syncthreads();
      bool sing;
      if (n <= 32) {  // one warp eliminates, without CTA barriers per pivot
        if (threadIdx.x < 32 && gepp_solve_warp32<double>(J, n, n, R, piv) && threadIdx.x == 0)
          red[0] = 1.0;
        else if (threadIdx.x == 0)
          red[0] = 0.0;
        __syncthreads();
        sing = red[0] != 0.0;
        __syncthreads();
      } else {
        sing = gepp_solve_block<double>(J, n, n, R, red);
      }
      if (sing) { status = RB_Q_SINGULAR; break; }
      double dl = 0.0;
      for (int i = tid; i < n; i += blockDim.x) {
        dl += R[i] * R[i];
        u[i] += R[i];
      }
      dn = sqrt(block_sum(dl, red));
      if (!isfinite(dn)) { status = RB_Q_NONFINITE; break; }
      if (dn <= p.tol_upd && rn <= p.tol_res * fscale) { status = RB_Q_OK; break; }
    }
    __syncthreads();
    for (int i = tid; i < o.n_max; i += blockDim.x) urow[i] = (i < n) ? u[i] : 0.0;
    if (tid == 0 && p.info) {
      rb_query_info q = {status, it0 + iters, RB_PREC_FP64, 0, rn, dn};
      p.info[b] = q;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Pressure recovery, one CTA per query:
//   r[k'] = sum_q th^f_q fs_q[k'] - sum_q th^a_q (As_q u)[k'] - sum_q th^c_q sum_{j,l}
//           Cs_q[j][l][k'] u_j u_l,  B(mu) = sum_q th^b_q B_q,  B(mu) p = r.
struct PresSmem {
  int th, u, r, red, part, Bm, total, groups, gw;
  __host__ __device__ PresSmem(const DevOps &o) {
    gw = ((o.m + 31) / 32) * 32;                 // lanes per group
    groups = kThreads / gw > 0 ? kThreads / gw : 1;
    int p = 0;
    th = p; p += (o.n_theta + 1) & ~1;
    u = p; p += o.n_max;
    r = p; p += o.m;
    red = p; p += 4 * kWarps;
    part = p; p += groups * gw;
    Bm = p; p += o.m * o.m;
    total = p;
  }
};

size_t pressure_smem_bytes(const DevOps &o) { return sizeof(double) * (size_t)PresSmem(o).total; }

__global__ void __launch_bounds__(kThreads) k_pressure(PressureParams p) {
  extern __shared__ double sm[];
  const DevOps &o = p.o;
  const PresSmem L(o);
  double *th = sm + L.th, *u = sm + L.u, *r = sm + L.r, *red = sm + L.red, *part = sm + L.part;
  double *Bm = sm + L.Bm;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, m = o.m;
  const size_t nm = (size_t)o.n_max;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    double *prow = p.p_out + (size_t)b * m;
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    const bool ok = (n >= 1 && n <= o.n_max) && (!p.info || p.info[b].status == RB_Q_OK);
    if (!ok) {
      for (int i = tid; i < m; i += blockDim.x) prow[i] = 0.0;
      continue;
    }
    load_theta(o, p.mu, p.theta, b, th);
    for (int i = tid; i < n; i += blockDim.x) u[i] = p.u[(size_t)b * nm + i];
    __syncthreads();
    const double *ta = th, *tc = th + o.q_a, *tf = th + o.q_a + o.q_c;
    const double *tb = tf + o.q_f;
    // convection part: group g handles pairs (q, j), lane k' accumulates over l
    {
      const int g = tid / L.gw, kk = tid % L.gw;
      double acc = 0.0;
      if (g < L.groups && kk < m) {
        for (int qj = g; qj < o.q_c * n; qj += L.groups) {
          const int q = qj / n, j = qj % n;
          const double *cs = o.Cs + ((size_t)q * nm + j) * nm * m;
          double s = 0.0;
          for (int l = 0; l < n; ++l) s = fma(__ldg(cs + (size_t)l * m + kk), u[l], s);
          acc = fma(tc[q] * u[j], s, acc);
        }
      }
      if (g < L.groups) part[g * L.gw + kk] = acc;
    }
    __syncthreads();
    // linear part, one warp per k'
    for (int k = w; k < m; k += kWarps) {
      double s = 0.0;
      for (int q = 0; q < o.q_a; ++q) {
        double sq = 0.0;
        for (int j = lane; j < n; j += 32) sq = fma(__ldg(o.As + ((size_t)q * m + k) * nm + j), u[j], sq);
        s = fma(ta[q], sq, s);
      }
      s = warp_sum(s);
      if (lane == 0) {
        double c = 0.0;
        for (int g = 0; g < L.groups; ++g) c += part[g * L.gw + k];
        double fsv = 0.0;
        for (int q = 0; q < o.q_f; ++q) fsv = fma(tf[q], o.fs[(size_t)q * m + k], fsv);
        r[k] = fsv - s - c;
      }
    }
    for (int e = tid; e < m * m; e += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < o.q_b; ++q) s = fma(tb[q], __ldg(o.B + (size_t)q * m * m + e), s);
      Bm[e] = s;
    }
    __syncthreads();
    const bool sing = gepp_solve_block<double>(Bm, m, m, r, red);
    for (int i = tid; i < m; i += blockDim.x) prow[i] = sing ? 0.0 : r[i];
    if (sing && tid == 0 && p.info) p.info[b].status = RB_Q_SINGULAR;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// R(u) and J(u) in FP64 at given u (all queries of size n), one CTA per query.
__global__ void __launch_bounds__(kThreads) k_eval_fp64(EvalParams p) {
  extern __shared__ double sm[];
  const DevOps &o = p.o;
  const Fp64Smem L(o, false);
  double *th = sm + L.th, *u = sm + L.u, *R = sm + L.R, *fm = sm + L.fm, *xs = sm + L.xs;
  const int tid = threadIdx.x, n = p.n;
  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    double *J = p.J_out + (size_t)b * n * n;
    load_theta(o, p.mu, nullptr, b, th);
    for (int i = tid; i < n; i += blockDim.x) u[i] = p.u[(size_t)b * n + i];
    __syncthreads();
    assemble_f(o, n, th, fm);
    const double *tc = th + o.q_a;
    for (int i = tid; i < o.q_c * n; i += blockDim.x) xs[i] = tc[i / n] * u[i % n];
    __syncthreads();
    contract_fp64(o, n, xs, J);
    __syncthreads();
    row_pass_fp64(o, n, th, u, fm, J, R, nullptr);
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) p.R_out[(size_t)b * n + i] = R[i];
    __syncthreads();
  }
}

// Batched FP64 GEPP on global matrices (modified in place), rhs -> x.
__global__ void __launch_bounds__(kThreads) k_gepp_fp64(double *M, double *rhs, int n, int batch,
                                                        int *status) {
  extern __shared__ double sm[];
  double *b = sm, *red = sm + ((n + 1) & ~1);
  for (int s = blockIdx.x; s < batch; s += gridDim.x) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = rhs[(size_t)s * n + i];
    __syncthreads();
    const bool sing = gepp_solve_block<double>(M + (size_t)s * n * n, n, n, b, red);
    for (int i = threadIdx.x; i < n; i += blockDim.x) rhs[(size_t)s * n + i] = b[i];
    if (threadIdx.x == 0) status[s] = sing ? RB_Q_SINGULAR : 0;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Load-time builders.
// Dt[q][l][k][j] = C[q][l][j][k] + C[q][j][l][k] (index [j][l][k] of C as stored).
// storage types of C and Cs (RB_F64, RB_F32, RB_BF16) to FP64, exactly
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <typename TC>
__global__ void k_build_dt(const TC *C, double *Dt, int nm, int qc) {
  const size_t nm1 = nm, total = (size_t)qc * nm1 * nm1 * nm1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e % nm1, k = (e / nm1) % nm1, l = (e / (nm1 * nm1)) % nm1;
    const size_t q = e / (nm1 * nm1 * nm1);
    const size_t cq = q * nm1 * nm1 * nm1;
    const double a = to_f64(C[cq + (l * nm1 + j) * nm1 + k]);
    const double c = to_f64(C[cq + (j * nm1 + l) * nm1 + k]);
    Dt[e] = a + c;
  }
}

template <typename TS>
__global__ void k_convert(const TS *src, double *dst, size_t count) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] = to_f64(src[e]);
}

// ---------------------------------------------------------------------------------------
// host-side launchers
static int grid_for(int nq, int per_sm, int sms) {
  const int g = per_sm * sms;
  return nq < g ? (nq > 0 ? nq : 1) : g;
}

cudaError_t launch_newton_fp64(const NewtonParams &p, int sms, cudaStream_t st) {
  const size_t smem = fp64_smem_bytes(p.o, p.j_in_smem != 0);
  cudaError_t e = cudaFuncSetAttribute(k_newton_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_newton_fp64<<<p.grid, kThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_pressure(const PressureParams &p, int sms, cudaStream_t st) {
  const size_t smem = pressure_smem_bytes(p.o);
  cudaError_t e = cudaFuncSetAttribute(k_pressure, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_pressure<<<grid_for(p.nq, 8, sms), kThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_eval_fp64(const EvalParams &p, int sms, cudaStream_t st) {
  const size_t smem = fp64_smem_bytes(p.o, false);
  cudaError_t e = cudaFuncSetAttribute(k_eval_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_eval_fp64<<<grid_for(p.nq, 8, sms), kThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_gepp_fp64(double *M, double *rhs, int n, int batch, int *status, int sms,
                             cudaStream_t st) {
  const size_t smem = sizeof(double) * (((n + 1) & ~1) + 4 * kWarps);
  k_gepp_fp64<<<grid_for(batch, 8, sms), kThreads, smem, st>>>(M, rhs, n, batch, status);
  return cudaGetLastError();
}

cudaError_t launch_build_dt(const void *C, int dtype, double *Dt, int nm, int qc, int sms,
                            cudaStream_t st) {
  if (dtype == RB_F32)
    k_build_dt<float><<<sms * 8, 256, 0, st>>>((const float *)C, Dt, nm, qc);
  else if (dtype == RB_BF16)
    k_build_dt<__nv_bfloat16><<<sms * 8, 256, 0, st>>>((const __nv_bfloat16 *)C, Dt, nm, qc);
  else
    k_build_dt<double><<<sms * 8, 256, 0, st>>>((const double *)C, Dt, nm, qc);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void *src, int dtype, double *dst, size_t count, int sms,
                           cudaStream_t st) {
  if (dtype == RB_F32)
    k_convert<float><<<sms * 8, 256, 0, st>>>((const float *)src, dst, count);
  else if (dtype == RB_BF16)
    k_convert<__nv_bfloat16><<<sms * 8, 256, 0, st>>>((const __nv_bfloat16 *)src, dst, count);
  else
    k_convert<double><<<sms * 8, 256, 0, st>>>((const double *)src, dst, count);
  return cudaGetLastError();
}

}  // namespace rb
