// k_small.cu -- the whole mixed-precision Newton solve of a small system (n <= 32) in one launch,
// one CTA per query, on the CUDA cores.
//
// For small reduced sizes the tensor-core pipeline (operand builds, two GEMMs, assembly and
// elimination launched per iteration) is bound by launch latency; a single query at n = 20 then
// costs far more than its arithmetic. Here one CTA keeps its query's state in shared memory and
// runs every Newton iteration (Sec. 3.6 tensor Jacobian, Sec. 4.1 dense solve, Sec. 6 stopping
// rule) without leaving the kernel:
//   J^c[k][j] = sum_{q,l} theta^c_q u_l D~_q[k][j][l]        (double-float, D~ from L2)
//   R[k]      = sum_j (A(mu)[k][j] + J^c[k][j] / 2) u_j - f(mu)[k]   (Euler identity of the
//               quadratic term: C_mu(u, u) = J^c(u) u / 2; double-float, FP64-accurate)
//   [fl32(A(mu) + J^c) | -R] eliminated in FP32 by one warp (partial pivoting), u += delta.
// The Jacobian is exact up to FP32 rounding and the residual FP64-accurate, so the iteration
// converges quadratically to the FP64 solution until the FP32 factorisation's rate ~kappa 2^-24
// takes over; the stopping rule is tested on the FP64 norms as on every other path.
#include <cuda_runtime.h>

#include "rb_ctx.h"
#include "rb_small.cuh"

namespace rb {

namespace {

#ifndef RB_SMALL_THREADS
#define RB_SMALL_THREADS 512
#endif
#ifndef RB_SMALL_UNROLL
#define RB_SMALL_UNROLL 8
#endif
constexpr int kSmallThreads = RB_SMALL_THREADS;
constexpr int kSmallUnroll = RB_SMALL_UNROLL;  // loads of D~ in flight per thread (L2 latency)
constexpr int kSmallWarps = kSmallThreads / 32;

// ld of the augmented matrix [J | -R] in shared memory (the warp elimination's layout)
__host__ __device__ inline int small_ld(int nb) {
  int ld = (nb + 1 + 3) & ~3;
  if (((ld >> 2) & 1) == 0) ld += 4;
  return ld;
}

// The contraction's work split: element e = t % E (E = nb^2 rounded up to a warp) and part
// t / E of the (q, l) range, P parts (P E >= the block when E is smaller than the block).
__host__ __device__ inline int small_elems(int nb) { return (nb * nb + 31) & ~31; }
__host__ __device__ inline int small_parts(int nb) {
  const int E = small_elems(nb);
  return kSmallThreads / E > 0 ? kSmallThreads / E : 1;
}

// shared-memory carve-up (bytes); every block 16-byte aligned
struct SmallSmem {
  int th, th2, u2, fm, rv, xs, am, t, jaug, part, pseq, red, total;
  __host__ __device__ SmallSmem(const DevOps &o, int nb) {
    auto al = [](int b) { return (b + 15) & ~15; };
    int p = 0;
    th = p; p += al(8 * o.n_theta);
    th2 = p; p += al(8 * o.n_theta);        // theta as double-float
    u2 = p; p += al(8 * nb);                // u as double-float
    fm = p; p += al(8 * nb);
    rv = p; p += al(8 * nb);                // the residual R (double-float)
    xs = p; p += al(8 * o.q_c * nb);        // theta^c_q u_l as double-float
    am = p; p += al(8 * nb * nb);           // A(mu) as double-float
    t = p; p += al(8 * nb * nb);            // A(mu) + J^c / 2 as double-float
    jaug = p; p += al(4 * nb * small_ld(nb));
    part = p; p += al(8 * small_parts(nb) * small_elems(nb));  // partial sums of J^c
    pseq = p; p += al(4 * ((nb + 3) & ~3));
    red = p; p += al(8 * 4);                 // the step's norms and status
    total = p;
  }
};

}  // namespace

size_t small_smem_bytes(const DevOps &o, int nb) { return (size_t)SmallSmem(o, nb).total; }

__global__ void __launch_bounds__(kSmallThreads) k_newton_small(SmallParams p) {
  extern __shared__ __align__(16) uint8_t sm[];
  const DevOps &o = p.o;
  const int nb = p.nb;
  const SmallSmem L(o, nb);
  double *th = reinterpret_cast<double *>(sm + L.th);
  float2 *th2 = reinterpret_cast<float2 *>(sm + L.th2);
  float2 *u2 = reinterpret_cast<float2 *>(sm + L.u2);
  float2 *fm2 = reinterpret_cast<float2 *>(sm + L.fm);  // f(mu) as double-float
  float2 *rv = reinterpret_cast<float2 *>(sm + L.rv);   // R as double-float
  float2 *xs = reinterpret_cast<float2 *>(sm + L.xs);
  float2 *am = reinterpret_cast<float2 *>(sm + L.am);
  float2 *tm = reinterpret_cast<float2 *>(sm + L.t);
  float *J = reinterpret_cast<float *>(sm + L.jaug);
  float2 *part = reinterpret_cast<float2 *>(sm + L.part);
  int *pseq = reinterpret_cast<int *>(sm + L.pseq);
  double *red = reinterpret_cast<double *>(sm + L.red);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ld = small_ld(nb);
  const size_t nn = (size_t)nb * nb;
  // J^c: thread t sums element e = t % E over part t / E of the (q, l) range (E = nn rounded up
  // to a warp; P parts fill the block), then the parts add up in a fixed order
  const int E = small_elems(nb), P = small_parts(nb);
  const float tol_upd = (float)p.tol_upd, tol_res = (float)p.tol_res;
  const int Kc = o.q_c * nb;

  for (int b = blockIdx.x; b < p.nq; b += gridDim.x) {
    const int n = p.nsz ? p.nsz[b] : o.n_max;
    if (n < 1 || n > nb) {  // outside this launch's size range: rejected, untouched otherwise
      if (tid == 0 && p.info) {
        rb_query_info q = {RB_Q_REJECTED, 0, RB_PREC_MIXED, 0, 0.0, 0.0};
        p.info[b] = q;
      }
      for (int i = tid; i < o.n_max; i += blockDim.x) p.u[(size_t)b * o.n_max + i] = 0.0;
      continue;
    }
    // per-query data: theta, f(mu), A(mu) (Sec. 2.4, Sec. 3.5), u = 0
    if (p.theta) {
      for (int i = tid; i < o.n_theta; i += blockDim.x) th[i] = p.theta[(size_t)b * o.n_theta + i];
    } else {
      theta_eval(o, p.mu[2 * b], p.mu[2 * b + 1], th);
    }
    __syncthreads();
    // the FP64 pipe is narrow: every later product works on double-float copies
    for (int i = tid; i < o.n_theta; i += blockDim.x) {
      float h, lo;
      df_split(th[i], h, lo);
      th2[i] = make_float2(h, lo);
    }
    for (int k = tid; k < nb; k += blockDim.x) {
      double s = 0.0;
      if (k < n)
        for (int q = 0; q < o.q_f; ++q) s = fma(th[o.q_a + o.q_c + q], o.f[(size_t)q * o.n_max + k], s);
      float h, lo;
      df_split(s, h, lo);
      fm2[k] = make_float2(h, lo);
      u2[k] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (size_t e = tid; e < nn; e += blockDim.x) {
      float h = 0.f, l = 0.f;
      const int k = (int)(e / nb), j = (int)(e - (size_t)k * nb);
      if (k < n && j < n)
        for (int q = 0; q < o.q_a; ++q) {
          const float2 t = th2[q];
          const float2 a = p.A2[(size_t)q * nn + e];
          df_fma(h, l, a.x, a.y, t.x, t.y);
        }
      float s, ee;
      two_sum(h, l, s, ee);
      am[e] = make_float2(s, ee);
    }
    // norms for the stopping test in FP32 (relative accuracy 1e-7 of a norm is ample for a test
    // against 1e-10), by warp 0 (n <= 32: one entry per lane): the FP64 pipe is narrow
    float fscale = 1.f;
    if (w == 0) {
      const float fk = lane < n ? fm2[lane].x : 0.f;
      fscale = fmaxf(1.f, sqrtf(warp_sum(fk * fk)));
    }
    rb_query_info qi = {RB_Q_NOT_CONVERGED, 0, RB_PREC_MIXED, 0, 0.0, 0.0};
    bool done = false;
    while (!done) {
      // xs = theta^c (x) u in double-float
      for (int i = tid; i < o.q_c * nb; i += blockDim.x) {
        const int q = i / nb, l = i - q * nb;
        float h = 0.f, lo = 0.f;
        if (l < n) {
          const float2 t = th2[o.q_a + q], v = u2[l];
          df_fma(h, lo, t.x, t.y, v.x, v.y);
        }
        xs[i] = make_float2(h, lo);
      }
      __syncthreads();
      // J^c and T = A(mu) + J^c / 2; J = fl32(A(mu) + J^c) into the augmented matrix
      const bool zero = qi.iters == 0;  // u = 0: J^c = 0
      if (!zero) {
        for (int t = tid; t < P * E; t += blockDim.x) {
          const int e = t % E, pt = t / E;
          const int k = e / nb, j = e - k * nb;
          float h = 0.f, l = 0.f;
          if (e < (int)nn && k < n && j < n) {
            const int i0 = (int)(((long long)Kc * pt) / P), i1 = (int)(((long long)Kc * (pt + 1)) / P);
            const float2 *D = p.Dt2 + e;
#pragma unroll kSmallUnroll
            for (int i = i0; i < i1; ++i) {
              const float2 x = xs[i];
              const float2 d = __ldg(D + (size_t)i * nn);
              df_fma(h, l, d.x, d.y, x.x, x.y);
            }
          }
          part[t] = make_float2(h, l);
        }
        __syncthreads();
      }
      for (size_t e = tid; e < nn; e += blockDim.x) {
        const int k = (int)(e / nb), j = (int)(e - (size_t)k * nb);
        float h = 0.f, l = 0.f;
        if (!zero)
          for (int pt = 0; pt < P; ++pt) {
            const float2 v = part[pt * E + e];
            df_add(h, l, v.x, v.y);
          }
        float s, ee;
        two_sum(h, l, s, ee);  // J^c[k][j] = s + ee
        const float2 a = am[e];
        float th2 = a.x, tl2 = a.y;
        df_add(th2, tl2, 0.5f * s, 0.5f * ee);
        tm[e] = make_float2(th2, tl2);
        float jh = a.x, jl = a.y;
        df_add(jh, jl, s, ee);
        if (k < n && j < n) J[k * ld + j] = jh + jl;
      }
      __syncthreads();
      // R[k] = sum_j T[k][j] u_j - f[k], one warp per row; -R into column n
      for (int k = w; k < n; k += kSmallWarps) {
        float h = 0.f, l = 0.f;
        for (int j = lane; j < n; j += 32) {
          const float2 uu = u2[j];
          const float2 t = tm[(size_t)k * nb + j];
          df_fma(h, l, t.x, t.y, uu.x, uu.y);
        }
        // (h, l) summed over the warp in double-float, minus f(mu)[k]
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
          const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
          df_add(h, l, h2, l2);
        }
        if (lane == 0) {
          const float2 f = fm2[k];
          df_add(h, l, -f.x, -f.y);
          float rh, rl;
          two_sum(h, l, rh, rl);
          J[k * ld + n] = -rh;
          rv[k] = make_float2(rh, rl);
        }
      }
      __syncthreads();
      qi.iters += 1;
      // residual norm, elimination and update by warp 0 (n <= 32: one row per lane)
      if (w == 0) {
        int status = RB_Q_NOT_CONVERGED;
        float dn = 0.f;
        const float rk = lane < n ? rv[lane].x : 0.f;
        const float rn = sqrtf(warp_sum(rk * rk));
        if (!isfinite(rn)) {
          status = RB_Q_NONFINITE;
        } else {
          float x[1];
          if (gepp_aug_warp<1>(J, ld, n, x, pseq)) {
            status = RB_Q_SINGULAR;
          } else {
            const float d = lane < n ? x[0] : 0.f;
            if (lane < n) {  // u += delta in double-float
              float2 uu = u2[lane];
              df_add(uu.x, uu.y, d, 0.f);
              float s2, e2;
              two_sum(uu.x, uu.y, s2, e2);
              u2[lane] = make_float2(s2, e2);
            }
            dn = sqrtf(warp_sum(d * d));
            if (!isfinite(dn)) status = RB_Q_NONFINITE;
            else if (dn <= tol_upd && rn <= tol_res * fscale) status = RB_Q_OK;
          }
        }
        if (lane == 0) {
          red[0] = dn;
          red[1] = rn;
          reinterpret_cast<int *>(red + 2)[0] = status;
        }
      }
      __syncthreads();
      qi.upd_norm = red[0];
      qi.res_norm = red[1];
      qi.status = reinterpret_cast<const int *>(red + 2)[0];
      done = qi.status != RB_Q_NOT_CONVERGED || qi.iters >= p.max_iter;
      __syncthreads();  // red and the shared state are reused
    }
    for (int i = tid; i < o.n_max; i += blockDim.x)
      p.u[(size_t)b * o.n_max + i] = i < n ? (double)u2[i].x + (double)u2[i].y : 0.0;
    if (tid == 0 && p.info) p.info[b] = qi;
    __syncthreads();
  }
}

cudaError_t launch_newton_small(const SmallParams &p, int sms, cudaStream_t st) {
  const size_t smem = small_smem_bytes(p.o, p.nb);
  cudaError_t e = cudaFuncSetAttribute(k_newton_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = p.nq < 4 * sms ? (p.nq > 0 ? p.nq : 1) : 4 * sms;
  k_newton_small<<<grid, kSmallThreads, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace rb
