// rb_internal.cuh -- device-side layouts and block-level building blocks shared by the
// kernels of librb (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rb.h"

namespace rb {

constexpr int kThreads = 256;  // block size of the per-query kernels (8 warps)
constexpr int kWarps = kThreads / 32;

// Device-resident operator layouts (all owned by the context, built at load time).
struct DevOps {
  int n_max, m, q_a, q_c, q_f, q_b, n_theta;
  int theta_family;   // RB_THETA_POLY: monomials phi^q, otherwise the trigonometric family
  const double *A;    // [q_a][n_max][n_max]          row = test k
  const double *Dt;   // [q_c][n_max(l)][n_max(k)][n_max(j)]  D~_q[k][j][l] =
                      //   C_q[l][j][k] + C_q[j][l][k]  (both orders of Sec. 3.6 pre-summed)
  const double *f;    // [q_f][n_max]
  const double *B;    // [q_b][m][m]
  const double *As;   // [q_a][m][n_max]
  const double *Cs;   // [q_c][n_max][n_max][m]   index [j][l][k'] (FP64 copy)
  const double *fs;   // [q_f][m]
};

// Parameter functions of the trigonometric family (Sec. 2.4 affine split): trig_q(a) is
// cos(q a) for even q and sin(q a) for odd q; theta^a carries 1/Re.
__device__ __forceinline__ double trig_q(int q, double a) {
  return (q & 1) ? sin((double)q * a) : cos((double)q * a);
}

// theta row of one query into th[0..n_theta): [a | c | f | b], entries start, start + stride, ...
__device__ __forceinline__ void theta_eval_strided(const DevOps &o, double alpha_deg, double re,
                                                   double *th, int start, int stride) {
  const double a = alpha_deg * 0.017453292519943295769;  // pi / 180
  for (int i = start; i < o.n_theta; i += stride) {
    int q = i;
    double scale = 1.0;
    if (q < o.q_a) {
      scale = 1.0 / re;
    } else {
      q -= o.q_a;
      if (q >= o.q_c) {
        q -= o.q_c;
        if (q >= o.q_f) q -= o.q_f;
      }
    }
    if (o.theta_family == RB_THETA_POLY) {
      // monomial phi^q of the truncated rotation series (Sec. 5, Eq. rotsum), by repeated
      // multiplication
      double v = 1.0;
      for (int k = 0; k < q; ++k) v *= a;
      th[i] = v * scale;
    } else {
      th[i] = trig_q(q, a) * scale;
    }
  }
}

// theta row of one query, all threads of the block
__device__ __forceinline__ void theta_eval(const DevOps &o, double alpha_deg, double re,
                                           double *th) {
  theta_eval_strided(o, alpha_deg, re, th, threadIdx.x, blockDim.x);
}

// Asynchronous 16-byte copies global -> shared (cp.async, cached in L2 only): every copy of a
// thread is in flight at once; cp_async_wait_all waits for the calling thread's copies (a warp
// or block barrier then makes them visible to the others). Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; red must hold kWarps doubles. Result valid in all threads.
__device__ __forceinline__ double block_sum(double v, double *red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) s += red[i];
  return s;
}

// ---- double-float ("float-float") arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2 ----
// Used where FP64 accuracy is needed for O(n^2) work per query: GB300's FP64 pipe is narrow.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (ah, al) += (xh + xl) (yh + yl), the product's error kept by an FMA split
__device__ __forceinline__ void df_fma(float &ah, float &al, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float pe = fmaf(xh, yh, -p);
  pe = fmaf(xh, yl, pe);
  pe = fmaf(xl, yh, pe);
  float s, e;
  two_sum(ah, p, s, e);
  ah = s;
  al += e + pe;
}

// v = h + l with h = v rounded to FP32 (nearest, ties to even) and l = v - h rounded to FP32,
// from v's bit pattern with integer operations. GB300's FP64 pipe issues about 1/64 of the FP32
// rate and a warp instruction on it occupies it for the whole warp, so the two FP64 conversions
// and the subtraction of the plain split cost far more than these integer steps. The significand
// 1.m (53 bits) is t (its top 24 bits) followed by r (29 bits); rounding t up leaves r - 2^29, and
// l = +-r 2^(e - 52) is r rounded to 24 bits by the integer conversion, scaled by a power of two
// that is a normal FP32 value for 2^-74 <= |v| < 2^127. Zero is exact; other magnitudes,
// infinities and NaN take the FP64 conversions (same results: the split is unique).
__device__ __forceinline__ void df_split(double v, float &h, float &l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sgn = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023;
  if (e >= -74 && e <= 126) {
    unsigned t = 0x800000u | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    int r = (int)(lo & 0x1FFFFFFFu);
    if (r > 0x10000000 || (r == 0x10000000 && (t & 1u))) {
      t += 1u;
      r -= 0x20000000;
    }
    int eh = e;
    if (t == 0x1000000u) {  // rounded up into the next binade
      t = 0x800000u;
      eh += 1;
    }
    h = __uint_as_float(sgn | ((unsigned)(eh + 127) << 23) | (t & 0x7FFFFFu));
    l = __int2float_rn(sgn ? -r : r) * __uint_as_float((unsigned)(e + 75) << 23);
  } else if ((b << 1) == 0ull) {
    h = __uint_as_float(sgn);
    l = 0.f;
  } else {
    h = (float)v;
    l = (float)(v - (double)h);
  }
}

// The FP32 value x as a double, from its bit pattern (exact; zero and normal x by integer
// operations, other values by the FP64 conversion).
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned ex = (u >> 23) & 0xFFu;
  if (ex != 0u && ex != 0xFFu) {
    const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
    const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
    return __longlong_as_double((long long)(s | ((unsigned long long)(ex + 896u) << 52) | m));
  }
  if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
  return (double)x;
}

// warp-wide sum of double-float values, result in every lane as a double
__device__ __forceinline__ double df_warp_sum(float h, float l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    two_sum(h, h2, s, e);
    h = s;
    l = l + l2 + e;
  }
  return (double)h + (double)l;
}

// (h1, l1) += (h2, l2) in double-float
__device__ __forceinline__ void df_add(float &h1, float &l1, float h2, float l2) {
  float s, e;
  two_sum(h1, h2, s, e);
  h1 = s;
  l1 = l1 + l2 + e;
}

// Reduce-scatter of 8 double-float values per lane (one per row r = 0..7) over the warp:
// after it, the lanes 4 r .. 4 r + 3 hold the warp total of row r in (h[0], l[0]).
// 18 shuffle pairs instead of 8 full butterflies.
__device__ __forceinline__ void df_warp_reduce8(float (&h)[8], float (&l)[8]) {
  const int lane = threadIdx.x & 31;
  // level xor 16: lanes with bit 4 set keep rows 4..7 (moved to slots 0..3), the others 0..3
  {
    const bool up = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float sh = up ? h[i] : h[i + 4], sl = up ? l[i] : l[i + 4];
      const float kh = up ? h[i + 4] : h[i], kl = up ? l[i + 4] : l[i];
      const float rh = __shfl_xor_sync(0xffffffffu, sh, 16);
      const float rl = __shfl_xor_sync(0xffffffffu, sl, 16);
      h[i] = kh;
      l[i] = kl;
      df_add(h[i], l[i], rh, rl);
    }
  }
  // level xor 8: bit 3 selects slots 2..3 or 0..1
  {
    const bool up = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float sh = up ? h[i] : h[i + 2], sl = up ? l[i] : l[i + 2];
      const float kh = up ? h[i + 2] : h[i], kl = up ? l[i + 2] : l[i];
      const float rh = __shfl_xor_sync(0xffffffffu, sh, 8);
      const float rl = __shfl_xor_sync(0xffffffffu, sl, 8);
      h[i] = kh;
      l[i] = kl;
      df_add(h[i], l[i], rh, rl);
    }
  }
  // level xor 4: bit 2 selects slot 1 or 0
  {
    const bool up = lane & 4;
    const float sh = up ? h[0] : h[1], sl = up ? l[0] : l[1];
    const float kh = up ? h[1] : h[0], kl = up ? l[1] : l[0];
    const float rh = __shfl_xor_sync(0xffffffffu, sh, 4);
    const float rl = __shfl_xor_sync(0xffffffffu, sl, 4);
    h[0] = kh;
    l[0] = kl;
    df_add(h[0], l[0], rh, rl);
  }
  // levels xor 2, 1: the group of four lanes holding one row
#pragma unroll
  for (int o = 2; o > 0; o >>= 1) {
    const float rh = __shfl_xor_sync(0xffffffffu, h[0], o);
    const float rl = __shfl_xor_sync(0xffffffffu, l[0], o);
    df_add(h[0], l[0], rh, rl);
  }
}

// (|value|, row) argmax with the first row winning ties.
template <typename T>
__device__ __forceinline__ void argmax_merge(T &v, int &r, T v2, int r2) {
  if (v2 > v || (v2 == v && r2 < r)) { v = v2; r = r2; }
}

// Solve M x = b in place by Gaussian elimination with partial pivoting (pivot = first row
// of largest magnitude), block-cooperative, every operation in the precision T (FP32 work
// stays off the FP64 pipe). M: n x n with row stride ld (shared or global), b: shared,
// overwritten by x. red: >= 2 * kWarps + 2 doubles of shared scratch.
// Returns true if a pivot was zero or not finite (b is then unspecified).
template <typename T>
__device__ bool gepp_solve_block(T *M, int ld, int n, T *b, double *red) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  T *tred = reinterpret_cast<T *>(red);
  int *ired = reinterpret_cast<int *>(red + kWarps + 1);
  for (int p = 0; p < n; ++p) {
    // pivot search over rows p..n-1 of column p, only by the warps that hold rows
    const int rows = n - p;
    if (w * 32 < rows) {
      T best = T(-1);
      int brow = n;
      for (int i = p + tid; i < n; i += blockDim.x) argmax_merge<T>(best, brow, fabs(M[(size_t)i * ld + p]), i);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int r2 = __shfl_xor_sync(0xffffffffu, brow, o);
        argmax_merge<T>(best, brow, v2, r2);
      }
      if (lane == 0) { tred[w] = best; ired[w] = brow; }
    }
    __syncthreads();
    if (tid == 0) {
      T bv = tred[0];
      int br = ired[0];
      const int nw = min(kWarps, (rows + 31) / 32);
      for (int i = 1; i < nw; ++i) argmax_merge<T>(bv, br, tred[i], ired[i]);
      tred[kWarps] = bv;
      ired[kWarps] = br;
    }
    __syncthreads();
    const T pv = tred[kWarps];
    const int r = ired[kWarps];
    if (!(pv > T(0)) || !isfinite(pv)) return true;
    if (r != p) {
      for (int j = p + tid; j < n; j += blockDim.x) {
        T t = M[(size_t)p * ld + j];
        M[(size_t)p * ld + j] = M[(size_t)r * ld + j];
        M[(size_t)r * ld + j] = t;
      }
      if (tid == 0) { T t = b[p]; b[p] = b[r]; b[r] = t; }
    }
    __syncthreads();
    const T piv = M[(size_t)p * ld + p];
    for (int i = p + 1 + tid; i < n; i += blockDim.x) M[(size_t)i * ld + p] = M[(size_t)i * ld + p] / piv;
    __syncthreads();
    const T bp = b[p];
    // trailing update, one warp per row
    for (int i = p + 1 + w; i < n; i += kWarps) {
      const T lip = M[(size_t)i * ld + p];
      T *Mi = M + (size_t)i * ld;
      const T *Mp = M + (size_t)p * ld;
      for (int j = p + 1 + lane; j < n; j += 32) Mi[j] -= lip * Mp[j];
      if (lane == 0) b[i] -= lip * bp;
    }
    __syncthreads();
  }
  // back substitution by warp 0
  if (w == 0) {
    for (int i = n - 1; i >= 0; --i) {
      T s = T(0);
      for (int j = i + 1 + lane; j < n; j += 32) s += M[(size_t)i * ld + j] * b[j];
      s = warp_sum(s);
      if (lane == 0) b[i] = (b[i] - s) / M[(size_t)i * ld + i];
      __syncwarp();
    }
  }
  __syncthreads();
  return false;
}

// Solve M x = b in place for n <= 32 by the calling warp alone (no CTA barriers): Gaussian
// elimination with partial pivoting (pivot = first row of largest magnitude), rows left in place
// and owned by lane r; the elimination order goes to pseq (n ints of shared scratch), then back
// substitution in that order; b (shared) receives x. Every operation in precision T. Returns
// true (all lanes) if a pivot was zero or not finite.
template <typename T>
__device__ bool gepp_solve_warp32(T *M, int ld, int n, T *b, int *pseq) {
  const int lane = threadIdx.x & 31;
  T *row = M + (size_t)lane * ld;
  int step = lane < n ? n : -1;  // step at which the row was the pivot
  for (int p = 0; p < n; ++p) {
    T best = step == n ? fabs(row[p]) : T(-1);
    int brow = step == n ? lane : n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int r2 = __shfl_xor_sync(0xffffffffu, brow, o);
      argmax_merge<T>(best, brow, v2, r2);
    }
    if (!(best > T(0)) || !isfinite(best)) return true;  // uniform after the butterfly
    const T *prow = M + (size_t)brow * ld;
    const T pv = prow[p];
    if (lane == brow) step = p;
    if (lane == 0) pseq[p] = brow;
    if (step == n) {
      const T l = row[p] / pv;
      for (int j = p + 1; j < n; ++j) row[j] -= l * prow[j];
      b[lane] -= l * b[brow];
    }
    __syncwarp();
  }
  // back substitution in step order: unknown p from row pseq[p]
  for (int p = n - 1; p >= 0; --p) {
    const int r = pseq[p];
    const T xp = b[r] / M[(size_t)r * ld + p];
    __syncwarp();
    if (step >= 0 && step < p) b[lane] -= M[(size_t)lane * ld + p] * xp;
    if (lane == r) b[lane] = xp;
    __syncwarp();
  }
  // b[pseq[p]] holds x_p: gather into column order
  T xv = T(0);
  if (lane < n) xv = b[pseq[lane]];
  __syncwarp();
  if (lane < n) b[lane] = xv;
  __syncwarp();
  return false;
}

// ---- warp-level elimination for small systems (one warp per system, FP32) ----------------
// Lane r % 32 owns row r of the register-held vectors below: up to kWarpRows slots per lane.
constexpr int kWarpRows = 3;  // n <= 96

// Pivot key of |v| in row i (i < 256): the magnitude's leading 15 mantissa bits, then the lower
// row index on ties, so that one unsigned warp maximum picks the pivot (partial pivoting, up to
// a relative 2^-15 preference for the first row).
__device__ __forceinline__ unsigned pivot_key(float v, int i) {
  return (__float_as_uint(fabsf(v)) & 0xFFFFFF00u) | (unsigned)(255 - i);
}

// Element s of a register vector of R lane slots (s warp-uniform or per lane), without local
// memory: a chain of selects.
template <typename T, int R>
__device__ __forceinline__ T pick(const T (&a)[R], int s) {
  T v = a[0];
#pragma unroll
  for (int i = 1; i < R; ++i)
    if (s == i) v = a[i];
  return v;
}

__device__ __forceinline__ float comp4(const float4 &a, int t) {
  return t == 0 ? a.x : (t == 1 ? a.y : (t == 2 ? a.z : a.w));
}

__device__ __forceinline__ void set4(float4 &a, int t, float v) {
  if (t == 0) a.x = v; else if (t == 1) a.y = v; else if (t == 2) a.z = v; else a.w = v;
}

__device__ __forceinline__ float4 shfl4(const float4 &v, int src) {
  return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                     __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

__device__ __forceinline__ float4 fms4(float4 a, float l, const float4 &u) {  // a - l u
  a.x = fmaf(-l, u.x, a.x);
  a.y = fmaf(-l, u.y, a.y);
  a.z = fmaf(-l, u.z, a.z);
  a.w = fmaf(-l, u.w, a.w);
  return a;
}

// Solve the n x n system stored with its right-hand side as the augmented matrix M = [A | b]
// (column n holds b; row stride ld a multiple of 4 with ld / 4 odd and M 16-byte aligned, so
// that lanes reading float4 chunks of rows i, i + 1, ... hit distinct banks) by one warp:
// Gaussian elimination with partial pivoting (pivot_key over the rows not yet used as pivots),
// b eliminated along, then back substitution. Rows stay in place (implicit pivoting): row r is
// owned by lane r % 32. The elimination goes by panels of 4 columns (one float4 chunk): the
// lanes factor the panel in registers (4 pivot steps), finish the 4 pivot rows right of the
// panel (U rows, lanes over chunks), then apply one rank-4 update to every other row, so each
// trailing element passes through shared memory once per 4 steps. pseq (shared, n ints rounded
// up to 4) receives the pivot row of every step. Row k of the solution is returned in
// x[k / 32] of lane k % 32 (n <= 32 R). Returns true if a pivot was zero or not finite.
template <int R>
__device__ __forceinline__ void backsub_warp_steps(const float *M, int ld, int n, const int *pseq,
                                                   const int (&step)[R], const float (&dinv)[R],
                                                   float (&y)[R], float (&x)[R]);

template <int R>
__device__ __forceinline__ bool gepp_aug_warp(float *M, int ld, int n, float (&x)[R], int *pseq) {
  const int lane = threadIdx.x & 31;
  const int c_end = n >> 2;  // last float4 chunk: the one holding column n
  float4 *M4 = reinterpret_cast<float4 *>(M);
  const int ld4 = ld >> 2;
  float dinv[R];
  int step[R];       // step at which the row was the pivot; n: not yet; -1: no row
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = lane + 32 * s;
    step[s] = r < n ? n : -1;
    dinv[s] = 0.f;
  }
  for (int c0 = 0; 4 * c0 < n; ++c0) {
    float4 pc[R];    // own rows' panel chunk
    float lm[R][4];  // own rows' multipliers of the panel's steps
#pragma unroll
    for (int s = 0; s < R; ++s) {
      pc[s] = step[s] >= 0 ? M4[(lane + 32 * s) * ld4 + c0] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int t = 0; t < 4; ++t) lm[s][t] = 0.f;
    }
    int prow[4] = {0, 0, 0, 0};
    const int steps = min(4, n - 4 * c0);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= steps) break;
      const int p = 4 * c0 + t;
      unsigned key = 0;
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const unsigned k = pivot_key(comp4(pc[s], t), lane + 32 * s);
        if (step[s] == n && k > key) key = k;
      }
      key = __reduce_max_sync(0xffffffffu, key);
      const int piv = 255 - (int)(key & 255u), ps = piv >> 5;
      const float4 pp = shfl4(pick(pc, ps), piv & 31);
      const float pv = comp4(pp, t);
      // (the fast reciprocal is within 2 ulp below 2^126 in magnitude)
      if (!(fabsf(pv) > 0.f) || !(fabsf(pv) < 0x1p126f)) return true;
      const float rinv = __fdividef(1.0f, pv);
      prow[t] = piv;
      if (lane == 0) pseq[p] = piv;
#pragma unroll
      for (int s = 0; s < R; ++s) {
        if (lane + 32 * s == piv) {
          step[s] = p;
          dinv[s] = rinv;
        } else if (step[s] == n) {
          const float l = comp4(pc[s], t) * rinv;
          lm[s][t] = l;
#pragma unroll
          for (int t2 = t + 1; t2 < 4; ++t2) set4(pc[s], t2, fmaf(-l, comp4(pp, t2), comp4(pc[s], t2)));
          set4(pc[s], t, l);  // the eliminated entry keeps its multiplier (L, for later solves)
        }
      }
    }
    // panel chunks back (U entries of the pivot rows, the remaining rows' next values)
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (step[s] >= 0) M4[(lane + 32 * s) * ld4 + c0] = pc[s];
    // multipliers of the later pivot rows with respect to the earlier ones, in all lanes
    float lp[4][4];
#pragma unroll
    for (int t = 1; t < 4; ++t) {
      const int pr = prow[t], ps = pr >> 5;
#pragma unroll
      for (int t2 = 0; t2 < t; ++t2) {
        float v = lm[0][t2];
#pragma unroll
        for (int s = 1; s < R; ++s)
          if (ps == s) v = lm[s][t2];
        lp[t][t2] = __shfl_sync(0xffffffffu, v, pr & 31);
      }
    }
    __syncwarp();
    // U rows right of the panel, lanes over chunks: U_t = row_t - sum_{t2 < t} l(t, t2) U_t2
    for (int c = c0 + 1 + lane; c <= c_end; c += 32) {
      float4 u[4];
      u[0] = M4[prow[0] * ld4 + c];
#pragma unroll
      for (int t = 1; t < 4; ++t) {
        if (t >= steps) break;
        float4 a = M4[prow[t] * ld4 + c];
#pragma unroll
        for (int t2 = 0; t2 < t; ++t2) a = fms4(a, lp[t][t2], u[t2]);
        u[t] = a;
        M4[prow[t] * ld4 + c] = a;
      }
    }
    __syncwarp();
    // rank-`steps` update of the rows not yet used as pivots
#pragma unroll
    for (int s = 0; s < R; ++s) {
      if (step[s] != n) continue;
      float4 *row = M4 + (lane + 32 * s) * ld4;
#pragma unroll 2
      for (int c = c0 + 1; c <= c_end; ++c) {
        float4 a = row[c];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < steps) a = fms4(a, lm[s][t], M4[prow[t] * ld4 + c]);
        row[c] = a;
      }
    }
    __syncwarp();
  }
  float y[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = lane + 32 * s;
    y[s] = r < n ? M[r * ld + n] : 0.f;
  }
  backsub_warp_steps<R>(M, ld, n, pseq, step, dinv, y, x);
  return false;
}

// Back substitution in step order on the U rows left in place by gepp_aug_warp (row r pivoted
// step[r], 1 / pivot in dinv), the eliminated right-hand side in y: the solution entry of
// column j comes from row pseq[j]. Row k of the solution goes to x[k / 32] of lane k % 32.
template <int R>
__device__ __forceinline__ void backsub_warp_steps(const float *M, int ld, int n, const int *pseq,
                                                   const int (&step)[R], const float (&dinv)[R],
                                                   float (&y)[R], float (&x)[R]) {
  const int lane = threadIdx.x & 31;
  const float4 *M4 = reinterpret_cast<const float4 *>(M);
  const int ld4 = ld >> 2;
  for (int c = (n - 1) >> 2; c >= 0; --c) {
    float4 mc[R];
#pragma unroll
    for (int s = 0; s < R; ++s)
      mc[s] = step[s] >= 0 ? M4[(lane + 32 * s) * ld4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int4 pq = reinterpret_cast<const int4 *>(pseq)[c];
#pragma unroll
    for (int t = 3; t >= 0; --t) {
      const int j = 4 * c + t;
      if (j >= n) continue;
      const int pr = t == 0 ? pq.x : (t == 1 ? pq.y : (t == 2 ? pq.z : pq.w));
      float own[R];
#pragma unroll
      for (int s = 0; s < R; ++s) own[s] = y[s] * dinv[s];
      const float xj = __shfl_sync(0xffffffffu, pick(own, pr >> 5), pr & 31);
#pragma unroll
      for (int s = 0; s < R; ++s)
        if (step[s] >= 0 && step[s] < j) y[s] = fmaf(-comp4(mc[s], t), xj, y[s]);
    }
  }
  // row r holds the solution entry of the column it pivoted; gather by column
  float xr[R];
#pragma unroll
  for (int s = 0; s < R; ++s) xr[s] = y[s] * dinv[s];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int k = lane + 32 * s;
    const int pr = k < n ? pseq[k] : 0;
    float v = 0.f;
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) {
      const float t = __shfl_sync(0xffffffffu, xr[s2], pr & 31);
      if ((pr >> 5) == s2) v = t;
    }
    x[s] = v;
  }
}

// Solve with factors that gepp_aug_warp left in place (chord step: a new right-hand side in
// column n, the same Jacobian): forward elimination of the right-hand side in step order with
// the stored multipliers (row r, column p < step[r]), then back substitution on U. pseq from
// the factorisation; `stp` is shared scratch of n ints (the step of every row).
template <int R>
__device__ __forceinline__ bool chord_solve_warp(const float *M, int ld, int n, const int *pseq,
                                                 int *stp, float (&x)[R]) {
  const int lane = threadIdx.x & 31;
  const float4 *M4 = reinterpret_cast<const float4 *>(M);
  const int ld4 = ld >> 2;
  for (int p = lane; p < n; p += 32) stp[pseq[p]] = p;
  __syncwarp();
  int step[R];
  float dinv[R], y[R];
  bool bad = false;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = lane + 32 * s;
    step[s] = r < n ? stp[r] : -1;
    y[s] = r < n ? M[r * ld + n] : 0.f;
    const float pv = r < n ? M[r * ld + step[s]] : 1.f;
    bad |= !(fabsf(pv) > 0.f) || !(fabsf(pv) < 0x1p126f);
    dinv[s] = r < n ? __fdividef(1.0f, pv) : 0.f;
  }
  if (__any_sync(0xffffffffu, bad)) return true;
  // forward: b[r] -= l(r, p) b[pseq[p]] for the rows pivoted after step p
  for (int c = 0; 4 * c < n; ++c) {
    float4 mc[R];
#pragma unroll
    for (int s = 0; s < R; ++s)
      mc[s] = step[s] >= 0 ? M4[(lane + 32 * s) * ld4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int4 pq = reinterpret_cast<const int4 *>(pseq)[c];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int p = 4 * c + t;
      if (p >= n) break;
      const int pr = t == 0 ? pq.x : (t == 1 ? pq.y : (t == 2 ? pq.z : pq.w));
      const float bp = __shfl_sync(0xffffffffu, pick(y, pr >> 5), pr & 31);
#pragma unroll
      for (int s = 0; s < R; ++s)
        if (step[s] > p) y[s] = fmaf(-comp4(mc[s], t), bp, y[s]);
    }
  }
  backsub_warp_steps<R>(M, ld, n, pseq, step, dinv, y, x);
  return false;
}

// The same elimination by a CTA of W = ceil(n / 32) warps, one row per thread (row r owned by
// thread r; n <= 128): the matrix in shared memory as for gepp_aug_warp, panels of 4 columns.
// Each pivot step takes one CTA barrier: every warp's maximum key (redux) goes to `keys`
// (double-buffered by step parity), after the barrier every thread takes the maximum over the
// warps and reads the pivot row's current panel chunk from shared memory (every non-pivot row
// writes its updated chunk back after each step). After the panel's pivot steps the pivot rows'
// multipliers go through `lmp`, the threads finish the pivot rows right of the panel (threads
// over chunks) and every remaining row takes its rank-4 update. Back substitution runs in warp 0
// (rows in 4 lane slots, the pivot steps and reciprocals from `stepv` / `dinvv`); the solution
// entry of column k is left in xs[k]. Every thread must call this; returns true (all threads)
// if a pivot was zero or not finite. Scratch: pseq[n rounded to 4], keys[2 W], lmp[16],
// stepv[n], dinvv[n], xs[n].
__device__ __forceinline__ bool gepp_aug_cta(float *M, int ld, int n, int *pseq, unsigned *keys,
                                             float *lmp, int *stepv, float *dinvv, float *xs) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, W = blockDim.x >> 5;
  const int c_end = n >> 2;
  float4 *M4 = reinterpret_cast<float4 *>(M);
  const int ld4 = ld >> 2;
  int step = tid < n ? n : -1;  // step at which the row was the pivot; n: not yet; -1: no row
  float dinv = 0.f;
  for (int c0 = 0; 4 * c0 < n; ++c0) {
    float4 pc = step >= 0 ? M4[tid * ld4 + c0] : make_float4(0.f, 0.f, 0.f, 0.f);
    float lm[4] = {0.f, 0.f, 0.f, 0.f};
    int prow[4] = {0, 0, 0, 0};
    const int steps = min(4, n - 4 * c0);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= steps) break;
      const int p = 4 * c0 + t;
      unsigned key = step == n ? pivot_key(comp4(pc, t), tid) : 0u;
      key = __reduce_max_sync(0xffffffffu, key);
      if (lane == 0) keys[(p & 1) * W + w] = key;
      __syncthreads();
      unsigned kmax = 0;
      for (int i = 0; i < W; ++i) kmax = max(kmax, keys[(p & 1) * W + i]);
      const int piv = 255 - (int)(kmax & 255u);
      const float4 pp = M4[piv * ld4 + c0];
      const float pv = comp4(pp, t);
      // (the fast reciprocal is within 2 ulp below 2^126 in magnitude)
      if (!(fabsf(pv) > 0.f) || !(fabsf(pv) < 0x1p126f)) return true;  // uniform
      const float rinv = __fdividef(1.0f, pv);
      prow[t] = piv;
      if (tid == 0) pseq[p] = piv;
      if (tid == piv) {
        step = p;
        dinv = rinv;
      } else if (step == n) {
        const float l = comp4(pc, t) * rinv;
        lm[t] = l;
#pragma unroll
        for (int t2 = t + 1; t2 < 4; ++t2) set4(pc, t2, fmaf(-l, comp4(pp, t2), comp4(pc, t2)));
        set4(pc, t, l);           // the eliminated entry keeps its multiplier (L, for chord solves)
        M4[tid * ld4 + c0] = pc;  // current chunk for the next pivot step
      }
    }
    // multipliers of the panel's pivot rows with respect to its earlier pivots
    if (step >= 4 * c0 && step < 4 * c0 + steps) {
      const int t = step - 4 * c0;
      for (int t2 = 0; t2 < t; ++t2) lmp[4 * t + t2] = lm[t2];
    }
    __syncthreads();
    // U rows right of the panel, threads over chunks: U_t = row_t - sum_{t2 < t} l(t, t2) U_t2
    for (int c = c0 + 1 + tid; c <= c_end; c += blockDim.x) {
      float4 u[4];
      u[0] = M4[prow[0] * ld4 + c];
#pragma unroll
      for (int t = 1; t < 4; ++t) {
        if (t >= steps) break;
        float4 a = M4[prow[t] * ld4 + c];
#pragma unroll
        for (int t2 = 0; t2 < t; ++t2) a = fms4(a, lmp[4 * t + t2], u[t2]);
        u[t] = a;
        M4[prow[t] * ld4 + c] = a;
      }
    }
    __syncthreads();
    // rank-`steps` update of the rows not yet used as pivots
    if (step == n) {
      float4 *row = M4 + tid * ld4;
#pragma unroll 2
      for (int c = c0 + 1; c <= c_end; ++c) {
        float4 a = row[c];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < steps) a = fms4(a, lm[t], M4[prow[t] * ld4 + c]);
        row[c] = a;
      }
    }
    // the next panel reads other rows only after its first pivot barrier
  }
  if (tid < n) {
    stepv[tid] = step;
    dinvv[tid] = dinv;
  }
  __syncthreads();
  if (w == 0) {  // back substitution in step order, rows r = lane + 32 s
    constexpr int RS = 4;
    int st[RS];
    float y[RS], dv[RS];
#pragma unroll
    for (int s = 0; s < RS; ++s) {
      const int r = lane + 32 * s;
      st[s] = r < n ? stepv[r] : -1;
      dv[s] = r < n ? dinvv[r] : 0.f;
      y[s] = r < n ? M[r * ld + n] : 0.f;
    }
    for (int c = (n - 1) >> 2; c >= 0; --c) {
      float4 mc[RS];
#pragma unroll
      for (int s = 0; s < RS; ++s)
        mc[s] = st[s] >= 0 ? M4[(lane + 32 * s) * ld4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
      const int4 pq = reinterpret_cast<const int4 *>(pseq)[c];
#pragma unroll
      for (int t = 3; t >= 0; --t) {
        const int j = 4 * c + t;
        if (j >= n) continue;
        const int pr = t == 0 ? pq.x : (t == 1 ? pq.y : (t == 2 ? pq.z : pq.w));
        float own[RS];
#pragma unroll
        for (int s = 0; s < RS; ++s) own[s] = y[s] * dv[s];
        const float xj = __shfl_sync(0xffffffffu, pick(own, pr >> 5), pr & 31);
        if (lane == 0) xs[j] = xj;
#pragma unroll
        for (int s = 0; s < RS; ++s)
          if (st[s] >= 0 && st[s] < j) y[s] = fmaf(-comp4(mc[s], t), xj, y[s]);
      }
    }
  }
  __syncthreads();
  return false;
}

}  // namespace rb
