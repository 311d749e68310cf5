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
    th[i] = trig_q(q, a) * scale;
  }
}

// theta row of one query, all threads of the block
__device__ __forceinline__ void theta_eval(const DevOps &o, double alpha_deg, double re,
                                           double *th) {
  theta_eval_strided(o, alpha_deg, re, th, threadIdx.x, blockDim.x);
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

__device__ __forceinline__ void df_split(double v, float &h, float &l) {
  h = (float)v;
  l = (float)(v - (double)h);
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

// Warp-cooperative variant of gepp_solve_block for one small system per warp (no block
// barriers): same pivoting rule, same operation order per entry.
template <typename T>
__device__ bool gepp_solve_warp(T *M, int ld, int n, T *b) {
  const int lane = threadIdx.x & 31;
  for (int p = 0; p < n; ++p) {
    T best = T(-1);
    int brow = n;
    for (int i = p + lane; i < n; i += 32) argmax_merge<T>(best, brow, fabs(M[(size_t)i * ld + p]), i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int r2 = __shfl_xor_sync(0xffffffffu, brow, o);
      argmax_merge<T>(best, brow, v2, r2);
    }
    if (!(best > T(0)) || !isfinite(best)) return true;
    if (brow != p) {
      for (int j = p + lane; j < n; j += 32) {
        const T t = M[(size_t)p * ld + j];
        M[(size_t)p * ld + j] = M[(size_t)brow * ld + j];
        M[(size_t)brow * ld + j] = t;
      }
      if (lane == 0) { const T t = b[p]; b[p] = b[brow]; b[brow] = t; }
    }
    __syncwarp();
    const T piv = M[(size_t)p * ld + p];
    for (int i = p + 1 + lane; i < n; i += 32) M[(size_t)i * ld + p] = M[(size_t)i * ld + p] / piv;
    __syncwarp();
    const T bp = b[p];
    // trailing update: lanes over rows, 4 columns per step (independent loads in flight)
    for (int i = p + 1 + lane; i < n; i += 32) {
      T *Mi = M + (size_t)i * ld;
      const T *Mp = M + (size_t)p * ld;
      const T lip = Mi[p];
      int j = p + 1;
      for (; j + 4 <= n; j += 4) {
        const T a0 = Mi[j], a1 = Mi[j + 1], a2 = Mi[j + 2], a3 = Mi[j + 3];
        const T p0 = Mp[j], p1 = Mp[j + 1], p2 = Mp[j + 2], p3 = Mp[j + 3];
        Mi[j] = a0 - lip * p0;
        Mi[j + 1] = a1 - lip * p1;
        Mi[j + 2] = a2 - lip * p2;
        Mi[j + 3] = a3 - lip * p3;
      }
      for (; j < n; ++j) Mi[j] -= lip * Mp[j];
      b[i] -= lip * bp;
    }
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = T(0);
    for (int j = i + 1 + lane; j < n; j += 32) s += M[(size_t)i * ld + j] * b[j];
    s = warp_sum(s);
    if (lane == 0) b[i] = (b[i] - s) / M[(size_t)i * ld + i];
    __syncwarp();
  }
  return false;
}

}  // namespace rb
