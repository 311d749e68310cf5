// k_reconstruct.cu -- pressure reconstruction with a combined velocity-pressure basis (Sec. 4.2).
//
// Every velocity basis function j carries pressure data p^_j (the "second approach" of Sec. 4.2:
// the pressure functions are combined with the same snapshot coefficients as the velocity
// functions), so a solution with velocity coefficients u has the pressure p = sum_j u_j p^_j.
// The velocity system of Sec. 4.1 (Eq. blocksolve-1) is untouched; this replaces the recovery
// of Eq. sup-vvar by one batched matrix-vector product per query. The pressure modes are kept
// transposed, PT [n_max][m_r], so that the threads of a CTA, one pressure coefficient k each,
// read consecutive addresses of one row j and write consecutive entries of p.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "rb_ctx.h"

namespace rb {

constexpr int kRecQ = 8;    // queries per CTA (their u rows staged in shared memory)
constexpr int kRecT = 256;  // threads per CTA: one pressure coefficient each

// p[b][k] = sum_{j < n_b} PT[j][k] u[b][j], j ascending; n_b outside 1..n_max: NaN.
// grid.x: tiles of kRecQ queries; grid.y (grid-stride): tiles of kRecT coefficients.
__global__ void __launch_bounds__(kRecT) k_reconstruct(const double *__restrict__ PT, int n_max,
                                                       int m_r, const double *__restrict__ u,
                                                       int nq, const int *__restrict__ nsz,
                                                       double *__restrict__ p) {
  __shared__ double us[kRecQ][RB_N_MAX];
  __shared__ int nn[kRecQ];
  const long long b0 = (long long)blockIdx.x * kRecQ;
  if (threadIdx.x < kRecQ) {
    const long long b = b0 + threadIdx.x;
    int n = 0;  // 0: no query in this row of the tile
    if (b < nq) {
      n = nsz ? nsz[b] : n_max;
      if (n < 1 || n > n_max) n = -1;  // rejected size
    }
    nn[threadIdx.x] = n;
  }
  __syncthreads();
  int nt = 0;
#pragma unroll
  for (int q = 0; q < kRecQ; ++q) nt = max(nt, nn[q]);
  for (int i = threadIdx.x; i < kRecQ * n_max; i += kRecT) {
    const int q = i / n_max, j = i - q * n_max;
    us[q][j] = j < nn[q] ? u[(size_t)(b0 + q) * n_max + j] : 0.0;
  }
  __syncthreads();
  for (long long k = (long long)blockIdx.y * kRecT + threadIdx.x; k < m_r;
       k += (long long)gridDim.y * kRecT) {
    double acc[kRecQ];
#pragma unroll
    for (int q = 0; q < kRecQ; ++q) acc[q] = 0.0;
    const double *col = PT + k;
#pragma unroll 16
    for (int j = 0; j < nt; ++j) {  // 16 independent loads in flight per thread
      const double a = __ldg(col + (size_t)j * m_r);
#pragma unroll
      for (int q = 0; q < kRecQ; ++q) acc[q] = fma(a, us[q][j], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kRecQ; ++q)
      if (nn[q] != 0) p[(size_t)(b0 + q) * m_r + k] = nn[q] > 0 ? acc[q] : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// Small pressure spaces (m_r <= kRecFlatMax): one thread per (query, coefficient) with the
// coefficient fastest, so a launch keeps nq m_r threads in flight (the tiled kernel would leave
// most of its 256 threads idle); the same sums in the same order as k_reconstruct.
constexpr int kRecFlatMax = 128;
__global__ void __launch_bounds__(256) k_reconstruct_flat(const double *__restrict__ PT,
                                                          int n_max, int m_r,
                                                          const double *__restrict__ u, int nq,
                                                          const int *__restrict__ nsz,
                                                          double *__restrict__ p) {
  const long long total = (long long)nq * m_r;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / m_r;
    const int k = (int)(i - b * m_r);
    const int n = nsz ? nsz[b] : n_max;
    if (n < 1 || n > n_max) {
      p[i] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    const double *ub = u + (size_t)b * n_max;
    const double *col = PT + k;
    double acc = 0.0;
#pragma unroll 8
    for (int j = 0; j < n; ++j) acc = fma(__ldg(col + (size_t)j * m_r), __ldg(ub + j), acc);
    p[i] = acc;
  }
}

// PT[j][k] = P[k][j] for P [m_r][n_max], 32 x 32 tiles through shared memory.
__global__ void k_transpose_modes(const double *__restrict__ P, int m_r, int n_max,
                                  double *__restrict__ PT) {
  __shared__ double t[32][33];
  const long long k0 = (long long)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const long long k = k0 + r;
    const int j = j0 + threadIdx.x;
    if (k < m_r && j < n_max) t[r][threadIdx.x] = P[(size_t)k * n_max + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r;
    const long long k = k0 + threadIdx.x;
    if (k < m_r && j < n_max) PT[(size_t)j * m_r + k] = t[threadIdx.x][r];
  }
}

void drop_pressure_modes(rb_ctx *ctx) {
  if (ctx->d_PT) ctx_free(ctx, ctx->d_PT);
  ctx->d_PT = nullptr;
  ctx->m_r = 0;
}

int reconstruct_impl(rb_ctx *ctx, const double *d_u, int nq, const int *d_n, double *d_p,
                     cudaStream_t st) {
  if (!ctx->d_PT) return set_error(ctx, RB_ERR_STATE, "no pressure modes loaded");
  if (nq == 0) return RB_OK;
  const int mk = prof_begin(ctx, RB_K_RECONSTRUCT, st);
  if (ctx->m_r <= kRecFlatMax) {
    const long long total = (long long)nq * ctx->m_r;
    const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)ctx->sms * 16);
    k_reconstruct_flat<<<blocks, 256, 0, st>>>(ctx->d_PT, ctx->ops.n_max, ctx->m_r, d_u, nq, d_n, d_p);
  } else {
    const long long k_tiles = (ctx->m_r + kRecT - 1) / kRecT;
    dim3 grid((unsigned)((nq + kRecQ - 1) / kRecQ), (unsigned)std::min<long long>(k_tiles, 65535));
    k_reconstruct<<<grid, kRecT, 0, st>>>(ctx->d_PT, ctx->ops.n_max, ctx->m_r, d_u, nq, d_n, d_p);
  }
  prof_end(ctx, mk, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_reconstruct");
  return RB_OK;
}

}  // namespace rb

using namespace rb;

extern "C" {

int rb_load_pressure_modes(rb_ctx *ctx, const double *P_hat, int m_r) {
  if (!ctx) return RB_ERR_ARG;
  if (!ctx->loaded) return set_error(ctx, RB_ERR_STATE, "no operators loaded");
  if (!P_hat || m_r < 1 || m_r > RB_MR_MAX)
    return set_error(ctx, RB_ERR_ARG, "pressure modes: P_hat NULL or m_r outside 1..%d", RB_MR_MAX);
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  drop_pressure_modes(ctx);
  const int n = ctx->ops.n_max;
  const size_t bytes = sizeof(double) * (size_t)m_r * n;
  void *pt = nullptr;
  int rc = ctx_alloc(ctx, &pt, bytes, "pressure modes");
  if (rc != RB_OK) return rc;
  if ((rc = ctx->stage.reserve(ctx, bytes, "pressure modes upload")) != RB_OK) {
    ctx_free(ctx, pt);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(ctx->stage.ptr, P_hat, bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    dim3 grid((unsigned)((m_r + 31) / 32), (unsigned)((n + 31) / 32));
    k_transpose_modes<<<grid, dim3(32, 8), 0, ctx->stream>>>((const double *)ctx->stage.ptr, m_r, n,
                                                             (double *)pt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    ctx_free(ctx, pt);
    return cuda_fail(ctx, e, "rb_load_pressure_modes");
  }
  ctx->d_PT = (double *)pt;
  ctx->m_r = m_r;
  return RB_OK;
}

int rb_reconstruct_pressure_device(rb_ctx *ctx, const double *d_u, int n_queries, const int *d_n,
                                   double *d_p, void *cuda_stream) {
  if (!ctx) return RB_ERR_ARG;
  if (n_queries < 0 || (n_queries > 0 && (!d_u || !d_p)))
    return set_error(ctx, RB_ERR_ARG, "bad arguments to rb_reconstruct_pressure_device");
  cudaSetDevice(ctx->device);
  return reconstruct_impl(ctx, d_u, n_queries, d_n, d_p, (cudaStream_t)cuda_stream);
}

int rb_reconstruct_pressure(rb_ctx *ctx, const double *u, int n_queries, const int *n,
                            double *p_out) {
  if (!ctx) return RB_ERR_ARG;
  if (n_queries < 0 || (n_queries > 0 && (!u || !p_out)))
    return set_error(ctx, RB_ERR_ARG, "bad arguments to rb_reconstruct_pressure");
  if (!ctx->d_PT) return set_error(ctx, RB_ERR_STATE, "no pressure modes loaded");
  if (n_queries == 0) return RB_OK;
  cudaSetDevice(ctx->device);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_u = al(sizeof(double) * (size_t)n_queries * ctx->ops.n_max);
  const size_t b_n = al(sizeof(int) * (size_t)n_queries);
  const size_t b_p = sizeof(double) * (size_t)n_queries * ctx->m_r;
  int rc = ctx->stage.reserve(ctx, b_u + b_n + b_p, "reconstruction staging");
  if (rc != RB_OK) return rc;
  char *base = (char *)ctx->stage.ptr;
  double *d_u = (double *)base;
  int *d_n = n ? (int *)(base + b_u) : nullptr;
  double *d_p = (double *)(base + b_u + b_n);
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(d_u, u, sizeof(double) * (size_t)n_queries * ctx->ops.n_max,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n)
    e = cudaMemcpyAsync(d_n, n, sizeof(int) * (size_t)n_queries, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_reconstruct_pressure upload");
  if ((rc = reconstruct_impl(ctx, d_u, n_queries, d_n, d_p, st)) != RB_OK) return rc;
  e = cudaMemcpyAsync(p_out, d_p, b_p, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_reconstruct_pressure");
  return RB_OK;
}

}  // extern "C"
