// rb_offline.cu -- the offline stage: reduced operators from high-fidelity data, in FP64 on the GPU.
//
//  * POD by the method of snapshots (Sec. 3.2): the covariance matrix C_ij = z(phi_i, phi_j)
//    (Eq. covmx) as S^T (Z S) with a CSR product and a split-K Gram kernel, its eigenpairs by a
//    cyclic Jacobi method in one CTA (the matrix in shared memory, disjoint rotations applied in
//    parallel), and the modes psi_j = lambda_j^(-1/2) sum_i v^j_i phi_i (Eq. spd).
//  * Galerkin projection (Sec. 3.5, Eq. redorth-final): M^R = V^T (M V), f^R = V^T f.
//  * The third-order tensor of a trilinear form given by pointwise quadrature terms (Sec. 3.6,
//    Eq. tensor): C[j][l][k] = sum_terms sum_x w(x) (P psi_j)(x) (Q psi_l)(x) (R psi_k)(x), the
//    evaluated modes from CSR products, then a tiled triple contraction over the points, split
//    over point chunks whose partial tensors add in a fixed order (deterministic).
// Everything is FP64: the results are the operators of the online stage, which takes them as exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rb_ctx.h"

namespace rb {

namespace {

// ---- CSR times dense: Y[r][c] = sum_e val[e] X[col[e]][c], X [cols][m], Y [rows][m] ----------
__global__ void k_csr_dense(int rows, int m, const int *indptr, const int *indices,
                            const double *values, const double *X, double *Y) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += nw) {
    const int e0 = indptr[r], e1 = indptr[r + 1];
    for (int c0 = 0; c0 < m; c0 += 32) {
      const int c = c0 + lane;
      double s = 0.0;
      for (int e = e0; e < e1; ++e) {
        const double v = values[e];
        if (c < m) s = fma(v, X[(size_t)indices[e] * m + c], s);
      }
      if (c < m) Y[(size_t)r * m + c] = s;
    }
  }
}

// out[c][r] = in[r][c] for in [rows][cols] (32 x 32 tiles through shared memory)
__global__ void k_transpose(int rows, int cols, const double *in, double *out) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = by + i, c = bx + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = bx + i, r = by + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * rows + r] = t[threadIdx.x][i];
  }
}

// Gram of two tall matrices over one chunk of rows: part[chunk][i][j] = sum_{r in chunk}
// A[r][i] B[r][j], A [N][m1], B [N][m2] (m1, m2 <= kGramMax); 256 threads, each an 8 x 8 block
// of outputs, rows staged through shared memory 16 at a time.
constexpr int kGramMax = 128, kGramRows = 16;
__global__ void __launch_bounds__(256) k_gram_part(int N, int m1, int m2, int chunk_rows,
                                                   const double *A, const double *B, double *part) {
  __shared__ double sa[kGramRows][kGramMax], sb[kGramRows][kGramMax];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.x * chunk_rows, r1 = min(N, r0 + chunk_rows);
  double acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
  for (int rb = r0; rb < r1; rb += kGramRows) {
    const int cnt = min(kGramRows, r1 - rb);
    __syncthreads();
    for (int e = threadIdx.x; e < kGramRows * kGramMax; e += blockDim.x) {
      const int r = e / kGramMax, c = e - r * kGramMax;
      sa[r][c] = (r < cnt && c < m1) ? A[(size_t)(rb + r) * m1 + c] : 0.0;
      sb[r][c] = (r < cnt && c < m2) ? B[(size_t)(rb + r) * m2 + c] : 0.0;
    }
    __syncthreads();
    for (int r = 0; r < cnt; ++r) {
      double x[8], y[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) x[a] = sa[r][ty * 8 + a];
#pragma unroll
      for (int b = 0; b < 8; ++b) y[b] = sb[r][tx * 8 + b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
    }
  }
  double *out = part + (size_t)blockIdx.x * m1 * m2;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = ty * 8 + a, j = tx * 8 + b;
      if (i < m1 && j < m2) out[(size_t)i * m2 + j] = acc[a][b];
    }
}

// out[e] = sum_{c < chunks} part[c][e] in chunk order
__global__ void k_sum_parts(size_t count, int chunks, const double *part, double *out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[(size_t)c * count + e];
    out[e] = s;
  }
}

// ---- symmetric eigenproblem by the cyclic Jacobi method (one CTA) ---------------------------
// A (K x K, symmetric, K <= RB_POD_K_MAX) in shared memory; every round rotates K/2 disjoint
// index pairs (a round-robin tournament covers all pairs in K - 1 rounds: one sweep): for each
// pair (p, q) the rotation of the symmetric Schur decomposition of the 2 x 2 block that zeroes
// A[p][q] (Golub and Van Loan, Algorithm 8.4.1), then rows p, q of A, columns p, q of A and of
// the accumulated rotations W. Sweeps until the off-diagonal part falls below 1e-15 of the norm.
// Output: lam (the diagonal) and W [K][K] (columns = eigenvectors).
constexpr int kJacThreads = 512;
__global__ void __launch_bounds__(kJacThreads) k_jacobi(int K, const double *Ain, double *W,
                                                        double *lam, int max_sweeps, int *sweeps) {
  extern __shared__ double smj[];
  const int Kp = K + (K & 1);                // even: a dummy index K when K is odd
  double *A = smj;                           // [K][K]
  double *cs = A + (size_t)K * K;            // [Kp / 2][2] cos, sin
  int *order = reinterpret_cast<int *>(cs + Kp);  // [Kp] tournament positions
  double *red = reinterpret_cast<double *>(order + Kp + (Kp & 1));  // [2 * warps]
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int half = Kp / 2;
  for (int e = tid; e < K * K; e += nthr) {
    A[e] = Ain[e];
    W[e] = (e / K == e % K) ? 1.0 : 0.0;
  }
  for (int i = tid; i < Kp; i += nthr) order[i] = i;
  __syncthreads();
  int sw = 0;
  for (; sw < max_sweeps; ++sw) {
    // convergence: off-diagonal and total Frobenius norms
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < K * K; e += nthr) {
      const double v = A[e] * A[e];
      tot += v;
      if (e / K != e % K) off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) {
      red[2 * (tid >> 5)] = off;
      red[2 * (tid >> 5) + 1] = tot;
    }
    __syncthreads();
    double so = 0.0, st = 0.0;
    for (int w = 0; w < nthr / 32; ++w) {
      so += red[2 * w];
      st += red[2 * w + 1];
    }
    __syncthreads();
    if (!(so > 1e-30 * st)) break;  // off-diagonal below 1e-15 of the norm (also all zero)
    for (int round = 0; round < Kp - 1; ++round) {
      // pair k: positions k and Kp - 1 - k of the tournament order
      for (int k = tid; k < half; k += nthr) {
        int p = order[k], q = order[Kp - 1 - k];
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < K) {
          const double apq = A[p * K + q];
          if (apq != 0.0) {
            const double tau = (A[q * K + q] - A[p * K + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // rows p, q of A: A <- J^T A
      for (int e = tid; e < half * K; e += nthr) {
        const int k = e / K, col = e - k * K;
        int p = order[k], q = order[Kp - 1 - k];
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= K) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1];
        const double a = A[p * K + col], b = A[q * K + col];
        A[p * K + col] = c * a - s * b;
        A[q * K + col] = s * a + c * b;
      }
      __syncthreads();
      // columns p, q of A and of W: A <- A J, W <- W J
      for (int e = tid; e < half * K; e += nthr) {
        const int k = e / K, row = e - k * K;
        int p = order[k], q = order[Kp - 1 - k];
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= K) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1];
        const double a = A[row * K + p], b = A[row * K + q];
        A[row * K + p] = c * a - s * b;
        A[row * K + q] = s * a + c * b;
        const double wa = W[(size_t)row * K + p], wb = W[(size_t)row * K + q];
        W[(size_t)row * K + p] = c * wa - s * wb;
        W[(size_t)row * K + q] = s * wa + c * wb;
      }
      __syncthreads();
      // next round of the tournament: position 0 stays, the others rotate by one
      if (tid == 0) {
        const int last = order[Kp - 1];
        for (int i = Kp - 1; i > 1; --i) order[i] = order[i - 1];
        order[1] = last;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < K; i += nthr) lam[i] = A[i * K + i];
  if (tid == 0) *sweeps = sw;
}

// Modes of Eq. spd: VT[r][m] = sum_i ST[r][i] W[i][perm[m]] / sqrt(lam[perm[m]]), the
// eigenvalues in decreasing order (perm from their ranks, ties by index). One warp per row r.
__global__ void k_modes(int N, int K, int n, const double *ST, const double *W, const double *lam,
                        const int *perm, double *VT) {
  extern __shared__ double wn[];  // [K][n]
  for (int e = threadIdx.x; e < K * n; e += blockDim.x) {
    const int i = e / n, m = e - i * n;
    wn[e] = W[(size_t)i * K + perm[m]] / sqrt(lam[perm[m]]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N; r += nw) {
    const double *s = ST + (size_t)r * K;
    for (int m0 = 0; m0 < n; m0 += 32) {
      const int m = m0 + lane;
      double acc = 0.0;
      for (int i = 0; i < K; ++i) {
        const double x = s[i];
        if (m < n) acc = fma(x, wn[i * n + m], acc);
      }
      if (m < n) VT[(size_t)r * n + m] = acc;
    }
  }
}

// ranks of the eigenvalues: perm[rank] = i, decreasing, ties by index
__global__ void k_rank(int K, const double *lam, int *perm, double *lam_sorted) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
    int r = 0;
    const double li = lam[i];
    for (int j = 0; j < K; ++j) {
      const double lj = lam[j];
      if (lj > li || (lj == li && j < i)) ++r;
    }
    perm[r] = i;
    lam_sorted[r] = li;
  }
}

// Triple contraction over one chunk of points: part[chunk][j][l][k] += sum_{x in chunk}
// EP[x][j] EQ[x][l] ER[x][k] (the weight already in EP). A CTA takes an 8 x 8 block of (j, l)
// and a block of up to 64 k; thread t: pair (j, l) = t / 4, k = k0 + t % 4 + 4 i. Points are
// staged through shared memory 32 at a time.
constexpr int kTriJ = 8, kTriK = 64, kTriPts = 32;
__global__ void __launch_bounds__(256) k_triple(int npts, int n, int chunk_pts, const double *EP,
                                                const double *EQ, const double *ER, double *part) {
  __shared__ double sp_[kTriPts][kTriJ], sq[kTriPts][kTriJ], sr[kTriPts][kTriK];
  const int jb = blockIdx.x * kTriJ, lb = blockIdx.y * kTriJ;
  const int kb = (blockIdx.z % ((n + kTriK - 1) / kTriK)) * kTriK;
  const int chunk = blockIdx.z / ((n + kTriK - 1) / kTriK);
  const int x0 = chunk * chunk_pts, x1 = min(npts, x0 + chunk_pts);
  const int t = threadIdx.x;
  const int pr = t >> 2, kq = t & 3;
  const int jj = pr >> 3, ll = pr & 7;
  const int j = jb + jj, l = lb + ll;
  double acc[kTriK / 4];
#pragma unroll
  for (int i = 0; i < kTriK / 4; ++i) acc[i] = 0.0;
  for (int xb = x0; xb < x1; xb += kTriPts) {
    const int cnt = min(kTriPts, x1 - xb);
    __syncthreads();
    for (int e = t; e < kTriPts * kTriJ; e += blockDim.x) {
      const int x = e / kTriJ, c = e - x * kTriJ;
      sp_[x][c] = (x < cnt && jb + c < n) ? EP[(size_t)(xb + x) * n + jb + c] : 0.0;
      sq[x][c] = (x < cnt && lb + c < n) ? EQ[(size_t)(xb + x) * n + lb + c] : 0.0;
    }
    for (int e = t; e < kTriPts * kTriK; e += blockDim.x) {
      const int x = e / kTriK, c = e - x * kTriK;
      sr[x][c] = (x < cnt && kb + c < n) ? ER[(size_t)(xb + x) * n + kb + c] : 0.0;
    }
    __syncthreads();
    for (int x = 0; x < cnt; ++x) {
      const double pq = sp_[x][jj] * sq[x][ll];
#pragma unroll
      for (int i = 0; i < kTriK / 4; ++i) acc[i] = fma(pq, sr[x][kq + 4 * i], acc[i]);
    }
  }
  if (j < n && l < n) {
    double *out = part + (size_t)chunk * n * n * n + ((size_t)j * n + l) * n;
#pragma unroll
    for (int i = 0; i < kTriK / 4; ++i) {
      const int k = kb + kq + 4 * i;
      if (k < n) out[k] += acc[i];
    }
  }
}

__global__ void k_scale_rows(int rows, int m, const double *w, double *Y) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)rows * m;
       e += (size_t)gridDim.x * blockDim.x)
    Y[e] *= w[e / m];
}

// ---- host helpers -------------------------------------------------------------------------
struct Buffers {  // device allocations of one call, freed at its end
  rb_ctx *ctx;
  std::vector<void *> ptrs;
  explicit Buffers(rb_ctx *c) : ctx(c) {}
  ~Buffers() {
    for (void *p : ptrs) ctx_free(ctx, p);
  }
  template <typename T>
  int get(T **p, size_t count, const char *what) {
    void *q = nullptr;
    const int rc = ctx_alloc(ctx, &q, sizeof(T) * std::max<size_t>(count, 1), what);
    if (rc == RB_OK) ptrs.push_back(q);
    *p = (T *)q;
    return rc;
  }
};

bool csr_ok(const rb_csr *M, int rows, int cols) {
  return M && M->indptr && (M->rows == 0 || M->indices) && M->rows >= 0 && M->cols == cols &&
         (rows < 0 || M->rows == rows);
}

// upload a CSR matrix (the caller's host arrays)
int upload_csr(rb_ctx *ctx, Buffers &B, const rb_csr *M, int **ip, int **ix, double **v,
               const char *what) {
  const int nnz = M->indptr[M->rows];
  if (M->indptr[0] != 0 || nnz < 0) return set_error(ctx, RB_ERR_ARG, "%s: indptr[0] must be 0", what);
  for (int r = 0; r < M->rows; ++r)
    if (M->indptr[r + 1] < M->indptr[r]) return set_error(ctx, RB_ERR_ARG, "%s: indptr not monotone", what);
  for (int e = 0; e < nnz; ++e)
    if (M->indices[e] < 0 || M->indices[e] >= M->cols)
      return set_error(ctx, RB_ERR_ARG, "%s: column index %d out of range", what, M->indices[e]);
  int rc;
  if ((rc = B.get(ip, (size_t)M->rows + 1, what)) != RB_OK) return rc;
  if ((rc = B.get(ix, (size_t)nnz, what)) != RB_OK) return rc;
  if ((rc = B.get(v, (size_t)nnz, what)) != RB_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(*ip, M->indptr, 4 * ((size_t)M->rows + 1), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && nnz)
    e = cudaMemcpyAsync(*ix, M->indices, 4 * (size_t)nnz, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && nnz)
    e = cudaMemcpyAsync(*v, M->values, 8 * (size_t)nnz, cudaMemcpyHostToDevice, ctx->stream);
  return e == cudaSuccess ? RB_OK : cuda_fail(ctx, e, what);
}

int spmm(rb_ctx *ctx, int rows, int m, const int *ip, const int *ix, const double *v,
         const double *X, double *Y) {
  const int grid = std::max(1, std::min((rows + 7) / 8, ctx->sms * 16));
  k_csr_dense<<<grid, 256, 0, ctx->stream>>>(rows, m, ip, ix, v, X, Y);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RB_OK : cuda_fail(ctx, e, "k_csr_dense");
}

int transpose(rb_ctx *ctx, int rows, int cols, const double *in, double *out) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, ctx->stream>>>(rows, cols, in, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RB_OK : cuda_fail(ctx, e, "k_transpose");
}

// G = A^T B for A [N][m1], B [N][m2] (m1, m2 <= kGramMax), split over row chunks
int gram(rb_ctx *ctx, Buffers &Bf, int N, int m1, int m2, const double *A, const double *B,
         double *G) {
  const int chunks = std::max(1, std::min(2 * ctx->sms, (N + 255) / 256));
  const int chunk_rows = (N + chunks - 1) / chunks;
  double *part;
  int rc;
  if ((rc = Bf.get(&part, (size_t)chunks * m1 * m2, "Gram partial sums")) != RB_OK) return rc;
  k_gram_part<<<chunks, 256, 0, ctx->stream>>>(N, m1, m2, chunk_rows, A, B, part);
  k_sum_parts<<<std::max(1, std::min(ctx->sms * 4, (m1 * m2 + 255) / 256)), 256, 0, ctx->stream>>>(
      (size_t)m1 * m2, chunks, part, G);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RB_OK : cuda_fail(ctx, e, "k_gram_part");
}

int finish(rb_ctx *ctx, const char *what) {
  const cudaError_t e = cudaStreamSynchronize(ctx->stream);
  return e == cudaSuccess ? RB_OK : cuda_fail(ctx, e, what);
}

}  // namespace

size_t jacobi_smem_bytes(int K) {
  const int Kp = K + (K & 1);
  return sizeof(double) * ((size_t)K * K + Kp) + sizeof(int) * (Kp + (Kp & 1)) +
         sizeof(double) * 2 * (kJacThreads / 32);
}

}  // namespace rb

using namespace rb;

extern "C" {

int rb_offline_pod(rb_ctx *ctx, const double *S, int K, int N, const rb_csr *Z, int n,
                   double *V_out, double *lambda_out) {
  if (!ctx) return RB_ERR_ARG;
  if (!S || !V_out || K < 1 || K > RB_POD_K_MAX || N < 1 || n < 1 || n > K || !csr_ok(Z, N, N))
    return set_error(ctx, RB_ERR_ARG, "rb_offline_pod: bad arguments (1 <= n <= K <= %d, Z N x N)",
                     RB_POD_K_MAX);
  cudaSetDevice(ctx->device);
  if ((size_t)jacobi_smem_bytes(K) > (size_t)ctx->max_smem)
    return set_error(ctx, RB_ERR_ARG, "rb_offline_pod: K = %d needs more shared memory", K);
  Buffers B(ctx);
  double *dS, *ST, *ZS, *C, *W, *lam, *lams, *VT, *V;
  int *ip, *ix, *perm, *sweeps;
  double *zv;
  int rc;
  if ((rc = B.get(&dS, (size_t)K * N, "snapshots")) != RB_OK) return rc;
  if ((rc = B.get(&ST, (size_t)K * N, "snapshots (transposed)")) != RB_OK) return rc;
  if ((rc = B.get(&ZS, (size_t)K * N, "Z S")) != RB_OK) return rc;
  if ((rc = B.get(&C, (size_t)K * K, "covariance")) != RB_OK) return rc;
  if ((rc = B.get(&W, (size_t)K * K, "eigenvectors")) != RB_OK) return rc;
  if ((rc = B.get(&lam, (size_t)K, "eigenvalues")) != RB_OK) return rc;
  if ((rc = B.get(&lams, (size_t)K, "eigenvalues (sorted)")) != RB_OK) return rc;
  if ((rc = B.get(&perm, (size_t)K, "eigenvalue order")) != RB_OK) return rc;
  if ((rc = B.get(&sweeps, 1, "sweep count")) != RB_OK) return rc;
  if ((rc = B.get(&VT, (size_t)N * n, "modes")) != RB_OK) return rc;
  if ((rc = B.get(&V, (size_t)N * n, "modes (rows)")) != RB_OK) return rc;
  if ((rc = upload_csr(ctx, B, Z, &ip, &ix, &zv, "Z")) != RB_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(dS, S, 8 * (size_t)K * N, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "snapshots upload");
  if ((rc = transpose(ctx, K, N, dS, ST)) != RB_OK) return rc;            // ST [N][K]
  if ((rc = spmm(ctx, N, K, ip, ix, zv, ST, ZS)) != RB_OK) return rc;      // Z S   [N][K]
  const size_t js = jacobi_smem_bytes(K);
  e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)js);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_jacobi attribute");
  const int mk = prof_begin(ctx, RB_K_OFFLINE_EIG, ctx->stream);
  if ((rc = gram(ctx, B, N, K, K, ST, ZS, C)) != RB_OK) return rc;         // S^T Z S (Eq. covmx)
  k_jacobi<<<1, kJacThreads, js, ctx->stream>>>(K, C, W, lam, 40, sweeps);
  k_rank<<<1, 256, 0, ctx->stream>>>(K, lam, perm, lams);
  prof_end(ctx, mk, ctx->stream);
  const size_t ms = 8 * (size_t)K * n;
  if (ms > (size_t)ctx->max_smem) return set_error(ctx, RB_ERR_ARG, "rb_offline_pod: K n too large");
  e = cudaFuncSetAttribute(k_modes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_modes attribute");
  // the modes need n positive eigenvalues (n at most the rank of the snapshots in z)
  std::vector<double> hl(K);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "rb_offline_pod kernels");
  e = cudaMemcpyAsync(hl.data(), lams, 8 * (size_t)K, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "eigenvalues");
  // an eigenvalue within rounding of zero (K eps of the largest) has no meaningful mode
  if (!(hl[n - 1] > (double)K * 2.220446049250313e-16 * hl[0]) || !std::isfinite(hl[0]))
    return set_error(ctx, RB_ERR_ARG, "rb_offline_pod: eigenvalue %d is %g (largest %g): n exceeds "
                     "the numerical rank of the snapshots", n, hl[n - 1], hl[0]);
  k_modes<<<std::max(1, std::min((N + 7) / 8, ctx->sms * 4)), 256, ms, ctx->stream>>>(N, K, n, ST, W,
                                                                                  lam, perm, VT);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "k_modes");
  if ((rc = transpose(ctx, N, n, VT, V)) != RB_OK) return rc;             // V [n][N]
  e = cudaMemcpyAsync(V_out, V, 8 * (size_t)n * N, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && lambda_out)
    e = cudaMemcpyAsync(lambda_out, lams, 8 * (size_t)K, cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_offline_pod download");
  return finish(ctx, "rb_offline_pod");
}

int rb_offline_project(rb_ctx *ctx, const double *V, int n, int N, const rb_csr *M, double *Mr_out) {
  if (!ctx) return RB_ERR_ARG;
  if (!V || !Mr_out || n < 1 || n > kGramMax || N < 1 || !csr_ok(M, N, N))
    return set_error(ctx, RB_ERR_ARG, "rb_offline_project: bad arguments (1 <= n <= %d, M N x N)",
                     kGramMax);
  cudaSetDevice(ctx->device);
  Buffers B(ctx);
  double *dV, *VT, *MV, *Mr, *mv;
  int *ip, *ix;
  int rc;
  if ((rc = B.get(&dV, (size_t)n * N, "modes")) != RB_OK) return rc;
  if ((rc = B.get(&VT, (size_t)n * N, "modes (transposed)")) != RB_OK) return rc;
  if ((rc = B.get(&MV, (size_t)n * N, "M V")) != RB_OK) return rc;
  if ((rc = B.get(&Mr, (size_t)n * n, "reduced matrix")) != RB_OK) return rc;
  if ((rc = upload_csr(ctx, B, M, &ip, &ix, &mv, "M")) != RB_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(dV, V, 8 * (size_t)n * N, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "modes upload");
  if ((rc = transpose(ctx, n, N, dV, VT)) != RB_OK) return rc;              // V^T [N][n]
  if ((rc = spmm(ctx, N, n, ip, ix, mv, VT, MV)) != RB_OK) return rc;       // M V [N][n]
  if ((rc = gram(ctx, B, N, n, n, VT, MV, Mr)) != RB_OK) return rc;         // V^T M V
  e = cudaMemcpyAsync(Mr_out, Mr, 8 * (size_t)n * n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_offline_project download");
  return finish(ctx, "rb_offline_project");
}

int rb_offline_project_vector(rb_ctx *ctx, const double *V, int n, int N, const double *f,
                              double *fr_out) {
  if (!ctx) return RB_ERR_ARG;
  if (!V || !f || !fr_out || n < 1 || n > kGramMax || N < 1)
    return set_error(ctx, RB_ERR_ARG, "rb_offline_project_vector: bad arguments");
  cudaSetDevice(ctx->device);
  Buffers B(ctx);
  double *dV, *VT, *df, *fr;
  int rc;
  if ((rc = B.get(&dV, (size_t)n * N, "modes")) != RB_OK) return rc;
  if ((rc = B.get(&VT, (size_t)n * N, "modes (transposed)")) != RB_OK) return rc;
  if ((rc = B.get(&df, (size_t)N, "f")) != RB_OK) return rc;
  if ((rc = B.get(&fr, (size_t)n, "reduced vector")) != RB_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(dV, V, 8 * (size_t)n * N, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(df, f, 8 * (size_t)N, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
  if ((rc = transpose(ctx, n, N, dV, VT)) != RB_OK) return rc;
  if ((rc = gram(ctx, B, N, n, 1, VT, df, fr)) != RB_OK) return rc;          // V^T f
  e = cudaMemcpyAsync(fr_out, fr, 8 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "download");
  return finish(ctx, "rb_offline_project_vector");
}

int rb_offline_tensor(rb_ctx *ctx, const double *V, int n, int N, const rb_trilinear_term *terms,
                      int n_terms, double *C_out) {
  if (!ctx) return RB_ERR_ARG;
  if (!V || !C_out || !terms || n_terms < 1 || n < 1 || n > RB_N_MAX || N < 1)
    return set_error(ctx, RB_ERR_ARG, "rb_offline_tensor: bad arguments (1 <= n <= %d)", RB_N_MAX);
  for (int t = 0; t < n_terms; ++t) {
    const int pts = terms[t].P.rows;
    if (!csr_ok(&terms[t].P, -1, N) || !csr_ok(&terms[t].Q, pts, N) || !csr_ok(&terms[t].R, pts, N))
      return set_error(ctx, RB_ERR_ARG, "rb_offline_tensor: term %d: P, Q, R must be points x N", t);
  }
  cudaSetDevice(ctx->device);
  Buffers B(ctx);
  double *dV, *VT, *part, *C;
  int rc;
  if ((rc = B.get(&dV, (size_t)n * N, "modes")) != RB_OK) return rc;
  if ((rc = B.get(&VT, (size_t)n * N, "modes (transposed)")) != RB_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(dV, V, 8 * (size_t)n * N, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "modes upload");
  if ((rc = transpose(ctx, n, N, dV, VT)) != RB_OK) return rc;
  // point chunks: partial tensors of at most about 1 GB in all
  const size_t n3 = (size_t)n * n * n;
  int max_pts = 0;
  for (int t = 0; t < n_terms; ++t) max_pts = std::max(max_pts, terms[t].P.rows);
  const int chunks = (int)std::max<size_t>(1, std::min<size_t>(16, ((size_t)1 << 27) / n3));
  if ((rc = B.get(&part, (size_t)chunks * n3, "tensor partial sums")) != RB_OK) return rc;
  if ((rc = B.get(&C, n3, "tensor")) != RB_OK) return rc;
  if ((e = cudaMemsetAsync(part, 0, 8 * (size_t)chunks * n3, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "memset");
  double *EP, *EQ, *ER, *w = nullptr;
  if ((rc = B.get(&EP, (size_t)std::max(max_pts, 1) * n, "P V")) != RB_OK) return rc;
  if ((rc = B.get(&EQ, (size_t)std::max(max_pts, 1) * n, "Q V")) != RB_OK) return rc;
  if ((rc = B.get(&ER, (size_t)std::max(max_pts, 1) * n, "R V")) != RB_OK) return rc;
  if ((rc = B.get(&w, (size_t)std::max(max_pts, 1), "weights")) != RB_OK) return rc;
  for (int t = 0; t < n_terms; ++t) {
    const rb_trilinear_term &T = terms[t];
    const int pts = T.P.rows;
    if (pts == 0) continue;
    Buffers Bt(ctx);  // this term's sparse operators
    int *ip[3], *ix[3];
    double *vv[3];
    const rb_csr *ops[3] = {&T.P, &T.Q, &T.R};
    double *outs[3] = {EP, EQ, ER};
    for (int a = 0; a < 3; ++a) {
      if ((rc = upload_csr(ctx, Bt, ops[a], &ip[a], &ix[a], &vv[a], "trilinear term")) != RB_OK) return rc;
      if ((rc = spmm(ctx, pts, n, ip[a], ix[a], vv[a], VT, outs[a])) != RB_OK) return rc;
    }
    if (T.weight) {
      e = cudaMemcpyAsync(w, T.weight, 8 * (size_t)pts, cudaMemcpyHostToDevice, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "weights upload");
      k_scale_rows<<<std::max(1, std::min(ctx->sms * 4, (pts * n + 255) / 256)), 256, 0, ctx->stream>>>(pts, n, w, EP);
    }
    const int kblocks = (n + kTriK - 1) / kTriK;
    const int chunk_pts = (pts + chunks - 1) / chunks;
    dim3 grid((n + kTriJ - 1) / kTriJ, (n + kTriJ - 1) / kTriJ, kblocks * chunks);
    const int mk = prof_begin(ctx, RB_K_OFFLINE_TENSOR, ctx->stream);
    k_triple<<<grid, 256, 0, ctx->stream>>>(pts, n, chunk_pts, EP, EQ, ER, part);
    prof_end(ctx, mk, ctx->stream);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "k_triple");
    // the term's buffers are freed after its kernels have run
    if ((rc = finish(ctx, "rb_offline_tensor term")) != RB_OK) return rc;
  }
  const int sgrid = (int)std::max<size_t>(1, std::min<size_t>((size_t)ctx->sms * 8, (n3 + 255) / 256));
  k_sum_parts<<<sgrid, 256, 0, ctx->stream>>>(n3, chunks, part, C);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "k_sum_parts");
  e = cudaMemcpyAsync(C_out, C, 8 * n3, cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_offline_tensor download");
  return finish(ctx, "rb_offline_tensor");
}

}  // extern "C"
