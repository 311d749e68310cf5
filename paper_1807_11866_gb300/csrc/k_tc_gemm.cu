// k_tc_gemm.cu -- the tensor-Jacobian contraction of Sec. 3.6 as a dense GEMM on the tcgen05
// tensor cores, for a whole batch of queries.
//
// GEMM form: rows b = queries (M), columns c = (k, j) of the n_b x n_b Jacobian (N),
// reduction kappa = (q, l) (K):
//     T[b][c] = sum_kappa X[b][kappa] * W[c][kappa],
//     X[b][(q,l)] = s * theta^c_q(mu_b) u_b[l],   W[(k,j)][(q,l)] = D~_q[k][j][l]
// with D~_q[k][j][l] = C_q[l][j][k] + C_q[j][l][k] (both index orders of Sec. 3.6 summed once at
// load). With s = 1, T is the convection Jacobian J^c(u_b); with s = 1/2, sum_j T[b][(k,j)] u_b[j]
// is the convection term C_mu(u_b, u_b)[k] (Euler identity of a quadratic form).
//
// Two epilogues:
//  * kPlain: X, W rounded to BF16, FP32 accumulation; writes T (FP32) -> Jacobian for the LU.
//  * kSliced: error-free sliced product (after Ozaki et al., 2012) for the FP64-accurate
//    residual. X rows and W are split into S signed 7-bit digit slices on fixed-point grids
//    (per-row exponent for X, one exponent for W): X = 2^ex sum_i x_i 2^-7i, W = 2^ew sum_j w_j 2^-7j.
//    Products of two digits are below 2^14, so up to 1024 of them add exactly in an FP32
//    accumulator. Pairs (i, j) with i + j = L share the scale 2^(ex + ew - 7L); the kernel
//    accumulates each level in TMEM chunks of at most 1024 terms, drains every chunk exactly,
//    contracts it with u_b[j] in double-float arithmetic, and adds the level-scaled result into
//    the FP64 output R^c[b][k]. Pairs with i + j > S + 1 are dropped (truncation 2^-7S relative).
//
// Roles (192 threads): warp 0 issues TMA loads into a STAGES-deep shared-memory ring, warp 1
// allocates TMEM and issues tcgen05.mma (one elected lane), warps 2-5 drain the two TMEM
// accumulator buffers (128 lanes = 128 query rows). Persistent over output tiles.
#include <cuda.h>

#include "rb_mixed.cuh"
#include "tc_ptx.cuh"

namespace rb {

using namespace tc;

constexpr int kBM = 128, kBK = 64;
constexpr int kStages = 4;
constexpr int kChunkSteps = 16;  // 16 k-blocks of 64 = 1024 exact terms per chunk (7-bit digits)

template <int BN>
struct TcSmem {
  static constexpr int kTileA = kBM * kBK * 2;
  static constexpr int kTileB = BN * kBK * 2;
  static constexpr int kStage = kTileA + kTileB;
  static constexpr int kBarOff = kStages * kStage;
  static constexpr int kBytes = kBarOff + 256 + 1024;  // barriers + alignment slack
};

struct Level {
  int L, ilo, npairs;
};

__device__ __forceinline__ Level level_of(int mode, int S, int li) {
  Level v;
  if (mode == kPlain) {
    v.L = 0; v.ilo = 1; v.npairs = 1;
  } else {
    v.L = li + 2;
    v.ilo = max(1, v.L - S);
    v.npairs = min(S, v.L - 1) - v.ilo + 1;
  }
  return v;
}

template <int MODE, int BN>
__global__ void __launch_bounds__(192, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW,
              TcGemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  using SM = TcSmem<BN>;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + SM::kBarOff);
  uint64_t *empty = full + kStages;
  uint64_t *tfull = empty + kStages;   // [2]
  uint64_t *tempty = tfull + 2;        // [2]
  uint64_t *mdone = tempty + 2;        // [1]
  uint32_t *tmem_slot = (uint32_t *)(mdone + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_levels = (MODE == kPlain) ? 1 : p.S;
  const int chunk_steps = (MODE == kPlain) ? (1 << 30) : kChunkSteps;
  const int num_tiles = p.m_tiles * p.n_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(mdone, 1);
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 2 * BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      tma_prefetch_desc(&tmX);
      tma_prefetch_desc(&tmW);
      uint32_t step = 0;
      bool bad = false;
      for (int t = blockIdx.x; t < num_tiles && !bad; t += gridDim.x) {
        const int m0 = (t % p.m_tiles) * kBM, n0 = (t / p.m_tiles) * BN;
        for (int li = 0; li < n_levels && !bad; ++li) {
          const Level lv = level_of(MODE, p.S, li);
          const int nsteps = lv.npairs * p.kb;
          for (int idx = 0; idx < nsteps; ++idx, ++step) {
            const int s = step % kStages;
            const uint32_t ph = (step / kStages) & 1;
            if (!mbar_wait(&empty[s], ph ^ 1, p.err, 1)) { bad = true; break; }
            uint8_t *sa = smem + s * SM::kStage;
            uint8_t *sb = sa + SM::kTileA;
            const int pr = idx / p.kb, kk = idx % p.kb;
            const int xi = (MODE == kPlain) ? 0 : (lv.ilo + pr - 1);
            const int wj = (MODE == kPlain) ? 0 : (lv.L - (lv.ilo + pr) - 1);
            mbar_expect_tx(&full[s], SM::kStage);
            tma_load_2d(sa, &tmX, &full[s], kk * kBK, xi * p.b_pad + m0);
            tma_load_2d(sb, &tmW, &full[s], kk * kBK, wj * p.n_pad + n0);
          }
        }
      }
      if (bad) {  // let loads already in flight land before the CTA exits
        const uint32_t last = step;
        for (uint32_t st = (last > (uint32_t)kStages ? last - kStages : 0); st < last; ++st) {
          mbar_wait(&full[st % kStages], (st / kStages) & 1, nullptr, 1);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(kBM, BN);
      uint32_t step = 0, chunk = 0;
      bool bad = false;
      for (int t = blockIdx.x; t < num_tiles && !bad; t += gridDim.x) {
        for (int li = 0; li < n_levels && !bad; ++li) {
          const Level lv = level_of(MODE, p.S, li);
          const int nsteps = lv.npairs * p.kb;
          for (int c0 = 0; c0 < nsteps && !bad; c0 += chunk_steps, ++chunk) {
            const int buf = chunk & 1;
            const uint32_t tph = (chunk >> 1) & 1;
            if (!mbar_wait(&tempty[buf], tph ^ 1, p.err, 2)) { bad = true; break; }
            tc_fence_after();
            const uint32_t dt = tmem_base + buf * BN;
            const int c1 = min(nsteps, c0 + chunk_steps);
            for (int idx = c0; idx < c1; ++idx, ++step) {
              const int s = step % kStages;
              const uint32_t ph = (step / kStages) & 1;
              if (!mbar_wait(&full[s], ph, p.err, 3)) { bad = true; break; }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + s * SM::kStage);
              const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + SM::kTileA);
#pragma unroll
              for (int k4 = 0; k4 < kBK / 16; ++k4)
                mma_bf16(dt, ad + 2 * k4, bd + 2 * k4, idesc, (idx > c0 || k4 > 0) ? 1u : 0u);
              mma_commit(&empty[s]);
            }
            mma_commit(&tfull[buf]);
          }
        }
      }
      // all issued MMAs complete before TMEM is released
      mma_commit(mdone);
      mbar_wait(mdone, 0, nullptr, 4);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;              // TMEM lane quarter of this warp
    const int row = q * 32 + lane;       // row of the tile
    uint32_t chunk = 0;
    bool bad = false;
    for (int t = blockIdx.x; t < num_tiles && !bad; t += gridDim.x) {
      const int m0 = (t % p.m_tiles) * kBM, n0 = (t / p.m_tiles) * BN;
      const int b = m0 + row;
      for (int li = 0; li < n_levels && !bad; ++li) {
        const Level lv = level_of(MODE, p.S, li);
        const int nsteps = lv.npairs * p.kb;
        for (int c0 = 0; c0 < nsteps; c0 += chunk_steps, ++chunk) {
          const int buf = chunk & 1;
          const uint32_t tph = (chunk >> 1) & 1;
          // warp-uniform outcome: tcgen05.ld below is a warp-collective instruction
          const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], tph, p.err, 5));
          if (!ok) { bad = true; break; }
          tc_fence_after();
          const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + buf * BN;
          if (MODE == kPlain) {
            float *out = p.Jc + (size_t)b * p.ldj + n0;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
              uint32_t r[32];
              tmem_ld_x32(taddr + c, r);
              tmem_ld_wait();
              float4 *o4 = reinterpret_cast<float4 *>(out + c);
#pragma unroll
              for (int v = 0; v < 8; ++v)
                o4[v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                    __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
            }
          } else {
            // contract the exact chunk with u_b[j] over the tile's columns (k, j)
            const bool live = b < p.nq;
            const int nb = p.nb, nn = nb * nb;
            const double scale = live ? ldexp(1.0, p.xexp[b] + p.wexp - 7 * lv.L) : 0.0;
            const float2 *ub = p.uf + (size_t)b * nb;
            int g = n0, k = n0 / nb, j = n0 - (n0 / nb) * nb;
            float ah = 0.f, al = 0.f;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
              uint32_t r[32];
              tmem_ld_x32(taddr + c, r);
              tmem_ld_wait();
              if (live) {
#pragma unroll
                for (int v = 0; v < 32; ++v, ++g) {
                  if (g < nn) {
                    const float x = __uint_as_float(r[v]);
                    const float2 u2 = ub[j];
                    // x * (uh + ul) as p + e + x*ul, p = fl(x*uh) and e its exact error
                    const float pp = x * u2.x;
                    const float e = fmaf(x, u2.x, -pp);
                    const float tl = fmaf(x, u2.y, e);
                    // two-sum (ah, pp)
                    const float s = ah + pp;
                    const float bb = s - ah;
                    const float er = (ah - (s - bb)) + (pp - bb);
                    ah = s;
                    al += er + tl;
                    if (++j == nb) {
                      atomicAdd(p.Rc + (size_t)b * nb + k, ((double)ah + (double)al) * scale);
                      ah = al = 0.f;
                      j = 0;
                      ++k;
                    }
                  }
                }
              }
            }
            if (live && (ah != 0.f || al != 0.f) && k < nb)
              atomicAdd(p.Rc + (size_t)b * nb + k, ((double)ah + (double)al) * scale);
          }
          tc_fence_before();
          mbar_arrive(&tempty[buf]);
        }
        if (bad) break;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem_base, 2 * BN);
  }
}

// ---------------------------------------------------------------------------------------
template <int MODE, int BN>
static cudaError_t launch_impl(const CUtensorMap &tmX, const CUtensorMap &tmW,
                               const TcGemmParams &p, int grid, cudaStream_t st) {
  const int smem = TcSmem<BN>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<MODE, BN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_tc_gemm<MODE, BN><<<grid, 192, smem, st>>>(tmX, tmW, p);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(int mode, const CUtensorMap &tmX, const CUtensorMap &tmW,
                           const TcGemmParams &p, int sms, cudaStream_t st) {
  const int tiles = p.m_tiles * p.n_tiles;
  const int grid = tiles < sms ? tiles : sms;
  if (mode == kPlain) return launch_impl<kPlain, kTcBN>(tmX, tmW, p, grid, st);
  return launch_impl<kSliced, kTcBN>(tmX, tmW, p, grid, st);
}

}  // namespace rb
