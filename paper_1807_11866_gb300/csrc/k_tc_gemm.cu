// k_tc_gemm.cu -- the tensor-Jacobian contraction of Sec. 3.6 as a dense GEMM on the tcgen05
// tensor cores, for a whole batch of queries.
//
// GEMM form: rows b = queries (M), columns c = (k, j) (N), reduction kappa (K):
//     T[b][c] = sum_kappa X[b][kappa] * W[c][kappa].
// Jacobian/residual: kappa = (q, l), X[b][(q,l)] = s theta^c_q(mu_b) u_b[l],
// W[(k,j)][(q,l)] = D~_q[k][j][l] = C_q[l][j][k] + C_q[j][l][k] (both index orders of Sec. 3.6
// summed once at load). With s = 1, T is the convection Jacobian J^c(u_b); with s = 1/2,
// sum_j T[b][(k,j)] u_b[j] = C_mu(u_b, u_b)[k] (Euler identity of the quadratic term).
// A second K segment kappa = q with X[b][q] = theta^a_q(mu_b), W[(k,j)][q] = A_q[k][j] adds
// A(mu)[k][j], so the contraction with u gives A(mu) u + C_mu(u, u) (Eq. velonly without f).
// The pressure right-hand side (Eq. sup-vvar) uses the same X with W = (2 Cs, As).
//
// Two epilogues:
//  * kPlain: X, W split into BF16 hi + lo parts, x_hi w_hi + x_hi w_lo + x_lo w_hi accumulated in
//    FP32 (about 16 significant bits); writes T (FP32) -> Jacobian for the LU.
//  * kSliced: error-free sliced product (after Ozaki, Ogita, Oishi and Rump, 2012). Per segment,
//    X rows and W are split into S balanced base-128 digit slices (|digit| <= 64) on fixed-point
//    grids (per-row exponent for X, one exponent for W): X = 2^ex sum_i x_i 2^-7i,
//    W = 2^ew sum_j w_j 2^-7j (S may differ per segment).
//    A product of two digits is at most 2^12, so up to 4096 of them add exactly in FP32. Pairs
//    (i, j) with i + j = L share the scale 2^(ex + ew - 7L); each level is accumulated in TMEM
//    in chunks of at most 4096 terms, every chunk is drained exactly and added, scaled by its
//    power of two, into per-column double-float sums held in registers; at the end of the tile
//    the sums are contracted with u_b[j] (double-float) and added into the FP64 output. Pairs
//    with i + j > S + 1 are dropped (relative truncation ~2^-7S of the fixed-point range).
//
// Roles (576 threads): warp 0 issues TMA loads into a STAGES-deep shared-memory ring, warp 1
// allocates TMEM and issues tcgen05.mma (one lane), warps 2-17 drain the two TMEM accumulator
// buffers (128 lanes = 128 query rows; four warps per lane quarter split the columns, so that
// a chunk drains in a quarter of the MMA time it took to fill).
// Persistent over output tiles, in groups of kGroupM row tiles (rows fastest inside a group).
// The sliced epilogue reads u_b[j] straight from L2 at the end of a tile, so all shared memory
// but the barriers goes to the TMA ring; the plain epilogue adds a small staging area for
// coalesced stores where the ring leaves room.
#include <cuda.h>

#include <algorithm>

#include "rb_mixed.cuh"
#include "tc_ptx.cuh"

namespace rb {

using namespace tc;

constexpr int kBM = 128, kBK = 64;
constexpr int kChunkSteps = 64;  // 64 k-blocks of 64 = 4096 exact terms per chunk (|digit| <= 64)
constexpr int kEpiWarps = 16;    // epilogue warps: kEpiParts per TMEM lane quarter
constexpr int kEpiParts = kEpiWarps / 4;  // column parts of a tile, one per warp of a quarter
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreadsTc = 64 + kEpiThreads;
constexpr int kGroupM = 8;  // row tiles per group of the tile order

// PAIR: the CTA holds half of the B tile (the pair's MMA reads the other half from the peer).
template <int BN, int STAGES, bool PAIR>
struct TcSmem {
  static constexpr int kTileA = kBM * kBK * 2;
  static constexpr int kTileB = (PAIR ? BN / 2 : BN) * kBK * 2;
  static constexpr int kStage = kTileA + kTileB;
  static constexpr int kBarOff = STAGES * kStage;
  static constexpr int kBytes = kBarOff + 256 + 1024;  // barriers + alignment slack
};

// The plain epilogue stages each warp's 16 x 32 blocks of T through shared memory (rows padded
// to 33 floats: conflict-free both ways), so that a global store writes 4 rows x 128 bytes
// instead of 32 rows x 16 bytes; only where it fits beside the ring (not with 7 stages of 32 KB,
// which then store from registers).
constexpr int kEpiStageBytes = kEpiWarps * 16 * 33 * 4;
constexpr int kMaxSmem = 232448;  // 227 KB per CTA
template <int MODE, int BN, int STAGES, bool PAIR>
struct TcLaunchSmem {
  static constexpr bool kStaged =
      MODE == kPlain && TcSmem<BN, STAGES, PAIR>::kBytes + kEpiStageBytes <= kMaxSmem;
  static constexpr int kBytes = TcSmem<BN, STAGES, PAIR>::kBytes + (kStaged ? kEpiStageBytes : 0);
};

// Output tile t -> (first row, first column). Tiles run in groups of group_m row tiles, rows
// fastest inside a group: the CTAs resident at one time share the operand tiles of a few row
// and column tiles, so both operands stream from L2 when neither fits in it.
// bm: rows of an output tile (128, or 256 for a CTA pair).
__device__ __forceinline__ void tile_origin(int t, const TcGemmParams &p, int bm, int bn, int &m0,
                                            int &n0) {
  const int G = p.group_m;
  const int per = G * p.n_tiles;
  const int g = t / per, r = t - g * per;
  const int gsz = min(G, p.m_tiles - g * G);
  m0 = (g * G + r % gsz) * bm;
  n0 = (r / gsz) * bn;
}

struct Level {
  int seg, kb_off, kb, L, ilo, npairs;
};

// The (segment, level) sequence every role walks through for one output tile.
__host__ __device__ __forceinline__ int num_levels(int mode, const TcGemmParams &p) {
  if (mode == kPlain) return 1;
  return (p.kb[0] > 0 ? p.S[0] : 0) + (p.kb[1] > 0 ? p.S[1] : 0);
}

__host__ __device__ __forceinline__ Level level_of(int mode, const TcGemmParams &p, int idx) {
  Level v;
  if (mode == kPlain) {  // products of the split operands, one accumulator
    v.seg = 0; v.kb_off = 0; v.kb = p.kb[0]; v.L = 0; v.ilo = 1; v.npairs = p.nsplit;
    return v;
  }
  const int n0 = p.kb[0] > 0 ? p.S[0] : 0;  // levels of segment 0
  v.seg = idx < n0 ? 0 : 1;
  const int S = p.S[v.seg];
  v.kb_off = v.seg == 0 ? 0 : p.kb[0];
  v.kb = p.kb[v.seg];
  v.L = (idx - (v.seg ? n0 : 0)) + 2;
  v.ilo = v.L - S > 1 ? v.L - S : 1;
  v.npairs = (S < v.L - 1 ? S : v.L - 1) - v.ilo + 1;
  return v;
}

// PAIR: clusters of two CTAs share each 256-row output tile through tcgen05 .cta_group::2
// (the leader, rank 0, issues the M = 256 MMAs; each CTA loads its 128 rows of X and half of
// the W tile into its own shared memory, signalling the leader's barriers, and drains its own
// TMEM). p.m_tiles then counts 256-row tiles.
// Level range [lo, hi) of part `part` of a tile split into `split` work units: contiguous
// levels, each in the part that holds the midpoint of its cost (pairs x K blocks), so the parts
// carry about equal work. Their contributions add up in the output (atomics).
__device__ __forceinline__ void level_range(int mode, const TcGemmParams &p, int n_levels, int part,
                                            int split, int &lo, int &hi) {
  if (split <= 1) {
    lo = 0;
    hi = n_levels;
    return;
  }
  int total = 0;
  for (int li = 0; li < n_levels; ++li) {
    const Level v = level_of(mode, p, li);
    total += v.npairs * v.kb;
  }
  lo = n_levels;
  hi = 0;
  int cum = 0;
  for (int li = 0; li < n_levels; ++li) {
    const Level v = level_of(mode, p, li);
    const int c = v.npairs * v.kb;
    const int owner = (int)(((long long)(2 * cum + c) * split) / (2LL * total));
    if (owner == part) {
      lo = min(lo, li);
      hi = max(hi, li + 1);
    }
    cum += c;
  }
  if (hi < lo) hi = lo;  // empty part
}

template <int MODE, int BN, int STAGES, bool PAIR>
__global__ void __launch_bounds__(kThreadsTc, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW,
              TcGemmParams p) {
  if (p.run_if && *(volatile const int *)p.run_if == 0) return;  // uniform over the grid
  extern __shared__ uint8_t smem_raw[];
  using SM = TcSmem<BN, STAGES, PAIR>;
  constexpr int kBMT = PAIR ? 2 * kBM : kBM;  // rows of an output tile
  constexpr int kBH = PAIR ? BN / 2 : BN;     // W rows this CTA loads per tile
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + SM::kBarOff);
  uint64_t *empty = full + STAGES;
  uint64_t *tfull = empty + STAGES;  // [2]
  uint64_t *tempty = tfull + 2;      // [2]
  uint64_t *mdone = tempty + 2;      // [1]
  uint32_t *tmem_slot = (uint32_t *)(mdone + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int n_levels = num_levels(MODE, p);
  if (MODE != kPlain && p.lmax && p.kb[1] == 0)  // a truncated launch: levels 2 .. *lmax
    n_levels = min(n_levels, max(1, *(volatile const int *)p.lmax - 1));
  const int chunk_steps = (MODE == kPlain) ? (1 << 30) : kChunkSteps;
  // work units: tiles [0, full) whole, the tail tiles split into lsplit level parts each
  const int num_tiles = p.m_tiles * p.n_tiles;
  const int lsplit = p.lsplit > 1 ? p.lsplit : 1;
  const int whole = lsplit > 1 ? p.full_tiles : num_tiles;
  const int num_units = whole + (num_tiles - whole) * lsplit;
  auto unit = [&](int t, int &tile, int &l0, int &l1) {
    if (t < whole) {
      tile = t;
      level_range(MODE, p, n_levels, 0, 1, l0, l1);
    } else {
      tile = whole + (t - whole) / lsplit;
      level_range(MODE, p, n_levels, (t - whole) % lsplit, lsplit, l0, l1);
    }
  };
  const uint32_t rank = PAIR ? cluster_rank() : 0u;  // 0: the pair's leader
  const int t_first = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int t_step = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], PAIR ? 2 * kEpiWarps : kEpiThreads);  // pair: one arrive per warp
    }
    mbar_init(mdone, 1);
    fence_barrier_init();
    fence_proxy_async();
  }
  // TMEM columns: [0, 2 BN) two accumulator buffers; sliced mode adds [2 BN, 4 BN) for the
  // per-column double-float sums (hi, lo) of each epilogue column part
  constexpr uint32_t kTmemCols = MODE == kSliced ? 4 * BN : 2 * BN;
  if (warp == 1) {
    if (PAIR) {
      tmem_alloc_pair(tmem_slot, kTmemCols);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(tmem_slot, kTmemCols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncwarp();
  if (PAIR) cluster_sync();  // barriers initialised and TMEM allocated in both CTAs
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      tma_prefetch_desc(&tmX);
      tma_prefetch_desc(&tmW);
      uint32_t step = 0;
      bool bad = false;
      for (int t = t_first; t < num_units && !bad; t += t_step) {
        int m0, n0, l0, l1, tile;
        unit(t, tile, l0, l1);
        tile_origin(tile, p, kBMT, BN, m0, n0);
        const int mr = m0 + (int)rank * kBM, nr = n0 + (int)rank * kBH;  // this CTA's part
        for (int li = l0; li < l1 && !bad; ++li) {
          const Level lv = level_of(MODE, p, li);
          const int nsteps = lv.npairs * lv.kb;
          for (int idx = 0; idx < nsteps; ++idx, ++step) {
            const int s = step % STAGES;
            const uint32_t ph = (step / STAGES) & 1;
            if (!mbar_wait(&empty[s], ph ^ 1, p.err, 1)) { bad = true; break; }
            uint8_t *sa = smem + s * SM::kStage;
            uint8_t *sb = sa + SM::kTileA;
            const int pr = idx / lv.kb, kk = lv.kb_off + idx % lv.kb;
            // plain split products: (x_hi, w_hi), (x_hi, w_lo), (x_lo, w_hi)
            const int xi = (MODE == kPlain) ? pr : (lv.ilo + pr - 1);
            const int wj = (MODE == kPlain) ? (pr == 1 ? 1 : 0) : (lv.L - (lv.ilo + pr) - 1);
            if (PAIR) {
              // both CTAs' loads complete on the leader's barrier, which expects all the bytes
              const uint32_t cbar = mapa_shared(smem_u32(&full[s]), 0);
              if (rank == 0) mbar_expect_tx(&full[s], 2 * SM::kStage);
              tma_load_2d_pair(sa, &tmX, cbar, kk * kBK, xi * p.b_pad + mr);
              tma_load_2d_pair(sb, &tmW, cbar, kk * kBK, wj * p.n_pad + nr);
            } else {
              mbar_expect_tx(&full[s], SM::kStage + ((step == 0 && blockIdx.x == 0) ? p.tx_extra : 0u));
              tma_load_2d(sa, &tmX, &full[s], kk * kBK, xi * p.b_pad + mr);
              tma_load_2d(sb, &tmW, &full[s], kk * kBK, wj * p.n_pad + nr);
            }
          }
        }
      }
      if (bad) {  // let loads already in flight land before the CTA exits
        if (PAIR) {  // they complete on the leader's barriers: give them a fixed grace time
          const uint64_t t0 = globaltimer();
          while (globaltimer() - t0 < 100000ull) {
          }
        } else {
          const uint32_t last = step;
          for (uint32_t st = (last > (uint32_t)STAGES ? last - STAGES : 0); st < last; ++st)
            mbar_wait(&full[st % STAGES], (st / STAGES) & 1, nullptr, 1);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && rank == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(kBMT, BN);
      uint32_t step = 0, chunk = 0;
      bool bad = false;
      for (int t = t_first; t < num_units && !bad; t += t_step) {
        int l0, l1, tile;
        unit(t, tile, l0, l1);
        for (int li = l0; li < l1 && !bad; ++li) {
          const Level lv = level_of(MODE, p, li);
          const int nsteps = lv.npairs * lv.kb;
          for (int c0 = 0; c0 < nsteps && !bad; c0 += chunk_steps, ++chunk) {
            const int buf = chunk & 1;
            const uint32_t tph = (chunk >> 1) & 1;
            if (!mbar_wait(&tempty[buf], tph ^ 1, p.err, 2)) { bad = true; break; }
            tc_fence_after();
            const uint32_t dt = tmem_base + buf * BN;
            const int c1 = min(nsteps, c0 + chunk_steps);
            for (int idx = c0; idx < c1; ++idx, ++step) {
              const int s = step % STAGES;
              const uint32_t ph = (step / STAGES) & 1;
              if (!mbar_wait(&full[s], ph, p.err, 3)) { bad = true; break; }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + s * SM::kStage);
              const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + SM::kTileA);
#pragma unroll
              for (int k4 = 0; k4 < kBK / 16; ++k4) {
                if (PAIR) mma_bf16_pair(dt, ad + 2 * k4, bd + 2 * k4, idesc, (idx > c0 || k4 > 0) ? 1u : 0u);
                else mma_bf16(dt, ad + 2 * k4, bd + 2 * k4, idesc, (idx > c0 || k4 > 0) ? 1u : 0u);
              }
              if (PAIR) mma_commit_pair(&empty[s]);  // frees the stage in both CTAs
              else mma_commit(&empty[s]);
            }
            if (PAIR) mma_commit_pair(&tfull[buf]);
            else mma_commit(&tfull[buf]);
          }
        }
      }
      // the tensor work this CTA (pair) issued: 2 kBMT BN kBK FLOPs per K step
      if (p.issued && step) atomicAdd(p.issued, (unsigned long long)step * (2ull * kBMT * BN * kBK));
      // all issued MMAs complete before TMEM is released (pair: in both CTAs)
      if (PAIR) mma_commit_pair(mdone);
      else mma_commit(mdone);
      mbar_wait(mdone, 0, nullptr, 4);
    } else if (PAIR && lane == 0) {
      mbar_wait(mdone, 0, nullptr, 4);  // the peer: the leader's last MMAs have completed
    }
  } else {
    // ---------------- epilogue (warps 2..17) ----------------
    const int q = warp & 3;                  // TMEM lane quarter of this warp
    const int half = (warp - 2) >> 2;        // which column part of the tile this warp drains
    const int row = q * 32 + lane;           // row of the tile owned by this thread
    constexpr int HC = BN / kEpiParts;       // columns per thread
    uint32_t chunk = 0;
    bool bad = false;
    for (int t = t_first; t < num_units && !bad; t += t_step) {
      int m0, n0, l0, l1, tile;
      unit(t, tile, l0, l1);
      tile_origin(tile, p, kBMT, BN, m0, n0);
      const int b = m0 + (int)rank * kBM + row;  // b < b_pad (a multiple of the tile rows)
      const int nj = p.nj, total = p.nk * p.nj;
      // wide sliced mode: the thread's HC <= 2 nj columns hold rows k_first .. k_first + 2
      const int c_begin = n0 + half * HC;
      const int k_first = c_begin / nj, j_first = c_begin - k_first * nj;
      float kah = 0.f, kal = 0.f, kbh = 0.f, kbl = 0.f, kch = 0.f, kcl = 0.f;
      // sliced mode: per-column double-float sums over all level chunks of this tile, in TMEM
      // columns [2 BN + half 2 HC, +HC) (hi) and [+HC, +2 HC) (lo) of this thread's lane
      const uint32_t tsum = tmem_base + ((uint32_t)(q * 32) << 16) + 2 * BN + half * 2 * HC;
      if (MODE == kSliced) {
        uint32_t z[16];
#pragma unroll
        for (int v = 0; v < 16; ++v) z[v] = 0u;
#pragma unroll
        for (int g = 0; g < 2 * HC / 16; ++g) tmem_st_x16(tsum + g * 16, z);
        tmem_st_wait();
      }
      for (int li = l0; li < l1 && !bad; ++li) {
        const Level lv = level_of(MODE, p, li);
        const int nsteps = lv.npairs * lv.kb;
        for (int c0 = 0; c0 < nsteps; c0 += chunk_steps, ++chunk) {
          const int buf = chunk & 1;
          const uint32_t tph = (chunk >> 1) & 1;
          // warp-uniform outcome: tcgen05.ld below is a warp-collective instruction
          const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], tph, p.err, 5));
          if (!ok) { bad = true; break; }
          tc_fence_after();
          const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + buf * BN + half * HC;
          if (MODE == kPlain && TcLaunchSmem<MODE, BN, STAGES, PAIR>::kStaged) {
            // columns past n_pad (a ragged last tile of a 256-column pair tile) are not stored;
            // cend is a multiple of 32 (n_pad and n0 are multiples of 128, HC of 32)
            const int cend = min(HC, p.n_pad - (n0 + half * HC));
            float *stg = reinterpret_cast<float *>(smem + SM::kBarOff + 256) + (warp - 2) * (16 * 33);
            // this warp's rows b - lane .. b - lane + 31 (within b_pad)
            float *out = p.Jc + (size_t)(b - lane) * p.ldj + n0 + half * HC;
#pragma unroll 1
            for (int c = 0; c < cend; c += 32) {
              uint32_t r[32];
              tmem_ld_x32(taddr + c, r);
              tmem_ld_wait();
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                if ((lane >> 4) == h) {
                  float *sr = stg + (lane & 15) * 33;
#pragma unroll
                  for (int v = 0; v < 32; ++v) sr[v] = __uint_as_float(r[v]);
                }
                __syncwarp();
                // lane l: row 4 i + l / 8 of the half, columns 4 (l % 8) .. + 3
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const int rr = 4 * i + (lane >> 3), cc = 4 * (lane & 7);
                  const float *sr = stg + rr * 33 + cc;
                  *reinterpret_cast<float4 *>(out + (size_t)(16 * h + rr) * p.ldj + c + cc) =
                      make_float4(sr[0], sr[1], sr[2], sr[3]);
                }
                __syncwarp();
              }
            }
          } else if (MODE == kPlain) {
            float *out = p.Jc + (size_t)b * p.ldj + n0 + half * HC;
            // columns past n_pad (a ragged last tile of a 256-column pair tile) are not stored
            const int cend = min(HC, p.n_pad - (n0 + half * HC));
#pragma unroll 1
            for (int c = 0; c < cend; c += 32) {
              uint32_t r[32];
              tmem_ld_x32(taddr + c, r);
              tmem_ld_wait();
              float4 *o4 = reinterpret_cast<float4 *>(out + c);
#pragma unroll
              for (int v = 0; v < 8; ++v)
                o4[v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                    __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
            }
          } else if (MODE == kSlicedWide) {
            // contract the exact chunk, scaled by its level (and segment) relative to segment 0,
            // with u_b[j] at once: three double-float row sums per thread (k_first + 0, 1, 2)
            const int d = (lv.seg ? (p.xexp[p.b_pad + b] + p.wexp[1] - p.xexp[b] - p.wexp[0]) : 0) -
                          kDigitBits * lv.L;
            const float sc = ldexpf(1.0f, d);
            const float2 *ub = p.ufT + b;  // u_b[j] at ub[j b_pad] (L2-resident)
#pragma unroll 1
            for (int g = 0; g < HC / 8; ++g) {
              float2 u2[8];
#pragma unroll
              for (int v = 0; v < 8; ++v) {
                int j = j_first + g * 8 + v;
                if (j >= nj) j -= nj;  // HC <= 2 nj: at most two wraps
                if (j >= nj) j -= nj;
                u2[v] = ub[(size_t)j * p.b_pad];
              }
              uint32_t r[8];
              tmem_ld_x8(taddr + g * 8, r);
              tmem_ld_wait();
#pragma unroll
              for (int v = 0; v < 8; ++v) {
                const int cl = g * 8 + v;
                if (c_begin + cl < total) {  // warp-uniform, as is the row below
                  const float x = __uint_as_float(r[v]) * sc;
                  const int js = j_first + cl;
                  if (js < nj) df_fma(kah, kal, x, 0.f, u2[v].x, u2[v].y);
                  else if (js < 2 * nj) df_fma(kbh, kbl, x, 0.f, u2[v].x, u2[v].y);
                  else df_fma(kch, kcl, x, 0.f, u2[v].x, u2[v].y);
                }
              }
            }
            float s, e;  // renormalise the sums once per chunk
            two_sum(kah, kal, s, e);
            kah = s;
            kal = e;
            two_sum(kbh, kbl, s, e);
            kbh = s;
            kbl = e;
            two_sum(kch, kcl, s, e);
            kch = s;
            kcl = e;
          } else {
            // add the exact chunk, scaled by its level (and segment) relative to segment 0, into
            // this thread's per-column double-float sums (exact power-of-two scaling)
            const int d = (lv.seg ? (p.xexp[p.b_pad + b] + p.wexp[1] - p.xexp[b] - p.wexp[0]) : 0) -
                          kDigitBits * lv.L;
            const float sc = ldexpf(1.0f, d);
#pragma unroll 1
            for (int g = 0; g < HC / 16; ++g) {
              uint32_t r[16], hi[16], lo[16];
              tmem_ld_x16(taddr + g * 16, r);
              tmem_ld_x16(tsum + g * 16, hi);
              tmem_ld_x16(tsum + HC + g * 16, lo);
              tmem_ld_wait();
#pragma unroll
              for (int v = 0; v < 16; ++v) {
                const float x = __uint_as_float(r[v]) * sc;
                float sh, e;
                two_sum(__uint_as_float(hi[v]), x, sh, e);
                hi[v] = __float_as_uint(sh);
                lo[v] = __float_as_uint(__uint_as_float(lo[v]) + e);
              }
              tmem_st_x16(tsum + g * 16, hi);
              tmem_st_x16(tsum + HC + g * 16, lo);
            }
            tmem_st_wait();
          }
          tc_fence_before();
          if (PAIR) {  // one arrival per warp on the leader's barrier
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(mapa_shared(smem_u32(&tempty[buf]), 0));
          } else {
            mbar_arrive(&tempty[buf]);
          }
        }
      }
      if (MODE == kSlicedWide && !bad && b < p.nq && c_begin < total) {
        // out[b][k] += 2^(ex + ew) sum_j T[(k,j)] u_j over this thread's columns
        const double scale = ldexp(1.0, p.xexp[b] + p.wexp[0]);
        atomicAdd(p.out + (size_t)b * p.nk + k_first, ((double)kah + (double)kal) * scale);
        const int cnt = min(HC, total - c_begin);
        if (j_first + cnt > nj)
          atomicAdd(p.out + (size_t)b * p.nk + k_first + 1, ((double)kbh + (double)kbl) * scale);
        if (j_first + cnt > 2 * nj)
          atomicAdd(p.out + (size_t)b * p.nk + k_first + 2, ((double)kch + (double)kcl) * scale);
      }
      if (MODE == kSliced && !bad) {
        // contract the tile's column sums with u_b[j]: out[b][k] += 2^(ex + ew) sum_j T[(k,j)] u_j
        // every lane executes the warp-collective TMEM loads; rows beyond the batch only skip the
        // arithmetic and the stores
        const bool live = b < p.nq;
        const double scale = live ? ldexp(1.0, p.xexp[b] + p.wexp[0]) : 0.0;
        int k = k_first, j = j_first;
        const int cend = min(HC, total - c_begin);
        const float2 *ub = p.ufT + b;  // u_b[j] at ub[j b_pad] (row b < b_pad: in bounds)
        float ah = 0.f, al = 0.f;
#pragma unroll 1
        for (int g = 0; g < HC / 16; ++g) {
          // u_b[j] of the group's columns: L2-resident, coalesced over the warp's rows
          float2 u2[16];
          int jj = j;
#pragma unroll
          for (int v = 0; v < 16; ++v) {
            u2[v] = ub[(size_t)jj * p.b_pad];
            if (++jj == nj) jj = 0;
          }
          uint32_t hi[16], lo[16];
          tmem_ld_x16(tsum + g * 16, hi);
          tmem_ld_x16(tsum + HC + g * 16, lo);
          tmem_ld_wait();
#pragma unroll
          for (int v = 0; v < 16; ++v) {
            if (g * 16 + v < cend) {
              df_fma(ah, al, __uint_as_float(hi[v]), __uint_as_float(lo[v]), u2[v].x, u2[v].y);
              if (++j == nj) {
                if (live) atomicAdd(p.out + (size_t)b * p.nk + k, ((double)ah + (double)al) * scale);
                ah = al = 0.f;
                j = 0;
                ++k;
              }
            }
          }
        }
        if (live && k < p.nk && cend > 0 && (ah != 0.f || al != 0.f))
          atomicAdd(p.out + (size_t)b * p.nk + k, ((double)ah + (double)al) * scale);
      }
    }
  }
  tc_fence_before();
  __syncwarp();
  if (PAIR) cluster_sync();  // no arrivals or MMAs target a CTA of the pair after this
  else __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    if (PAIR) tmem_dealloc_pair(tmem_base, kTmemCols);
    else tmem_dealloc(tmem_base, kTmemCols);
  }
}

// ---------------------------------------------------------------------------------------
// Tail split of a sliced GEMM: with `slots` work units resident at once, the tiles of the last,
// partly filled round are split into up to six level parts each (as many as the idle slots
// take), so that the round's work spreads over the whole GPU; the whole tiles before them run
// unsplit. Sets p.full_tiles and p.lsplit (1: no split).
static void choose_tail_split(int mode, TcGemmParams &p, int tiles, int slots) {
  p.lsplit = 1;
  p.full_tiles = tiles;
  if (mode == kPlain || slots < 1) return;
  const int tail = tiles % slots;
  if (tail == 0) return;
  const int s = std::min(std::min(6, num_levels(mode, p)), slots / tail);
  if (s < 2) return;
  p.lsplit = s;
  p.full_tiles = tiles - tail;
}

template <int MODE, int BN, int STAGES, bool PAIR>
static cudaError_t launch_impl(const CUtensorMap &tmX, const CUtensorMap &tmW,
                               const TcGemmParams &p0, int sms, cudaStream_t st) {
  const int smem = TcLaunchSmem<MODE, BN, STAGES, PAIR>::kBytes;
  auto kern = k_tc_gemm<MODE, BN, STAGES, PAIR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  TcGemmParams p = p0;
  const int tiles = p.m_tiles * p.n_tiles;
  if (!PAIR) {
    choose_tail_split(MODE, p, tiles, sms);
    const int units = p.full_tiles + (tiles - p.full_tiles) * p.lsplit;
    kern<<<std::min(units, sms), kThreadsTc, smem, st>>>(tmX, tmW, p);
    return cudaGetLastError();
  }
  // persistent clusters of two: no more than can be resident at once
  static int max_clusters = 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kThreadsTc);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (max_clusters == 0) {
    cfg.gridDim = dim3(2 * (sms / 2));
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    max_clusters = n;
  }
  choose_tail_split(MODE, p, tiles, max_clusters);
  const int units = p.full_tiles + (tiles - p.full_tiles) * p.lsplit;
  cfg.gridDim = dim3(2 * std::min(units, max_clusters));
  e = cudaLaunchKernelEx(&cfg, kern, tmX, tmW, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int MODE, int BN, bool PAIR>
static cudaError_t launch_stages(const CUtensorMap &tmX, const CUtensorMap &tmW,
                                 const TcGemmParams &p, int sms, cudaStream_t st, int stages) {
  if (stages == 4) return launch_impl<MODE, BN, 4, PAIR>(tmX, tmW, p, sms, st);
  if (stages == 7) return launch_impl<MODE, BN, 7, PAIR>(tmX, tmW, p, sms, st);
  return launch_impl<MODE, BN, 6, PAIR>(tmX, tmW, p, sms, st);
}

// stages: depth of the TMA ring, 4, 6 (default) or 7 (7 x 32 KB: the shared-memory limit of
// the single-CTA tiles). pair: CTA pairs on 256-row tiles; the plain mode then uses 256-column
// tiles (tmW with 128-row boxes), the sliced mode 128-column tiles (tmW with 64-row boxes). The
// batch stride b_pad must then be a multiple of 256.
cudaError_t launch_tc_gemm(int mode, const CUtensorMap &tmX, const CUtensorMap &tmW,
                           const TcGemmParams &p, int sms, cudaStream_t st, int stages, bool pair) {
  if (p.m_tiles < 1 || p.n_tiles < 1) return cudaErrorInvalidValue;
  TcGemmParams q = p;
  if (!pair) {
    if (mode == kSlicedWide) return cudaErrorInvalidValue;  // pairs only
    q.group_m = std::min(q.m_tiles, kGroupM);
    return mode == kPlain ? launch_stages<kPlain, kTcBN, false>(tmX, tmW, q, sms, st, stages)
                          : launch_stages<kSliced, kTcBN, false>(tmX, tmW, q, sms, st, stages);
  }
  if (p.b_pad % (2 * kBM) != 0) return cudaErrorInvalidValue;
  q.m_tiles = (p.m_tiles + 1) / 2;
  q.group_m = std::min(q.m_tiles, kGroupM / 2);
  if (mode == kPlain || mode == kSlicedWide) {
    if (mode == kSlicedWide && 2 * p.nj < 2 * kTcBN / kEpiParts) return cudaErrorInvalidValue;
    q.n_tiles = (p.n_pad + 2 * kTcBN - 1) / (2 * kTcBN);
    return mode == kPlain ? launch_stages<kPlain, 2 * kTcBN, true>(tmX, tmW, q, sms, st, stages)
                          : launch_stages<kSlicedWide, 2 * kTcBN, true>(tmX, tmW, q, sms, st, stages);
  }
  return launch_stages<kSliced, kTcBN, true>(tmX, tmW, q, sms, st, stages);
}

}  // namespace rb
