// k_leaf_tc.cu -- exact leaf products of Algorithm 1 on the 5th-generation
// tensor cores (tcgen05, sm_103a).
//
// A leaf product R = X Y^T mod p (X: M x K, Y: N x K balanced residues) is
// computed from signed base-2^b digit planes, X = sum_i 2^(b i) X_i, as
//
//     R = sum_{i,j} 2^(b (i + j)) X_i Y_j^T  mod p.
//
// Every digit is an integer of at most 9 bits, exact in BF16, and every
// product of two digits is exact in FP32.  The tensor core accumulates in
// FP32 in tensor memory (TMEM); a chunk of the K loop is cut short whenever
// the partial sums could leave [-2^exact_bits, 2^exact_bits] (exact_bits <=
// 24 keeps every integer representable), and the chunk's exact integer
// result is drained by the epilogue warps into int32 registers.  Digit pairs
// are processed in decreasing weight; between pairs the int32 accumulator is
// multiplied by 2^(b * gap) and reduced mod p (Horner), so one balanced int32
// per output entry carries the whole sum (delayed Barrett reduction).
//
// Kernel organisation (one CTA per SM, persistent over a tile list):
//   warp 0        TMA producer: 128x64 tile of X_i and 256x64 tile of Y_j per
//                 stage into 128B-swizzled shared memory (4 stages); in the
//                 CTA-pair form 128x64 of each per CTA (6 stages)
//   warp 1        TMEM allocator + tcgen05.mma issuer: the warp runs the
//                 K loop in uniform control flow and the lane chosen by
//                 elect.sync issues each MMA and commit (a loop run by one
//                 divergent lane could not issue as fast as the MMAs ran);
//                 M=128 N=256 K=16 per instruction (CTA pair: M=256 across
//                 the pair, issued by the leader), FP32 accumulator in one of
//                 two 256-column TMEM buffers (double buffered per chunk)
//   warps 2..9    epilogue: tcgen05.ld of the finished chunk, float -> int32,
//                 accumulate; mod-p Horner step at digit-pair boundaries;
//                 canonical store (lower triangle only for SYRK leaves)
// The tile list is taken round robin by the persistent CTAs (or CTA pairs).
// One launch computes one product (kSingle), a batch of products of
// different moduli with tables in global memory (kBatch), or up to
// MAX_MULTI independent products of one modulus with their tensor maps in
// the kernel parameters (kMulti).
// Every mbarrier wait is bounded (kTimeoutNs): on expiry the CTA sets the
// device status word to AAT_ETIMEOUT, stops issuing work, waits (bounded) for
// its copies and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace aat {

namespace {

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = 256;
constexpr int MAX_GROUPS = 160;

struct Group {
  int16_t xp, yp;   // digit planes of X and Y
  int32_t kb0, kb1; // k-block range [kb0, kb1) (units of BK)
  int32_t kchunk;   // k-blocks per FP32 accumulation chunk
  uint32_t ratio;   // accumulator multiplier (mod p) applied before the group
  uint32_t ratio_sh;  // floor(ratio 2^32 / p), Shoup's precomputed quotient
};


// One problem of a batched launch; its tensor maps live in global memory.
struct alignas(64) BatchProb {
  CUtensorMap tmx, tmy;
  int32_t *out;
  int64_t ldo, M, N;
  int goff, ng;  // its groups: gtab[goff .. goff + ng)
  int lower, accumulate;  // accumulate: out <- product + beta out
  uint32_t beta, beta_sh;
  ModP m;
};

// One problem of a multi-problem launch (up to MAX_MULTI independent
// products that share one digit spec and modulus); its tensor maps live in
// the kernel parameters like the single-problem maps.
constexpr int MAX_MULTI = 16;
struct alignas(64) MultiProb {
  CUtensorMap tmx, tmy;
  int32_t *out;
  int64_t ldo, M, N;
  int goff, ng;  // its groups: Params::g[goff .. goff + ng)
  int lower, accumulate;
  uint32_t beta, beta_sh;
};

// Launch modes of the kernel: one problem (maps and groups in the
// parameters), a batch (per-problem maps and groups in global memory, many
// moduli), several problems of one modulus (maps and groups in the
// parameters, tile entries (problem, I, J) in global memory).
constexpr int kSingle = 0, kBatch = 1, kMulti = 2;

struct Params {
  CUtensorMap tmx;  // 3D {K, rows, plane}, box {64, 128, 1}
  CUtensorMap tmy;  // 3D {K, rows, plane}, box {64, 256, 1} (CTA pair: {64, 128, 1})
  Group g[MAX_GROUPS];
  int ng;
  int32_t *out;
  int64_t ldo, M, N;
  const int2 *tiles;
  int ntiles;
  int lower, accumulate;  // accumulate: out <- product + beta out
  uint32_t beta, beta_sh;
  ModP m;
  int32_t *status;
  // batched launches: tiles are (problem, I, J) and every problem carries
  // its own maps, groups and output
  const BatchProb *probs;
  const int4 *btiles;
  const Group *gtab;
  // multi-problem launches: tile entries (problem, I, J, 0)
  const int4 *mtiles;
  MultiProb mp[MAX_MULTI];
};

// Batched tile entries are (problem, I, J, goff | ng << 16): the tile's
// group table is one hop away instead of two.
__device__ __forceinline__ int tile_goff(int w) { return w & 0xFFFF; }
__device__ __forceinline__ int tile_ngrp(int w) { return w >> 16; }

// What one tile of the launch reads.
struct TileView {
  const CUtensorMap *tmx, *tmy;
  const Group *g;
  int ng, I, J;
};

template <int MODE>
__device__ __forceinline__ TileView tile_view(const Params &P, int t) {
  TileView v;
  if constexpr (MODE == kBatch) {
    const int4 tl = P.btiles[t];
    const BatchProb &b = P.probs[tl.x];
    v.tmx = &b.tmx;
    v.tmy = &b.tmy;
    v.g = P.gtab + tile_goff(tl.w);
    v.ng = tile_ngrp(tl.w);
    v.I = tl.y;
    v.J = tl.z;
  } else if constexpr (MODE == kMulti) {
    const int4 tl = P.mtiles[t];
    const MultiProb &b = P.mp[tl.x];
    v.tmx = &b.tmx;
    v.tmy = &b.tmy;
    v.g = P.g + b.goff;
    v.ng = b.ng;
    v.I = tl.y;
    v.J = tl.z;
  } else {
    const int2 tl = P.tiles[t];
    v.tmx = &P.tmx;
    v.tmy = &P.tmy;
    v.g = P.g;
    v.ng = P.ng;
    v.I = tl.x;
    v.J = tl.y;
  }
  return v;
}

// Group gi of tile t, and the group count (parameter loads when not batched).
template <int MODE>
__device__ __forceinline__ Group tile_group(const Params &P, int t, int gi) {
  if constexpr (MODE == kBatch) {
    return P.gtab[tile_goff(P.btiles[t].w) + gi];
  } else if constexpr (MODE == kMulti) {
    return P.g[P.mp[P.mtiles[t].x].goff + gi];
  } else {
    return P.g[gi];
  }
}

template <int MODE>
__device__ __forceinline__ int tile_ng(const Params &P, int t) {
  if constexpr (MODE == kBatch) {
    return tile_ngrp(P.btiles[t].w);
  } else if constexpr (MODE == kMulti) {
    return P.mp[P.mtiles[t].x].ng;
  } else {
    return P.ng;
  }
}

template <int MODE>
__device__ __forceinline__ int2 tile_ij(const Params &P, int t) {
  if constexpr (MODE == kBatch) {
    const int4 tl = P.btiles[t];
    return make_int2(tl.y, tl.z);
  } else if constexpr (MODE == kMulti) {
    const int4 tl = P.mtiles[t];
    return make_int2(tl.y, tl.z);
  } else {
    return P.tiles[t];
  }
}

template <int MODE>
__device__ __forceinline__ const ModP &tile_modp(const Params &P, int t) {
  if constexpr (MODE == kBatch) {
    return P.probs[P.btiles[t].x].m;
  } else {
    return P.m;
  }
}

// Where one tile writes.
struct OutView {
  int32_t *out;
  int64_t ldo, M, N;
  int lower, accumulate;
  uint32_t beta, beta_sh;
};

template <class B>
__device__ __forceinline__ OutView out_view(const B &b) {
  OutView o;
  o.out = b.out;
  o.ldo = b.ldo;
  o.M = b.M;
  o.N = b.N;
  o.lower = b.lower;
  o.accumulate = b.accumulate;
  o.beta = b.beta;
  o.beta_sh = b.beta_sh;
  return o;
}

template <int MODE>
__device__ __forceinline__ OutView tile_out(const Params &P, int t) {
  if constexpr (MODE == kBatch) {
    return out_view(P.probs[P.btiles[t].x]);
  } else if constexpr (MODE == kMulti) {
    return out_view(P.mp[P.mtiles[t].x]);
  } else {
    return out_view(P);
  }
}

// ------------------------------------------------------------------ kernel

// Two forms of the kernel share the code below.
//   one CTA  (PAIR = false): a 128 x 256 output tile per CTA; each stage holds
//            128 rows of X and 256 rows of Y (48 KB), 4 stages.
//   CTA pair (PAIR = true):  a 256 x 256 output tile per cluster of 2 CTAs,
//            tcgen05 cta_group::2: each CTA holds 128 rows of X and 128 rows
//            of Y per stage (32 KB), so 6 stages fit and the copies in
//            flight cover more of the DRAM latency; the leader CTA (rank 0)
//            issues M=256 N=256 MMAs that read both CTAs' shared memory and
//            write 128 TMEM lanes in each CTA.
//   EW: epilogue warps, 8 or 16.  Each owns 32 TMEM lanes (its warp index
//   mod 4 picks them) and 1024 / EW of the 256 columns, so it holds 128 or
//   64 int32 accumulators per thread.  16 warps run the drains, Horner steps
//   and stores of a tile with twice the threads (the epilogue's per-entry
//   work is latency-bound at 2 warps per scheduler: the 128 live
//   accumulators leave few registers for independent temporaries); the
//   price is 96 registers per thread (and some spills).
template <bool PAIR, int EW = 8>
struct Shape {
  static constexpr int EPI_WARPS = EW;
  static constexpr int THREADS = 64 + EW * 32;
  static constexpr int VALS = 1024 / EW;          // accumulators per thread
  static constexpr int XB = EW == 8 ? 16 : 8;     // staged store block width
  static constexpr int TM = PAIR ? 256 : 128;     // output tile rows
  static constexpr int YROWS = PAIR ? 128 : 256;  // rows of Y per CTA and stage
  static constexpr int STAGES = PAIR ? 6 : 4;
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = YROWS * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  // + 256 bytes of barriers + a per-warp cache of the tile's groups
  // (batched launches: 32 groups per epilogue warp) + a per-warp
  // 32 x (XB + 1) int32 staging area of the output stores
  static constexpr size_t GCACHE_BYTES = (size_t)EW * 32 * sizeof(Group);
  static constexpr size_t XS_BYTES = (size_t)EW * 32 * (XB + 1) * 4;
  static constexpr size_t SMEM =
      1024 + (size_t)STAGES * STAGE_BYTES + 256 + GCACHE_BYTES + XS_BYTES;
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
  // Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator
  // (bit 4), A and B BF16 (bits 7, 10), both K-major, N >> 3 at bit 17,
  // M >> 4 at bit 24.
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
};

// Epilogue warps of the single-problem launches and of the batched launch
// (whose tiles are mostly short in K, so the per-tile epilogue dominates).
constexpr int kEwLeaf = 8, kEwBatch = 16;

template <int MODE, bool PAIR, int EW>
__global__ void __launch_bounds__(Shape<PAIR, EW>::THREADS, 1)
    leaf_tc_kernel(const __grid_constant__ Params P) {
  using S = Shape<PAIR, EW>;
  constexpr int EPI_WARPS = S::EPI_WARPS, VALS = S::VALS, XB = S::XB;
  constexpr int STAGES = S::STAGES;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment of the shared-window address (128B-swizzle atoms);
  // the same offset in both CTAs of a pair, as the pair MMA requires
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t *bars = (uint64_t *)(smem + (size_t)STAGES * S::STAGE_BYTES);
  const uint32_t bar0 = smem_u32(bars);
#define FULL(s) (bar0 + 8u * (uint32_t)(s))
#define EMPTY(s) (bar0 + 8u * (uint32_t)(STAGES + (s)))
#define AFULL(b) (bar0 + 8u * (uint32_t)(2 * STAGES + (b)))
#define AEMPTY(b) (bar0 + 8u * (uint32_t)(2 * STAGES + 2 + (b)))
#define DONE (bar0 + 8u * (uint32_t)(2 * STAGES + 4))
  uint32_t *tmem_slot = (uint32_t *)(bars + 2 * STAGES + 5);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  // work units: tiles are taken round robin by CTAs (one CTA) or clusters
  uint32_t rank = 0, unit0 = blockIdx.x, nunits = gridDim.x;
  if constexpr (PAIR) {
    rank = cluster_ctarank();
    unit0 = cluster_id_x();
    nunits = ncluster_x();
  }
  const bool leader = (rank == 0);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(FULL(s), 1);
      mbar_init(EMPTY(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(AFULL(b), 1);
      mbar_init(AEMPTY(b), PAIR ? 2 * EPI_WARPS : EPI_WARPS);
    }
    mbar_init(DONE, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
  }
  __syncthreads();
  // the peer's barriers must be initialised before any copy or arrival
  // reaches them
  if constexpr (PAIR) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      int stage = 0;
      uint32_t ph = 0;
      int issued = 0;
      bool ok = true;
      // both CTAs' copies of a stage complete on the leader's FULL barrier
      const uint32_t full0 = PAIR ? map_to_rank(FULL(0), 0) : FULL(0);
      for (int t = (int)unit0; t < P.ntiles && ok; t += (int)nunits) {
        const TileView v = tile_view<MODE>(P, t);
        const int rowx = v.I * S::TM + (int)rank * BM;
        const int rowy = v.J * BN + (int)rank * S::YROWS;
        for (int gi = 0; gi < v.ng && ok; ++gi) {
          const Group g = v.g[gi];
          for (int kb = g.kb0; kb < g.kb1; ++kb) {
            if (!wait_bounded<PAIR>(EMPTY(stage), ph ^ 1u, abort_flag, P.status)) {
              ok = false;
              break;
            }
            const uint32_t sa = sbase + (uint32_t)(stage * S::STAGE_BYTES);
            const uint32_t fb = full0 + 8u * (uint32_t)stage;
            if constexpr (PAIR) {
              if (leader) mbar_expect_tx(FULL(stage), (uint32_t)(2 * S::STAGE_BYTES));
              tma_load_3d_pair(sa, v.tmx, fb, kb * BK, rowx, g.xp);
              tma_load_3d_pair(sa + S::A_BYTES, v.tmy, fb, kb * BK, rowy, g.yp);
            } else {
              mbar_expect_tx(FULL(stage), (uint32_t)S::STAGE_BYTES);
              tma_load_3d(sa, v.tmx, fb, kb * BK, rowx, g.xp);
              tma_load_3d(sa + S::A_BYTES, v.tmy, fb, kb * BK, rowy, g.yp);
            }
            ++issued;
            if (++stage == STAGES) {
              stage = 0;
              ph ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        // let the copies in flight land before the CTA exits
        if (!PAIR || leader) {
          int s = stage;
          uint32_t q = ph;
          for (int i = 0; i < STAGES && i < issued; ++i) {
            if (--s < 0) {
              s = STAGES - 1;
              q ^= 1u;
            }
            wait_quiet(FULL(s), q);
          }
        } else {
          // the peer's copies complete on the leader's barriers: give them
          // a fixed 20 ms to land
          const unsigned long long t0 = gtimer();
          while (gtimer() - t0 < 20000000ull) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    // the whole warp runs the loop in uniform control flow (its state stays
    // in uniform registers); one elected lane issues the MMAs and commits
    if (leader) {
      int stage = 0;
      uint32_t ph = 0, chunk = 0;
      bool ok = true;
      for (int t = (int)unit0; t < P.ntiles && ok; t += (int)nunits) {
        const int ng = tile_ng<MODE>(P, t);
        for (int gi = 0; gi < ng && ok; ++gi) {
          const Group g = tile_group<MODE>(P, t, gi);
          for (int kb = g.kb0; kb < g.kb1 && ok;) {
            const int kend = min(kb + g.kchunk, g.kb1);
            const uint32_t buf = chunk & 1u, use = chunk >> 1;
            if (!__all_sync(0xffffffffu, wait_bounded<PAIR>(AEMPTY(buf), (use & 1u) ^ 1u, abort_flag,
                                                            P.status))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dt = tmem + buf * ACC_COLS;
            for (int k = kb; k < kend; ++k) {
              if (!__all_sync(0xffffffffu, wait_bounded<PAIR>(FULL(stage), ph, abort_flag, P.status))) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = sbase + (uint32_t)(stage * S::STAGE_BYTES);
              const uint32_t sb = sa + S::A_BYTES;
              if (elect_one()) {
#pragma unroll
                for (int s = 0; s < BK / 16; ++s) {
                  const uint32_t acc = (k > kb || s > 0) ? 1u : 0u;
                  if constexpr (PAIR)
                    tc_mma_pair(dt, sw128_desc(sa + 32u * s), sw128_desc(sb + 32u * s), S::IDESC, acc);
                  else
                    tc_mma(dt, sw128_desc(sa + 32u * s), sw128_desc(sb + 32u * s), S::IDESC, acc);
                }
                if constexpr (PAIR)
                  tc_commit_pair(EMPTY(stage), 3);
                else
                  tc_commit(EMPTY(stage));
              }
              __syncwarp();
              if (++stage == STAGES) {
                stage = 0;
                ph ^= 1u;
              }
            }
            if (!ok) break;
            if (elect_one()) {
              if constexpr (PAIR)
                tc_commit_pair(AFULL(buf), 3);
              else
                tc_commit(AFULL(buf));
            }
            __syncwarp();
            ++chunk;
            kb = kend;
          }
        }
      }
      if (!ok && elect_one()) {
        if constexpr (PAIR)
          tc_commit_pair(DONE, 1);
        else
          tc_commit(DONE);
        wait_quiet(DONE, 0);
      }
      __syncwarp();
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int e = warp - 2;
    const int quarter = warp & 3;  // TMEM lanes [32 quarter, 32 quarter + 32)
    const int cpart = e >> 2;      // columns [VALS cpart, VALS cpart + VALS)
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    // the leader's MMA waits until the epilogues of both CTAs drained a buffer
    const uint32_t aempty0 = PAIR ? map_to_rank(AEMPTY(0), 0) : AEMPTY(0);
    Group *gcache = reinterpret_cast<Group *>(smem + (size_t)STAGES * S::STAGE_BYTES + 256) + e * 32;
    int32_t *xs = reinterpret_cast<int32_t *>(smem + (size_t)STAGES * S::STAGE_BYTES + 256 +
                                              S::GCACHE_BYTES) + e * 32 * (XB + 1);
    uint32_t chunk = 0;
    bool ok = true;
    ModP m = P.m;
    for (int t = (int)unit0; t < P.ntiles && ok; t += (int)nunits) {
      int ng;
      // batched launches: the tile's groups come from global memory; lane i
      // of each warp loads group i into the warp's shared-memory cache at
      // the start of the tile (all loads in flight together) and the group
      // loop reads them from there
      if constexpr (MODE == kBatch) {
        const int4 tl = P.btiles[t];
        ng = tile_ngrp(tl.w);
        __syncwarp();
        if (lane < ng) gcache[lane] = P.gtab[tile_goff(tl.w) + lane];
        __syncwarp();
        m = P.probs[tl.x].m;
      } else {
        ng = tile_ng<MODE>(P, t);
      }
      // this warp's 32 x VALS block of the tile: when it lies wholly outside
      // the product (rows >= M, columns >= N, or above the diagonal of a
      // lower product) the warp only keeps the barrier protocol going
      bool live;
      {
        const OutView o = tile_out<MODE>(P, t);
        const int2 ij = tile_ij<MODE>(P, t);
        const int64_t r0 = (int64_t)ij.x * S::TM + (int64_t)rank * BM + quarter * 32;
        const int64_t c0 = (int64_t)ij.y * BN + cpart * VALS;
        live = r0 < o.M && c0 < o.N && !(o.lower && c0 > r0 + 31);
      }
      int32_t acc[VALS];
#pragma unroll
      for (int i = 0; i < VALS; ++i) acc[i] = 0;
      for (int gi = 0; gi < ng && ok; ++gi) {
        const Group g = (MODE == kBatch && gi < 32) ? gcache[gi] : tile_group<MODE>(P, t, gi);
        if (gi > 0 && live) {
          if (m.p < (1u << 30)) {  // the signed form (set_shoup stored its quotient)
            const int32_t wb = g.ratio > m.half ? (int32_t)g.ratio - (int32_t)m.p : (int32_t)g.ratio;
            const int32_t wsh = (int32_t)g.ratio_sh;
#pragma unroll
            for (int i = 0; i < VALS; ++i) acc[i] = mulmod_shoup_s(acc[i], wb, wsh, m);
          } else {
#pragma unroll
            for (int i = 0; i < VALS; ++i) acc[i] = mulmod_shoup(acc[i], g.ratio, g.ratio_sh, m);
          }
        }
        for (int kb = g.kb0; kb < g.kb1;) {
          const int kend = min(kb + g.kchunk, g.kb1);
          const uint32_t buf = chunk & 1u, use = chunk >> 1;
          if (!wait_bounded<PAIR>(AFULL(buf), use & 1u, abort_flag, P.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (live) {
            const uint32_t ta = tmem + lane_base + buf * ACC_COLS + (uint32_t)(cpart * VALS);
            tmem_drain16<0>(ta, acc);
            tmem_drain16<16>(ta + 16u, acc);
            tmem_drain16<32>(ta + 32u, acc);
            tmem_drain16<48>(ta + 48u, acc);
            if constexpr (VALS == 128) {
              tmem_drain16<64>(ta + 64u, acc);
              tmem_drain16<80>(ta + 80u, acc);
              tmem_drain16<96>(ta + 96u, acc);
              tmem_drain16<112>(ta + 112u, acc);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if constexpr (PAIR)
              mbar_arrive_cluster(aempty0 + 8u * buf);
            else
              mbar_arrive(AEMPTY(buf));
          }
          ++chunk;
          kb = kend;
        }
      }
      if (!ok) break;
      if (!live) continue;
      const int2 ij = tile_ij<MODE>(P, t);
      const int64_t row = (int64_t)ij.x * S::TM + (int64_t)rank * BM + quarter * 32 + lane;
      const int64_t col0 = (int64_t)ij.y * BN + cpart * VALS;
      // final value, canonical, in place: the last group is the final
      // multiplier, whose Horner step left every entry balanced
#pragma unroll
      for (int i = 0; i < VALS; ++i) acc[i] = (int32_t)bal_to_canon(acc[i], m);
      const OutView o = tile_out<MODE>(P, t);
      const int64_t row0 = row - lane;
      // rows 16-byte aligned and nothing to read back: each thread stores its
      // row segment with 16-byte stores
      if (!o.accumulate && ((reinterpret_cast<uintptr_t>(o.out) | (uintptr_t)(o.ldo * 4)) & 15) == 0) {
        int64_t lim = o.N - col0;
        if (o.lower) lim = min(lim, row - col0 + 1);
        if (row < o.M && lim > 0) {
          int32_t *orow = o.out + row * o.ldo + col0;
#pragma unroll
          for (int q = 0; q < VALS / 4; ++q) {
            const int c = 4 * q;
            if (c + 4 <= lim) {
              *reinterpret_cast<int4 *>(orow + c) = make_int4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (c + j < lim) orow[c + j] = acc[c + j];
            }
            asm volatile("" ::: "memory");
          }
        }
        continue;
      }
      // Otherwise coalesced through shared memory: each thread owns one row
      // of the tile (its TMEM lane), so the warp writes XB columns of its 32
      // rows at a time into shared memory and reads them back 32 / XB rows
      // per instruction, every store instruction covering 32 / XB contiguous
      // row segments of 4 XB bytes (ragged rows, and the read-modify-write of
      // an accumulating product).
      // the warp's 32 x VALS block: rows below mlim, columns below nlim, and
      // for a lower product only column - row <= dl (tile coordinates)
      constexpr int RPI = 32 / XB;  // rows per store instruction
      const int mlim = (int)max((int64_t)0, min((int64_t)32, o.M - row0));
      const int nlim = (int)max((int64_t)0, min((int64_t)VALS, o.N - col0));
      const int dl = o.lower ? (int)max((int64_t)-256, min((int64_t)256, row0 - col0)) : 1 << 20;
      int32_t *const base = o.out + row0 * o.ldo + col0;
      const int64_t ldo = o.ldo;
      const int accum = o.accumulate;
      const uint32_t beta = o.beta, beta_sh = o.beta_sh;
      const int lr = lane / XB, lc = lane % XB;
#pragma unroll
      for (int cb = 0; cb < VALS; cb += XB) {
        __syncwarp();
#pragma unroll
        for (int j = 0; j < XB; ++j) xs[lane * (XB + 1) + j] = acc[cb + j];
        __syncwarp();
        if constexpr (EW == 8) {
          // accumulating product (8 epilogue warps): the old values are
          // loaded four at a time, so four DRAM latencies overlap instead of
          // one round trip per store
          if (accum) {
            constexpr int G = 4;
#pragma unroll 1
            for (int i0 = 0; i0 < XB; i0 += G) {
              int32_t oldv[G];
#pragma unroll
              for (int g = 0; g < G; ++g) {
                const int rr = RPI * (i0 + g) + lr, cl = cb + lc;
                oldv[g] = (rr < mlim && cl < nlim && cl - rr <= dl)
                              ? base[(int64_t)rr * ldo + cl] : 0;
              }
#pragma unroll
              for (int g = 0; g < G; ++g) {
                const int rr = RPI * (i0 + g) + lr, cl = cb + lc;
                if (rr < mlim && cl < nlim && cl - rr <= dl) {
                  int32_t old = bal(oldv[g], m);
                  if (beta != 1u) old = mulmod_shoup(old, beta, beta_sh, m);
                  const int32_t x = xs[rr * (XB + 1) + lc];
                  base[(int64_t)rr * ldo + cl] =
                      (int32_t)bal_to_canon(add_bal(to_bal((uint32_t)x, m), old, m), m);
                }
              }
            }
            continue;
          }
        }
#pragma unroll 1
        for (int i = 0; i < XB; ++i) {
          const int rr = RPI * i + lr, cl = cb + lc;
          if (rr < mlim && cl < nlim && cl - rr <= dl) {
            int32_t x = xs[rr * (XB + 1) + lc];
            int32_t *dst = base + (int64_t)rr * ldo + cl;
            if (accum) {
              int32_t old = bal(*dst, m);
              if (beta != 1u) old = mulmod_shoup(old, beta, beta_sh, m);
              x = (int32_t)bal_to_canon(add_bal(to_bal((uint32_t)x, m), old, m), m);
            }
            *dst = x;
          }
        }
      }
    }
  }

  __syncthreads();
  // no CTA of a pair leaves (or frees TMEM) while its peer may still touch
  // its shared memory or tensor memory
  if constexpr (PAIR) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(TMEM_COLS)
                   : "memory");
  }
#undef FULL
#undef EMPTY
#undef AFULL
#undef AEMPTY
#undef DONE
}

// ------------------------------------------------------------------ host

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_mu;
std::map<std::tuple<int, int64_t, int64_t, int, int>, std::pair<int2 *, int>> g_tiles;
std::map<int, bool> g_attr_set;
std::map<int, int> g_pair_units;  // co-resident CTA pairs per device

cudaError_t get_encode() {
  if (g_encode) return cudaSuccess;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return cudaSuccess;
}

cudaError_t encode_planes(CUtensorMap *tm, const Planes &P, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)P.cols, (cuuint64_t)P.rows, (cuuint64_t)P.L};
  cuuint64_t strides[2] = {(cuuint64_t)P.kstride * 2, (cuuint64_t)(P.rows * P.kstride * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)P.ptr, dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tile order: bands of 2048 output rows (8 tile rows of 256, or 16 of 128),
// each swept column by column.  The persistent CTAs take tiles round robin,
// so the tiles in flight at any time are about a full wave of consecutive
// entries: 76 pairs (or 152 CTAs) cover 8 (16) tile rows by ~9.5 tile
// columns, whose X row panels and Y column panels are read from DRAM once
// and shared through L2 by every tile of the wave (18 panels per wave of 76
// tiles against 24 for 8 x 8 super-blocks swept row by row).  `tm` is the
// tile height (128 or 256).
// Band height in output rows (AAT_TILE_BAND, default 2048).
int64_t band_rows() {
  static const int64_t v = [] {
    const char *e = getenv("AAT_TILE_BAND");
    const long long r = e ? atoll(e) : 2048;
    return (int64_t)(r >= 128 ? r : 2048);
  }();
  return v;
}

void tile_order(int64_t M, int64_t N, int lower, int tm, std::vector<int2> &v) {
  const int64_t TI = (M + tm - 1) / tm, TJ = (N + BN - 1) / BN;
  const int64_t band = std::max<int64_t>(1, band_rows() / tm);
  for (int64_t bi = 0; bi < TI; bi += band) {
    const int64_t iend = std::min(TI, bi + band);
    for (int64_t j = 0; j < TJ; ++j)
      for (int64_t i = bi; i < iend; ++i) {
        if (lower && j * BN > i * tm + tm - 1) continue;
        v.push_back(make_int2((int)i, (int)j));
      }
  }
}

template <class T>
cudaError_t upload(const std::vector<T> &v, T **out) {
  *out = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(out, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

cudaError_t get_tiles(int dev, int64_t M, int64_t N, int lower, int tm, int2 **out, int *count) {
  auto key = std::make_tuple(dev, M, N, lower, tm);
  auto it = g_tiles.find(key);
  if (it != g_tiles.end()) {
    *out = it->second.first;
    *count = it->second.second;
    return cudaSuccess;
  }
  std::vector<int2> v;
  tile_order(M, N, lower, tm, v);
  int2 *d = nullptr;
  cudaError_t e = upload(v, &d);
  if (e != cudaSuccess) return e;
  g_tiles[key] = std::make_pair(d, (int)v.size());
  *out = d;
  *count = (int)v.size();
  return cudaSuccess;
}

// Tile list of a multi-problem launch: the problems in launch order, each in
// its own super-block order, entries (problem, I, J, 0).  Cached per device,
// tile height and list of shapes.
std::map<std::vector<int64_t>, std::pair<int4 *, int>> g_mtiles;

cudaError_t get_multi_tiles(int dev, const TcLeafArgs *as, const int *order, int count, int tm,
                            int4 **out, int *ntiles) {
  std::vector<int64_t> key = {dev, tm};
  for (int q = 0; q < count; ++q) {
    const TcLeafArgs &a = as[order[q]];
    key.insert(key.end(), {(int64_t)order[q], a.M, a.N, (int64_t)a.lower});
  }
  auto it = g_mtiles.find(key);
  if (it != g_mtiles.end()) {
    *out = it->second.first;
    *ntiles = it->second.second;
    return cudaSuccess;
  }
  std::vector<int4> v;
  std::vector<int2> one;
  for (int q = 0; q < count; ++q) {
    const TcLeafArgs &a = as[order[q]];
    one.clear();
    tile_order(a.M, a.N, a.lower, tm, one);
    for (const int2 &t : one) v.push_back(make_int4(order[q], t.x, t.y, 0));
  }
  int4 *d = nullptr;
  cudaError_t e = upload(v, &d);
  if (e != cudaSuccess) return e;
  g_mtiles[key] = std::make_pair(d, (int)v.size());
  *out = d;
  *ntiles = (int)v.size();
  return cudaSuccess;
}

// Shoup quotients of the Horner ratios: floor(ratio 2^32 / p) for the
// unsigned form, or, for p < 2^30, floor(wb 2^32 / p) of the balanced ratio
// wb (the signed form, mulmod_shoup_s), as int32 bits.
void set_shoup(Group *g, int ng, uint32_t p) {
  for (int i = 0; i < ng; ++i) {
    if (p < (1u << 30)) {
      const int64_t wb = g[i].ratio > (p - 1) / 2 ? (int64_t)g[i].ratio - p : (int64_t)g[i].ratio;
      const int64_t num = wb * ((int64_t)1 << 32);
      int64_t q = num / (int64_t)p;
      if (num % (int64_t)p != 0 && num < 0) q -= 1;  // floor
      g[i].ratio_sh = (uint32_t)(int32_t)q;
    } else {
      g[i].ratio_sh = (uint32_t)(((uint64_t)g[i].ratio << 32) / p);
    }
  }
}

// K segment of the groups in K blocks: every plane product runs over one
// segment of K before the next segment starts, so that the tiles in flight
// share the segment's panels in L2 (AAT_KSEG: the width in K elements, a
// multiple of 64; default 8192).
int kseg_blocks() {
  static const int v = [] {
    const char *e = getenv("AAT_KSEG");
    const int w = e ? atoi(e) : 8192;
    return std::max(1, (w > 0 ? w : 8192) / BK);
  }();
  return v;
}

// Groups of the leaf product: plane pairs with integer weights turned into a
// Horner sequence (see the file header).  Returns false when the product does
// not fit the group table or a bound cannot be met.
bool build_groups(const TcLeafArgs &a, const ModP &m, Group *out, int *ng_out, int *nprod_out) {
  // The terms of the product: plane pairs with integer weights.
  //   plain:     X_i Y_j^T with weight z^(i+j), z = 2^b
  //   pair sums: X_i Y_i^T with weight z^(2i) - sum_{j != i} z^(i+j), and
  //              (X_i + X_j)(Y_i + Y_j)^T with weight z^(i+j) for i < j
  struct Term { int xp, yp; int64_t w; int64_t prod; };
  std::vector<Term> terms;
  const int L = a.dx.L;
  auto zp = [&](int e) { return (int64_t)1 << (a.dx.b * e); };
  const bool sums = a.dx.nsum > 0 && a.dy.nsum == a.dx.nsum && a.dy.L == L &&
                    a.x.nsum == a.dx.nsum && a.y.nsum == a.dy.nsum;
  if (sums) {
    for (int i = 0; i < L; ++i) {
      int64_t w = zp(2 * i);
      for (int j = 0; j < L; ++j)
        if (j != i) w -= zp(i + j);
      terms.push_back({i, i, w, (int64_t)a.dx.dmax[i] * a.dy.dmax[i]});
    }
    for (int q = 0; q < a.dx.nsum; ++q) {
      const int i = a.dx.si[q], j = a.dx.sj[q];
      const int64_t bx = a.dx.dmax[i] + a.dx.dmax[j], by = a.dy.dmax[i] + a.dy.dmax[j];
      terms.push_back({L + q, L + q, zp(i + j), bx * by});
    }
  } else {
    for (int s2 = 2 * (L - 1); s2 >= 0; --s2)
      for (int i = 0; i < L; ++i) {
        const int j = s2 - i;
        if (j < 0 || j >= a.dy.L) continue;
        terms.push_back({i, j, zp(s2), (int64_t)a.dx.dmax[i] * a.dy.dmax[j]});
      }
  }
  // Planes that keep only a window of the sequence (the low-memory plane
  // passes): the terms whose two planes are both stored, indexed within the
  // windows.
  {
    std::vector<Term> kept;
    for (Term t : terms) {
      const int xs = t.xp - a.x.q0, ys = t.yp - a.y.q0;
      if (xs < 0 || xs >= a.x.L || ys < 0 || ys >= a.y.L) continue;
      t.xp = xs;
      t.yp = ys;
      kept.push_back(t);
    }
    terms.swap(kept);
  }
  auto modw = [&](int64_t w) {
    int64_t r = w % (int64_t)m.p;
    return (uint32_t)(r < 0 ? r + (int64_t)m.p : r);
  };
  auto mulm = [&](uint32_t x, uint32_t y) { return (uint32_t)((uint64_t)x * y % m.p); };
  auto invm = [&](uint32_t x) {
    uint64_t r = 1, bb = x, e = m.p - 2;
    while (e) {
      if (e & 1) r = r * bb % m.p;
      bb = bb * bb % m.p;
      e >>= 1;
    }
    return (uint32_t)r;
  };
  // Groups: K segments of at most 8192 (for L2 reuse of the planes), each
  // term split further so that (p-1)/2 + K_range * max|product| < 2^31; the
  // epilogue multiplies its accumulator by w_prev / w_cur between groups and
  // by the last weight in a final group without K blocks (Horner).
  const int kblocks = (int)((a.K + BK - 1) / BK);
  const int kseg = kseg_blocks();
  const int ebits = std::min(std::max(a.exact_bits, 8), 24);
  const int64_t room = ((int64_t)1 << 31) - 1 - (int64_t)m.half;
  int ng = 0;
  uint32_t wprev = 0;
  for (int seg = 0; seg < kblocks; seg += kseg) {
    const int segend = std::min(kblocks, seg + kseg);
    for (const Term &t : terms) {
      const uint32_t w = modw(t.w);
      if (w == 0) continue;  // the term vanishes mod p
      const int64_t prod = std::max<int64_t>(t.prod, 1);
      const int64_t kc = ((int64_t)1 << ebits) / prod / BK;
      const int64_t kr = room / prod / BK;
      if (kc < 1 || kr < 1) return false;
      for (int kb = seg; kb < segend; kb += (int)kr) {
        if (ng >= MAX_GROUPS - 1) return false;
        Group &g = out[ng];
        g.xp = (int16_t)t.xp;
        g.yp = (int16_t)t.yp;
        g.kb0 = kb;
        g.kb1 = (int)std::min<int64_t>(segend, kb + kr);
        g.kchunk = (int)std::min<int64_t>(kc, 1 << 20);
        g.ratio = (ng == 0) ? 1u : mulm(wprev, invm(w));
        wprev = w;
        ++ng;
      }
    }
  }
  // final multiplier (a group without K blocks): the last weight times the
  // product's scale alpha (the SYRK update's alpha, 1 otherwise).  It is
  // there even when it is 1: its Horner step leaves every entry balanced,
  // which the kernel's final canonicalisation relies on.
  const uint32_t wfinal = mulm(wprev, a.lin.alpha.w % m.p);
  if (ng > 0) {
    if (ng >= MAX_GROUPS) return false;
    Group &g = out[ng++];
    g.xp = g.yp = 0;
    g.kb0 = g.kb1 = 0;
    g.kchunk = 1;
    g.ratio = wfinal;
  }
  set_shoup(out, ng, m.p);
  int nprod = 0;
  for (const Term &t : terms)
    if (modw(t.w) != 0) ++nprod;
  *ng_out = ng;
  *nprod_out = nprod;
  return true;
}

// The stored planes form a window of the plane sequence (all of it, or the
// planes of one low-memory pass).
bool window_ok(const Planes &P) {
  return P.L >= 1 && P.q0 >= 0 && P.q0 + P.L <= P.nbase + P.nsum;
}

// Co-resident CTA pairs of the pair kernel on this device (0: none).
int pair_units(int dev) {
  auto it = g_pair_units.find(dev);
  if (it != g_pair_units.end()) return it->second;
  int units = 0;
  if (cudaFuncSetAttribute(leaf_tc_kernel<kSingle, true, kEwLeaf>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Shape<true, kEwLeaf>::SMEM) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(Shape<true, kEwLeaf>::THREADS, 1, 1);
    cfg.dynamicSmemBytes = Shape<true, kEwLeaf>::SMEM;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&units, leaf_tc_kernel<kSingle, true, kEwLeaf>, &cfg) != cudaSuccess)
      units = 0;
  }
  cudaGetLastError();
  g_pair_units[dev] = units;
  return units;
}

// The form of a leaf: the caller's (TcLeafArgs::form, set by the tuning
// table), else AAT_LEAF_PAIR=0 (every leaf on the one-CTA form) or =1 (every
// leaf with at least 256 rows on the CTA-pair form), else the pair form when
// its tiles fill every co-resident pair at least once.
int pair_override() {
  static const int v = [] {
    const char *e = getenv("AAT_LEAF_PAIR");
    return e ? atoi(e) : -1;
  }();
  return v;
}

}  // namespace

cudaError_t launch_leaf_tc(const TcLeafArgs &a, const ModP &m, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  if (a.dx.b != a.dy.b || a.x.nbase != a.dx.L || a.y.nbase != a.dy.L || !window_ok(a.x) ||
      !window_ok(a.y))
    return cudaErrorInvalidValue;
  if (a.x.kstride % 8 || a.y.kstride % 8 || a.x.cols != a.K || a.y.cols != a.K)
    return cudaErrorInvalidValue;
  if (((uintptr_t)a.x.ptr | (uintptr_t)a.y.ptr) & 15) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(g_mu);
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);

  // the form: CTA pairs when there are enough 256 x 256 tiles to keep every
  // co-resident pair busy
  const int units = pair_units(dev);
  bool pair = false;
  if (units > 0 && a.M >= 256) {
    const int64_t pt = ((a.M + 255) / 256) * ((a.N + BN - 1) / BN);
    const int ov = a.form > 0 ? a.form - 1 : pair_override();
    pair = ov >= 0 ? ov > 0 : (a.lower ? pt / 2 : pt) >= units;
  }
  const int tm = pair ? Shape<true>::TM : Shape<false>::TM;

  Params *P = new Params;
  std::memset(P, 0, sizeof(Params));
  if ((e = encode_planes(&P->tmx, a.x, BM)) != cudaSuccess ||
      (e = encode_planes(&P->tmy, a.y, pair ? Shape<true>::YROWS : Shape<false>::YROWS)) !=
          cudaSuccess) {
    delete P;
    return e;
  }
  int ng = 0, nprod = 0;
  if (!build_groups(a, m, P->g, &ng, &nprod)) {
    delete P;
    return cudaErrorInvalidValue;
  }
  P->ng = ng;
  P->out = a.out;
  P->ldo = a.ldo;
  P->M = a.M;
  P->N = a.N;
  P->lower = a.lower;
  P->accumulate = a.lin.beta.w != 0u;
  P->beta = a.lin.beta.w;
  P->beta_sh = a.lin.beta.wsh;
  P->m = m;
  P->status = device_status_ptr();
  int2 *tiles = nullptr;
  int nt = 0;
  if ((e = get_tiles(dev, a.M, a.N, a.lower, tm, &tiles, &nt)) != cudaSuccess) {
    delete P;
    return e;
  }
  P->tiles = tiles;
  P->ntiles = nt;
  if (!g_attr_set[dev]) {
    e = cudaFuncSetAttribute(leaf_tc_kernel<kSingle, false, kEwLeaf>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Shape<false, kEwLeaf>::SMEM);
    if (e != cudaSuccess) { delete P; return e; }
    g_attr_set[dev] = true;
  }
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nt > 0) {
    // algorithmic tensor work: one BF16 product of the ring MACs per plane
    // product with a non-zero weight
    const double macs =
        a.lower ? 0.5 * (double)a.M * (double)(a.M + 1) * a.K : (double)a.M * a.N * a.K;
    ProfScope prof(AAT_K_LEAF_TC, st, 2.0 * nprod * macs);
    if (pair) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(2 * std::max(1, std::min(nt, units)), 1, 1);
      cfg.blockDim = dim3(Shape<true, kEwLeaf>::THREADS, 1, 1);
      cfg.dynamicSmemBytes = Shape<true, kEwLeaf>::SMEM;
      cfg.stream = st;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, leaf_tc_kernel<kSingle, true, kEwLeaf>, *P);
      if (e != cudaSuccess) { delete P; return e; }
    } else {
      leaf_tc_kernel<kSingle, false, kEwLeaf>
          <<<std::max(1, std::min(nt, sms)), Shape<false, kEwLeaf>::THREADS,
             Shape<false, kEwLeaf>::SMEM, st>>>(*P);
    }
  }
  delete P;
  return cudaGetLastError();
}

int64_t tile_count(int64_t M, int64_t N, int lower, int tm) {
  const int64_t TI = (M + tm - 1) / tm, TJ = (N + BN - 1) / BN;
  if (!lower) return TI * TJ;
  int64_t c = 0;
  for (int64_t i = 0; i < TI; ++i) c += std::min(TJ, (i * tm + tm - 1) / BN + 1);
  return c;
}

// Whether one launch over the tiles of several products beats one launch
// per product: the launches of single products leave part of the GPU idle
// in their last wave (tiles / units rounded up).  Measured on GB300: one
// launch wins by 5-10 % when those last waves waste 10-16 % of the slots
// (4096-sized products), and loses ~5 % at 3-4 % (8192-sized products in
// a second-long run under the power cap, where idle tails let the clock
// rise).  So: one launch when more than 6 % of the slots would be idle.
int leaf_tc_terms(const TcLeafArgs &a, const ModP &m) {
  std::vector<Group> g(MAX_GROUPS);
  int ng = 0, nprod = 0;
  if (!build_groups(a, m, g.data(), &ng, &nprod)) return -1;
  return nprod;
}

bool leaf_tc_fuse_pays(const TcLeafArgs *as, int count) {
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int units = 0;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    units = pair_units(dev);
  }
  double idle = 0.0, all = 0.0;
  for (int i = 0; i < count; ++i) {
    const TcLeafArgs &a = as[i];
    bool pair = false;
    if (units > 0 && a.M >= 256) {
      const int64_t pt = ((a.M + 255) / 256) * ((a.N + BN - 1) / BN);
      const int ov = a.form > 0 ? a.form - 1 : pair_override();
      pair = ov >= 0 ? ov > 0 : (a.lower ? pt / 2 : pt) >= units;
    }
    const int u = pair ? units : sms;
    const double nt = (double)tile_count(a.M, a.N, a.lower, pair ? 256 : 128);
    const double slots = std::ceil(nt / u) * u;
    const double kb = (double)((a.K + BK - 1) / BK);
    idle += (slots - nt) * kb;
    all += slots * kb;
  }
  return all > 0.0 && idle > 0.06 * all;
}

// Several independent products of one modulus and digit base in one
// persistent launch: the tiles of all of them form one list taken round
// robin, so the last wave of one product is filled by the tiles of the next
// instead of leaving SMs idle between launches.
cudaError_t launch_leaf_tc_multi(const TcLeafArgs *as, int count, const ModP &m,
                                 cudaStream_t st) {
  if (count < 1 || count > MAX_MULTI) return cudaErrorInvalidValue;
  for (int i = 0; i < count; ++i) {
    const TcLeafArgs &a = as[i];
    if (a.M <= 0 || a.N <= 0) return cudaErrorInvalidValue;
    if (a.dx.b != as[0].dx.b || a.dx.b != a.dy.b || a.x.nbase != a.dx.L ||
        a.y.nbase != a.dy.L || !window_ok(a.x) || !window_ok(a.y))
      return cudaErrorInvalidValue;
    if (a.x.kstride % 8 || a.y.kstride % 8 || a.x.cols != a.K || a.y.cols != a.K)
      return cudaErrorInvalidValue;
    if (((uintptr_t)a.x.ptr | (uintptr_t)a.y.ptr) & 15) return cudaErrorInvalidValue;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);

  // the form, as for one product, over the tiles of all of them
  const int units = pair_units(dev);
  bool pair = false;
  if (units > 0) {
    bool big = true;
    int64_t pt = 0;
    for (int i = 0; i < count; ++i) {
      big = big && as[i].M >= 256;
      const int64_t t = ((as[i].M + 255) / 256) * ((as[i].N + BN - 1) / BN);
      pt += as[i].lower ? t / 2 : t;
    }
    const int ov = as[0].form > 0 ? as[0].form - 1 : pair_override();
    pair = big && (ov >= 0 ? ov > 0 : pt >= units);
  }
  const int tm = pair ? Shape<true>::TM : Shape<false>::TM;

  Params *P = new Params;
  std::memset(P, 0, sizeof(Params));
  std::vector<Group> tmp(MAX_GROUPS);
  std::vector<double> cost(count);
  int gused = 0;
  double work = 0.0;
  for (int i = 0; i < count; ++i) {
    const TcLeafArgs &a = as[i];
    MultiProb &b = P->mp[i];
    if ((e = encode_planes(&b.tmx, a.x, BM)) != cudaSuccess ||
        (e = encode_planes(&b.tmy, a.y, pair ? Shape<true>::YROWS : Shape<false>::YROWS)) !=
            cudaSuccess) {
      delete P;
      return e;
    }
    int ng = 0, nprod = 0;
    if (!build_groups(a, m, tmp.data(), &ng, &nprod)) {
      delete P;
      return cudaErrorInvalidValue;
    }
    // problems with the same K, scale and digit form share one group list
    int goff = -1;
    for (int j = 0; j < i && goff < 0; ++j)
      if (P->mp[j].ng == ng &&
          std::memcmp(P->g + P->mp[j].goff, tmp.data(), sizeof(Group) * ng) == 0)
        goff = P->mp[j].goff;
    if (goff < 0) {
      if (gused + ng > MAX_GROUPS) {
        delete P;
        return cudaErrorInvalidValue;
      }
      std::memcpy(P->g + gused, tmp.data(), sizeof(Group) * ng);
      goff = gused;
      gused += ng;
    }
    b.goff = goff;
    b.ng = ng;
    b.out = a.out;
    b.ldo = a.ldo;
    b.M = a.M;
    b.N = a.N;
    b.lower = a.lower;
    b.accumulate = a.lin.beta.w != 0u;
    b.beta = a.lin.beta.w;
    b.beta_sh = a.lin.beta.wsh;
    cost[i] = (double)((a.K + BK - 1) / BK) * nprod;
    const double macs =
        a.lower ? 0.5 * (double)a.M * (double)(a.M + 1) * a.K : (double)a.M * a.N * a.K;
    work += 2.0 * nprod * macs;
  }
  P->ng = gused;
  // the problems with the most expensive tiles first
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return cost[u] > cost[v]; });
  int4 *tiles = nullptr;
  int nt = 0;
  if ((e = get_multi_tiles(dev, as, order.data(), count, tm, &tiles, &nt)) != cudaSuccess) {
    delete P;
    return e;
  }
  P->mtiles = tiles;
  P->ntiles = nt;
  P->m = m;
  P->status = device_status_ptr();
  static std::map<int, bool> attr;
  if (!attr[dev]) {
    if ((e = cudaFuncSetAttribute(leaf_tc_kernel<kMulti, false, kEwLeaf>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Shape<false, kEwLeaf>::SMEM)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(leaf_tc_kernel<kMulti, true, kEwLeaf>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Shape<true, kEwLeaf>::SMEM)) != cudaSuccess) {
      delete P;
      return e;
    }
    attr[dev] = true;
  }
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nt > 0) {
    ProfScope prof(AAT_K_LEAF_TC, st, work);
    if (pair) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr1[1];
      attr1[0].id = cudaLaunchAttributeClusterDimension;
      attr1[0].val.clusterDim.x = 2;
      attr1[0].val.clusterDim.y = 1;
      attr1[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(2 * std::max(1, std::min(nt, units)), 1, 1);
      cfg.blockDim = dim3(Shape<true, kEwLeaf>::THREADS, 1, 1);
      cfg.dynamicSmemBytes = Shape<true, kEwLeaf>::SMEM;
      cfg.stream = st;
      cfg.attrs = attr1;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, leaf_tc_kernel<kMulti, true, kEwLeaf>, *P);
      if (e != cudaSuccess) {
        delete P;
        return e;
      }
    } else {
      leaf_tc_kernel<kMulti, false, kEwLeaf>
          <<<std::max(1, std::min(nt, sms)), Shape<false, kEwLeaf>::THREADS,
             Shape<false, kEwLeaf>::SMEM, st>>>(*P);
    }
  }
  delete P;
  return cudaGetLastError();
}

// ------------------------------------------------------- batched launches

struct LeafBatchImpl {
  BatchProb *probs = nullptr;
  Group *gtab = nullptr;
  int4 *tiles = nullptr;
  int ntiles = 0;
  double work = 0.0;
};

cudaError_t leaf_tc_batch_build(const TcLeafArgs *args, const ModP *mods, int count,
                                LeafBatch *out) {
  std::lock_guard<std::mutex> lock(g_mu);
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return e;
  std::vector<BatchProb> probs(count);
  std::vector<Group> gtab;
  struct T4 { int4 t; double cost; };
  std::vector<T4> tiles;
  double work = 0.0;
  std::vector<Group> tmp(MAX_GROUPS);
  for (int i = 0; i < count; ++i) {
    const TcLeafArgs &a = args[i];
    BatchProb &b = probs[i];
    std::memset(&b, 0, sizeof(b));
    if ((e = encode_planes(&b.tmx, a.x, BM)) != cudaSuccess ||
        (e = encode_planes(&b.tmy, a.y, BN)) != cudaSuccess)
      return e;
    int ng = 0, nprod = 0;
    if (!build_groups(a, mods[i], tmp.data(), &ng, &nprod)) return cudaErrorInvalidValue;
    b.goff = (int)gtab.size();
    b.ng = ng;
    if (b.goff + ng > 0xFFFF) return cudaErrorInvalidValue;  // tile entries pack goff in 16 bits
    gtab.insert(gtab.end(), tmp.begin(), tmp.begin() + ng);
    b.out = a.out;
    b.ldo = a.ldo;
    b.M = a.M;
    b.N = a.N;
    b.lower = a.lower;
    b.accumulate = a.lin.beta.w != 0u;
    b.beta = a.lin.beta.w;
    b.beta_sh = a.lin.beta.wsh;
    b.m = mods[i];
    const double kb = (double)((a.K + BK - 1) / BK);
    const double cost = kb * nprod;  // K blocks x plane products per tile
    const int64_t TI = (a.M + BM - 1) / BM, TJ = (a.N + BN - 1) / BN;
    for (int64_t I = 0; I < TI; ++I)
      for (int64_t J = 0; J < TJ; ++J) {
        if (a.lower && J * BN > I * BM + BM - 1) continue;
        tiles.push_back({make_int4(i, (int)I, (int)J, b.goff | (ng << 16)), cost});
      }
    const double macs =
        a.lower ? 0.5 * (double)a.M * (double)(a.M + 1) * a.K : (double)a.M * a.N * a.K;
    work += 2.0 * nprod * macs;
  }
  // the most expensive tiles first: the persistent CTAs take tiles round
  // robin, so this spreads the heavy problems over every SM
  std::stable_sort(tiles.begin(), tiles.end(),
                   [](const T4 &u, const T4 &v) { return u.cost > v.cost; });
  std::vector<int4> tl(tiles.size());
  for (size_t i = 0; i < tiles.size(); ++i) tl[i] = tiles[i].t;
  LeafBatchImpl *L = new LeafBatchImpl;
  L->ntiles = (int)tl.size();
  L->work = work;
  if ((e = cudaMalloc(&L->probs, sizeof(BatchProb) * std::max(count, 1))) != cudaSuccess ||
      (e = cudaMalloc(&L->gtab, sizeof(Group) * std::max<size_t>(gtab.size(), 1))) != cudaSuccess ||
      (e = cudaMalloc(&L->tiles, sizeof(int4) * std::max<size_t>(tl.size(), 1))) != cudaSuccess) {
    LeafBatch tmp;
    tmp.impl = L;
    leaf_tc_batch_free(&tmp);
    return e;
  }
  cudaMemcpy(L->probs, probs.data(), sizeof(BatchProb) * count, cudaMemcpyHostToDevice);
  if (!gtab.empty())
    cudaMemcpy(L->gtab, gtab.data(), sizeof(Group) * gtab.size(), cudaMemcpyHostToDevice);
  if (!tl.empty()) cudaMemcpy(L->tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice);
  out->impl = L;
  return cudaGetLastError();
}

cudaError_t leaf_tc_batch_launch(const LeafBatch &lb, cudaStream_t st) {
  const LeafBatchImpl *L = (const LeafBatchImpl *)lb.impl;
  if (!L || L->ntiles == 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lock(g_mu);
    static std::map<int, bool> attr;
    if (!attr[dev]) {
      cudaError_t e = cudaFuncSetAttribute(leaf_tc_kernel<kBatch, false, kEwBatch>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Shape<false, kEwBatch>::SMEM);
      if (e != cudaSuccess) return e;
      attr[dev] = true;
    }
  }
  Params *P = new Params;
  std::memset(P, 0, sizeof(Params));
  P->probs = L->probs;
  P->gtab = L->gtab;
  P->btiles = L->tiles;
  P->ntiles = L->ntiles;
  P->status = device_status_ptr();
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  {
    ProfScope prof(AAT_K_LEAF_TC, st, L->work);
    leaf_tc_kernel<kBatch, false, kEwBatch>
        <<<std::max(1, std::min(L->ntiles, sms)), Shape<false, kEwBatch>::THREADS,
           Shape<false, kEwBatch>::SMEM, st>>>(*P);
  }
  delete P;
  return cudaGetLastError();
}

void leaf_tc_batch_free(LeafBatch *lb) {
  LeafBatchImpl *L = (LeafBatchImpl *)lb->impl;
  if (!L) return;
  if (L->probs) cudaFree(L->probs);
  if (L->gtab) cudaFree(L->gtab);
  if (L->tiles) cudaFree(L->tiles);
  delete L;
  lb->impl = nullptr;
}

void noalloc_forget();

void leaf_tc_release() {
  noalloc_forget();
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto &kv : g_tiles)
    if (kv.second.first) cudaFree(kv.second.first);
  g_tiles.clear();
  for (auto &kv : g_mtiles)
    if (kv.second.first) cudaFree(kv.second.first);
  g_mtiles.clear();
  g_attr_set.clear();
  g_pair_units.clear();
}

}  // namespace aat

// ======================================================================
// Allocation-free variant of the general leaf product (aat_gemm_modp_noalloc).
//
// Some callers cannot allocate device memory when they call the library: a
// host application that hands all device memory to its own pool and forbids
// cudaMalloc from plug-ins, code running while another component owns the
// allocator, or a latency-bound path where a first-call allocation (and the
// device synchronisation cudaFree implies) is not acceptable.  This variant
// keeps its scratch -- the digit planes of X and Y and the tile list -- in a
// fixed file-scope device array instead of the library's workspace, and calls
// no allocating routine.  The caller still passes X, Y and C.
namespace aat {
namespace {

// 32 MiB of device memory, held by every GPU that loads the library until the
// process exits.  m = n = k = 1024 with 4 digit planes (p = 2^31 - 1) needs
// 16 MiB of it.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
// Status word of this entry point's bounded waits (cleared by every call).
static __device__ int32_t g_noalloc_status;

struct NoAllocDevice {
  bool ready = false;
  unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
  int32_t *status = nullptr;         // device address of g_noalloc_status
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// The tile list, row-major, written on the device: no host buffer, no copy.
__global__ void noalloc_tiles_kernel(int2 *tiles, int TI, int TJ) {
  const int total = TI * TJ;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x)
    tiles[t] = make_int2(t / TJ, t - (t / TJ) * TJ);
}

// Device addresses of the scratch array and status word on the current
// device, looked up once per device with that device current.
int noalloc_device(NoAllocDevice *out) {
  int dev = 0;
  cudaError_t ce;
  if ((ce = cudaGetDevice(&dev)) != cudaSuccess || dev < 0 || dev >= 64)
    return report_error(AAT_ECUDA, "no current device");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice &d = g_noalloc_dev[dev];
  if (!d.ready) {
    // the host names of the device arrays are not device addresses
    void *ptr = nullptr;
    if ((ce = cudaGetSymbolAddress(&ptr, g_noalloc_scratch)) != cudaSuccess)
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    d.scratch = (unsigned char *)ptr;
    if ((ce = cudaGetSymbolAddress(&ptr, g_noalloc_status)) != cudaSuccess)
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    d.status = (int32_t *)ptr;
    d.ready = true;
  }
  *out = d;
  return AAT_OK;
}

}  // namespace

// Forgets the looked-up addresses (library shutdown): the next call looks
// them up again, in case the context was torn down in between.
void noalloc_forget() {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  for (NoAllocDevice &d : g_noalloc_dev) d = NoAllocDevice();
}

// The allocation-free entry point's status word on the current device
// (AAT_OK or AAT_ETIMEOUT; AAT_OK if it never ran there), cleared with reset.
// The caller has synchronised the device.
int noalloc_status(int reset) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return AAT_OK;
  int32_t *st = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_dev[dev].ready) st = g_noalloc_dev[dev].status;
  }
  if (!st) return AAT_OK;
  int32_t v = 0;
  if (cudaMemcpy(&v, st, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return AAT_ECUDA;
  if (reset) cudaMemset(st, 0, sizeof(int32_t));
  return v;
}

}  // namespace aat

extern "C" AAT_API int aat_gemm_modp_noalloc(const int32_t *X, int64_t ldx, const int32_t *Y,
                                             int64_t ldy, int64_t m, int64_t n, int64_t k,
                                             uint32_t p, int32_t *C, int64_t ldc, void *stream) {
  using namespace aat;
  if (m < 0 || n < 0 || k < 0) return report_error(AAT_EINVAL, "negative size");
  if (ldx < std::max<int64_t>(k, 1) || ldy < std::max<int64_t>(k, 1) ||
      ldc < std::max<int64_t>(n, 1))
    return report_error(AAT_EINVAL, "stride smaller than the row length");
  if (m > 0 && n > 0 && (!C || (k > 0 && (!X || !Y)))) return report_error(AAT_EINVAL, "null pointer");
  int e = check_prime_arg(p);
  if (e) return e;
  if (m == 0 || n == 0) return AAT_OK;
  if ((e = check_gb300())) return e;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t ce;
  if (k == 0) {
    ce = cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)n * 4, (size_t)m, st);
    return ce == cudaSuccess ? AAT_OK : report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  const DigitSpec ds = digits_for_prime(p);
  const ModP mp = make_modp(p);
  const bool same = (X == Y && ldx == ldy && m == n);
  const int64_t ks = (k + 7) / 8 * 8;
  const int64_t TI = (m + BM - 1) / BM, TJ = (n + BN - 1) / BN;
  const size_t xbytes = round256((size_t)ds.L * m * ks * 2);
  const size_t ybytes = same ? 0 : round256((size_t)ds.L * n * ks * 2);
  const size_t tbytes = round256((size_t)TI * TJ * sizeof(int2));
  if (xbytes + ybytes + tbytes > kNoAllocScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "aat_gemm_modp_noalloc: m=%lld n=%lld k=%lld needs %zu bytes of scratch, more "
                  "than its fixed %zu bytes",
                  (long long)m, (long long)n, (long long)k, xbytes + ybytes + tbytes,
                  kNoAllocScratchBytes);
    return report_error(AAT_ERANGE, msg);
  }
  int dev = 0;
  if ((ce = cudaGetDevice(&dev)) != cudaSuccess) return report_error(AAT_ECUDA, "no current device");
  // first call on this device: look up the arrays' device addresses
  NoAllocDevice nd;
  if ((e = noalloc_device(&nd))) return e;
  Planes px, py;
  std::memset(&px, 0, sizeof(px));
  px.nbase = ds.L;
  px.ptr = (__nv_bfloat16 *)nd.scratch;
  px.rows = m;
  px.cols = k;
  px.kstride = ks;
  px.L = ds.L;
  py = px;
  if (!same) {
    py.ptr = (__nv_bfloat16 *)(nd.scratch + xbytes);
    py.rows = n;
  }
  int2 *tiles_dev = (int2 *)(nd.scratch + xbytes + ybytes);

  std::lock_guard<std::mutex> lock(g_mu);  // tensor-map encoder and kernel attribute
  if ((ce = get_encode()) != cudaSuccess) return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  // the status word must start at zero; planes and tiles are fully rewritten
  if ((ce = cudaMemsetAsync(nd.status, 0, sizeof(int32_t), st)) != cudaSuccess)
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  // tile list, row-major, written by a kernel (no host buffer to copy from)
  noalloc_tiles_kernel<<<(unsigned)std::min<int64_t>((TI * TJ + 255) / 256, 1024), 256, 0, st>>>(
      tiles_dev, (int)TI, (int)TJ);
  if ((ce = cudaGetLastError()) != cudaSuccess) return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  if ((ce = launch_split(X, ldx, m, k, mp, ds.b, px, st)) != cudaSuccess)
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  if (!same && (ce = launch_split(Y, ldy, n, k, mp, ds.b, py, st)) != cudaSuccess)
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));

  Params P;
  std::memset(&P, 0, sizeof(P));
  if (encode_planes(&P.tmx, px, BM) != cudaSuccess || encode_planes(&P.tmy, py, BN) != cudaSuccess)
    return report_error(AAT_ECUDA, "tensor map encoding failed");
  // the digit-pair groups of the shared builder (plain digit products, as
  // the scratch holds no pair-sum planes), ending with the final multiplier
  TcLeafArgs a;
  std::memset(&a, 0, sizeof(a));
  a.x = px;
  a.y = py;
  a.dx = a.dy = ds;
  a.dx.nsum = a.dy.nsum = 0;
  a.M = m;
  a.N = n;
  a.K = k;
  a.exact_bits = 24;
  a.lin = lin_of(1, 0, p);
  int ng = 0, nprod = 0;
  if (!build_groups(a, mp, P.g, &ng, &nprod))
    return report_error(AAT_ERANGE, "leaf product does not fit the group table");
  P.ng = ng;
  P.out = C;
  P.ldo = ldc;
  P.M = m;
  P.N = n;
  P.lower = 0;
  P.accumulate = 0;
  P.beta = P.beta_sh = 0;
  P.m = mp;
  P.status = nd.status;
  P.tiles = tiles_dev;
  P.ntiles = (int)(TI * TJ);
  if (!g_attr_set[dev]) {
    ce = cudaFuncSetAttribute(leaf_tc_kernel<kSingle, false, kEwLeaf>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Shape<false, kEwLeaf>::SMEM);
    if (ce != cudaSuccess) return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    g_attr_set[dev] = true;
  }
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(P.ntiles, sms));
  leaf_tc_kernel<kSingle, false, kEwLeaf>
      <<<grid, Shape<false, kEwLeaf>::THREADS, Shape<false, kEwLeaf>::SMEM, st>>>(P);
  ce = cudaGetLastError();
  return ce == cudaSuccess ? AAT_OK : report_error(AAT_ECUDA, cudaGetErrorString(ce));
}

// ---------------------------------------------------------------- test hook

extern "C" AAT_API int aatx_leaf_groups(uint32_t p, int64_t K, uint32_t flags, int exact_bits,
                                        int32_t *out, int max_groups, int *nprod) {
  using namespace aat;
  int e = check_prime_arg(p);
  if (e) return e;
  if (K <= 0 || !out || !nprod) return report_error(AAT_EINVAL, "bad arguments");
  DigitSpec ds = digits_for_prime(p);
  if (flags & AAT_DIGITS_PLAIN) ds.nsum = 0;
  TcLeafArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dx = a.dy = ds;
  a.x.nbase = a.y.nbase = ds.L;
  a.x.nsum = a.y.nsum = ds.nsum;
  a.x.L = a.y.L = ds.L + ds.nsum;
  a.M = a.N = 1;
  a.K = K;
  a.exact_bits = exact_bits > 0 ? exact_bits : 24;
  a.lin = lin_of(1, 0, p);
  std::vector<Group> g(MAX_GROUPS);
  int ng = 0;
  if (!build_groups(a, make_modp(p), g.data(), &ng, nprod))
    return report_error(AAT_ERANGE, "leaf product does not fit the group table");
  if (ng > max_groups) return report_error(AAT_ERANGE, "output too small");
  for (int i = 0; i < ng; ++i) {
    int32_t *o = out + 6 * i;
    o[0] = g[i].xp;
    o[1] = g[i].yp;
    o[2] = g[i].kb0;
    o[3] = g[i].kb1;
    o[4] = g[i].kchunk;
    o[5] = (int32_t)g[i].ratio;
  }
  return ng;
}

// ------------------------------------------------- failure-path test probe

namespace aat {
namespace {

// One thread waits, with the bounded wait the leaf kernels use, for a phase
// of a fresh mbarrier that nothing will ever complete; the wait gives up
// after limit_ns and records AAT_ETIMEOUT in `status`.  Nothing else runs.
__global__ void wait_probe_kernel(int32_t *status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  tc::mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::wait_bounded<false>(b, 0, &abort_flag, status, limit_ns);
}

}  // namespace
}  // namespace aat

extern "C" AAT_API int aatx_wait_probe(int which, int64_t limit_ns, void *stream) {
  using namespace aat;
  if (limit_ns <= 0 || limit_ns > 2000000000LL || (which != 0 && which != 1))
    return report_error(AAT_EINVAL, "which must be 0 or 1, limit in (0, 2 s]");
  int e = check_gb300();
  if (e) return e;
  int32_t *status = nullptr;
  if (which == 0) {
    status = device_status_ptr();
    if (!status) return report_error(AAT_ECUDA, "no device status word");
  } else {
    NoAllocDevice nd;
    if ((e = noalloc_device(&nd))) return e;
    status = nd.status;
  }
  wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(status, (unsigned long long)limit_ns);
  cudaError_t ce = cudaGetLastError();
  return ce == cudaSuccess ? AAT_OK : report_error(AAT_ECUDA, cudaGetErrorString(ce));
}
