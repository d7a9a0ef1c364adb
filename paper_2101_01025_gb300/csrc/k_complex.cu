// k_complex.cu -- the product of a complex matrix by its adjoint (Sec. 6.1,
// Algorithm 2, the "2M" method) on the tensor cores.
//
// A = Ar + i Ai (complex64, row-major).  With phi the conjugate transposition
// eps = i phi(i) = 1, and Algorithm 2 gives, from two real products
//     H = Ar Ai^T            (general, all n x n entries)
//     G = (Ar + Ai)(Ar + Ai)^T  (only Low(G) is needed),
// A A^H = (G - H - H^T) + i (H^T - H).  With phi the transposition,
// eps = i i = -1: G = (Ar + Ai)(Ar - Ai)^T (Low only) and
// A A^T = (G + H - H^T) + i (H + H^T).
//
// Real products run on tcgen05 with BF16 operands: every real input is split
// into P BF16 pieces x = x0 + x1 + x2 (x1 = bf16(x - x0), ...), and the
// product keeps the piece products of weight >= 2^-16: P = 3 gives x0y0,
// x0y1, x1y0, x0y2, x1y1, x2y0 (close to FP32), P = 2 gives x0y0, x0y1, x1y0,
// P = 1 is plain BF16.  The piece products of a tile accumulate in FP32 in
// TMEM (sign per product from the instruction's negate bit), drained every
// 8 K blocks into FP32 registers (round to nearest) while the next chunk
// accumulates in the other TMEM buffer.  The Hermitian diagonal sum_l |a_il|^2 is
// computed in FP64 (real and >= 0).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/aat.h"
#include "common.cuh"
#include "tc_ptx.cuh"

namespace aat {

namespace {

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + EPI_WARPS * 32;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = 256;
constexpr int MAX_FGROUPS = 48;
// bit 13 of the instruction descriptor negates A
constexpr uint32_t NEG_A = 1u << 13;

struct FGroup {
  int16_t xp, yp;  // planes of X and Y
  int32_t neg;     // subtract this product
};

// One product of a batched launch (its maps live in global memory).
struct alignas(64) FJobDesc {
  CUtensorMap tmx, tmy;
  float *out;
  int64_t ldo, M, N;
  int lower, kblocks, goff, ng;  // its groups: gtab[goff .. goff + ng)
};

struct FParams {
  CUtensorMap tmx;  // 3D {K, rows, plane}, box {64, 128, 1}
  CUtensorMap tmy;  // 3D {K, rows, plane}, box {64, 256, 1} (CTA pair: {64, 128, 1})
  FGroup g[MAX_FGROUPS];
  int ng;
  int kblocks;
  int kchunk;  // K blocks per FP32 TMEM accumulation before it is drained
  float *out;
  int64_t ldo, M, N;
  const int2 *tiles;
  int ntiles;
  int lower;
  int32_t *status;
  // batched launches: tiles are (job, I, J) and every job carries its own
  // maps, groups, K and output
  const FJobDesc *jobs;
  const int4 *btiles;
  const FGroup *gtab;
};

// What one tile of a launch works on.
struct FJob {
  const CUtensorMap *tmx, *tmy;
  const FGroup *g;
  int ng, kblocks, lower, I, J;
  float *out;
  int64_t ldo, M, N;
};

template <bool BATCH>
__device__ __forceinline__ FJob fjob(const FParams &P, int t) {
  FJob j;
  if constexpr (BATCH) {
    const int4 tl = P.btiles[t];
    const FJobDesc &d = P.jobs[tl.x];
    j.tmx = &d.tmx;
    j.tmy = &d.tmy;
    j.g = P.gtab + d.goff;
    j.ng = d.ng;
    j.kblocks = d.kblocks;
    j.lower = d.lower;
    j.out = d.out;
    j.ldo = d.ldo;
    j.M = d.M;
    j.N = d.N;
    j.I = tl.y;
    j.J = tl.z;
  } else {
    const int2 tl = P.tiles[t];
    j.tmx = &P.tmx;
    j.tmy = &P.tmy;
    j.g = P.g;
    j.ng = P.ng;
    j.kblocks = P.kblocks;
    j.lower = P.lower;
    j.out = P.out;
    j.ldo = P.ldo;
    j.M = P.M;
    j.N = P.N;
    j.I = tl.x;
    j.J = tl.y;
  }
  return j;
}

// out = sum_g (+-) X_{xp(g)} Y_{yp(g)}^T in FP32, one TMEM accumulation per
// output tile.  Same CTA organisation as the modular leaf kernel, in the
// same two forms: one CTA per 128 x 256 tile (4 stages of 48 KB), or a CTA
// pair per 256 x 256 tile (tcgen05 cta_group::2; each CTA holds 128 rows of
// X and 128 rows of Y per stage, 6 stages of 32 KB; the leader issues the
// M=256 MMAs, both CTAs' copies complete on its barrier, its commits
// multicast to both, and the epilogues of both release a buffer on its
// barrier).
template <bool PAIR>
struct FShape {
  static constexpr int TM = PAIR ? 256 : 128;
  static constexpr int YROWS = PAIR ? 128 : 256;
  static constexpr int STAGES = PAIR ? 6 : 4;
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = YROWS * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  // + 256 bytes of barriers + a per-warp 32 x 17 FP32 staging area of the
  // output stores
  static constexpr size_t XS_BYTES = (size_t)EPI_WARPS * 32 * 17 * 4;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 256 + XS_BYTES;
  // kind::f16, FP32 accumulator, BF16 A and B, K-major, N = 256, M = TM
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
};

template <bool PAIR, bool BATCH>
__global__ void __launch_bounds__(THREADS, 1) leaf_f32_kernel(const __grid_constant__ FParams P) {
  using S = FShape<PAIR>;
  constexpr int STAGES = S::STAGES;
  extern __shared__ uint8_t smem_raw[];
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
  if constexpr (PAIR) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int stage = 0, issued = 0;
      uint32_t ph = 0;
      bool ok = true;
      const uint32_t full0 = PAIR ? map_to_rank(FULL(0), 0) : FULL(0);
      for (int t = (int)unit0; t < P.ntiles && ok; t += (int)nunits) {
        const FJob jb = fjob<BATCH>(P, t);
        const int rowx = jb.I * S::TM + (int)rank * BM;
        const int rowy = jb.J * BN + (int)rank * S::YROWS;
        for (int gi = 0; gi < jb.ng && ok; ++gi) {
          const FGroup g = jb.g[gi];
          for (int kb = 0; kb < jb.kblocks; ++kb) {
            if (!wait_bounded<PAIR>(EMPTY(stage), ph ^ 1u, abort_flag, P.status)) {
              ok = false;
              break;
            }
            const uint32_t sa = sbase + (uint32_t)(stage * S::STAGE_BYTES);
            const uint32_t fb = full0 + 8u * (uint32_t)stage;
            if constexpr (PAIR) {
              if (leader) mbar_expect_tx(FULL(stage), (uint32_t)(2 * S::STAGE_BYTES));
              tma_load_3d_pair(sa, jb.tmx, fb, kb * BK, rowx, g.xp);
              tma_load_3d_pair(sa + S::A_BYTES, jb.tmy, fb, kb * BK, rowy, g.yp);
            } else {
              mbar_expect_tx(FULL(stage), (uint32_t)S::STAGE_BYTES);
              tma_load_3d(sa, jb.tmx, fb, kb * BK, rowx, g.xp);
              tma_load_3d(sa + S::A_BYTES, jb.tmy, fb, kb * BK, rowy, g.yp);
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
    if (leader) {  // MMA issuer: the whole warp runs the loop, one elected lane issues
      int stage = 0;
      uint32_t ph = 0, chunk = 0;
      bool ok = true;
      // shared-memory descriptors: stage and K step move the start-address
      // field (16-byte units) only, so they are formed by adds
      const uint64_t da0 = sw128_desc(sbase);
      for (int t = (int)unit0; t < P.ntiles && ok; t += (int)nunits) {
        const FJob jb = fjob<BATCH>(P, t);
        // chunks of kchunk K blocks over the flattened (group, K block)
        // sequence: a chunk may span two groups (one FP32 sum)
        const int total = jb.ng * jb.kblocks;
        int gi = 0, kbi = 0;
        uint32_t idesc = S::IDESC | ((jb.ng > 0 && jb.g[0].neg) ? NEG_A : 0u);
        for (int q0 = 0; q0 < total && ok; q0 += P.kchunk) {
          const int q1 = min(q0 + P.kchunk, total);
          const uint32_t buf = chunk & 1u, use = chunk >> 1;
          if (!__all_sync(0xffffffffu, wait_bounded<PAIR>(AEMPTY(buf), (use & 1u) ^ 1u, abort_flag,
                                                          P.status))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dt = tmem + buf * ACC_COLS;
          for (int q = q0; q < q1; ++q) {
            if (!__all_sync(0xffffffffu, wait_bounded<PAIR>(FULL(stage), ph, abort_flag, P.status))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t da = da0 + (uint64_t)((uint32_t)(stage * S::STAGE_BYTES) >> 4);
            const uint64_t db = da + (uint64_t)(S::A_BYTES >> 4);
            if (elect_one()) {
#pragma unroll
              for (int s = 0; s < BK / 16; ++s) {
                const uint32_t acc = (q > q0 || s > 0) ? 1u : 0u;
                if constexpr (PAIR)
                  tc_mma_pair(dt, da + 2u * s, db + 2u * s, idesc, acc);
                else
                  tc_mma(dt, da + 2u * s, db + 2u * s, idesc, acc);
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
            if (++kbi == jb.kblocks) {
              kbi = 0;
              if (++gi < jb.ng) idesc = S::IDESC | (jb.g[gi].neg ? NEG_A : 0u);
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
  } else {  // epilogue: chunks -> FP32 registers -> global (lower if asked)
    const int e = warp - 2;
    const int quarter = warp & 3;
    const int chalf = e >> 2;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;

    const uint32_t aempty0 = PAIR ? map_to_rank(AEMPTY(0), 0) : AEMPTY(0);
    float *xs = reinterpret_cast<float *>(smem + (size_t)STAGES * S::STAGE_BYTES + 256) + e * 32 * 17;
    uint32_t chunk = 0;
    bool ok = true;
    for (int t = (int)unit0; t < P.ntiles && ok; t += (int)nunits) {
      const FJob jb = fjob<BATCH>(P, t);
      const int nchunks = (jb.ng * jb.kblocks + P.kchunk - 1) / P.kchunk;
      float acc[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
      for (int c = 0; c < nchunks; ++c) {
        const uint32_t buf = chunk & 1u, use = chunk >> 1;
        if (!wait_bounded<PAIR>(AFULL(buf), use & 1u, abort_flag, P.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + lane_base + buf * ACC_COLS + (uint32_t)(chalf * 128);
        tmem_accum16f<0>(ta, acc);
        tmem_accum16f<16>(ta + 16u, acc);
        tmem_accum16f<32>(ta + 32u, acc);
        tmem_accum16f<48>(ta + 48u, acc);
        tmem_accum16f<64>(ta + 64u, acc);
        tmem_accum16f<80>(ta + 80u, acc);
        tmem_accum16f<96>(ta + 96u, acc);
        tmem_accum16f<112>(ta + 112u, acc);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR)
            mbar_arrive_cluster(aempty0 + 8u * buf);
          else
            mbar_arrive(AEMPTY(buf));
        }
        ++chunk;
      }
      if (!ok) break;
      const int64_t row = (int64_t)jb.I * S::TM + (int64_t)rank * BM + quarter * 32 + lane;
      const int64_t col0 = (int64_t)jb.J * BN + chalf * 128;
      // rows 16-byte aligned: each thread stores its row segment with
      // 16-byte stores
      if (((reinterpret_cast<uintptr_t>(jb.out) | (uintptr_t)(jb.ldo * 4)) & 15) == 0) {
        int64_t lim = jb.N - col0;
        if (jb.lower) lim = min(lim, row - col0 + 1);
        if (row < jb.M && lim > 0) {
          float *orow = jb.out + row * jb.ldo + col0;
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int cc = 4 * q;
            if (cc + 4 <= lim) {
              *reinterpret_cast<float4 *>(orow + cc) =
                  make_float4(acc[cc], acc[cc + 1], acc[cc + 2], acc[cc + 3]);
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (cc + j < lim) orow[cc + j] = acc[cc + j];
            }
            asm volatile("" ::: "memory");
          }
        }
        continue;
      }
      // otherwise coalesced through shared memory: 16 columns of the warp's
      // 32 rows at a time, two contiguous 64-byte row segments per store
      const int64_t row0 = row - lane;
      const int mlim = (int)max((int64_t)0, min((int64_t)32, jb.M - row0));
      const int nlim = (int)max((int64_t)0, min((int64_t)128, jb.N - col0));
      const int dl = jb.lower ? (int)max((int64_t)-256, min((int64_t)256, row0 - col0)) : 1 << 20;
      float *const base = jb.out + row0 * jb.ldo + col0;
      const int64_t ldo = jb.ldo;
#pragma unroll
      for (int cb = 0; cb < 128; cb += 16) {
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 16; ++j) xs[lane * 17 + j] = acc[cb + j];
        __syncwarp();
#pragma unroll 1
        for (int i = 0; i < 16; ++i) {
          const int rr = 2 * i + (lane >> 4), cl = cb + (lane & 15);
          if (rr < mlim && cl < nlim && cl - rr <= dl) base[(int64_t)rr * ldo + cl] = xs[rr * 17 + (lane & 15)];
        }
      }
    }
  }

  __syncthreads();
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

// ----------------------------------------------------------- split / combine

struct CSplitOut {
  Planes re, im, s, d;  // pieces of Re, Im, Re + Im, Re - Im (each optional)
};

// Up to 4 consecutive values of a row (zeros past nv), 16-byte loads when the
// row is aligned.
__device__ __forceinline__ void cload4(const float2 *__restrict__ a_row, int64_t c0, int nv,
                                       float2 (&a)[4]) {
  if (nv == 4 && (reinterpret_cast<uintptr_t>(a_row) & 15) == 0) {
    const float4 u0 = reinterpret_cast<const float4 *>(a_row + c0)[0];
    const float4 u1 = reinterpret_cast<const float4 *>(a_row + c0)[1];
    a[0] = make_float2(u0.x, u0.y);
    a[1] = make_float2(u0.z, u0.w);
    a[2] = make_float2(u1.x, u1.y);
    a[3] = make_float2(u1.z, u1.w);
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v) a[v] = v < nv ? a_row[c0 + v] : make_float2(0.f, 0.f);
  }
}

// The pieces of 4 consecutive values a[0..nv) of row r, columns c0.., into
// every plane set of o: one 8-byte store per plane (kstride is a multiple of
// 8); a ragged last quad stores element by element.
__device__ __forceinline__ void csplit_store(const float2 (&a)[4], int64_t r, int64_t c0, int nv,
                                             int np, const CSplitOut &o) {
  const Planes *outs[4] = {&o.re, &o.im, &o.s, &o.d};
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const Planes &P = *outs[w];
    if (!P.ptr) continue;
    float x[4];
#pragma unroll
    for (int v = 0; v < 4; ++v)
      x[v] = w == 0 ? a[v].x : w == 1 ? a[v].y : w == 2 ? a[v].x + a[v].y : a[v].x - a[v].y;
    // pieces of two values per conversion instruction (round to nearest),
    // the rest carried in FP32 (exact: each rest is an FP32 difference of a
    // value and its BF16 rounding)
    __nv_bfloat162 lo[3], hi[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q < np) {
        lo[q] = __floats2bfloat162_rn(x[0], x[1]);
        hi[q] = __floats2bfloat162_rn(x[2], x[3]);
        const float2 fl = __bfloat1622float2(lo[q]), fh = __bfloat1622float2(hi[q]);
        x[0] -= fl.x;
        x[1] -= fl.y;
        x[2] -= fh.x;
        x[3] -= fh.y;
      }
    }
    const int64_t plane = P.rows * P.kstride;
    __nv_bfloat16 *dst = P.ptr + r * P.kstride + c0;
    for (int q = 0; q < np; ++q) {
      if (nv == 4) {
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&lo[q]);
        u.y = *reinterpret_cast<uint32_t *>(&hi[q]);
        *reinterpret_cast<uint2 *>(dst + q * plane) = u;
      } else {
        const __nv_bfloat16 pv[4] = {lo[q].x, lo[q].y, hi[q].x, hi[q].y};
        for (int v = 0; v < nv; ++v) dst[q * plane + v] = pv[v];
      }
    }
  }
}

// One thread per 4 consecutive columns of a row (rows over blockIdx.y, a
// grid-stride loop over column quads).
__device__ __forceinline__ void csplit_quad(const float2 *__restrict__ a_row, int64_t r,
                                            int64_t q4, int64_t cols, int np, const CSplitOut &o) {
  const int64_t c0 = 4 * q4;
  const int nv = (int)min((int64_t)4, cols - c0);
  float2 a[4];
  cload4(a_row, c0, nv, a);
  csplit_store(a, r, c0, nv, np, o);
}

__global__ void csplit_kernel(const float2 *__restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                              int np, CSplitOut o) {
  const int64_t cq = (cols + 3) / 4;
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y)
    for (int64_t q4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q4 < cq;
         q4 += (int64_t)gridDim.x * blockDim.x)
      csplit_quad(A + r * lda, r, q4, cols, np, o);
}

// ------------------------------------------------ batched A A^H / A A^T (2M)

// One problem of the batched 2M sequence: its input, pieces, plane sets,
// the products H and G and the output, and the first block it owns in each
// of the batched element-wise launches.
struct CBProb {
  const float2 *A;
  int64_t lda, n, k;
  int np, herm;
  CSplitOut ox, oy;
  float *H, *G;
  float2 *C;
  int64_t ldc;
  int split_first, comb_first, diag_first;
};

constexpr int kCSplitRows = 8, kDiagRows = 8;

__device__ __forceinline__ int cb_find(const CBProb *pr, int count, int b, int which) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    const int f = which == 0 ? pr[mid].split_first : which == 1 ? pr[mid].comb_first
                                                                : pr[mid].diag_first;
    if (f <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// both plane sets of kCSplitRows rows of one problem per block
__global__ void csplit_batch_kernel(const CBProb *__restrict__ pr, int count) {
  const CBProb &q = pr[cb_find(pr, count, blockIdx.x, 0)];
  const int64_t r0 = (int64_t)(blockIdx.x - q.split_first) * kCSplitRows;
  const uint32_t nr = (uint32_t)min((int64_t)kCSplitRows, q.n - r0);
  const uint32_t cq = (uint32_t)((q.k + 3) / 4);
  // the block's rows x column quads as one index: every thread has work
  // when the rows are short (32-bit index arithmetic: nr * cq < 8 * 2^28)
  for (uint32_t t = threadIdx.x; t < nr * cq; t += blockDim.x) {
    const uint32_t ri = t / cq;
    const int64_t r = r0 + ri, q4 = t - ri * cq;
    csplit_quad(q.A + r * q.lda, r, q4, q.k, q.np, q.ox);
    csplit_quad(q.A + r * q.lda, r, q4, q.k, q.np, q.oy);
  }
}

// The combination of Algorithm 2 for one tile pair {(I, J), (J, I)}, I >= J,
// writing Low(C) (complex64):  herm: Re = G - H - H^T, Im = H^T - H;
// otherwise Re = G + H - H^T, Im = H + H^T.
constexpr int T = 32;
__device__ __forceinline__ void combine2m_tile(const float *__restrict__ G,
                                               const float *__restrict__ H, int64_t ldw,
                                               int64_t n, float2 *C, int64_t ldc, int herm,
                                               int64_t pid, float (&hij)[T][T + 1],
                                               float (&hji)[T][T + 1]) {
  const int64_t ntiles = (n + T - 1) / T;
  int64_t I, J;
  tri_index(pid, I, J);
  if (I >= ntiles) return;
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  const int64_t r0 = I * T, c0 = J * T;
  for (int yy = ty; yy < T; yy += 8) {
    int64_t r = r0 + yy, c = c0 + tx;
    if (r < n && c < n) hij[yy][tx] = H[r * ldw + c];
    int64_t r2 = c0 + yy, c2 = r0 + tx;
    if (r2 < n && c2 < n) hji[yy][tx] = H[r2 * ldw + c2];
  }
  __syncthreads();
  for (int yy = ty; yy < T; yy += 8) {
    int64_t r = r0 + yy, c = c0 + tx;
    if (r < n && c < n && c <= r) {
      const float h = hij[yy][tx], ht = hji[tx][yy], g = G[r * ldw + c];
      float2 v;
      if (herm) {
        v.x = g - h - ht;
        v.y = ht - h;
      } else {
        v.x = g + h - ht;
        v.y = h + ht;
      }
      C[r * ldc + c] = v;
    }
  }
}

__global__ void combine2m_kernel(const float *__restrict__ G, const float *__restrict__ H,
                                 int64_t ldw, int64_t n, float2 *C, int64_t ldc, int herm) {
  __shared__ float hij[T][T + 1];
  __shared__ float hji[T][T + 1];
  combine2m_tile(G, H, ldw, n, C, ldc, herm, blockIdx.x, hij, hji);
}

__global__ void combine2m_batch_kernel(const CBProb *__restrict__ pr, int count) {
  __shared__ float hij[T][T + 1];
  __shared__ float hji[T][T + 1];
  const CBProb &q = pr[cb_find(pr, count, blockIdx.x, 1)];
  combine2m_tile(q.G, q.H, q.n, q.n, q.C, q.ldc, q.herm, (int64_t)(blockIdx.x - q.comb_first),
                 hij, hji);
}

// x·x added to the unevaluated float pair hi + lo without rounding error:
// the product by its FMA residual (x·x = p + e exactly) and the sum by
// Knuth's TwoSum (hi + p = s + err exactly).  The _rn intrinsics keep the
// compiler from contracting any of these steps into an FMA.
__device__ __forceinline__ void sq_acc(float x, float &hi, float &lo) {
  const float p = __fmul_rn(x, x);
  const float e = fmaf(x, x, -p);
  const float s = __fadd_rn(hi, p);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// Re C[row][row] = Σ_l |a_l|², one warp per row.  Each lane sums its
// columns' squares as a float pair (about 48 significant bits: the only
// rounding is in lo, whose terms are each below ulp(hi)), two pairs per lane
// for the real and imaginary parts so the two dependency chains overlap;
// the lanes' pairs are added in FP64.  This part's FP64 pipe is a small
// fraction of its FP32 pipe: an FP64 multiply-add per square (and two
// conversions) held the kernel far below the memory rate.
__device__ __forceinline__ void herm_diag_row(const float2 *__restrict__ A, int64_t lda,
                                              int64_t n, int64_t k, float2 *C, int64_t ldc,
                                              int64_t row) {
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float2 *a_row = A + row * lda;
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
  int64_t l = 0;
  if ((reinterpret_cast<uintptr_t>(a_row) & 15) == 0) {
    // two complex values per lane per 16-byte load, four loads in flight
    const float4 *a4 = reinterpret_cast<const float4 *>(a_row);
    const int64_t k2 = k / 2;
    int64_t q = lane;
    for (; q + 96 < k2; q += 128) {
      const float4 v0 = a4[q], v1 = a4[q + 32], v2 = a4[q + 64], v3 = a4[q + 96];
      sq_acc(v0.x, h0, l0); sq_acc(v0.y, h1, l1); sq_acc(v0.z, h0, l0); sq_acc(v0.w, h1, l1);
      sq_acc(v1.x, h0, l0); sq_acc(v1.y, h1, l1); sq_acc(v1.z, h0, l0); sq_acc(v1.w, h1, l1);
      sq_acc(v2.x, h0, l0); sq_acc(v2.y, h1, l1); sq_acc(v2.z, h0, l0); sq_acc(v2.w, h1, l1);
      sq_acc(v3.x, h0, l0); sq_acc(v3.y, h1, l1); sq_acc(v3.z, h0, l0); sq_acc(v3.w, h1, l1);
    }
    for (; q < k2; q += 32) {
      const float4 v = a4[q];
      sq_acc(v.x, h0, l0); sq_acc(v.y, h1, l1); sq_acc(v.z, h0, l0); sq_acc(v.w, h1, l1);
    }
    l = 2 * k2;  // an odd last column is left to the loop below
  }
  for (l += lane; l < k; l += 32) {
    const float2 a = a_row[l];
    sq_acc(a.x, h0, l0);
    sq_acc(a.y, h1, l1);
  }
  double s = ((double)h0 + (double)l0) + ((double)h1 + (double)l1);
  for (int off = 16; off; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) C[row * ldc + row] = make_float2((float)s, 0.0f);
}

__global__ void herm_diag_kernel(const float2 *__restrict__ A, int64_t lda, int64_t n, int64_t k,
                                 float2 *C, int64_t ldc) {
  herm_diag_row(A, lda, n, k, C, ldc, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32);
}

// one warp per row, kDiagRows rows of one Hermitian problem per block
__global__ void herm_diag_batch_kernel(const CBProb *__restrict__ pr, int count) {
  const CBProb &q = pr[cb_find(pr, count, blockIdx.x, 2)];
  const int64_t row = (int64_t)(blockIdx.x - q.diag_first) * kDiagRows + threadIdx.x / 32;
  herm_diag_row(q.A, q.lda, q.n, q.k, q.C, q.ldc, row);
}

// ------------------------------------------------------------------ host

PFN_cuTensorMapEncodeTiled_v12000 g_encode_c = nullptr;
std::mutex g_mu_c;
std::map<std::tuple<int, int64_t, int64_t, int, int>, std::pair<int2 *, int>> g_tiles_c;
std::map<int, bool> g_attr_c;
std::map<int, int> g_pair_units_c;

cudaError_t encode_c(CUtensorMap *tm, const Planes &P, int box_rows) {
  if (!g_encode_c) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode_c = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  cuuint64_t dims[3] = {(cuuint64_t)P.cols, (cuuint64_t)P.rows, (cuuint64_t)P.L};
  cuuint64_t strides[2] = {(cuuint64_t)P.kstride * 2, (cuuint64_t)(P.rows * P.kstride * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode_c(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)P.ptr, dims, strides,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// tm: tile height (128, or 256 for CTA pairs).  Bands of 2048 output rows
// swept column by column: the tiles in flight at one time (about a wave of
// consecutive entries) span few row and column panels, which they share
// through L2.
cudaError_t tiles_c(int dev, int64_t M, int64_t N, int lower, int tm, int2 **out, int *count) {
  auto key = std::make_tuple(dev, M, N, lower, tm);
  auto it = g_tiles_c.find(key);
  if (it != g_tiles_c.end()) {
    *out = it->second.first;
    *count = it->second.second;
    return cudaSuccess;
  }
  const int64_t TI = (M + tm - 1) / tm, TJ = (N + BN - 1) / BN;
  const int64_t band = std::max<int64_t>(1, 2048 / tm);
  std::vector<int2> v;
  for (int64_t bi = 0; bi < TI; bi += band)
    for (int64_t j = 0; j < TJ; ++j)
      for (int64_t i = bi; i < std::min(TI, bi + band); ++i) {
        if (lower && j * BN > i * tm + tm - 1) continue;
        v.push_back(make_int2((int)i, (int)j));
      }
  int2 *d = nullptr;
  if (!v.empty()) {
    cudaError_t e = cudaMalloc(&d, v.size() * sizeof(int2));
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpy(d, v.data(), v.size() * sizeof(int2), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return e;
  }
  g_tiles_c[key] = std::make_pair(d, (int)v.size());
  *out = d;
  *count = (int)v.size();
  return cudaSuccess;
}

int grid_c(int64_t total, int threads) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (total + threads - 1) / threads;
  want = std::min<int64_t>(want, (int64_t)sms * 16);
  return (int)std::max<int64_t>(want, 1);
}

// Co-resident CTA pairs of the pair kernel on this device (0: none).
int pair_units_c(int dev) {
  auto it = g_pair_units_c.find(dev);
  if (it != g_pair_units_c.end()) return it->second;
  int units = 0;
  if (cudaFuncSetAttribute(leaf_f32_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)FShape<true>::SMEM) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = FShape<true>::SMEM;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&units, leaf_f32_kernel<true, false>, &cfg) != cudaSuccess)
      units = 0;
  }
  cudaGetLastError();
  g_pair_units_c[dev] = units;
  return units;
}

}  // namespace

// The piece products kept for P pieces per operand (weight >= 2^-16).
static int piece_pairs(int np, int (*pairs)[2]) {
  static const int all[6][2] = {{0, 0}, {0, 1}, {1, 0}, {0, 2}, {1, 1}, {2, 0}};
  const int cnt = np == 3 ? 6 : (np == 2 ? 3 : 1);
  for (int i = 0; i < cnt; ++i) {
    pairs[i][0] = all[i][0];
    pairs[i][1] = all[i][1];
  }
  return cnt;
}

// out (M x N fp32) = sum over terms (+-) X_a Y_b^T, each term expanded into its
// piece products.  terms: (x plane set, y plane set, negate).
struct FTerm {
  const Planes *x, *y;
  bool neg;
};

// np: pieces stored per plane set; keep: pieces whose pair products are kept
// (keep <= np: the leading pieces of a longer split are the same values).
static cudaError_t launch_leaf_f32(const std::vector<FTerm> &terms, int np, int keep, int64_t M,
                                   int64_t N, int64_t K, float *out, int64_t ldo, int lower,
                                   cudaStream_t st) {
  if (M <= 0 || N <= 0 || terms.empty()) return cudaSuccess;
  // every term must use the same two plane buffers: X planes in one
  // tensor map, Y planes in the other (plane index = set * np + piece)
  std::lock_guard<std::mutex> lock(g_mu_c);
  int dev = 0;
  cudaGetDevice(&dev);
  // the form: CTA pairs when the 256 x 256 tiles keep every co-resident pair
  // busy (AAT_LEAF_PAIR=0/1 forces one form, as for the modular leaf)
  const int units = pair_units_c(dev);
  bool pair = false;
  if (units > 0 && M >= 256) {
    const int64_t pt = ((M + 255) / 256) * ((N + BN - 1) / BN);
    const char *ev = getenv("AAT_LEAF_PAIR");
    pair = ev ? atoi(ev) > 0 : (lower ? pt / 2 : pt) >= units;
  }
  FParams *P = new FParams;
  std::memset(P, 0, sizeof(FParams));
  cudaError_t e;
  const Planes &X = *terms[0].x, &Y = *terms[0].y;
  if ((e = encode_c(&P->tmx, X, BM)) != cudaSuccess ||
      (e = encode_c(&P->tmy, Y, pair ? FShape<true>::YROWS : FShape<false>::YROWS)) !=
          cudaSuccess) {
    delete P;
    return e;
  }
  int pairs[6][2];
  const int npairs = piece_pairs(std::min(keep, np), pairs);
  int ng = 0;
  for (const FTerm &t : terms) {
    const int xs = (int)((t.x->ptr - X.ptr) / (X.rows * X.kstride));  // plane offset
    const int ys = (int)((t.y->ptr - Y.ptr) / (Y.rows * Y.kstride));
    for (int q = 0; q < npairs; ++q) {
      if (ng >= MAX_FGROUPS) {
        delete P;
        return cudaErrorInvalidValue;
      }
      P->g[ng].xp = (int16_t)(xs + pairs[q][0]);
      P->g[ng].yp = (int16_t)(ys + pairs[q][1]);
      P->g[ng].neg = t.neg ? 1 : 0;
      ++ng;
    }
  }
  P->ng = ng;
  P->kblocks = (int)((K + BK - 1) / BK);
  // The tensor core's FP32 accumulation is drained into round-to-nearest
  // FP32 registers every 8 K blocks (512 products).  Measured at n = k =
  // 8192 (A A^H, 3 pieces, N(0,1) entries, 3000 sampled entries against the
  // FP64 oracle): relative error 6.9e-7 / 5.2e-7 / 5.9e-7 / 1.0e-6 draining
  // every 2 / 4 / 8 / 16 K blocks, time 9.23 / 8.41 / 8.01 / 7.82 ms.
  P->kchunk = 8;
  P->out = out;
  P->ldo = ldo;
  P->M = M;
  P->N = N;
  P->lower = lower;
  P->status = device_status_ptr();
  int2 *tiles = nullptr;
  int nt = 0;
  if ((e = tiles_c(dev, M, N, lower, pair ? 256 : 128, &tiles, &nt)) != cudaSuccess) {
    delete P;
    return e;
  }
  P->tiles = tiles;
  P->ntiles = nt;
  if (!g_attr_c[dev]) {
    if ((e = cudaFuncSetAttribute(leaf_f32_kernel<false, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)FShape<false>::SMEM)) != cudaSuccess) {
      delete P;
      return e;
    }
    g_attr_c[dev] = true;
  }
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nt > 0) {
    const double macs = lower ? 0.5 * (double)M * (double)(M + 1) * K : (double)M * N * K;
    ProfScope prof(AAT_K_LEAF_F32, st, 2.0 * ng * macs);
    if (pair) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(2 * std::max(1, std::min(nt, units)), 1, 1);
      cfg.blockDim = dim3(THREADS, 1, 1);
      cfg.dynamicSmemBytes = FShape<true>::SMEM;
      cfg.stream = st;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, leaf_f32_kernel<true, false>, *P);
      if (e != cudaSuccess) {
        delete P;
        return e;
      }
    } else {
      leaf_f32_kernel<false, false><<<std::max(1, std::min(nt, sms)), THREADS, FShape<false>::SMEM, st>>>(*P);
    }
  }
  delete P;
  return cudaGetLastError();
}

// ------------------------------------ several real products in one launch

// One real product of a fused launch: out (M x N FP32, row stride ldo) =
// X_xs Y_ys^T over the piece pairs of `keep` pieces, where X_xs is plane set
// xs of the plane buffer X (np pieces per set), likewise Y; lower: only the
// tiles on or below the diagonal.
struct FusedJob {
  const Planes *X, *Y;
  int xs, ys, keep;
  float *out;
  int64_t ldo, M, N;
  int lower;
};

constexpr int MAX_FUSED = 16;
constexpr int MAX_FUSED_GROUPS = MAX_FUSED * 6;

// The job table of a fused launch, passed by value to one small kernel that
// writes it into device memory (no host buffer, no copy).
struct FusedTable {
  FJobDesc jobs[MAX_FUSED];
  FGroup g[MAX_FUSED_GROUPS];
  int njobs, ng;
};

size_t fused_table_bytes() {
  return ((sizeof(FJobDesc) * MAX_FUSED + 255) & ~(size_t)255) + sizeof(FGroup) * MAX_FUSED_GROUPS;
}

namespace {

__global__ void fused_table_kernel(const __grid_constant__ FusedTable T, FJobDesc *jobs,
                                   FGroup *gtab) {
  for (int i = threadIdx.x; i < T.njobs; i += blockDim.x) jobs[i] = T.jobs[i];
  for (int i = threadIdx.x; i < T.ng; i += blockDim.x) gtab[i] = T.g[i];
}

// Tile lists of fused launches, per device, tile height and job shapes: each
// job's tiles in bands of 2048 rows swept column by column, jobs in order.
std::map<std::vector<int64_t>, std::pair<int4 *, int>> g_ftiles;
std::map<int, bool> g_fattr[2];

}  // namespace

// All jobs in one persistent launch of the FP32 leaf (tcgen05, CTA pairs when
// the tiles fill every co-resident pair), so that no product's last wave
// leaves SMs idle.  table_mem: fused_table_bytes() of device memory, 256-byte
// aligned, for the job table.
static cudaError_t launch_leaf_f32_fused(const std::vector<FusedJob> &jobs, int np, int64_t K,
                                         void *table_mem, cudaStream_t st) {
  const int nj = (int)jobs.size();
  if (nj < 1 || nj > MAX_FUSED || K <= 0) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(g_mu_c);
  int dev = 0;
  cudaGetDevice(&dev);
  const int units = pair_units_c(dev);
  bool pair = units > 0;
  int64_t pt = 0;
  for (const FusedJob &j : jobs) {
    pair = pair && j.M >= 256;
    const int64_t t = ((j.M + 255) / 256) * ((j.N + BN - 1) / BN);
    pt += j.lower ? t / 2 : t;
  }
  const char *ev = getenv("AAT_LEAF_PAIR");
  pair = ev ? (atoi(ev) > 0 && units > 0) : (pair && pt >= units);
  const int tm = pair ? FShape<true>::TM : FShape<false>::TM;
  FusedTable *T = new FusedTable;
  std::memset(T, 0, sizeof(FusedTable));
  cudaError_t e = cudaSuccess;
  double work = 0.0;
  const int kblocks = (int)((K + BK - 1) / BK);
  for (int i = 0; i < nj && e == cudaSuccess; ++i) {
    const FusedJob &j = jobs[i];
    FJobDesc &d = T->jobs[i];
    if ((e = encode_c(&d.tmx, *j.X, BM)) != cudaSuccess ||
        (e = encode_c(&d.tmy, *j.Y, pair ? FShape<true>::YROWS : FShape<false>::YROWS)) !=
            cudaSuccess)
      break;
    d.out = j.out;
    d.ldo = j.ldo;
    d.M = j.M;
    d.N = j.N;
    d.lower = j.lower;
    d.kblocks = kblocks;
    d.goff = T->ng;
    int pairs[6][2];
    const int npairs = piece_pairs(std::min(j.keep, np), pairs);
    d.ng = npairs;
    for (int q = 0; q < npairs; ++q) {
      FGroup &g = T->g[T->ng++];
      g.xp = (int16_t)(j.xs * np + pairs[q][0]);
      g.yp = (int16_t)(j.ys * np + pairs[q][1]);
      g.neg = 0;
    }
    const double macs = j.lower ? 0.5 * (double)j.M * (double)(j.M + 1) * K : (double)j.M * j.N * K;
    work += 2.0 * npairs * macs;
  }
  T->njobs = nj;
  // the tile list, cached per shape list
  std::vector<int64_t> key = {dev, tm};
  for (const FusedJob &j : jobs) key.insert(key.end(), {j.M, j.N, (int64_t)j.lower});
  int4 *tiles = nullptr;
  int nt = 0;
  if (e == cudaSuccess) {
    auto it = g_ftiles.find(key);
    if (it != g_ftiles.end()) {
      tiles = it->second.first;
      nt = it->second.second;
    } else {
      std::vector<int4> v;
      for (int i = 0; i < nj; ++i) {
        const FusedJob &j = jobs[i];
        const int64_t TI = (j.M + tm - 1) / tm, TJ = (j.N + BN - 1) / BN;
        const int64_t band = std::max<int64_t>(1, 2048 / tm);
        for (int64_t bi = 0; bi < TI; bi += band)
          for (int64_t jj = 0; jj < TJ; ++jj)
            for (int64_t ii = bi; ii < std::min(TI, bi + band); ++ii) {
              if (j.lower && jj * BN > ii * tm + tm - 1) continue;
              v.push_back(make_int4(i, (int)ii, (int)jj, 0));
            }
      }
      if ((e = cudaMalloc(&tiles, std::max<size_t>(v.size(), 1) * sizeof(int4))) == cudaSuccess &&
          (e = cudaMemcpy(tiles, v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice)) ==
              cudaSuccess) {
        nt = (int)v.size();
        g_ftiles[key] = std::make_pair(tiles, nt);
      }
    }
  }
  if (e == cudaSuccess && !g_fattr[pair][dev]) {
    e = pair ? cudaFuncSetAttribute(leaf_f32_kernel<true, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)FShape<true>::SMEM)
             : cudaFuncSetAttribute(leaf_f32_kernel<false, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)FShape<false>::SMEM);
    if (e == cudaSuccess) g_fattr[pair][dev] = true;
  }
  if (e != cudaSuccess) {
    delete T;
    return e;
  }
  FJobDesc *jobs_dev = (FJobDesc *)table_mem;
  FGroup *gtab_dev =
      (FGroup *)((char *)table_mem + ((sizeof(FJobDesc) * MAX_FUSED + 255) & ~(size_t)255));
  fused_table_kernel<<<1, 64, 0, st>>>(*T, jobs_dev, gtab_dev);
  delete T;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  FParams *P = new FParams;
  std::memset(P, 0, sizeof(FParams));
  P->kchunk = 8;  // as launch_leaf_f32
  P->ntiles = nt;
  P->status = device_status_ptr();
  P->jobs = jobs_dev;
  P->btiles = tiles;
  P->gtab = gtab_dev;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nt > 0) {
    ProfScope prof(AAT_K_LEAF_F32, st, work);
    if (pair) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(2 * std::max(1, std::min(nt, units)), 1, 1);
      cfg.blockDim = dim3(THREADS, 1, 1);
      cfg.dynamicSmemBytes = FShape<true>::SMEM;
      cfg.stream = st;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, leaf_f32_kernel<true, true>, *P);
    } else {
      leaf_f32_kernel<false, true><<<std::max(1, std::min(nt, sms)), THREADS, FShape<false>::SMEM,
                                     st>>>(*P);
      e = cudaGetLastError();
    }
  }
  delete P;
  return e;
}

void leaf_f32_release() {
  std::lock_guard<std::mutex> lock(g_mu_c);
  for (auto &kv : g_tiles_c)
    if (kv.second.first) cudaFree(kv.second.first);
  g_tiles_c.clear();
  for (auto &kv : g_ftiles)
    if (kv.second.first) cudaFree(kv.second.first);
  g_ftiles.clear();
  g_fattr[0].clear();
  g_fattr[1].clear();
  g_attr_c.clear();
  g_pair_units_c.clear();
}

// BF16 pieces stored per value.  Plain BF16 (AAT_C_BF16) stores two: the
// 2M form's sum operand Ar +- Ai keeps both, because rounding it to one piece
// puts an error of the size of the result's entries into G, which Re C = G
// -+ H -+ H^T carries whole (measured 3.3e-3 for A A^T, against 2.3e-3 when
// only the inputs Ar, Ai are rounded).
static int pieces_for(uint32_t flags) {
  switch (flags & AAT_C_PREC_MASK) {
    case AAT_C_BF16X3: return 2;
    case AAT_C_BF16: return 2;
    default: return 3;
  }
}

// Pieces whose pair products are kept for products of plain operands (Ar,
// Ai, the 3M sums): one for AAT_C_BF16, all stored pieces otherwise.
static int pieces_kept(uint32_t flags) {
  return (flags & AAT_C_PREC_MASK) == AAT_C_BF16 ? 1 : pieces_for(flags);
}

// ---------------------------------------------- complex elementwise kernels

namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiplication by Y = i I: (x + iy) i = -y + ix
__device__ __forceinline__ float2 ci(float2 a) { return make_float2(-a.y, a.x); }

// The four additions of Algorithm 1 over C with Y = i I (Sec. 4.1):
// S1 = (A21 - A11) i, S2 = A22 - A21 i, S3 = S1 - A22, S4 = S3 + A12.
__global__ void csblocks_kernel(const float2 *__restrict__ A, int64_t lda, int64_t h, int64_t kap,
                                float2 *S1, float2 *S2, float2 *S3, float2 *S4, int64_t ld1,
                                int64_t ld2, int64_t ld3, int64_t ld4) {
  const int64_t total = h * kap;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / kap, j = t - (t / kap) * kap;
    const float2 a11 = A[i * lda + j], a12 = A[i * lda + kap + j];
    const float2 a21 = A[(h + i) * lda + j], a22 = A[(h + i) * lda + kap + j];
    const float2 s1 = ci(csub(a21, a11));
    const float2 s2 = csub(a22, ci(a21));
    const float2 s3 = csub(s1, a22);
    const float2 s4 = cadd(s3, a12);
    if (S1) S1[i * ld1 + j] = s1;
    if (S2) S2[i * ld2 + j] = s2;
    if (S3) S3[i * ld3 + j] = s3;
    if (S4) S4[i * ld4 + j] = s4;
  }
}

// The last level of Algorithm 1 over C (Y = i I) in one pass over A: the S
// blocks S1 = (A21 - A11) i, S2 = A22 - A21 i, S3 = S1 - A22, S4 = S3 + A12
// are formed in registers and, with A11, A12, A22, written straight out as
// the BF16 pieces of the operand sets of the level's fused products.
struct CLevelOut {
  CSplitOut s2, s1, a22, s4, s3, a11, a12;
};

__global__ void csblocks_split_kernel(const float2 *__restrict__ A, int64_t lda, int64_t h,
                                      int64_t kap, int np, CLevelOut o) {
  const int64_t cq = (kap + 3) / 4;
  for (int64_t r = blockIdx.y; r < h; r += gridDim.y)
    for (int64_t q4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q4 < cq;
         q4 += (int64_t)gridDim.x * blockDim.x) {
      const int64_t c0 = 4 * q4;
      const int nv = (int)min((int64_t)4, kap - c0);
      float2 a11[4], a12[4], a21[4], a22[4], s[4];
      cload4(A + r * lda, c0, nv, a11);
      cload4(A + r * lda + kap, c0, nv, a12);
      cload4(A + (h + r) * lda, c0, nv, a21);
      cload4(A + (h + r) * lda + kap, c0, nv, a22);
      csplit_store(a11, r, c0, nv, np, o.a11);
      csplit_store(a12, r, c0, nv, np, o.a12);
      csplit_store(a22, r, c0, nv, np, o.a22);
#pragma unroll
      for (int v = 0; v < 4; ++v) s[v] = csub(a22[v], ci(a21[v]));  // S2
      csplit_store(s, r, c0, nv, np, o.s2);
#pragma unroll
      for (int v = 0; v < 4; ++v) s[v] = ci(csub(a21[v], a11[v]));  // S1
      csplit_store(s, r, c0, nv, np, o.s1);
#pragma unroll
      for (int v = 0; v < 4; ++v) s[v] = csub(s[v], a22[v]);  // S3
      csplit_store(s, r, c0, nv, np, o.s3);
#pragma unroll
      for (int v = 0; v < 4; ++v) s[v] = cadd(s[v], a12[v]);  // S4
      csplit_store(s, r, c0, nv, np, o.s4);
    }
}

// Post-additions of Algorithm 1 over C (phi = transposition, so Up(U1) is
// the plain transpose of Low(U1)); same tile-pair scheme as over F_p.
__global__ void cpostadd_kernel(const float2 *__restrict__ C11, const float2 *__restrict__ C12,
                                float2 *C21, float2 *C22, int64_t ldc, int64_t h) {
  __shared__ float2 p4t_ij[T][T + 1];
  __shared__ float2 p4t_ji[T][T + 1];
  __shared__ float2 u1_ij[T][T + 1];
  const int64_t ntiles = (h + T - 1) / T;
  int64_t pid = blockIdx.x;
  int64_t I, J;
  tri_index(pid, I, J);
  if (I >= ntiles) return;
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  const int64_t r0 = I * T, c0 = J * T;
  for (int yy = ty; yy < T; yy += 8) {
    int64_t r = r0 + yy, c = c0 + tx;
    if (r < h && c < h) {
      p4t_ij[yy][tx] = C22[r * ldc + c];
      const int64_t lr = r >= c ? r : c, lc = r >= c ? c : r;
      u1_ij[yy][tx] = cadd(C11[lr * ldc + lc], C12[lr * ldc + lc]);
    }
    int64_t r2 = c0 + yy, c2 = r0 + tx;
    if (r2 < h && c2 < h) p4t_ji[yy][tx] = C22[r2 * ldc + c2];
  }
  __syncthreads();
  for (int yy = ty; yy < T; yy += 8) {
    int64_t r = r0 + yy, c = c0 + tx;
    if (r < h && c < h) {
      const float2 u2 = cadd(u1_ij[yy][tx], p4t_ji[tx][yy]);
      C21[r * ldc + c] = cadd(u2, C21[r * ldc + c]);
      if (r >= c) C22[r * ldc + c] = cadd(u2, p4t_ij[yy][tx]);
    }
  }
  if (I == J) return;
  for (int yy = ty; yy < T; yy += 8) {
    int64_t r = c0 + yy, c = r0 + tx;
    if (r < h && c < h) {
      const float2 u2 = cadd(u1_ij[tx][yy], p4t_ij[tx][yy]);
      C21[r * ldc + c] = cadd(u2, C21[r * ldc + c]);
    }
  }
}

__global__ void cadd_low_kernel(float2 *C11, const float2 *__restrict__ C12, int64_t ldc,
                                int64_t h) {
  const int64_t total = h * h;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / h, c = t - (t / h) * h;
    if (c <= r) C11[r * ldc + c] = cadd(C11[r * ldc + c], C12[r * ldc + c]);
  }
}

// 3M: X Y^T = (T1 - T2) + i (T3 - T1 - T2) with T1 = Xr Yr^T, T2 = Xi Yi^T,
// T3 = (Xr + Xi)(Yr + Yi)^T.
__global__ void combine3m_kernel(const float *__restrict__ T1, const float *__restrict__ T2,
                                 const float *__restrict__ T3, int64_t ldt, int64_t M, int64_t N,
                                 float2 *C, int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / N, c = t - (t / N) * N;
    const float t1 = T1[r * ldt + c], t2 = T2[r * ldt + c], t3 = T3[r * ldt + c];
    C[r * ldc + c] = make_float2(t1 - t2, t3 - t1 - t2);
  }
}

__global__ void cpad_kernel(const float2 *__restrict__ src, int64_t lds, int64_t rows, int64_t cols,
                            float2 *dst, int64_t ldd, int64_t rows_d, int64_t cols_d) {
  const int64_t total = rows_d * cols_d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / cols_d, c = t - (t / cols_d) * cols_d;
    dst[r * ldd + c] = (r < rows && c < cols) ? src[r * lds + c] : make_float2(0.f, 0.f);
  }
}

__global__ void ccopy_low_kernel(const float2 *__restrict__ src, int64_t lds, float2 *dst,
                                 int64_t ldd, int64_t n) {
  const int64_t total = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, c = t - (t / n) * n;
    if (c <= r) dst[r * ldd + c] = src[r * lds + c];
  }
}

}  // namespace

// ------------------------------------------------------------ host plans

// Bump allocator over the workspace; the dry run only measures.
struct CArena {
  char *base = nullptr;
  size_t used = 0, peak = 0;
  bool dry = true;
  void *get(size_t bytes) {
    const size_t off = (used + 255) & ~(size_t)255;
    used = off + bytes;
    peak = std::max(peak, used);
    return dry ? nullptr : (void *)(base + off);
  }
};

struct CCtx {
  int np;    // pieces stored per value
  int keep;  // pieces kept for products of plain operands
  cudaStream_t st;
  CArena ar;
  int err = AAT_OK;
};

static bool cchk(CCtx &c, cudaError_t e, const char *where) {
  if (e != cudaSuccess && c.err == AAT_OK) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    c.err = report_error(AAT_ECUDA, m.c_str());
  }
  return c.err == AAT_OK;
}

static Planes cplanes(CCtx &c, int64_t rows, int64_t cols, int sets) {
  Planes P;
  std::memset(&P, 0, sizeof(P));
  P.rows = rows;
  P.cols = cols;
  P.kstride = (cols + 7) / 8 * 8;
  P.L = c.np * sets;
  P.nbase = P.L;
  P.ptr = (__nv_bfloat16 *)c.ar.get((size_t)P.L * rows * P.kstride * 2);
  return P;
}

static Planes subset(const Planes &P, int set, int np) {
  Planes Q = P;
  Q.L = Q.nbase = np;
  if (Q.ptr) Q.ptr = P.ptr + (size_t)set * np * P.rows * P.kstride;
  return Q;
}

static void csplit(CCtx &c, const float2 *A, int64_t lda, int64_t rows, int64_t cols,
                   const CSplitOut &o) {
  if (c.ar.dry) return;
  int nsets = (o.re.ptr != nullptr) + (o.im.ptr != nullptr) + (o.s.ptr != nullptr) +
              (o.d.ptr != nullptr);
  ProfScope prof(AAT_K_SPLIT, c.st, (double)rows * cols * (8.0 + 2.0 * c.np * nsets));
  const int64_t cq = (cols + 3) / 4;
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((cq + 255) / 256, 64)),
                  (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, 65535)));
  csplit_kernel<<<grid, 256, 0, c.st>>>(A, lda, rows, cols, c.np, o);
  cchk(c, cudaGetLastError(), "complex split");
}

// Algorithm 2: Low(X phi(X)) into C (herm: phi = conjugate transposition).
static void c_two_m(CCtx &c, const float2 *A, int64_t lda, int64_t n, int64_t k, float2 *C,
                    int64_t ldc, int herm) {
  if (c.err) return;
  const size_t mark = c.ar.used;
  // A A^H: G's two operands are both Ar + Ai, so its pieces are split once
  Planes X = cplanes(c, n, k, 2), Y = cplanes(c, n, k, herm ? 1 : 2);
  Planes Xr = subset(X, 0, c.np), Xs = subset(X, 1, c.np);
  Planes Yi = subset(Y, 0, c.np), Ysd = herm ? Xs : subset(Y, 1, c.np);
  float *H = (float *)c.ar.get((size_t)n * n * 4);
  float *G = (float *)c.ar.get((size_t)n * n * 4);
  void *table = c.ar.get(fused_table_bytes());
  if (!c.ar.dry) {
    // every piece set in one pass over A
    CSplitOut o;
    std::memset(&o, 0, sizeof(o));
    o.re = Xr;
    o.s = Xs;
    o.im = Yi;
    if (!herm) o.d = Ysd;
    csplit(c, A, lda, n, k, o);
    // H = Ar Ai^T (all entries) and G = (Ar + Ai)(Ar +- Ai)^T (lower tiles)
    // in one launch; G's sum operands keep every stored piece
    if (c.err == AAT_OK) {
      const std::vector<FusedJob> jobs = {
          FusedJob{&X, &Y, 0, 0, c.keep, H, n, n, n, 0},
          FusedJob{&X, herm ? &X : &Y, 1, 1, c.np, G, n, n, n, 1}};
      cchk(c, launch_leaf_f32_fused(jobs, c.np, k, table, c.st), "2M H and G");
    }
    if (c.err == AAT_OK) {
      const int64_t nt = (n + T - 1) / T;
      ProfScope prof(AAT_K_POSTADD, c.st, (double)n * n * (4.0 * 1.5 + 8.0 * 0.5));
      combine2m_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, c.st>>>(G, H, n, n, C, ldc,
                                                                           herm);
      cchk(c, cudaGetLastError(), "2M combine");
    }
    if (herm && c.err == AAT_OK) {
      ProfScope prof(AAT_K_COPY, c.st, (double)n * k * 8.0);
      herm_diag_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, c.st>>>(A, lda, n, k, C, ldc);
      cchk(c, cudaGetLastError(), "Hermitian diagonal");
    }
  }
  c.ar.used = mark;
}

// 3M: C = X Y^T (complex, M x N, inner K), all entries.
static void c_gen_leaf(CCtx &c, const float2 *X, int64_t ldx, const float2 *Y, int64_t ldy,
                       int64_t M, int64_t N, int64_t K, float2 *C, int64_t ldc) {
  if (c.err) return;
  const size_t mark = c.ar.used;
  Planes PX = cplanes(c, M, K, 3), PY = cplanes(c, N, K, 3);
  Planes Xr = subset(PX, 0, c.np), Xi = subset(PX, 1, c.np), Xs = subset(PX, 2, c.np);
  Planes Yr = subset(PY, 0, c.np), Yi = subset(PY, 1, c.np), Ys = subset(PY, 2, c.np);
  float *T1 = (float *)c.ar.get((size_t)M * N * 4);
  float *T2 = (float *)c.ar.get((size_t)M * N * 4);
  float *T3 = (float *)c.ar.get((size_t)M * N * 4);
  if (!c.ar.dry) {
    CSplitOut ox, oy;
    std::memset(&ox, 0, sizeof(ox));
    std::memset(&oy, 0, sizeof(oy));
    ox.re = Xr;
    ox.im = Xi;
    ox.s = Xs;
    oy.re = Yr;
    oy.im = Yi;
    oy.s = Ys;
    csplit(c, X, ldx, M, K, ox);
    csplit(c, Y, ldy, N, K, oy);
    if (c.err == AAT_OK)
      cchk(c, launch_leaf_f32({FTerm{&Xr, &Yr, false}}, c.np, c.keep, M, N, K, T1, N, 0, c.st), "3M T1");
    if (c.err == AAT_OK)
      cchk(c, launch_leaf_f32({FTerm{&Xi, &Yi, false}}, c.np, c.keep, M, N, K, T2, N, 0, c.st), "3M T2");
    if (c.err == AAT_OK)
      cchk(c, launch_leaf_f32({FTerm{&Xs, &Ys, false}}, c.np, c.keep, M, N, K, T3, N, 0, c.st), "3M T3");
    if (c.err == AAT_OK) {
      ProfScope prof(AAT_K_POSTADD, c.st, (double)M * N * (12.0 + 8.0));
      combine3m_kernel<<<grid_c(M * N, 256), 256, 0, c.st>>>(T1, T2, T3, N, M, N, C, ldc);
      cchk(c, cudaGetLastError(), "3M combine");
    }
  }
  c.ar.used = mark;
}

// The last level of Algorithm 1 over C (Sec. 4.1, Y = i I) with the twelve
// real products of its leaves in ONE launch: P4^T = S2 S1^T and P3 = A22 S4^T
// by 3M (T1 = Xr Yr^T, T2 = Xi Yi^T, T3 = (Xr + Xi)(Yr + Yi)^T each), P5 =
// Low(S3 S3^T), P1 = Low(A11 A11^T) and P2 = Low(A12 A12^T) by 2M with eps =
// -1 (H = Re Im^T, G = Low((Re + Im)(Re - Im)^T) each).  One pass over A
// forms the S blocks in registers and writes the BF16 pieces of every
// operand; every product reads only its operands' pieces and writes its own
// buffer, so all of them run as one persistent launch; the combines then form
// P4^T -> C22, P3 -> C21, P5 -> C12, P1 -> C11, the post-additions run, and
// P2's combine (into C12, free after them) and U3 = P1 + P2 close.
static void c_last_level_fused(CCtx &c, const float2 *A, int64_t lda, int64_t n, int64_t k,
                               float2 *C, int64_t ldc) {
  const int64_t h = n / 2, kap = k / 2;
  float2 *C11 = C, *C12 = C + h, *C21 = C + h * ldc, *C22 = C + h * ldc + h;
  const size_t mark = c.ar.used;
  // the pieces: 3M operands in 3 sets (re, im, re + im), 2M operands in 2
  // sets per side (re, re + im | im, re - im); the S blocks themselves exist
  // only in registers (one pass over A writes every set)
  Planes PX4 = cplanes(c, h, kap, 3), PY4 = cplanes(c, h, kap, 3);  // S2, S1
  Planes PX3 = cplanes(c, h, kap, 3), PY3 = cplanes(c, h, kap, 3);  // A22, S4
  Planes X2[3], Y2[3];                                              // S3, A11, A12
  for (int q = 0; q < 3; ++q) {
    X2[q] = cplanes(c, h, kap, 2);
    Y2[q] = cplanes(c, h, kap, 2);
  }
  float *T4[3], *T3[3], *Hb[3], *Gb[3];
  for (int q = 0; q < 3; ++q) {
    T4[q] = (float *)c.ar.get((size_t)h * h * 4);
    T3[q] = (float *)c.ar.get((size_t)h * h * 4);
    Hb[q] = (float *)c.ar.get((size_t)h * h * 4);
    Gb[q] = (float *)c.ar.get((size_t)h * h * 4);
  }
  void *table = c.ar.get(fused_table_bytes());
  if (!c.ar.dry && c.err == AAT_OK) {
    auto three = [&](const Planes &P) {
      CSplitOut o;
      std::memset(&o, 0, sizeof(o));
      o.re = subset(P, 0, c.np);
      o.im = subset(P, 1, c.np);
      o.s = subset(P, 2, c.np);
      return o;
    };
    auto two = [&](const Planes &X, const Planes &Y) {
      CSplitOut o;
      std::memset(&o, 0, sizeof(o));
      o.re = subset(X, 0, c.np);
      o.s = subset(X, 1, c.np);
      o.im = subset(Y, 0, c.np);
      o.d = subset(Y, 1, c.np);
      return o;
    };
    CLevelOut lo;
    lo.s2 = three(PX4);
    lo.s1 = three(PY4);
    lo.a22 = three(PX3);
    lo.s4 = three(PY3);
    lo.s3 = two(X2[0], Y2[0]);
    lo.a11 = two(X2[1], Y2[1]);
    lo.a12 = two(X2[2], Y2[2]);
    {
      // 4 blocks read, 24 sets of c.np pieces written
      ProfScope prof(AAT_K_SBLOCKS, c.st, (double)h * kap * (32.0 + 24.0 * 2.0 * c.np));
      const int64_t cq = (kap + 3) / 4;
      const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((cq + 255) / 256, 64)),
                      (unsigned)std::max<int64_t>(1, std::min<int64_t>(h, 65535)));
      csblocks_split_kernel<<<grid, 256, 0, c.st>>>(A, lda, h, kap, c.np, lo);
      cchk(c, cudaGetLastError(), "complex S blocks and pieces");
    }
    std::vector<FusedJob> jobs;
    for (int q = 0; q < 3; ++q) {
      jobs.push_back(FusedJob{&PX4, &PY4, q, q, c.keep, T4[q], h, h, h, 0});
      jobs.push_back(FusedJob{&PX3, &PY3, q, q, c.keep, T3[q], h, h, h, 0});
    }
    for (int q = 0; q < 3; ++q) {
      jobs.push_back(FusedJob{&X2[q], &Y2[q], 0, 0, c.keep, Hb[q], h, h, h, 0});
      jobs.push_back(FusedJob{&X2[q], &Y2[q], 1, 1, c.np, Gb[q], h, h, h, 1});
    }
    if (c.err == AAT_OK)
      cchk(c, launch_leaf_f32_fused(jobs, c.np, kap, table, c.st), "fused complex leaves");
    const int64_t nt = (h + T - 1) / T;
    if (c.err == AAT_OK) {
      ProfScope prof(AAT_K_POSTADD, c.st, (double)h * h * 2.0 * (12.0 + 8.0));
      combine3m_kernel<<<grid_c(h * h, 256), 256, 0, c.st>>>(T4[0], T4[1], T4[2], h, h, h, C22,
                                                            ldc);
      combine3m_kernel<<<grid_c(h * h, 256), 256, 0, c.st>>>(T3[0], T3[1], T3[2], h, h, h, C21,
                                                            ldc);
      cchk(c, cudaGetLastError(), "3M combine");
    }
    if (c.err == AAT_OK) {
      ProfScope prof(AAT_K_POSTADD, c.st, 2.0 * (double)h * h * (4.0 * 1.5 + 8.0 * 0.5));
      combine2m_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, c.st>>>(Gb[0], Hb[0], h, h, C12,
                                                                          ldc, 0);
      combine2m_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, c.st>>>(Gb[1], Hb[1], h, h, C11,
                                                                          ldc, 0);
      cchk(c, cudaGetLastError(), "2M combine");
    }
    if (c.err == AAT_OK) {  // U4 -> C21, Low(U5) -> C22
      ProfScope prof(AAT_K_POSTADD, c.st, (double)h * h * 8.0 * 4.5);
      cpostadd_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, c.st>>>(C11, C12, C21, C22, ldc,
                                                                         h);
      cchk(c, cudaGetLastError(), "complex post-additions");
    }
    if (c.err == AAT_OK) {  // P2 -> C12, Low(U3) = Low(P1 + P2) -> C11
      ProfScope prof(AAT_K_POSTADD, c.st, (double)h * h * (4.0 * 1.5 + 8.0 * 0.5));
      combine2m_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, c.st>>>(Gb[2], Hb[2], h, h, C12,
                                                                          ldc, 0);
      cchk(c, cudaGetLastError(), "2M combine");
    }
    if (c.err == AAT_OK) {
      ProfScope prof(AAT_K_ADD_LOW, c.st, (double)h * h * 8.0 * 1.5);
      cadd_low_kernel<<<grid_c(h * h, 256), 256, 0, c.st>>>(C11, C12, ldc, h);
      cchk(c, cudaGetLastError(), "complex U3");
    }
  }
  c.ar.used = mark;
}

// Algorithm 1 over C with phi = transposition and Y = i I (Sec. 4.1):
// Low(A A^T) -> Low(C).  n divisible by 2^levels, k by 2^levels.
static void c_rec(CCtx &c, const float2 *A, int64_t lda, int64_t n, int64_t k, float2 *C,
                  int64_t ldc, int levels) {
  if (c.err) return;
  if (levels == 0 || n < 2 || k < 2) {
    c_two_m(c, A, lda, n, k, C, ldc, 0);
    return;
  }
  static const bool unfused = [] {
    const char *e = getenv("AAT_C_UNFUSED");  // 1: one launch per real product
    return e && atoi(e) != 0;
  }();
  if (levels == 1 && !unfused) {
    c_last_level_fused(c, A, lda, n, k, C, ldc);
    return;
  }
  const int64_t h = n / 2, kap = k / 2;
  float2 *C11 = C, *C12 = C + h, *C21 = C + h * ldc, *C22 = C + h * ldc + h;
  const float2 *A11 = A, *A12 = A + kap, *A22 = A + h * lda + kap;
  const size_t mark = c.ar.used;
  float2 *S1 = (float2 *)c.ar.get((size_t)h * kap * 8);
  float2 *S2 = (float2 *)c.ar.get((size_t)h * kap * 8);
  float2 *S4 = (float2 *)c.ar.get((size_t)h * kap * 8);
  float2 *S3;
  int64_t ld3;
  if (kap <= h) {  // Table 3: S3 in C21
    S3 = C21;
    ld3 = ldc;
  } else {
    S3 = (float2 *)c.ar.get((size_t)h * kap * 8);
    ld3 = kap;
  }
  if (!c.ar.dry) {
    ProfScope prof(AAT_K_SBLOCKS, c.st, (double)h * kap * 8.0 * 8.0);
    csblocks_kernel<<<grid_c(h * kap, 256), 256, 0, c.st>>>(A, lda, h, kap, S1, S2, S3, S4, kap,
                                                            kap, ld3, kap);
    cchk(c, cudaGetLastError(), "complex S blocks");
  }
  c_gen_leaf(c, S2, kap, S1, kap, h, h, kap, C22, ldc);  // P4^T = S2 S1^T
  c_rec(c, S3, ld3, h, kap, C12, ldc, levels - 1);       // P5 = Low(S3 S3^T)
  c_gen_leaf(c, A22, lda, S4, kap, h, h, kap, C21, ldc);  // P3 = A22 S4^T
  c_rec(c, A11, lda, h, kap, C11, ldc, levels - 1);      // P1 = Low(A11 A11^T)
  if (!c.ar.dry && c.err == AAT_OK) {                    // U4 -> C21, Low(U5) -> C22
    const int64_t nt = (h + T - 1) / T;
    ProfScope prof(AAT_K_POSTADD, c.st, (double)h * h * 8.0 * 4.5);
    cpostadd_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, c.st>>>(C11, C12, C21, C22, ldc,
                                                                       h);
    cchk(c, cudaGetLastError(), "complex post-additions");
  }
  c_rec(c, A12, lda, h, kap, C12, ldc, levels - 1);  // P2 = Low(A12 A12^T)
  if (!c.ar.dry && c.err == AAT_OK) {                // Low(U3) = Low(P1 + P2)
    ProfScope prof(AAT_K_ADD_LOW, c.st, (double)h * h * 8.0 * 1.5);
    cadd_low_kernel<<<grid_c(h * h, 256), 256, 0, c.st>>>(C11, C12, ldc, h);
    cchk(c, cudaGetLastError(), "complex U3");
  }
  c.ar.used = mark;
}

// Runs (or measures, with dry) a complex product: method 0 = 2M A A^H,
// 1 = 2M A A^T, 2 = Algorithm 1 A A^T with `levels`.
static size_t c_plan(CCtx &c, int method, const float2 *A, int64_t n, int64_t k, int64_t lda,
                     float2 *C, int64_t ldc, int levels, bool dry, char *ws) {
  c.ar = CArena();
  c.ar.dry = dry;
  c.ar.base = ws;
  if (method < 2) {
    c_two_m(c, A, lda, n, k, C, ldc, method == 0 ? 1 : 0);
    return c.ar.peak;
  }
  const int64_t m = (int64_t)1 << levels;
  const int64_t np_ = (n + m - 1) / m * m, kp = (k + m - 1) / m * m;
  const bool pad = (np_ != n || kp != k) && levels > 0;
  const float2 *Aw = A;
  float2 *Cw = C;
  int64_t ldaw = lda, ldcw = ldc;
  if (pad) {
    float2 *Ap = (float2 *)c.ar.get((size_t)np_ * kp * 8);
    float2 *Cp = (float2 *)c.ar.get((size_t)np_ * np_ * 8);
    if (!dry) {
      cpad_kernel<<<grid_c(np_ * kp, 256), 256, 0, c.st>>>(A, lda, n, k, Ap, kp, np_, kp);
      cchk(c, cudaGetLastError(), "complex pad");
    }
    Aw = Ap;
    Cw = Cp;
    ldaw = kp;
    ldcw = np_;
  }
  c_rec(c, Aw, ldaw, pad ? np_ : n, pad ? kp : k, Cw, ldcw, levels);
  if (pad && !dry && c.err == AAT_OK) {
    ccopy_low_kernel<<<grid_c(n * n, 256), 256, 0, c.st>>>(Cw, ldcw, C, ldc, n);
    cchk(c, cudaGetLastError(), "complex unpad");
  }
  return c.ar.peak;
}

static int complex_levels(int64_t n, int64_t k, uint32_t flags) {
  const uint32_t lv = (flags & AAT_LEVELS_MASK) >> 8;
  if (lv) return (int)lv - 1;
  if ((flags & AAT_C_PREC_MASK) == AAT_C_BF16) return 0;  // see bf16_levels_ok
  int levels = 0;  // one level pays off once the leaves stay large
  while (levels < 4 && (n >> (levels + 1)) >= 4096 && (k >> (levels + 1)) >= 2048) ++levels;
  return levels;
}

// ----------------------------------------------- batched A A^H (2M), host

struct CBatchImpl {
  CBProb *probs = nullptr;
  FJobDesc *jobs = nullptr;
  FGroup *gtab = nullptr;
  int4 *tiles = nullptr;
  int count = 0, ntiles = 0;
  int split_blocks = 0, comb_blocks = 0, diag_blocks = 0;
  double leaf_work = 0.0, split_bytes = 0.0, comb_bytes = 0.0, diag_bytes = 0.0;
};

static size_t r256c(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t cb_planes_bytes(int64_t n, int64_t k, int np) {
  return r256c((size_t)2 * np * n * ((k + 7) / 8 * 8) * 2);
}

size_t cbatch_workspace(const CBInput *in, int count) {
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    const int np = pieces_for(in[i].flags);
    total += 2 * cb_planes_bytes(in[i].n, in[i].k, np) + 2 * r256c((size_t)in[i].n * in[i].n * 4);
  }
  return total;
}

void cbatch_free(CBatch *b) {
  CBatchImpl *L = (CBatchImpl *)b->impl;
  if (!L) return;
  if (L->probs) cudaFree(L->probs);
  if (L->jobs) cudaFree(L->jobs);
  if (L->gtab) cudaFree(L->gtab);
  if (L->tiles) cudaFree(L->tiles);
  delete L;
  b->impl = nullptr;
}

cudaError_t cbatch_build(const CBInput *in, int count, char *ws, CBatch *out) {
  std::lock_guard<std::mutex> lock(g_mu_c);
  std::vector<CBProb> probs(count);
  std::vector<FJobDesc> jobs;
  std::vector<FGroup> gtab;
  struct T4 { int4 t; double cost; };
  std::vector<T4> tiles;
  CBatchImpl *L = new CBatchImpl;
  L->count = count;
  char *w = ws;
  int sb = 0, cbk = 0, db = 0;
  for (int i = 0; i < count; ++i) {
    const CBInput &q = in[i];
    CBProb &b = probs[i];
    std::memset(&b, 0, sizeof(b));
    const int np = pieces_for(q.flags);
    Planes X, Y;
    std::memset(&X, 0, sizeof(X));
    X.rows = q.n;
    X.cols = q.k;
    X.kstride = (q.k + 7) / 8 * 8;
    X.L = X.nbase = 2 * np;
    Y = X;
    X.ptr = (__nv_bfloat16 *)w;
    w += cb_planes_bytes(q.n, q.k, np);
    Y.ptr = (__nv_bfloat16 *)w;
    w += cb_planes_bytes(q.n, q.k, np);
    b.H = (float *)w;
    w += r256c((size_t)q.n * q.n * 4);
    b.G = (float *)w;
    w += r256c((size_t)q.n * q.n * 4);
    b.A = q.A;
    b.lda = q.lda;
    b.n = q.n;
    b.k = q.k;
    b.np = np;
    b.herm = q.herm;
    b.ox.re = subset(X, 0, np);
    b.ox.s = subset(X, 1, np);
    b.oy.im = subset(Y, 0, np);
    if (!q.herm) b.oy.d = subset(Y, 1, np);  // A A^H: G reads Ar + Ai from X twice
    b.C = q.C;
    b.ldc = q.ldc;
    b.split_first = sb;
    sb += (int)((q.n + kCSplitRows - 1) / kCSplitRows);
    const int64_t nt = (q.n + T - 1) / T;
    b.comb_first = cbk;
    cbk += (int)(nt * (nt + 1) / 2);
    b.diag_first = db;
    if (q.herm) db += (int)((q.n + kDiagRows - 1) / kDiagRows);
    L->split_bytes += (double)q.n * q.k * (8.0 + 2.0 * np * (q.herm ? 3 : 4));
    L->comb_bytes += (double)q.n * q.n * (4.0 * 1.5 + 8.0 * 0.5);
    if (q.herm) L->diag_bytes += (double)q.n * q.k * 8.0;
    // two jobs: H = Ar Ai^T (all entries) from plane sets 0, G (lower) from
    // sets 1; G's sum operands keep every stored piece
    for (int jb = 0; jb < 2; ++jb) {
      int pairs[6][2];
      const int npairs = piece_pairs(jb == 0 ? pieces_kept(q.flags) : np, pairs);
      FJobDesc d;
      std::memset(&d, 0, sizeof(d));
      cudaError_t e;
      // A A^H's G job (jb 1): both operands are X's Ar + Ai pieces, which
      // sit at the same plane indices in X as Ar - Ai would in Y
      const Planes &ysrc = (jb == 1 && q.herm) ? X : Y;
      if ((e = encode_c(&d.tmx, X, BM)) != cudaSuccess ||
          (e = encode_c(&d.tmy, ysrc, FShape<false>::YROWS)) != cudaSuccess) {
        CBatch tmp;
        tmp.impl = L;
        cbatch_free(&tmp);
        return e;
      }
      d.out = jb == 0 ? b.H : b.G;
      d.ldo = q.n;
      d.M = d.N = q.n;
      d.lower = jb;
      d.kblocks = (int)((q.k + BK - 1) / BK);
      d.goff = (int)gtab.size();
      d.ng = npairs;
      for (int qq = 0; qq < npairs; ++qq) {
        FGroup g;
        g.xp = (int16_t)(jb * np + pairs[qq][0]);
        g.yp = (int16_t)(jb * np + pairs[qq][1]);
        g.neg = 0;
        gtab.push_back(g);
      }
      const int jobi = (int)jobs.size();
      jobs.push_back(d);
      const double cost = (double)d.kblocks * npairs;
      const int64_t TI = (q.n + BM - 1) / BM, TJ = (q.n + BN - 1) / BN;
      for (int64_t I = 0; I < TI; ++I)
        for (int64_t J = 0; J < TJ; ++J) {
          if (jb == 1 && J * BN > I * BM + BM - 1) continue;
          tiles.push_back({make_int4(jobi, (int)I, (int)J, 0), cost});
        }
      const double macs = jb == 1 ? 0.5 * (double)q.n * (q.n + 1) * q.k : (double)q.n * q.n * q.k;
      L->leaf_work += 2.0 * npairs * macs;
    }
  }
  std::stable_sort(tiles.begin(), tiles.end(),
                   [](const T4 &u, const T4 &v) { return u.cost > v.cost; });
  std::vector<int4> tl(tiles.size());
  for (size_t i = 0; i < tiles.size(); ++i) tl[i] = tiles[i].t;
  L->ntiles = (int)tl.size();
  L->split_blocks = sb;
  L->comb_blocks = cbk;
  L->diag_blocks = db;
  cudaError_t e;
  if ((e = cudaMalloc(&L->probs, sizeof(CBProb) * std::max(count, 1))) != cudaSuccess ||
      (e = cudaMalloc(&L->jobs, sizeof(FJobDesc) * std::max<size_t>(jobs.size(), 1))) != cudaSuccess ||
      (e = cudaMalloc(&L->gtab, sizeof(FGroup) * std::max<size_t>(gtab.size(), 1))) != cudaSuccess ||
      (e = cudaMalloc(&L->tiles, sizeof(int4) * std::max<size_t>(tl.size(), 1))) != cudaSuccess ||
      (e = cudaMemcpy(L->probs, probs.data(), sizeof(CBProb) * count, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(L->jobs, jobs.data(), sizeof(FJobDesc) * jobs.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(L->gtab, gtab.data(), sizeof(FGroup) * gtab.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (tl.size() && (e = cudaMemcpy(L->tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice)) != cudaSuccess)) {
    CBatch tmp;
    tmp.impl = L;
    cbatch_free(&tmp);
    return e;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if ((e = cudaFuncSetAttribute(leaf_f32_kernel<false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FShape<false>::SMEM)) != cudaSuccess) {
    CBatch tmp;
    tmp.impl = L;
    cbatch_free(&tmp);
    return e;
  }
  out->impl = L;
  return cudaSuccess;
}

cudaError_t cbatch_launch(const CBatch &b, cudaStream_t st) {
  const CBatchImpl *L = (const CBatchImpl *)b.impl;
  if (!L || L->count == 0) return cudaSuccess;
  cudaError_t e;
  if (L->split_blocks > 0) {
    ProfScope prof(AAT_K_SPLIT, st, L->split_bytes);
    csplit_batch_kernel<<<(unsigned)L->split_blocks, 256, 0, st>>>(L->probs, L->count);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (L->ntiles > 0) {
    FParams *P = new FParams;
    std::memset(P, 0, sizeof(FParams));
    P->kchunk = 8;  // as launch_leaf_f32
    P->ntiles = L->ntiles;
    P->status = device_status_ptr();
    P->jobs = L->jobs;
    P->btiles = L->tiles;
    P->gtab = L->gtab;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    {
      ProfScope prof(AAT_K_LEAF_F32, st, L->leaf_work);
      leaf_f32_kernel<false, true><<<std::max(1, std::min(L->ntiles, sms)), THREADS,
                                     FShape<false>::SMEM, st>>>(*P);
    }
    delete P;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (L->comb_blocks > 0) {
    ProfScope prof(AAT_K_POSTADD, st, L->comb_bytes);
    combine2m_batch_kernel<<<(unsigned)L->comb_blocks, T * 8, 0, st>>>(L->probs, L->count);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (L->diag_blocks > 0) {
    ProfScope prof(AAT_K_COPY, st, L->diag_bytes);
    herm_diag_batch_kernel<<<(unsigned)L->diag_blocks, 256, 0, st>>>(L->probs, L->count);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Plain BF16 through Algorithm 1: every level's S blocks and post-additions
// sum several products whose operands are larger than A's blocks, so the
// BF16 rounding of the leaf operands grows by about 2x per level (relative
// Frobenius error 8.7e-3 at one level, 1.8e-2 at two, n = k = 8192, N(0, 1)
// entries): above the 3e-3 that plain BF16 promises, so those depths are
// refused (2 pieces, AAT_C_BF16X3, stay near 1e-5).
static bool bf16_levels_ok(uint32_t flags, int levels) {
  return (flags & AAT_C_PREC_MASK) != AAT_C_BF16 || levels == 0;
}

int complex_run(int method, const void *A, int64_t n, int64_t k, int64_t lda, void *C,
                int64_t ldc, uint32_t flags, cudaStream_t st, char *ws, bool dry, size_t *need) {
  CCtx c;
  c.np = pieces_for(flags);
  c.keep = pieces_kept(flags);
  c.st = st;
  const int levels = method == 2 ? complex_levels(n, k, flags) : 0;
  if (!bf16_levels_ok(flags, levels))
    return report_error(AAT_EUNSUPPORTED,
                        "plain BF16 (AAT_C_BF16) with recursion levels exceeds its 3e-3 error "
                        "bound: use AAT_LEVELS(0) or AAT_C_BF16X3");
  const size_t peak = c_plan(c, method, (const float2 *)A, n, k, lda, (float2 *)C, ldc, levels,
                             dry, ws);
  if (need) *need = peak;
  return c.err;
}

static int complex_entry(const void *A, int64_t n, int64_t k, int64_t lda, void *C, int64_t ldc,
                         uint32_t flags, void *stream, int method) {
  if (n < 0 || k < 0) return report_error(AAT_EINVAL, "negative size");
  if (lda < std::max<int64_t>(k, 1) || ldc < std::max<int64_t>(n, 1))
    return report_error(AAT_EINVAL, "stride smaller than the row length");
  if (n > 0 && (!C || (k > 0 && !A))) return report_error(AAT_EINVAL, "null pointer");
  const uint32_t prec = flags & AAT_C_PREC_MASK;
  if (prec != AAT_C_FP32 && prec != AAT_C_BF16X3 && prec != AAT_C_BF16)
    return report_error(AAT_EUNSUPPORTED, "unknown precision");
  if (n == 0) return AAT_OK;
  int e = check_gb300();
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  if (k == 0) {
    cudaError_t ce = cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)n * 8, (size_t)n, st);
    return ce == cudaSuccess ? AAT_OK : report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  const char *a = (const char *)A, *cc = (const char *)C;
  if (a < cc + ((n - 1) * ldc + n) * 8 && cc < a + ((n - 1) * lda + k) * 8)
    return report_error(AAT_EINVAL, "C overlaps A");
  const int levels = method == 2 ? complex_levels(n, k, flags) : 0;
  if (!bf16_levels_ok(flags, levels))
    return report_error(AAT_EUNSUPPORTED,
                        "plain BF16 (AAT_C_BF16) with recursion levels exceeds its 3e-3 error "
                        "bound: use AAT_LEVELS(0) or AAT_C_BF16X3");
  CCtx c;
  c.np = pieces_for(flags);
  c.keep = pieces_kept(flags);
  c.st = st;
  const size_t need = c_plan(c, method, (const float2 *)A, n, k, lda, (float2 *)C, ldc, levels,
                             true, nullptr);
  void *ws = nullptr;
  if ((e = workspace_get(need, &ws))) return e;
  c.err = AAT_OK;
  c_plan(c, method, (const float2 *)A, n, k, lda, (float2 *)C, ldc, levels, false, (char *)ws);
  return c.err;
}

}  // namespace aat

using namespace aat;

extern "C" {

AAT_API int aah_complex_ex(const void *A, int64_t n, int64_t k, int64_t lda, void *C, int64_t ldc,
                           uint32_t flags, void *stream) {
  return complex_entry(A, n, k, lda, C, ldc, flags, stream, 0);
}

AAT_API int aah_complex(const void *A, int64_t n, int64_t k, void *C, void *stream) {
  return aah_complex_ex(A, n, k, k, C, n, 0u, stream);
}

AAT_API int aat_complex_2m(const void *A, int64_t n, int64_t k, int64_t lda, void *C, int64_t ldc,
                           uint32_t flags, void *stream) {
  return complex_entry(A, n, k, lda, C, ldc, flags, stream, 1);
}

AAT_API int aat_complex_ex(const void *A, int64_t n, int64_t k, int64_t lda, void *C, int64_t ldc,
                           uint32_t flags, void *stream) {
  return complex_entry(A, n, k, lda, C, ldc, flags, stream, 2);
}

AAT_API int aat_complex(const void *A, int64_t n, int64_t k, void *C, void *stream) {
  return aat_complex_ex(A, n, k, k, C, n, 0u, stream);
}

}  // extern "C"
