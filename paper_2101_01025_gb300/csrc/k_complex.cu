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
// 2 K blocks into FP32 registers (round to nearest) while the next chunk
// accumulates in the other TMEM buffer.  The Hermitian diagonal sum_l |a_il|^2 is
// computed in FP64 (real and >= 0).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/aat.h"
#include "common.cuh"
#include "tc_ptx.cuh"

namespace aat {

namespace {

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + EPI_WARPS * 32;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = 256;
constexpr int MAX_FGROUPS = 48;
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + 256;
// kind::f16, FP32 accumulator, BF16 A and B, K-major, N = 256, M = 128;
// bit 13 negates A.
constexpr uint32_t IDESC_F = (1u << 4) | (1u << 7) | (1u << 10) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t NEG_A = 1u << 13;

struct FGroup {
  int16_t xp, yp;  // planes of X and Y
  int32_t neg;     // subtract this product
};

struct FParams {
  CUtensorMap tmx;  // 3D {K, rows, plane}, box {64, 128, 1}
  CUtensorMap tmy;  // 3D {K, rows, plane}, box {64, 256, 1}
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
};

// out = sum_g (+-) X_{xp(g)} Y_{yp(g)}^T in FP32, one TMEM accumulation per
// output tile.  Same CTA organisation as the modular leaf kernel.
__global__ void __launch_bounds__(THREADS, 1) leaf_f32_kernel(const __grid_constant__ FParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t *bars = (uint64_t *)(smem + (size_t)STAGES * STAGE_BYTES);
  const uint32_t bar0 = smem_u32(bars);
#define FULL(s) (bar0 + 8u * (uint32_t)(s))
#define EMPTY(s) (bar0 + 8u * (uint32_t)(STAGES + (s)))
#define AFULL(b) (bar0 + 8u * (uint32_t)(2 * STAGES + (b)))
#define AEMPTY(b) (bar0 + 8u * (uint32_t)(2 * STAGES + 2 + (b)))
#define DONE (bar0 + 8u * (uint32_t)(2 * STAGES + 4))
  uint32_t *tmem_slot = (uint32_t *)(bars + 2 * STAGES + 5);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(FULL(s), 1);
      mbar_init(EMPTY(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(AFULL(b), 1);
      mbar_init(AEMPTY(b), EPI_WARPS);
    }
    mbar_init(DONE, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int stage = 0, issued = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
        const int2 tile = P.tiles[t];
        for (int gi = 0; gi < P.ng && ok; ++gi) {
          const FGroup g = P.g[gi];
          for (int kb = 0; kb < P.kblocks; ++kb) {
            if (!wait_bounded(EMPTY(stage), ph ^ 1u, abort_flag, P.status)) {
              ok = false;
              break;
            }
            mbar_expect_tx(FULL(stage), (uint32_t)STAGE_BYTES);
            const uint32_t sa = sbase + (uint32_t)(stage * STAGE_BYTES);
            tma_load_3d(sa, &P.tmx, FULL(stage), kb * BK, tile.x * BM, g.xp);
            tma_load_3d(sa + A_BYTES, &P.tmy, FULL(stage), kb * BK, tile.y * BN, g.yp);
            ++issued;
            if (++stage == STAGES) {
              stage = 0;
              ph ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        int s = stage;
        uint32_t q = ph;
        for (int i = 0; i < STAGES && i < issued; ++i) {
          if (--s < 0) {
            s = STAGES - 1;
            q ^= 1u;
          }
          wait_quiet(FULL(s), q);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer: chunks of kchunk K blocks over (group, K block)
      int stage = 0;
      uint32_t ph = 0, chunk = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
        int inchunk = 0;
        uint32_t dt = 0;
        for (int gi = 0; gi < P.ng && ok; ++gi) {
          const uint32_t idesc = IDESC_F | (P.g[gi].neg ? NEG_A : 0u);
          for (int kb = 0; kb < P.kblocks; ++kb) {
            if (inchunk == 0) {
              const uint32_t buf = chunk & 1u, use = chunk >> 1;
              if (!wait_bounded(AEMPTY(buf), (use & 1u) ^ 1u, abort_flag, P.status)) {
                ok = false;
                break;
              }
              tc_fence_after();
              dt = tmem + buf * ACC_COLS;
            }
            if (!wait_bounded(FULL(stage), ph, abort_flag, P.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = sbase + (uint32_t)(stage * STAGE_BYTES);
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int s = 0; s < BK / 16; ++s) {
              tc_mma(dt, sw128_desc(sa + 32u * s), sw128_desc(sb + 32u * s), idesc,
                     (inchunk == 0 && s == 0) ? 0u : 1u);
            }
            tc_commit(EMPTY(stage));
            if (++stage == STAGES) {
              stage = 0;
              ph ^= 1u;
            }
            const bool last = (gi == P.ng - 1) && (kb == P.kblocks - 1);
            if (++inchunk == P.kchunk || last) {
              tc_commit(AFULL(chunk & 1u));
              ++chunk;
              inchunk = 0;
            }
          }
        }
      }
      if (!ok) {
        tc_commit(DONE);
        wait_quiet(DONE, 0);
      }
    }
  } else {  // epilogue: chunks -> FP32 registers -> global (lower if asked)
    const int e = warp - 2;
    const int quarter = warp & 3;
    const int chalf = e >> 2;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int total_kb = P.ng * P.kblocks;
    const int nchunks = (total_kb + P.kchunk - 1) / P.kchunk;
    uint32_t chunk = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
      const int2 tile = P.tiles[t];
      float acc[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
      for (int c = 0; c < nchunks; ++c) {
        const uint32_t buf = chunk & 1u, use = chunk >> 1;
        if (!wait_bounded(AFULL(buf), use & 1u, abort_flag, P.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + lane_base + buf * ACC_COLS + (uint32_t)(chalf * 128);
        tmem_accum32f<0>(ta, acc);
        tmem_accum32f<32>(ta + 32u, acc);
        tmem_accum32f<64>(ta + 64u, acc);
        tmem_accum32f<96>(ta + 96u, acc);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(AEMPTY(buf));
        ++chunk;
      }
      if (!ok) break;
      const int64_t row = (int64_t)tile.x * BM + quarter * 32 + lane;
      const int64_t col0 = (int64_t)tile.y * BN + chalf * 128;
      int64_t lim = P.N - col0;
      if (P.lower) lim = min(lim, row - col0 + 1);
      if (row < P.M && lim > 0) {
        float *orow = P.out + row * P.ldo + col0;
        const bool vec = ((reinterpret_cast<uintptr_t>(orow) & 15) == 0);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int cc = 4 * q;
          if (vec && cc + 4 <= lim) {
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
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
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

// BF16 pieces of v: v = p0 + p1 + p2 + (rest), each p the BF16 rounding of
// what is left (the differences are exact in FP32).
__device__ __forceinline__ void pieces(float v, int np, __nv_bfloat16 (&o)[3]) {
  float r = v;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q < np) {
      o[q] = __float2bfloat16_rn(r);
      r = r - __bfloat162float(o[q]);
    }
  }
}

struct CSplitOut {
  Planes re, im, s, d;  // pieces of Re, Im, Re + Im, Re - Im (each optional)
};

__global__ void csplit_kernel(const float2 *__restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                              int np, CSplitOut o) {
  const int64_t total = rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / cols, c = t - (t / cols) * cols;
    const float2 a = A[r * lda + c];
    const float vals[4] = {a.x, a.y, a.x + a.y, a.x - a.y};
    const Planes *outs[4] = {&o.re, &o.im, &o.s, &o.d};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const Planes &P = *outs[w];
      if (!P.ptr) continue;
      __nv_bfloat16 pc[3];
      pieces(vals[w], np, pc);
      const int64_t plane = P.rows * P.kstride;
      for (int q = 0; q < np; ++q) P.ptr[q * plane + r * P.kstride + c] = pc[q];
    }
  }
}

// The combination of Algorithm 2 for one tile pair {(I, J), (J, I)}, I >= J,
// writing Low(C) (complex64):  herm: Re = G - H - H^T, Im = H^T - H;
// otherwise Re = G + H - H^T, Im = H + H^T.
constexpr int T = 32;
__global__ void combine2m_kernel(const float *__restrict__ G, const float *__restrict__ H,
                                 int64_t ldw, int64_t n, float2 *C, int64_t ldc, int herm) {
  __shared__ float hij[T][T + 1];
  __shared__ float hji[T][T + 1];
  const int64_t ntiles = (n + T - 1) / T;
  int64_t pid = blockIdx.x;
  int64_t I = (int64_t)((sqrt(8.0 * (double)pid + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > pid) --I;
  while ((I + 1) * (I + 2) / 2 <= pid) ++I;
  const int64_t J = pid - I * (I + 1) / 2;
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

// C[i,i] = sum_l |a_il|^2 in FP64 (A A^H: real and >= 0), one warp per row.
__global__ void herm_diag_kernel(const float2 *__restrict__ A, int64_t lda, int64_t n, int64_t k,
                                 float2 *C, int64_t ldc) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int64_t l = lane; l < k; l += 32) {
    const float2 a = A[row * lda + l];
    s += (double)a.x * a.x + (double)a.y * a.y;
  }
  for (int off = 16; off; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) C[row * ldc + row] = make_float2((float)s, 0.0f);
}

// ------------------------------------------------------------------ host

PFN_cuTensorMapEncodeTiled_v12000 g_encode_c = nullptr;
std::mutex g_mu_c;
std::map<std::tuple<int, int64_t, int64_t, int>, std::pair<int2 *, int>> g_tiles_c;
std::map<int, bool> g_attr_c;

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

cudaError_t tiles_c(int dev, int64_t M, int64_t N, int lower, int2 **out, int *count) {
  auto key = std::make_tuple(dev, M, N, lower);
  auto it = g_tiles_c.find(key);
  if (it != g_tiles_c.end()) {
    *out = it->second.first;
    *count = it->second.second;
    return cudaSuccess;
  }
  const int64_t TI = (M + BM - 1) / BM, TJ = (N + BN - 1) / BN;
  std::vector<int2> v;
  for (int64_t bi = 0; bi < TI; bi += 16)
    for (int64_t bj = 0; bj < TJ; bj += 8)
      for (int64_t i = bi; i < std::min(TI, bi + 16); ++i)
        for (int64_t j = bj; j < std::min(TJ, bj + 8); ++j) {
          if (lower && j * BN > i * BM + BM - 1) continue;
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

static cudaError_t launch_leaf_f32(const std::vector<FTerm> &terms, int np, int64_t M, int64_t N,
                                   int64_t K, float *out, int64_t ldo, int lower,
                                   cudaStream_t st) {
  if (M <= 0 || N <= 0 || terms.empty()) return cudaSuccess;
  // every term must use the same two plane buffers: X planes in one
  // tensor map, Y planes in the other (plane index = set * np + piece)
  std::lock_guard<std::mutex> lock(g_mu_c);
  FParams *P = new FParams;
  std::memset(P, 0, sizeof(FParams));
  cudaError_t e;
  const Planes &X = *terms[0].x, &Y = *terms[0].y;
  if ((e = encode_c(&P->tmx, X, BM)) != cudaSuccess || (e = encode_c(&P->tmy, Y, BN)) != cudaSuccess) {
    delete P;
    return e;
  }
  int pairs[6][2];
  const int npairs = piece_pairs(np, pairs);
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
  // FP32 accumulation in the tensor core drifts over long K loops (its
  // rounding is not to nearest); draining every 2 K blocks into FP32
  // registers keeps the error of a K = 8192 product near FP32 rounding.
  P->kchunk = 2;
  P->out = out;
  P->ldo = ldo;
  P->M = M;
  P->N = N;
  P->lower = lower;
  P->status = device_status_ptr();
  int dev = 0;
  cudaGetDevice(&dev);
  int2 *tiles = nullptr;
  int nt = 0;
  if ((e = tiles_c(dev, M, N, lower, &tiles, &nt)) != cudaSuccess) {
    delete P;
    return e;
  }
  P->tiles = tiles;
  P->ntiles = nt;
  if (!g_attr_c[dev]) {
    if ((e = cudaFuncSetAttribute(leaf_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SMEM_BYTES)) != cudaSuccess) {
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
    leaf_f32_kernel<<<std::max(1, std::min(nt, sms)), THREADS, SMEM_BYTES, st>>>(*P);
  }
  delete P;
  return cudaGetLastError();
}

void leaf_f32_release() {
  std::lock_guard<std::mutex> lock(g_mu_c);
  for (auto &kv : g_tiles_c)
    if (kv.second.first) cudaFree(kv.second.first);
  g_tiles_c.clear();
  g_attr_c.clear();
}

static int pieces_for(uint32_t flags) {
  switch (flags & AAT_C_PREC_MASK) {
    case AAT_C_BF16X3: return 2;
    case AAT_C_BF16: return 1;
    default: return 3;
  }
}

// Algorithm 2 for A (n x k complex64): Low(A A^H) (herm) or Low(A A^T).
static int two_m(const float2 *A, int64_t n, int64_t k, int64_t lda, float2 *C, int64_t ldc,
                 uint32_t flags, int herm, cudaStream_t st) {
  const int np = pieces_for(flags);
  const int64_t ks = (k + 7) / 8 * 8;
  // workspace: X planes [Ar pieces | Ar+Ai pieces], Y planes [Ai pieces |
  // Ar+Ai or Ar-Ai pieces], H and G in FP32
  const size_t set = (size_t)np * n * ks * 2;
  auto r256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t xbytes = r256(2 * set), ybytes = r256(2 * set), hbytes = r256((size_t)n * n * 4);
  void *ws = nullptr;
  int e = workspace_get(xbytes + ybytes + 2 * hbytes, &ws);
  if (e) return e;
  char *base = (char *)ws;
  auto planes_at = [&](char *p, int sets) {
    Planes P;
    std::memset(&P, 0, sizeof(P));
    P.ptr = (__nv_bfloat16 *)p;
    P.rows = n;
    P.cols = k;
    P.kstride = ks;
    P.L = np * sets;
    P.nbase = P.L;
    return P;
  };
  Planes X = planes_at(base, 2), Y = planes_at(base + xbytes, 2);
  Planes Xr = X, Xs = X, Yi = Y, Ysd = Y;
  Xr.L = Xs.L = Yi.L = Ysd.L = np;
  Xs.ptr = X.ptr + (size_t)np * n * ks;
  Ysd.ptr = Y.ptr + (size_t)np * n * ks;
  float *H = (float *)(base + xbytes + ybytes);
  float *G = (float *)(base + xbytes + ybytes + hbytes);
  CSplitOut ox, oy;
  std::memset(&ox, 0, sizeof(ox));
  std::memset(&oy, 0, sizeof(oy));
  ox.re = Xr;
  ox.s = Xs;
  oy.im = Yi;
  if (herm)
    oy.s = Ysd;
  else
    oy.d = Ysd;
  cudaError_t ce;
  {
    ProfScope prof(AAT_K_SPLIT, st, (double)n * k * (8.0 + 2.0 * 4 * np));
    csplit_kernel<<<grid_c(n * k, 256), 256, 0, st>>>(A, lda, n, k, np, ox);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  {
    ProfScope prof(AAT_K_SPLIT, st, (double)n * k * (8.0 + 2.0 * 4 * np));
    csplit_kernel<<<grid_c(n * k, 256), 256, 0, st>>>(A, lda, n, k, np, oy);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  // H = Ar Ai^T (all entries), G = (Ar + Ai)(Ar +- Ai)^T (lower tiles)
  if ((ce = launch_leaf_f32({FTerm{&Xr, &Yi, false}}, np, n, n, k, H, n, 0, st)) != cudaSuccess)
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  if ((ce = launch_leaf_f32({FTerm{&Xs, &Ysd, false}}, np, n, n, k, G, n, 1, st)) != cudaSuccess)
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  {
    const int64_t nt = (n + T - 1) / T;
    ProfScope prof(AAT_K_POSTADD, st, (double)n * n * (4.0 * 1.5 + 8.0 * 0.5));
    combine2m_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, st>>>(G, H, n, n, C, ldc, herm);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  if (herm) {
    ProfScope prof(AAT_K_COPY, st, (double)n * k * 8.0);
    herm_diag_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(A, lda, n, k, C, ldc);
    if ((ce = cudaGetLastError()) != cudaSuccess)
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  return AAT_OK;
}

static int complex_entry(const void *A, int64_t n, int64_t k, int64_t lda, void *C, int64_t ldc,
                         uint32_t flags, void *stream, int herm) {
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
  const char *a = (const char *)A, *c = (const char *)C;
  if (a < c + ((n - 1) * ldc + n) * 8 && c < a + ((n - 1) * lda + k) * 8)
    return report_error(AAT_EINVAL, "C overlaps A");
  return two_m((const float2 *)A, n, k, lda, (float2 *)C, ldc, flags, herm, st);
}

}  // namespace aat

using namespace aat;

extern "C" {

AAT_API int aah_complex_ex(const void *A, int64_t n, int64_t k, int64_t lda, void *C, int64_t ldc,
                           uint32_t flags, void *stream) {
  return complex_entry(A, n, k, lda, C, ldc, flags, stream, 1);
}

AAT_API int aah_complex(const void *A, int64_t n, int64_t k, void *C, void *stream) {
  return aah_complex_ex(A, n, k, k, C, n, 0u, stream);
}

AAT_API int aat_complex_2m(const void *A, int64_t n, int64_t k, int64_t lda, void *C, int64_t ldc,
                           uint32_t flags, void *stream) {
  return complex_entry(A, n, k, lda, C, ldc, flags, stream, 0);
}

}  // extern "C"
