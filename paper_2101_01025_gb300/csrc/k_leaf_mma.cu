// k_leaf_mma.cu -- the two other exact leaf kinds, on the warp-level
// mma.sync tensor instructions (sm_103a keeps them; tcgen05 has no integer
// kind there):
//
//   AAT_LEAF_I8   balanced residues split into signed 8-bit digits
//                 (X = sum_i 2^(8i) X_i, |digits| <= 127), one INT8 GEMM per
//                 digit pair with exact INT32 accumulation
//                 (mma.sync.m16n8k32.s32.s8.s8.s32), pairs folded into one
//                 int32 accumulator per entry by Horner steps mod p;
//   AAT_LEAF_F64  balanced residues as FP64, mma.sync.m8n8k4.f64: exact while
//                 every partial sum stays below 2^53, i.e. K ((p-1)/2)^2 <
//                 2^53 per chunk of K; the accumulator is reduced mod p
//                 between chunks (the leaf of Sec. 7's implementation, dsyrk
//                 plus a reduction, on the GPU's FP64 tensor path).
//
// Both read int32 residue blocks and are bound by their tensor rate, which
// on GB300 is far below the tcgen05 BF16 rate of the default leaf.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace aat {

namespace {

// ------------------------------------------------------------------ INT8

constexpr int I8_BM = 128, I8_BN = 128, I8_BK = 64;
constexpr int I8_THREADS = 256;        // 8 warps: 2 (M) x 4 (N), warp tile 64 x 32
constexpr int I8_LD = I8_BK + 16;      // padded smem row (bytes)

// int8 digit planes of an int32 residue block: plane d at
// P[(d * rows + r) * ks + c], ks = cols rounded up to 64, zero padded.
__global__ void split_i8_kernel(const int32_t *__restrict__ X, int64_t ldx, int64_t rows,
                                int64_t cols, int64_t ks, int L, ModP m, int8_t *P) {
  const int64_t total = rows * ks;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / ks, c = t - (t / ks) * ks;
    int32_t x = c < cols ? bal(X[r * ldx + c], m) : 0;
    for (int d = 0; d < L; ++d) {
      int32_t dig;
      if (d < L - 1) {
        dig = ((x + 128) & 255) - 128;
        x = (x - dig) >> 8;
      } else {
        dig = x;
      }
      P[((int64_t)d * rows + r) * ks + c] = (int8_t)dig;
    }
  }
}

__device__ __forceinline__ void mma_s8(int32_t (&d)[4], const uint32_t (&a)[4],
                                       const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct I8Args {
  const int8_t *xp, *yp;  // digit planes
  int64_t M, N, ks;       // rows of X, rows of Y, padded K
  int L;
  uint32_t w2;            // 2^8 mod p (Horner base)
  int32_t *out;
  int64_t ldo;
  int lower;
  Lin lin;
  ModP m;
};

// One 128 x 128 output tile per CTA; digit pairs (i, j) in decreasing i + j,
// each a full K loop into int32 registers, folded as acc = acc * 2^(8 gap) + D.
__global__ void __launch_bounds__(I8_THREADS) leaf_i8_kernel(I8Args a) {
  __shared__ __align__(16) int8_t sa[2][I8_BM * I8_LD];
  __shared__ __align__(16) int8_t sb[2][I8_BN * I8_LD];
  const int64_t r0 = (int64_t)blockIdx.y * I8_BM, c0 = (int64_t)blockIdx.x * I8_BN;
  if (a.lower && c0 > r0 + I8_BM - 1) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;  // warp tile rows wm*64, cols wn*32
  const int g = lane >> 2, tq = lane & 3;
  const ModP m = a.m;
  int32_t acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0;
  const int kt = (int)(a.ks / I8_BK);
  int prev_s = -1;
  for (int s = 2 * (a.L - 1); s >= 0; --s) {
    for (int di = 0; di < a.L; ++di) {
      const int dj = s - di;
      if (dj < 0 || dj >= a.L) continue;
      // Horner step between pairs: acc = acc * 2^(8 (prev_s - s)) mod p
      if (prev_s >= 0) {
        int64_t f = 1;
        for (int e = 0; e < prev_s - s; ++e) f = (f * a.w2) % m.p;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = red_s64((int64_t)acc[i][j][q] * f, m);
      }
      prev_s = s;
      const int8_t *X = a.xp + (int64_t)di * a.M * a.ks;
      const int8_t *Y = a.yp + (int64_t)dj * a.N * a.ks;
      int32_t d[4][4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) d[i][j][q] = 0;
      // cp.async double buffer: 128 rows x 64 bytes per operand per stage
      auto load = [&](int buf, int k0) {
        for (int c = tid; c < I8_BM * 4; c += I8_THREADS) {
          const int r = c >> 2, q = c & 3;
          const int64_t gr = r0 + r, gc = c0 + r;
          const uint32_t da = (uint32_t)__cvta_generic_to_shared(&sa[buf][r * I8_LD + 16 * q]);
          const uint32_t db = (uint32_t)__cvta_generic_to_shared(&sb[buf][r * I8_LD + 16 * q]);
          const int8_t *srca = X + (gr < a.M ? gr : 0) * a.ks + k0 + 16 * q;
          const int8_t *srcb = Y + (gc < a.N ? gc : 0) * a.ks + k0 + 16 * q;
          const int na = gr < a.M ? 16 : 0, nb = gc < a.N ? 16 : 0;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(da), "l"(srca),
                       "r"(na));
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(db), "l"(srcb),
                       "r"(nb));
        }
        asm volatile("cp.async.commit_group;");
      };
      load(0, 0);
      for (int k = 0; k < kt; ++k) {
        const int buf = k & 1;
        if (k + 1 < kt) {
          load(buf ^ 1, (k + 1) * I8_BK);
          asm volatile("cp.async.wait_group 1;");
        } else {
          asm volatile("cp.async.wait_group 0;");
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < I8_BK; kk += 32) {
          uint32_t af[4][4], bf[4][2];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int8_t *base = &sa[buf][(wm * 64 + i * 16 + g) * I8_LD + kk + 4 * tq];
            af[i][0] = *reinterpret_cast<const uint32_t *>(base);
            af[i][1] = *reinterpret_cast<const uint32_t *>(base + 8 * I8_LD);
            af[i][2] = *reinterpret_cast<const uint32_t *>(base + 16);
            af[i][3] = *reinterpret_cast<const uint32_t *>(base + 8 * I8_LD + 16);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int8_t *base = &sb[buf][(wn * 32 + j * 8 + g) * I8_LD + kk + 4 * tq];
            bf[j][0] = *reinterpret_cast<const uint32_t *>(base);
            bf[j][1] = *reinterpret_cast<const uint32_t *>(base + 16);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_s8(d[i][j], af[i], bf[j]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][j][q] += d[i][j][q];
    }
  }
  // canonical store; fragment (i, j): rows g, g+8 of the m16 tile, columns
  // 2 tq, 2 tq + 1 of the n8 tile
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t r = r0 + wm * 64 + i * 16 + g + (q >> 1) * 8;
        const int64_t c = c0 + wn * 32 + j * 8 + 2 * tq + (q & 1);
        if (r >= a.M || c >= a.N || (a.lower && c > r)) continue;
        const int32_t v = red_s64((int64_t)acc[i][j][q], m);
        const int32_t old = a.lin.beta.w ? a.out[r * a.ldo + c] : 0;
        a.out[r * a.ldo + c] = (int32_t)lin_apply(v, old, a.lin, m);
      }
}

// ------------------------------------------------------------------ FP64

constexpr int F_BM = 64, F_BN = 64, F_BK = 16;
constexpr int F_THREADS = 128;  // 4 warps: 2 x 2, warp tile 32 x 32

struct F64Args {
  const int32_t *X, *Y;
  int64_t ldx, ldy, M, N, K;
  int64_t kchunk;  // K steps per exact FP64 chunk (a multiple of F_BK)
  int32_t *out;
  int64_t ldo;
  int lower;
  Lin lin;
  ModP m;
};

__device__ __forceinline__ void mma_f64(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

__device__ __forceinline__ double reduce_f64(double x, double p) {
  return x - p * floor(x / p);  // exact for integers |x| < 2^53
}

__global__ void __launch_bounds__(F_THREADS) leaf_f64_kernel(F64Args a) {
  __shared__ double sa[F_BM][F_BK + 1];
  __shared__ double sb[F_BN][F_BK + 1];
  const int64_t r0 = (int64_t)blockIdx.y * F_BM, c0 = (int64_t)blockIdx.x * F_BN;
  if (a.lower && c0 > r0 + F_BM - 1) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, tq = lane & 3;
  const ModP m = a.m;
  const double pd = (double)m.p;
  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  int64_t inchunk = 0;
  for (int64_t k0 = 0; k0 < a.K; k0 += F_BK) {
    for (int c = tid; c < F_BM * F_BK; c += F_THREADS) {
      const int r = c / F_BK, kk = c % F_BK;
      const int64_t gr = r0 + r, gc = c0 + r, gk = k0 + kk;
      sa[r][kk] = (gr < a.M && gk < a.K) ? (double)bal(a.X[gr * a.ldx + gk], m) : 0.0;
      sb[r][kk] = (gc < a.N && gk < a.K) ? (double)bal(a.Y[gc * a.ldy + gk], m) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < F_BK; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) af[i] = sa[wm * 32 + i * 8 + g][kk + tq];
#pragma unroll
      for (int j = 0; j < 4; ++j) bf[j] = sb[wn * 32 + j * 8 + g][kk + tq];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_f64(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
    inchunk += F_BK;
    if (inchunk >= a.kchunk) {  // keep every partial sum an exact FP64 integer
      inchunk = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j][0] = reduce_f64(acc[i][j][0], pd);
          acc[i][j][1] = reduce_f64(acc[i][j][1], pd);
        }
    }
  }
  // fragment (i, j): row g of the m8 tile, columns 2 tq, 2 tq + 1
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int64_t r = r0 + wm * 32 + i * 8 + g;
        const int64_t c = c0 + wn * 32 + j * 8 + 2 * tq + q;
        if (r >= a.M || c >= a.N || (a.lower && c > r)) continue;
        const int32_t v = red_s64((int64_t)reduce_f64(acc[i][j][q], pd), m);
        const int32_t old = a.lin.beta.w ? a.out[r * a.ldo + c] : 0;
        a.out[r * a.ldo + c] = (int32_t)lin_apply(v, old, a.lin, m);
      }
}

int grid_mma(int64_t total) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)sms * 16));
}

}  // namespace

int i8_digits(uint32_t p) {
  int64_t X = (p - 1) / 2;
  int L = 1;
  while (X > 127 && L < 8) {
    X = (X + 128) >> 8;
    ++L;
  }
  return L;
}

size_t leaf_i8_workspace(int64_t M, int64_t N, int64_t K, uint32_t p) {
  const int64_t ks = (K + I8_BK - 1) / I8_BK * I8_BK;
  const int L = i8_digits(p);
  return (size_t)L * (M + N) * ks + 512;
}

cudaError_t launch_leaf_i8(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                           int64_t M, int64_t N, int64_t K, int32_t *out, int64_t ldo, int lower,
                           const Lin &lin, const ModP &m, void *ws, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int L = i8_digits(m.p);
  // int32 accumulation of one digit pair: (p-1)/2 + K 127^2 < 2^31
  if ((double)m.half + (double)K * 16384.0 >= 2147483647.0) return cudaErrorInvalidValue;
  const int64_t ks = (K + I8_BK - 1) / I8_BK * I8_BK;
  int8_t *xp = (int8_t *)ws;
  int8_t *yp = xp + (size_t)L * M * ks;
  yp = (int8_t *)(((uintptr_t)yp + 255) & ~(uintptr_t)255);
  {
    ProfScope prof(AAT_K_SPLIT, st, (double)M * K * (4.0 + L));
    split_i8_kernel<<<grid_mma(M * ks), 256, 0, st>>>(X, ldx, M, K, ks, L, m, xp);
  }
  {
    ProfScope prof(AAT_K_SPLIT, st, (double)N * K * (4.0 + L));
    split_i8_kernel<<<grid_mma(N * ks), 256, 0, st>>>(Y, ldy, N, K, ks, L, m, yp);
  }
  I8Args a;
  a.xp = xp;
  a.yp = yp;
  a.M = M;
  a.N = N;
  a.ks = ks;
  a.L = L;
  a.w2 = (uint32_t)(256u % m.p);
  a.out = out;
  a.ldo = ldo;
  a.lower = lower;
  a.lin = lin;
  a.m = m;
  dim3 grid((unsigned)((N + I8_BN - 1) / I8_BN), (unsigned)((M + I8_BM - 1) / I8_BM));
  const double macs = lower ? 0.5 * (double)M * (double)(M + 1) * K : (double)M * N * K;
  ProfScope prof(AAT_K_LEAF_MMA, st, 2.0 * L * L * macs);
  leaf_i8_kernel<<<grid, I8_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_leaf_f64(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                            int64_t M, int64_t N, int64_t K, int32_t *out, int64_t ldo, int lower,
                            const Lin &lin, const ModP &m, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  // partial sums: p (after a reduction) + kchunk ((p-1)/2)^2 < 2^53
  const double h = (double)m.half;
  const double room = 9007199254740992.0 - 2.0 * (double)m.p;
  int64_t kchunk = (int64_t)(room / (h * h > 1.0 ? h * h : 1.0));
  kchunk = kchunk / F_BK * F_BK;
  if (kchunk < F_BK) return cudaErrorInvalidValue;  // p too large for exact FP64
  F64Args a;
  a.X = X;
  a.Y = Y;
  a.ldx = ldx;
  a.ldy = ldy;
  a.M = M;
  a.N = N;
  a.K = K;
  a.kchunk = kchunk;
  a.out = out;
  a.ldo = ldo;
  a.lower = lower;
  a.lin = lin;
  a.m = m;
  dim3 grid((unsigned)((N + F_BN - 1) / F_BN), (unsigned)((M + F_BM - 1) / F_BM));
  const double macs = lower ? 0.5 * (double)M * (double)(M + 1) * K : (double)M * N * K;
  ProfScope prof(AAT_K_LEAF_MMA, st, 2.0 * macs);
  leaf_f64_kernel<<<grid, F_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------- peak rate of the instructions

namespace {

constexpr int kPeakChains = 8;  // independent accumulators per thread

// Each warp issues `iters` rounds of kPeakChains independent mma.sync on
// register operands (no memory traffic); the accumulators feed a store that
// a runtime flag (always 0) guards, so nothing is optimised away.
__global__ void __launch_bounds__(256) peak_s8_kernel(int64_t iters, int64_t *sink, int store) {
  uint32_t a[4], b[2];
  for (int i = 0; i < 4; ++i) a[i] = 0x01010101u * (uint32_t)((threadIdx.x + i) & 3);
  b[0] = 0x01010101u * (threadIdx.x & 1);
  b[1] = 0x01010101u * ((threadIdx.x >> 1) & 1);
  int32_t d[kPeakChains][4] = {};
  for (int64_t it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) mma_s8(d[c], a, b);
  int64_t acc = 0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) acc += (int64_t)d[c][0] + d[c][1] + d[c][2] + d[c][3];
  if (store) sink[0] = acc;
}

__global__ void __launch_bounds__(256) peak_f64_kernel(int64_t iters, int64_t *sink, int store) {
  const double a = 1.0 + 1e-3 * (threadIdx.x & 7), b = 1.0 - 1e-3 * (threadIdx.x & 3);
  double d[kPeakChains][2] = {};
  for (int64_t it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) mma_f64(d[c], a, b);
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) acc += d[c][0] + d[c][1];
  if (store) sink[0] = (int64_t)acc;
}

}  // namespace

}  // namespace aat

extern "C" AAT_API int aatx_mma_peak(int kind, int64_t iters, int blocks, void *sink,
                                     double *ops, void *stream) {
  using namespace aat;
  if ((kind != 0 && kind != 1) || iters <= 0 || blocks <= 0 || !sink || !ops)
    return report_error(AAT_EINVAL, "kind 0 (INT8) or 1 (FP64), iters > 0, blocks > 0, sink, ops");
  int e = check_gb300();
  if (e) return e;
  const double warps = (double)blocks * 8.0;
  // ops per warp-level instruction: 2 M N K (m16n8k32: 8192; m8n8k4: 512)
  const double per = kind == 0 ? 2.0 * 16 * 8 * 32 : 2.0 * 8 * 8 * 4;
  *ops = warps * (double)iters * kPeakChains * per;
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == 0)
    peak_s8_kernel<<<blocks, 256, 0, st>>>(iters, (int64_t *)sink, 0);
  else
    peak_f64_kernel<<<blocks, 256, 0, st>>>(iters, (int64_t *)sink, 0);
  cudaError_t ce = cudaGetLastError();
  return ce == cudaSuccess ? AAT_OK : report_error(AAT_ECUDA, cudaGetErrorString(ce));
}
