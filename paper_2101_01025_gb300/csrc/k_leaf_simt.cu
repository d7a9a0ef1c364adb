// k_leaf_simt.cu -- a plain CUDA-core leaf: out = X Y^T mod p in exact int64
// arithmetic.  It is the check path for the recursion (AAT_LEAF_SIMT): slow,
// simple, and independent of the digit planes of the tensor-core leaf.
#include "common.cuh"

namespace aat {

namespace {

constexpr int TS = 32;  // output tile TS x TS, 32 x 8 threads, 4 rows each
constexpr int TK = 32;

__global__ void leaf_simt_kernel(const int32_t *__restrict__ X, int64_t ldx,
                                 const int32_t *__restrict__ Y, int64_t ldy, int64_t M,
                                 int64_t N, int64_t K, int32_t *out, int64_t ldo, int lower,
                                 Lin lin, ModP m) {
  __shared__ int32_t xs[TS][TK + 1];
  __shared__ int32_t ys[TS][TK + 1];
  const int64_t r0 = (int64_t)blockIdx.y * TS, c0 = (int64_t)blockIdx.x * TS;
  if (lower && c0 > r0 + TS - 1) return;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  int32_t acc[4] = {0, 0, 0, 0};  // balanced partial sums
  for (int64_t k0 = 0; k0 < K; k0 += TK) {
    for (int yy = ty; yy < TS; yy += 8) {
      int64_t r = r0 + yy, c = c0 + yy, kk = k0 + tx;
      xs[yy][tx] = (r < M && kk < K) ? bal(X[r * ldx + kk], m) : 0;
      ys[yy][tx] = (c < N && kk < K) ? bal(Y[c * ldy + kk], m) : 0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      const int32_t yv = ys[tx][kk];
      for (int q = 0; q < 4; ++q) {
        // |acc| <= p/2, |x y| <= p^2 / 4 < 2^60: the sum stays below 2^62
        acc[q] = red_s64((int64_t)acc[q] + (int64_t)xs[ty + 8 * q][kk] * yv, m);
      }
    }
    __syncthreads();
  }
  for (int q = 0; q < 4; ++q) {
    int64_t r = r0 + ty + 8 * q, c = c0 + tx;
    if (r >= M || c >= N) continue;
    if (lower && c > r) continue;
    const int32_t old = lin.beta.w ? out[r * ldo + c] : 0;
    out[r * ldo + c] = (int32_t)lin_apply(acc[q], old, lin, m);
  }
}

}  // namespace

cudaError_t launch_leaf_simt(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                             int64_t M, int64_t N, int64_t K, int32_t *out, int64_t ldo,
                             int lower, const Lin &lin, const ModP &m, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((unsigned)((N + TS - 1) / TS), (unsigned)((M + TS - 1) / TS));
  const double macs = lower ? 0.5 * (double)M * (double)(M + 1) * K : (double)M * N * K;
  ProfScope prof(AAT_K_LEAF_SIMT, st, 2.0 * macs);
  leaf_simt_kernel<<<grid, 256, 0, st>>>(X, ldx, Y, ldy, M, N, K, out, ldo, lower, lin, m);
  return cudaGetLastError();
}

}  // namespace aat
