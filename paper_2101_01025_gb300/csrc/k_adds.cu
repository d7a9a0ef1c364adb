// k_adds.cu -- the block additions of Algorithm 1 (Sec. 3) on the GPU.
//
// These kernels are bound by HBM bandwidth: each reads and writes every
// element once, with consecutive threads on consecutive columns of a row so
// that every warp access is one contiguous segment.
#include <algorithm>

#include "common.cuh"

namespace aat {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int32_t ld_bal(const int32_t *p, const ModP &m) {
  return bal(__ldg(p), m);
}

__device__ __forceinline__ bool has(const Planes &P) { return P.ptr != nullptr; }

// Y applied to the pair (x_j, x_{j+kappa/2}) for kind 2, or to x_j for kind 1.
__device__ __forceinline__ void apply_y2(int32_t x0, int32_t x1, const YParams &y,
                                         const ModP &m, int32_t &o0, int32_t &o1) {
  // [x0 x1] [[a, b], [-b, a]] = [a x0 - b x1, b x0 + a x1]; a = 1 when
  // p = 3 mod 8 (two multiplications instead of three)
  if (y.a == 1) {
    o0 = red_s64((int64_t)x0 - (int64_t)y.b * x1, m);
    o1 = red_s64((int64_t)y.b * x0 + (int64_t)x1, m);
  } else {
    o0 = red_s64((int64_t)y.a * x0 - (int64_t)y.b * x1, m);
    o1 = red_s64((int64_t)y.b * x0 + (int64_t)y.a * x1, m);
  }
}

__device__ __forceinline__ void ld4_bal(const int32_t *p, const ModP &m, int32_t (&v)[4]) {
  const int4 q = __ldg(reinterpret_cast<const int4 *>(p));
  v[0] = bal(q.x, m);
  v[1] = bal(q.y, m);
  v[2] = bal(q.z, m);
  v[3] = bal(q.w, m);
}

__device__ __forceinline__ void st4_canon(int32_t *p, const int32_t (&v)[4], const ModP &m) {
  *reinterpret_cast<int4 *>(p) =
      make_int4((int32_t)bal_to_canon(v[0], m), (int32_t)bal_to_canon(v[1], m),
                (int32_t)bal_to_canon(v[2], m), (int32_t)bal_to_canon(v[3], m));
}

// Outputs of one group of V consecutive columns starting at column j.
template <int V, int NB>
__device__ __forceinline__ void sblocks_store(const SKernelOut &o, int64_t i, int64_t j,
                                              const int32_t (&sv)[4][V], const int32_t (&a11)[V],
                                              const int32_t (&a12)[V], const int32_t (&a22)[V],
                                              const ModP &m, int b) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (o.s[q]) {
      if constexpr (V == 4) {
        st4_canon(o.s[q] + i * o.lds[q] + j, sv[q], m);
      } else {
        o.s[q][i * o.lds[q] + j] = (int32_t)bal_to_canon(sv[q][0], m);
      }
    }
    if (has(o.sp[q])) store_digits_t<NB, V>(o.sp[q], i, j, sv[q], b);
  }
  if (has(o.a11)) store_digits_t<NB, V>(o.a11, i, j, a11, b);
  if (has(o.a12)) store_digits_t<NB, V>(o.a12, i, j, a12, b);
  if (has(o.a22)) store_digits_t<NB, V>(o.a22, i, j, a22, b);
}

template <int V>
__device__ __forceinline__ void ldv_bal(const int32_t *p, const ModP &m, int32_t (&v)[V]) {
  if constexpr (V == 4) {
    ld4_bal(p, m, v);
  } else {
    v[0] = ld_bal(p, m);
  }
}

// One thread per (row i, group of V columns at j): for kind 2, j < kappa/2
// and the thread also handles columns j + kappa/2; for kind 1, j < kappa.
// V = 4 needs kappa/2 (kind 2) or kappa (kind 1), lda, every output stride
// and every plane stride to be multiples of 4 and 16-byte aligned bases.
// NB: digits per residue of every plane output.
// Rows [r0, r1) of the blocks (all of them: r0 = 0, r1 = h).
template <int V, int NB>
__global__ void sblocks_kernel(const int32_t *__restrict__ A, int64_t lda, int64_t h,
                               int64_t kappa, ModP m, YParams y, int b, SKernelOut o,
                               int64_t r0, int64_t r1) {
  const int64_t ncols = ((y.kind == 2) ? kappa / 2 : kappa) / V;
  const int64_t total = (r1 - r0) * ncols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = r0 + t / ncols;
    const int64_t j = (t - (i - r0) * ncols) * V;
    const int32_t *r1 = A + i * lda;        // row i of [A11 A12]
    const int32_t *r2 = A + (h + i) * lda;  // row i of [A21 A22]
    if (y.kind == 2) {
      const int64_t jj = j + kappa / 2;
      int32_t a11_0[V], a11_1[V], a12_0[V], a12_1[V], a21_0[V], a21_1[V], a22_0[V], a22_1[V];
      ldv_bal<V>(r1 + j, m, a11_0);
      ldv_bal<V>(r1 + jj, m, a11_1);
      ldv_bal<V>(r1 + kappa + j, m, a12_0);
      ldv_bal<V>(r1 + kappa + jj, m, a12_1);
      ldv_bal<V>(r2 + j, m, a21_0);
      ldv_bal<V>(r2 + jj, m, a21_1);
      ldv_bal<V>(r2 + kappa + j, m, a22_0);
      ldv_bal<V>(r2 + kappa + jj, m, a22_1);
      int32_t sv0[4][V], sv1[4][V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        // S1 = (A21 - A11) Y
        apply_y2(sub_bal(a21_0[v], a11_0[v], m), sub_bal(a21_1[v], a11_1[v], m), y, m,
                 sv0[0][v], sv1[0][v]);
        // S2 = A22 - A21 Y
        int32_t t0, t1;
        apply_y2(a21_0[v], a21_1[v], y, m, t0, t1);
        sv0[1][v] = sub_bal(a22_0[v], t0, m);
        sv1[1][v] = sub_bal(a22_1[v], t1, m);
        // S3 = S1 - A22, S4 = S3 + A12
        sv0[2][v] = sub_bal(sv0[0][v], a22_0[v], m);
        sv1[2][v] = sub_bal(sv1[0][v], a22_1[v], m);
        sv0[3][v] = add_bal(sv0[2][v], a12_0[v], m);
        sv1[3][v] = add_bal(sv1[2][v], a12_1[v], m);
      }
      sblocks_store<V, NB>(o, i, j, sv0, a11_0, a12_0, a22_0, m, b);
      sblocks_store<V, NB>(o, i, jj, sv1, a11_1, a12_1, a22_1, m, b);
    } else {
      int32_t a11[V], a12[V], a21[V], a22[V];
      ldv_bal<V>(r1 + j, m, a11);
      ldv_bal<V>(r1 + kappa + j, m, a12);
      ldv_bal<V>(r2 + j, m, a21);
      ldv_bal<V>(r2 + kappa + j, m, a22);
      int32_t sv[4][V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        sv[0][v] = red_s64((int64_t)y.a * sub_bal(a21[v], a11[v], m), m);
        sv[1][v] = sub_bal(a22[v], red_s64((int64_t)y.a * a21[v], m), m);
        sv[2][v] = sub_bal(sv[0][v], a22[v], m);
        sv[3][v] = add_bal(sv[2][v], a12[v], m);
      }
      sblocks_store<V, NB>(o, i, j, sv, a11, a12, a22, m, b);
    }
  }
}

template <int V, int NB>
__global__ void split_kernel(const int32_t *__restrict__ X, int64_t ldx, int64_t rows,
                             int64_t cols, ModP m, int b, Planes P) {
  const int64_t ncol = cols / V;
  const int64_t total = rows * ncol;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / ncol, c = (t - (t / ncol) * ncol) * V;
    int32_t v[V];
    ldv_bal<V>(X + r * ldx + c, m, v);
    store_digits_t<NB, V>(P, r, c, v, b);
  }
}

// Winograd's form of Strassen's algorithm for a general product X Y^T: the
// seven operand blocks of one side from the 2 x 2 blocks Z11, Z12, Z21, Z22
// of an int32 residue block Z (2R x 2K), written as digit planes (R x K).
//   left operand (A = X):        X11, X12, X22, S1 = X21 + X22, S2 = S1 - X11,
//                                S3 = X11 - X21, S4 = X12 - S2
//   right operand (B = Y^T, kept in Y's row layout, so T_i = V_i^T):
//                                Y11, Y12, Y22, V1 = Y21 - Y11, V2 = Y22 - V1,
//                                V3 = Y22 - Y21, V4 = V2 - Y12
// The seven products are then X11 Y11^T, X12 Y12^T, S4 Y22^T, X22 V4^T,
// S1 V1^T, S2 V2^T, S3 V3^T.
template <int V, int NB>
__global__ void wino_operands_kernel(const int32_t *__restrict__ Z, int64_t ldz, int64_t R,
                                     int64_t K, ModP m, int b, int right, WinoPlanes o) {
  const int64_t ncols = K / V;
  const int64_t total = R * ncols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ncols;
    const int64_t j = (t - i * ncols) * V;
    const int32_t *r1 = Z + i * ldz, *r2 = Z + (R + i) * ldz;
    int32_t z11[V], z12[V], z21[V], z22[V];
    ldv_bal<V>(r1 + j, m, z11);
    ldv_bal<V>(r1 + K + j, m, z12);
    ldv_bal<V>(r2 + j, m, z21);
    ldv_bal<V>(r2 + K + j, m, z22);
    int32_t u[4][V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (right) {
        u[0][v] = sub_bal(z21[v], z11[v], m);   // V1
        u[1][v] = sub_bal(z22[v], u[0][v], m);  // V2
        u[2][v] = sub_bal(z22[v], z21[v], m);   // V3
        u[3][v] = sub_bal(u[1][v], z12[v], m);  // V4
      } else {
        u[0][v] = add_bal(z21[v], z22[v], m);   // S1
        u[1][v] = sub_bal(u[0][v], z11[v], m);  // S2
        u[2][v] = sub_bal(z11[v], z21[v], m);   // S3
        u[3][v] = sub_bal(z12[v], u[1][v], m);  // S4
      }
    }
    store_digits_t<NB, V>(o.q[0], i, j, z11, b);
    store_digits_t<NB, V>(o.q[1], i, j, z12, b);
    store_digits_t<NB, V>(o.q[2], i, j, z22, b);
#pragma unroll
    for (int q = 0; q < 4; ++q) store_digits_t<NB, V>(o.q[3 + q], i, j, u[q], b);
  }
}

// The seven additions after Winograd's products W1..W7 (canonical int32,
// R x N each, W_q at W + q wstride): C11 = W1 + W2, U2 = W1 + W6,
// U3 = U2 + W7, U4 = U2 + W5, C12 = U4 + W3, C21 = U3 - W4, C22 = U3 + W5;
// C (2R x 2N) canonical.
template <int V>
__global__ void wino_combine_kernel(const int32_t *__restrict__ W, int64_t ldw, int64_t wstride,
                                    int32_t *C, int64_t ldc, int64_t R, int64_t N, ModP m) {
  const int64_t ncols = N / V;
  const int64_t total = R * ncols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ncols;
    const int64_t j = (t - i * ncols) * V;
    int32_t w[7][V];
#pragma unroll
    for (int q = 0; q < 7; ++q) ldv_bal<V>(W + q * wstride + i * ldw + j, m, w[q]);
    int32_t c11[V], c12[V], c21[V], c22[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      c11[v] = add_bal(w[0][v], w[1][v], m);
      const int32_t u2 = add_bal(w[0][v], w[5][v], m);
      const int32_t u3 = add_bal(u2, w[6][v], m);
      const int32_t u4 = add_bal(u2, w[4][v], m);
      c12[v] = add_bal(u4, w[2][v], m);
      c21[v] = sub_bal(u3, w[3][v], m);
      c22[v] = add_bal(u3, w[4][v], m);
    }
    int32_t *o1 = C + i * ldc + j, *o2 = C + (R + i) * ldc + j;
    if constexpr (V == 4) {
      st4_canon(o1, c11, m);
      st4_canon(o1 + N, c12, m);
      st4_canon(o2, c21, m);
      st4_canon(o2 + N, c22, m);
    } else {
      o1[0] = (int32_t)bal_to_canon(c11[0], m);
      o1[N] = (int32_t)bal_to_canon(c12[0], m);
      o2[0] = (int32_t)bal_to_canon(c21[0], m);
      o2[N] = (int32_t)bal_to_canon(c22[0], m);
    }
  }
}

// Batched split: every problem owns ceil(rows / kSplitRows) consecutive
// blocks (first_block ascending), so the work of a block does not depend on
// how large its problem is; a block finds its problem by binary search and
// splits its kSplitRows rows, 4 columns per thread where rows are aligned.
constexpr int kSplitRows = 8;

template <int NB>
__device__ __forceinline__ void split_rows(const SplitDesc &d, int64_t r0) {
  // the block's rows x column quads as one index, so that every thread has
  // work when the rows are short; plane rows are 16-byte aligned (kstride is
  // a multiple of 8), so each quad leaves as one 8-byte store per plane,
  // the columns past the last one written as zeros into the row padding
  // (32-bit index arithmetic: nr * nq < 8 * 2^28)
  const uint32_t nr = (uint32_t)min((int64_t)kSplitRows, d.rows - r0);
  const uint32_t nq = (uint32_t)((d.cols + 3) / 4);
  for (uint32_t t = threadIdx.x; t < nr * nq; t += blockDim.x) {
    const uint32_t ri = t / nq;
    const int64_t c = 4 * (int64_t)(t - ri * nq);
    const int32_t *xr = d.X + (r0 + ri) * d.ldx;
    int32_t v[4];
    if (d.vec) {
      ldv_bal<4>(xr + c, d.m, v);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = c + j < d.cols ? ld_bal(xr + c + j, d.m) : 0;
    }
    store_digits_t<NB, 4>(d.P, r0 + ri, c, v, d.b);
  }
}

__global__ void split_batch_kernel(const SplitDesc *__restrict__ descs, int count) {
  const int b = blockIdx.x;
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (descs[mid].first_block <= b) lo = mid;
    else hi = mid - 1;
  }
  const SplitDesc &d = descs[lo];
  const int64_t r0 = (int64_t)(b - d.first_block) * kSplitRows;
  switch (d.P.nbase) {
    case 1: split_rows<1>(d, r0); break;
    case 2: split_rows<2>(d, r0); break;
    case 3: split_rows<3>(d, r0); break;
    case 4: split_rows<4>(d, r0); break;
    case 5: split_rows<5>(d, r0); break;
    default: break;
  }
}

// Post-additions of Algorithm 1 for one tile pair {(I, J), (J, I)}, I >= J,
// of T x T tiles:
//   U1 = Sym(P1 + P5)         (Low(U1) and Up(U1) = Low(U1)^T)
//   U2 = U1 + P4,  P4 = (P4^T)^T read transposed from C22
//   U4 = U2 + P3              -> C21 (both tiles of the pair)
//   U5 = Low(U2 + P4^T)       -> C22 (lower tile only)
// Both C22 tiles of the pair are read into shared memory before any write,
// and no other block touches them, so the in-place update is safe.
constexpr int T = 32;

// U1 = Sym(P1 + P5), U2 = U1 + P4, U4 = U2 + P3 -> C21 and
// Low(U5) = Low(U2 + P4^T) (+ beta Low(C22 before)) -> C22, one tile pair
// {(I, J), (J, I)} of the h x h blocks per CTA.  P1 is read from `P1` (C11
// in the Table 3 schedule, the temporary in the SYRK one); in the SYRK
// schedule (beta != 0) the strictly lower part of the original C22 is read
// back transposed from `up` (the upper triangle of C11) and its diagonal
// from `dg`.
template <bool SYRK>
__global__ void postadd_kernel(const int32_t *__restrict__ P1, int64_t ldp,
                               const int32_t *__restrict__ C12, int32_t *C21, int32_t *C22,
                               int64_t ldc, int64_t h, ModP m, const int32_t *__restrict__ up,
                               const int32_t *__restrict__ dg, uint32_t beta, uint32_t beta_sh) {
  __shared__ int32_t p4t_ij[T][T + 1];  // C22 tile (I, J) = P4^T block
  __shared__ int32_t p4t_ji[T][T + 1];  // C22 tile (J, I)
  __shared__ int32_t u1_ij[T][T + 1];   // U1 tile (I, J) (lower part source)
  __shared__ int32_t up_ji[SYRK ? T : 1][T + 1];  // saved C22, transposed (tile (J, I) of C11)
  const int64_t ntiles = (h + T - 1) / T;
  // map blockIdx.x to (I, J) with I >= J
  int64_t pid = blockIdx.x;
  int64_t I = (int64_t)((sqrt(8.0 * (double)pid + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > pid) --I;
  while ((I + 1) * (I + 2) / 2 <= pid) ++I;
  const int64_t J = pid - I * (I + 1) / 2;
  if (I >= ntiles) return;
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;  // 32 x 8 threads
  const int64_t r0 = I * T, c0 = J * T;
  // load
  for (int yy = ty; yy < T; yy += 8) {
    int64_t r = r0 + yy, c = c0 + tx;
    if (r < h && c < h) {
      p4t_ij[yy][tx] = bal(C22[r * ldc + c], m);
      // U1(r, c): lower entries from P1 + P5, upper ones by symmetry
      int64_t lr = r >= c ? r : c, lc = r >= c ? c : r;
      u1_ij[yy][tx] = add_bal(bal(P1[lr * ldp + lc], m), bal(C12[lr * ldc + lc], m), m);
    }
    int64_t r2 = c0 + yy, c2 = r0 + tx;  // tile (J, I)
    if (r2 < h && c2 < h) {
      p4t_ji[yy][tx] = bal(C22[r2 * ldc + c2], m);
      if constexpr (SYRK)
        if (r2 < c2) up_ji[yy][tx] = bal(up[r2 * ldc + c2], m);
    }
  }
  __syncthreads();
  // tile (I, J): U4 and U5
  for (int yy = ty; yy < T; yy += 8) {
    int64_t r = r0 + yy, c = c0 + tx;
    if (r < h && c < h) {
      int32_t u1 = u1_ij[yy][tx];
      int32_t p4 = p4t_ji[tx][yy];  // P4(r, c) = P4^T(c, r)
      int32_t u2 = add_bal(u1, p4, m);
      int32_t u4 = add_bal(u2, bal(C21[r * ldc + c], m), m);
      C21[r * ldc + c] = (int32_t)bal_to_canon(u4, m);
      if (r >= c) {
        int32_t u5 = add_bal(u2, p4t_ij[yy][tx], m);
        if constexpr (SYRK) {
          // C22 before the update: (r, c) was saved at (c, r) of C11
          int32_t old = r == c ? bal(dg[r], m) : up_ji[tx][yy];
          if (beta != 1u) old = mulmod_shoup(old, beta, beta_sh, m);
          u5 = add_bal(u5, old, m);
        }
        C22[r * ldc + c] = (int32_t)bal_to_canon(u5, m);
      }
    }
  }
  if (I == J) return;
  // tile (J, I): U4 only (upper tile of C22 is not part of Low(U5))
  for (int yy = ty; yy < T; yy += 8) {
    int64_t r = c0 + yy, c = r0 + tx;  // r < c here
    if (r < h && c < h) {
      int32_t u1 = u1_ij[tx][yy];      // U1(r, c) = U1(c, r)
      int32_t p4 = p4t_ij[tx][yy];     // P4(r, c) = P4^T(c, r)
      int32_t u2 = add_bal(u1, p4, m);
      int32_t u4 = add_bal(u2, bal(C21[r * ldc + c], m), m);
      C21[r * ldc + c] = (int32_t)bal_to_canon(u4, m);
    }
  }
}

// The SYRK schedule's first step (Table 4): Up(C11) <- Low(C22)^T on the
// strictly triangular parts (C11[c][r] = C22[r][c], r > c) and dg[r] =
// C22[r][r], so that C22 can receive P4^T.  One T x T tile of Low(C22) per
// CTA, transposed through shared memory.
__global__ void save_c22_kernel(int32_t *C11, const int32_t *__restrict__ C22, int64_t ldc,
                                int64_t h, int32_t *dg) {
  __shared__ int32_t t[T][T + 1];
  const int64_t ntiles = (h + T - 1) / T;
  int64_t pid = blockIdx.x;
  int64_t I = (int64_t)((sqrt(8.0 * (double)pid + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > pid) --I;
  while ((I + 1) * (I + 2) / 2 <= pid) ++I;
  const int64_t J = pid - I * (I + 1) / 2;
  if (I >= ntiles) return;
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  const int64_t r0 = I * T, c0 = J * T;
  for (int yy = ty; yy < T; yy += 8) {
    const int64_t r = r0 + yy, c = c0 + tx;
    if (r < h && c < h && r >= c) {
      const int32_t v = C22[r * ldc + c];
      t[yy][tx] = v;
      if (r == c) dg[r] = v;
    }
  }
  __syncthreads();
  for (int yy = ty; yy < T; yy += 8) {
    const int64_t rr = c0 + yy, cc = r0 + tx;  // C11 (rr, cc) <- C22 (cc, rr)
    if (rr < h && cc < h && cc > rr) C11[rr * ldc + cc] = t[tx][yy];
  }
}

// Low(C) <- beta Low(C) (the SYRK update with k = 0).
__global__ void scale_low_kernel(int32_t *C, int64_t ldc, int64_t n, uint32_t beta,
                                 uint32_t beta_sh, ModP m) {
  const int64_t total = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, c = t - (t / n) * n;
    if (c > r) continue;
    C[r * ldc + c] = (int32_t)bal_to_canon(mulmod_shoup(bal(C[r * ldc + c], m), beta, beta_sh, m), m);
  }
}

__global__ void add_low_kernel(int32_t *C11, int64_t ldc, const int32_t *__restrict__ S,
                               int64_t lds, int64_t h, ModP m) {
  const int64_t total = h * h;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / h, c = t - (t / h) * h;
    if (c > r) continue;
    int32_t v = add_bal(bal(C11[r * ldc + c], m), bal(S[r * lds + c], m), m);
    C11[r * ldc + c] = (int32_t)bal_to_canon(v, m);
  }
}

__global__ void pad_copy_kernel(const int32_t *__restrict__ src, int64_t lds, int64_t rows,
                                int64_t cols, int32_t *dst, int64_t ldd, int64_t rows_d,
                                int64_t cols_d) {
  const int64_t total = rows_d * cols_d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / cols_d, c = t - (t / cols_d) * cols_d;
    dst[r * ldd + c] = (r < rows && c < cols) ? src[r * lds + c] : 0;
  }
}

__global__ void copy_low_kernel(const int32_t *__restrict__ src, int64_t lds, int32_t *dst,
                                int64_t ldd, int64_t n) {
  const int64_t total = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, c = t - (t / n) * n;
    if (c <= r) dst[r * ldd + c] = src[r * lds + c];
  }
}

__global__ void zero_upper_kernel(int32_t *C, int64_t ldc, int64_t n) {
  const int64_t total = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, c = t - (t / n) * n;
    if (c > r) C[r * ldc + c] = 0;
  }
}

int grid_for(int64_t total) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (total + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sms * 16;  // 16 blocks of 256 threads per SM
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

}  // namespace

cudaError_t launch_sblocks(const int32_t *A, int64_t lda, int64_t h, int64_t kappa,
                           const ModP &m, const YParams &y, int b, const SKernelOut &o,
                           cudaStream_t st, int64_t r0, int64_t r1) {
  if (r1 < 0) r1 = h;
  if (r0 < 0 || r0 > r1 || r1 > h) return cudaErrorInvalidValue;
  const int64_t rows = r1 - r0;
  const int64_t ncols = (y.kind == 2) ? kappa / 2 : kappa;
  const int64_t total = rows * ncols;
  if (total <= 0) return cudaSuccess;
  double bytes = 16.0 * rows * kappa;  // A11, A12, A21, A22 read once
  for (int q = 0; q < 4; ++q) {
    if (o.s[q]) bytes += 4.0 * rows * kappa;
    if (o.sp[q].ptr) bytes += 2.0 * o.sp[q].L * rows * kappa;
  }
  for (const Planes *P : {&o.a11, &o.a12, &o.a22})
    if (P->ptr) bytes += 2.0 * P->L * rows * kappa;
  ProfScope prof(AAT_K_SBLOCKS, st, bytes);
  // 16-byte vector path when every address it touches is aligned
  auto al16 = [](const void *ptr) { return ((uintptr_t)ptr & 15) == 0; };
  bool vec = (ncols % 4 == 0) && (lda % 4 == 0) && al16(A) && (kappa % 4 == 0);
  for (int q = 0; q < 4; ++q) {
    if (o.s[q]) vec = vec && (o.lds[q] % 4 == 0) && al16(o.s[q]);
    if (o.sp[q].ptr) vec = vec && al16(o.sp[q].ptr);
  }
  for (const Planes *P : {&o.a11, &o.a12, &o.a22})
    if (P->ptr) vec = vec && al16(P->ptr);
  int nb = 0;
  for (const Planes *P : {&o.sp[0], &o.sp[1], &o.sp[2], &o.sp[3], &o.a11, &o.a12, &o.a22})
    if (P->ptr) {
      if (nb && P->nbase != nb) return cudaErrorInvalidValue;
      nb = P->nbase;
    }
  if (nb == 0) nb = 1;
  const int g = grid_for(vec ? total / 4 : total);
#define AAT_SB(NBV)                                                                     \
  case NBV:                                                                             \
    if (vec)                                                                            \
      sblocks_kernel<4, NBV><<<g, kThreads, 0, st>>>(A, lda, h, kappa, m, y, b, o, r0, r1); \
    else                                                                                    \
      sblocks_kernel<1, NBV><<<g, kThreads, 0, st>>>(A, lda, h, kappa, m, y, b, o, r0, r1); \
    break;
  switch (nb) {
    AAT_SB(1) AAT_SB(2) AAT_SB(3) AAT_SB(4) AAT_SB(5)
    default:
      return cudaErrorInvalidValue;
  }
#undef AAT_SB
  return cudaGetLastError();
}

cudaError_t launch_wino_operands(const int32_t *Z, int64_t ldz, int64_t R, int64_t K, const ModP &m,
                                 int b, bool right, const WinoPlanes &o, cudaStream_t st) {
  const int64_t total = R * K;
  if (total <= 0) return cudaSuccess;
  const int nb = o.q[0].nbase;
  for (int q = 0; q < 7; ++q)
    if (!o.q[q].ptr || o.q[q].nbase != nb || o.q[q].rows != R || o.q[q].cols != K)
      return cudaErrorInvalidValue;
  ProfScope prof(AAT_K_WINOGRAD, st, (double)total * (16.0 + 7.0 * 2.0 * o.q[0].L));
  bool vec = (K % 4 == 0) && (ldz % 4 == 0) && (((uintptr_t)Z & 15) == 0);
  for (int q = 0; q < 7; ++q) vec = vec && (((uintptr_t)o.q[q].ptr & 15) == 0);
  const int g = grid_for(vec ? total / 4 : total);
  const int rt = right ? 1 : 0;
#define AAT_WO(NBV)                                                                          \
  case NBV:                                                                                  \
    if (vec)                                                                                 \
      wino_operands_kernel<4, NBV><<<g, kThreads, 0, st>>>(Z, ldz, R, K, m, b, rt, o);       \
    else                                                                                     \
      wino_operands_kernel<1, NBV><<<g, kThreads, 0, st>>>(Z, ldz, R, K, m, b, rt, o);       \
    break;
  switch (nb) {
    AAT_WO(1) AAT_WO(2) AAT_WO(3) AAT_WO(4) AAT_WO(5)
    default:
      return cudaErrorInvalidValue;
  }
#undef AAT_WO
  return cudaGetLastError();
}

cudaError_t launch_wino_combine(const int32_t *W, int64_t ldw, int64_t wstride, int32_t *C,
                                int64_t ldc, int64_t R, int64_t N, const ModP &m,
                                cudaStream_t st) {
  const int64_t total = R * N;
  if (total <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_WINOGRAD, st, (double)total * (7.0 + 4.0) * 4.0);
  const bool vec = (N % 4 == 0) && (ldw % 4 == 0) && (wstride % 4 == 0) && (ldc % 4 == 0) &&
                   (((uintptr_t)W & 15) == 0) && (((uintptr_t)C & 15) == 0);
  const int g = grid_for(vec ? total / 4 : total);
  if (vec)
    wino_combine_kernel<4><<<g, kThreads, 0, st>>>(W, ldw, wstride, C, ldc, R, N, m);
  else
    wino_combine_kernel<1><<<g, kThreads, 0, st>>>(W, ldw, wstride, C, ldc, R, N, m);
  return cudaGetLastError();
}

cudaError_t launch_split(const int32_t *X, int64_t ldx, int64_t rows, int64_t cols,
                         const ModP &m, int b, const Planes &P, cudaStream_t st) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_SPLIT, st, (double)total * (4.0 + 2.0 * P.L));
  const bool vec = (cols % 4 == 0) && (ldx % 4 == 0) && (((uintptr_t)X & 15) == 0) &&
                   (((uintptr_t)P.ptr & 15) == 0);
  const int g = grid_for(vec ? total / 4 : total);
#define AAT_SP(NBV)                                                                     \
  case NBV:                                                                             \
    if (vec)                                                                            \
      split_kernel<4, NBV><<<g, kThreads, 0, st>>>(X, ldx, rows, cols, m, b, P);       \
    else                                                                                \
      split_kernel<1, NBV><<<g, kThreads, 0, st>>>(X, ldx, rows, cols, m, b, P);       \
    break;
  switch (P.nbase) {
    AAT_SP(1) AAT_SP(2) AAT_SP(3) AAT_SP(4) AAT_SP(5)
    default:
      return cudaErrorInvalidValue;
  }
#undef AAT_SP
  return cudaGetLastError();
}

int split_batch_blocks(SplitDesc *descs, int count) {
  int64_t nb = 0;
  for (int i = 0; i < count; ++i) {
    SplitDesc &d = descs[i];
    d.first_block = (int)nb;
    d.vec = (d.cols % 4 == 0) && (d.ldx % 4 == 0) && ((reinterpret_cast<uintptr_t>(d.X) & 15) == 0);
    nb += (d.rows + kSplitRows - 1) / kSplitRows;
  }
  return nb > INT32_MAX ? -1 : (int)nb;
}

cudaError_t launch_split_batch(const SplitDesc *descs_dev, int count, int nblocks, double bytes,
                               cudaStream_t st) {
  if (count <= 0 || nblocks <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_SPLIT, st, bytes);
  split_batch_kernel<<<(unsigned)nblocks, kThreads, 0, st>>>(descs_dev, count);
  return cudaGetLastError();
}

cudaError_t launch_postadd(const int32_t *P1, int64_t ldp, int32_t *C12, int32_t *C21,
                           int32_t *C22, int64_t ldc, int64_t h, const ModP &m, cudaStream_t st,
                           const SyrkSave *sv) {
  if (h <= 0) return cudaSuccess;
  const int64_t nt = (h + T - 1) / T;
  const int64_t pairs = nt * (nt + 1) / 2;
  const double tri = 0.5 * (double)h * (double)(h + 1), sq = (double)h * h;
  const bool b = sv && sv->beta.w;
  ProfScope prof(AAT_K_POSTADD, st, 4.0 * ((b ? 4.0 : 3.0) * tri + 3.0 * sq));
  if (b)
    postadd_kernel<true><<<(unsigned)pairs, T * 8, 0, st>>>(P1, ldp, C12, C21, C22, ldc, h, m,
                                                           sv->up, sv->dg, sv->beta.w,
                                                           sv->beta.wsh);
  else
    postadd_kernel<false><<<(unsigned)pairs, T * 8, 0, st>>>(P1, ldp, C12, C21, C22, ldc, h, m,
                                                            nullptr, nullptr, 0u, 0u);
  return cudaGetLastError();
}

cudaError_t launch_save_c22(int32_t *C11, const int32_t *C22, int64_t ldc, int64_t h, int32_t *dg,
                            cudaStream_t st) {
  if (h <= 0) return cudaSuccess;
  const int64_t nt = (h + T - 1) / T;
  ProfScope prof(AAT_K_COPY, st, 8.0 * 0.5 * (double)h * (double)(h + 1));
  save_c22_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, st>>>(C11, C22, ldc, h, dg);
  return cudaGetLastError();
}

cudaError_t launch_scale_low(int32_t *C, int64_t ldc, int64_t n, MulConst beta, const ModP &m,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_COPY, st, 8.0 * 0.5 * (double)n * (double)(n + 1));
  scale_low_kernel<<<grid_for(n * n), kThreads, 0, st>>>(C, ldc, n, beta.w, beta.wsh, m);
  return cudaGetLastError();
}

cudaError_t launch_add_low(int32_t *C11, int64_t ldc, const int32_t *S, int64_t lds, int64_t h,
                           const ModP &m, cudaStream_t st) {
  if (h <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_ADD_LOW, st, 4.0 * 3.0 * 0.5 * (double)h * (double)(h + 1));
  add_low_kernel<<<grid_for(h * h), kThreads, 0, st>>>(C11, ldc, S, lds, h, m);
  return cudaGetLastError();
}

cudaError_t launch_pad_copy(const int32_t *src, int64_t lds, int64_t rows, int64_t cols,
                            int32_t *dst, int64_t ldd, int64_t rows_d, int64_t cols_d,
                            cudaStream_t st) {
  if (rows_d * cols_d <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_COPY, st, 4.0 * ((double)rows * cols + (double)rows_d * cols_d));
  pad_copy_kernel<<<grid_for(rows_d * cols_d), kThreads, 0, st>>>(src, lds, rows, cols, dst,
                                                                  ldd, rows_d, cols_d);
  return cudaGetLastError();
}

cudaError_t launch_copy_low(const int32_t *src, int64_t lds, int32_t *dst, int64_t ldd,
                            int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_COPY, st, 8.0 * 0.5 * (double)n * (double)(n + 1));
  copy_low_kernel<<<grid_for(n * n), kThreads, 0, st>>>(src, lds, dst, ldd, n);
  return cudaGetLastError();
}

// U1 = A + B, U2 = C + D, U12 = U1 + U2 (balanced), the sums of the
// quaternion algorithm of Sec. 6.2 (M = A + B i + C j + D k).
__global__ void quat_sums_kernel(const int32_t *__restrict__ A, const int32_t *__restrict__ B,
                                 const int32_t *__restrict__ C, const int32_t *__restrict__ D,
                                 int64_t lda, int64_t n, int64_t k, int32_t *U1, int32_t *U2,
                                 int32_t *U12, int64_t ldu, ModP m) {
  const int64_t total = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k, c = t - r * k;
    const int64_t s = r * lda + c;
    const int32_t u1 = add_bal(bal(A[s], m), bal(B[s], m), m);
    const int32_t u2 = add_bal(bal(C[s], m), bal(D[s], m), m);
    U1[r * ldu + c] = u1;
    U2[r * ldu + c] = u2;
    U12[r * ldu + c] = add_bal(u1, u2, m);
  }
}

// The additions closing the quaternion algorithm of Sec. 6.2, on the lower
// triangle: T1 = Q1 - Q2, T2 = Q4 + Q5, T3 = (Q1 + Q2) - Q3,
// H1 = Q6 - (Q3^T + Q3) - (T2^T + T2), H2 = T2^T - T2, H3 = T1 - T1^T,
// H4 = T3^T - T3.  Low(Q6) arrives in H1.  One T x T tile (I, J), I >= J,
// per CTA, with tile (J, I) of every Q for the transposed terms.
__global__ void quat_combine_kernel(const int32_t *__restrict__ Q, int64_t ldq, int64_t qstride,
                                    int32_t *H1, int32_t *H2, int32_t *H3, int32_t *H4,
                                    int64_t ldh, int64_t n, ModP m) {
  __shared__ int32_t qt[5][T][T + 1];  // tile (J, I) of Q1..Q5
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
    const int64_t r2 = c0 + yy, c2 = r0 + tx;
    if (r2 < n && c2 < n)
#pragma unroll
      for (int q = 0; q < 5; ++q) qt[q][yy][tx] = bal(Q[q * qstride + r2 * ldq + c2], m);
  }
  __syncthreads();
  for (int yy = ty; yy < T; yy += 8) {
    const int64_t r = r0 + yy, c = c0 + tx;
    if (r >= n || c >= n || c > r) continue;
    int32_t q[5], qT[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      q[i] = bal(Q[i * qstride + r * ldq + c], m);
      qT[i] = qt[i][tx][yy];  // Q_i(c, r)
    }
    const int32_t t1 = sub_bal(q[0], q[1], m), t1T = sub_bal(qT[0], qT[1], m);
    const int32_t t2 = add_bal(q[3], q[4], m), t2T = add_bal(qT[3], qT[4], m);
    const int32_t t3 = sub_bal(add_bal(q[0], q[1], m), q[2], m);
    const int32_t t3T = sub_bal(add_bal(qT[0], qT[1], m), qT[2], m);
    int32_t h1 = sub_bal(bal(H1[r * ldh + c], m), add_bal(qT[2], q[2], m), m);
    h1 = sub_bal(h1, add_bal(t2T, t2, m), m);
    H1[r * ldh + c] = (int32_t)bal_to_canon(h1, m);
    H2[r * ldh + c] = (int32_t)bal_to_canon(sub_bal(t2T, t2, m), m);
    H3[r * ldh + c] = (int32_t)bal_to_canon(sub_bal(t1, t1T, m), m);
    H4[r * ldh + c] = (int32_t)bal_to_canon(sub_bal(t3T, t3, m), m);
  }
}

__global__ void fill_residues_kernel(int32_t *A, int64_t count, uint32_t p, uint64_t seed) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
    uint64_t z = seed + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull;  // SplitMix64
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const uint32_t r = (uint32_t)(((z >> 32) * (uint64_t)p) >> 32);
    A[t] = r > (p - 1) / 2 ? (int32_t)r - (int32_t)p : (int32_t)r;
  }
}

cudaError_t launch_quat_sums(const int32_t *A, const int32_t *B, const int32_t *C,
                             const int32_t *D, int64_t lda, int64_t n, int64_t k, int32_t *U1,
                             int32_t *U2, int32_t *U12, int64_t ldu, const ModP &m,
                             cudaStream_t st) {
  if (n * k <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_COPY, st, 4.0 * 7.0 * (double)n * k);
  quat_sums_kernel<<<grid_for(n * k), kThreads, 0, st>>>(A, B, C, D, lda, n, k, U1, U2, U12, ldu,
                                                          m);
  return cudaGetLastError();
}

cudaError_t launch_quat_combine(const int32_t *Q, int64_t ldq, int64_t qstride, int32_t *H1,
                                int32_t *H2, int32_t *H3, int32_t *H4, int64_t ldh, int64_t n,
                                const ModP &m, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t nt = (n + T - 1) / T;
  const double tri = 0.5 * (double)n * (double)(n + 1);
  ProfScope prof(AAT_K_POSTADD, st, 4.0 * (10.0 * tri + 4.0 * tri + tri));
  quat_combine_kernel<<<(unsigned)(nt * (nt + 1) / 2), T * 8, 0, st>>>(Q, ldq, qstride, H1, H2,
                                                                       H3, H4, ldh, n, m);
  return cudaGetLastError();
}

cudaError_t launch_fill_residues(int32_t *A, int64_t count, uint32_t p, uint64_t seed,
                                 cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  fill_residues_kernel<<<grid_for(count), kThreads, 0, st>>>(A, count, p, seed);
  return cudaGetLastError();
}

cudaError_t launch_zero_upper(int32_t *C, int64_t ldc, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(AAT_K_COPY, st, 4.0 * 0.5 * (double)n * (double)(n - 1));
  zero_upper_kernel<<<grid_for(n * n), kThreads, 0, st>>>(C, ldc, n);
  return cudaGetLastError();
}

}  // namespace aat
