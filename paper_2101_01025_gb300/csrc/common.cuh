// common.cuh -- shared definitions of the CUDA path: modular arithmetic on
// balanced residues, the digit-plane layout of the tensor-core leaves, the
// device status word and the internal launcher declarations.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/aat.h"

namespace aat {

// ---------------------------------------------------------------- F_p

// Constants of an odd prime p < 2^31.  Residues inside the library are
// int32 values congruent to the residue with |x| < p; "balanced" means
// |x| <= (p - 1) / 2.
struct ModP {
  uint32_t p;     // the prime
  uint32_t half;  // (p - 1) / 2
  uint64_t mu;    // floor(2^64 / p), Barrett constant
  uint64_t off;   // a multiple of p, >= 2^62: x + off >= 0 for |x| < 2^62
  uint32_t mu32;  // floor(2^32 / p)
};

ModP make_modp(uint32_t p);

// Barrett reduction (Barrett 1986) of x < 2^64: the estimate q is at most
// 2 below floor(x / p), so two conditional subtractions finish it.
__host__ __device__ __forceinline__ uint32_t red_u64(uint64_t x, const ModP &m) {
#ifdef __CUDA_ARCH__
  uint64_t q = __umul64hi(x, m.mu);
#else
  uint64_t q = (uint64_t)(((unsigned __int128)x * m.mu) >> 64);
#endif
  uint64_t r = x - q * (uint64_t)m.p;
  if (r >= m.p) r -= m.p;
  if (r >= m.p) r -= m.p;
  return (uint32_t)r;
}

__host__ __device__ __forceinline__ int32_t to_bal(uint32_t r, const ModP &m) {
  return r > m.half ? (int32_t)r - (int32_t)m.p : (int32_t)r;
}

// Any |x| < 2^62 to balanced.
__host__ __device__ __forceinline__ int32_t red_s64(int64_t x, const ModP &m) {
  return to_bal(red_u64((uint64_t)x + m.off, m), m);
}

// Any |x| < 2^62 to canonical [0, p).
__host__ __device__ __forceinline__ uint32_t red_s64_canon(int64_t x, const ModP &m) {
  return red_u64((uint64_t)x + m.off, m);
}

// Any int32 to canonical [0, p) with a 32-bit Barrett step: the estimate
// q = floor(|x| mu32 / 2^32) is at most 2 below floor(|x| / p).
__host__ __device__ __forceinline__ uint32_t red_i32_canon(int32_t x, const ModP &m) {
  const uint32_t ax = x < 0 ? (uint32_t)(-(int64_t)x) : (uint32_t)x;
#ifdef __CUDA_ARCH__
  const uint32_t q = __umulhi(ax, m.mu32);
#else
  const uint32_t q = (uint32_t)(((uint64_t)ax * m.mu32) >> 32);
#endif
  uint32_t r = ax - q * m.p;
  if (r >= m.p) r -= m.p;
  if (r >= m.p) r -= m.p;
  return (x < 0 && r) ? m.p - r : r;
}

// |x| < p to balanced.
__host__ __device__ __forceinline__ int32_t bal(int32_t x, const ModP &m) {
  if (x > (int32_t)m.half) return x - (int32_t)m.p;
  if (x < -(int32_t)m.half) return x + (int32_t)m.p;
  return x;
}

// a + b for balanced a, b (result balanced).
__host__ __device__ __forceinline__ int32_t add_bal(int32_t a, int32_t b, const ModP &m) {
  int32_t s = a + b;  // |s| <= p - 1 < 2^31
  return bal(s, m);
}

__host__ __device__ __forceinline__ int32_t sub_bal(int32_t a, int32_t b, const ModP &m) {
  int32_t s = a - b;
  return bal(s, m);
}

__host__ __device__ __forceinline__ uint32_t bal_to_canon(int32_t x, const ModP &m) {
  return x < 0 ? (uint32_t)(x + (int32_t)m.p) : (uint32_t)x;
}

// a * w mod p, balanced, for p < 2^30 and any int32 a, with the multiplier
// balanced (wb = w or w - p, |wb| <= (p - 1)/2) and wsh = floor(wb 2^32 / p)
// (|wsh| < 2^31; Shoup's method with signed operands): q = floor(a wsh /
// 2^32), the signed high word, leaves r = a wb - q p = a t / 2^32 + p s / 2^32
// with t = wb 2^32 - wsh p in [0, p) and s in [0, 2^32), so r lies in
// (-p/2, 3p/2) (inside int32 for p < 2^30) and one conditional subtraction
// makes it balanced.  Five instructions instead of the unsigned form's ten.
__host__ __device__ __forceinline__ int32_t mulmod_shoup_s(int32_t a, int32_t wb, int32_t wsh,
                                                           const ModP &m) {
#ifdef __CUDA_ARCH__
  const int32_t q = __mulhi(a, wsh);
#else
  const int32_t q = (int32_t)(((int64_t)a * wsh) >> 32);
#endif
  int32_t r = (int32_t)((uint32_t)a * (uint32_t)wb - (uint32_t)q * m.p);
  if (r > (int32_t)m.half) r -= (int32_t)m.p;
  return r;
}

// a * w mod p, balanced, for any int32 a and a fixed w in [0, p) with
// wsh = floor(w 2^32 / p) (Shoup's modular multiplication): with |a| < 2^32,
// |a| w - floor(|a| wsh / 2^32) p lies in [0, 2p), so 32-bit arithmetic and
// one conditional subtraction give the residue.
__host__ __device__ __forceinline__ int32_t mulmod_shoup(int32_t a, uint32_t w, uint32_t wsh,
                                                         const ModP &m) {
  const uint32_t ax = a < 0 ? 0u - (uint32_t)a : (uint32_t)a;
#ifdef __CUDA_ARCH__
  const uint32_t q = __umulhi(ax, wsh);
#else
  const uint32_t q = (uint32_t)(((uint64_t)ax * wsh) >> 32);
#endif
  uint32_t r = ax * w - q * m.p;
  if (r >= m.p) r -= m.p;
  const int32_t b = r > m.half ? (int32_t)r - (int32_t)m.p : (int32_t)r;
  return a < 0 ? -b : b;
}

// Shoup's quotient of a fixed multiplier w (reduced mod p first).
struct MulConst {
  uint32_t w, wsh;
};
inline MulConst mul_const(uint64_t w, uint32_t p) {
  MulConst c;
  c.w = (uint32_t)(w % p);
  c.wsh = (uint32_t)(((uint64_t)c.w << 32) / p);
  return c;
}

// The epilogue of a leaf product: out <- alpha * product + beta * out (mod p)
// (the SYRK update C <- alpha A A^T + beta C, Sec. 7; alpha = 1, beta = 0
// stores the product, beta = 1 accumulates).  Inputs in out must satisfy
// |x| < p; the stored value is canonical.
struct Lin {
  MulConst alpha, beta;
};
inline Lin lin_of(uint64_t alpha, uint64_t beta, uint32_t p) {
  Lin l;
  l.alpha = mul_const(alpha, p);
  l.beta = mul_const(beta, p);
  return l;
}

__host__ __device__ __forceinline__ uint32_t lin_apply(int32_t v, int32_t old, const Lin &L,
                                                       const ModP &m) {
  if (L.alpha.w != 1u) v = mulmod_shoup(v, L.alpha.w, L.alpha.wsh, m);
  if (L.beta.w != 0u) {
    int32_t o = bal(old, m);
    if (L.beta.w != 1u) o = mulmod_shoup(o, L.beta.w, L.beta.wsh, m);
    v = add_bal(v, o, m);
  }
  return bal_to_canon(v, m);
}

// ------------------------------------------------------ skew-unitary Y

// ykind 1: Y = i I, i^2 = -1 (Sec. 4.2).
// ykind 2: Y = [[a, b], [-b, a]] (x) I_{kappa/2} (Prop. 4.2): column j < kappa/2
// of X Y is a X_j - b X_{j+kappa/2}; column j + kappa/2 is b X_j + a X_{j+kappa/2}.
struct YParams {
  int kind;
  int32_t a;  // balanced: i for kind 1, a for kind 2
  int32_t b;  // balanced: 0 for kind 1
};

// ---------------------------------------------------- digit planes

// A residue block X (rows x cols) stored as digit planes in bf16: nbase
// planes of signed base-2^b digits, X = sum_d 2^(b d) D_d, followed by nsum
// planes of pair sums D_si[q] + D_sj[q]; every value is an integer of
// magnitude <= 256, exactly representable in bf16.  Plane d, row r, column c
// lives at ptr[(d * rows + r) * kstride + c]; kstride is a multiple of 8
// (16-byte rows for the tensor memory accelerator).
// (I, J), I >= J >= 0, of entry pid of a lower triangle numbered row by row
// (pid = I (I + 1) / 2 + J): a single-precision square root as the guess,
// made exact by integer steps (this GPU has few FP64 units, and every thread
// of a block computes it).
__device__ __forceinline__ void tri_index(int64_t pid, int64_t &I, int64_t &J) {
  int64_t i = (int64_t)((sqrtf(8.0f * (float)pid + 1.0f) - 1.0f) * 0.5f);
  if (i < 0) i = 0;
  while (i * (i + 1) / 2 > pid) --i;
  while ((i + 1) * (i + 2) / 2 <= pid) ++i;
  I = i;
  J = pid - i * (i + 1) / 2;
}

struct Planes {
  __nv_bfloat16 *ptr;
  int64_t rows;
  int64_t cols;
  int64_t kstride;
  int L;        // planes stored: planes q0 .. q0 + L - 1 of the sequence
  int nbase;    // digit planes of the sequence
  int nsum;     // pair-sum planes of the sequence (after the digit planes)
  int8_t si[8], sj[8];  // pair of plane nbase + q (always (0,1), (0,2), ...)
  int q0;       // first stored plane (0 unless only a window of the planes is kept)
};

struct DigitSpec {
  int b;          // digit width in bits
  int L;          // number of digits
  int dmax[8];    // bound on |digit| per position
  int nsum;       // pair-sum planes (0: every digit pair is its own product)
  int si[8], sj[8];
};

__device__ __forceinline__ uint2 pack4(float a, float b, float c, float d) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(a, b);
  __nv_bfloat162 hi = __floats2bfloat162_rn(c, d);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t *>(&lo);
  u.y = *reinterpret_cast<uint32_t *>(&hi);
  return u;
}

// Balanced digits of V consecutive balanced residues x[0..V-1] at columns
// c..c+V-1 (all digits but the last in [-2^(b-1), 2^(b-1) - 1], the last
// carries the rest), written to the NB digit planes; then, if P.nsum > 0,
// the pair sums d_i + d_j for i < j in the order (0,1), (0,2), ...,
// (NB-2,NB-1).  Only the planes of P's window [q0, q0 + L) of that sequence
// are stored.  V = 4 needs c % 4 == 0 and 8-byte aligned rows (one 8-byte
// store per plane).
template <int NB, int V>
__device__ __forceinline__ void store_digits_t(const Planes &P, int64_t r, int64_t c,
                                               const int32_t (&x0)[V], int b) {
  const int32_t half = 1 << (b - 1);
  const int32_t mask = (1 << b) - 1;
  const int64_t plane = P.rows * P.kstride;
  __nv_bfloat16 *dst = P.ptr + r * P.kstride + c;
  int32_t dig[NB][V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    int32_t x = x0[v];
#pragma unroll
    for (int d = 0; d < NB - 1; ++d) {
      dig[d][v] = ((x + half) & mask) - half;
      x = (x - dig[d][v]) >> b;
    }
    dig[NB - 1][v] = x;
  }
  // only the planes of the window [q0, q0 + L) are stored, at 0 .. L - 1
  auto put = [&](int pl, const int32_t (&w)[V]) {
    const int s = pl - P.q0;
    if ((unsigned)s >= (unsigned)P.L) return;
    if constexpr (V == 4) {
      *reinterpret_cast<uint2 *>(dst + s * plane) =
          pack4((float)w[0], (float)w[1], (float)w[2], (float)w[3]);
    } else {
      dst[s * plane] = __float2bfloat16_rn((float)w[0]);
    }
  };
#pragma unroll
  for (int d = 0; d < NB; ++d) put(d, dig[d]);
  if (P.nsum > 0) {
    int q = NB;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
      for (int j = i + 1; j < NB; ++j) {
        int32_t w[V];
#pragma unroll
        for (int v = 0; v < V; ++v) w[v] = dig[i][v] + dig[j][v];
        put(q++, w);
      }
  }
}

// --------------------------------------------------- device status

// Sticky status word written by kernels whose bounded waits give up.
int32_t *device_status_ptr();

// --------------------------------------------------- instrumentation

// Brackets one kernel launch with CUDA events on its stream while profiling
// is on (aat_profile_begin / aat_profile_end); `work` is the algorithmic
// FLOPs or bytes of the launch.
struct ProfScope {
  int idx;
  ProfScope(int cls, cudaStream_t st, double work);
  ~ProfScope();
};

// ------------------------------------------------ internal launchers

// K1: the four additions of Algorithm 1 with Y applied in registers.
// Reads the four h x kappa blocks of A once.  Every output is optional
// (a null pointer skips it): S1..S4 as int32 canonical residues, S1..S4 as
// digit planes, and digit planes of A11, A12, A22.
struct SKernelOut {
  int32_t *s[4];
  int64_t lds[4];
  Planes sp[4];
  Planes a11, a12, a22;
};
// Rows [r0, r1) of the four blocks (default: all h rows).
cudaError_t launch_sblocks(const int32_t *A, int64_t lda, int64_t h, int64_t kappa,
                           const ModP &m, const YParams &y, int b,
                           const SKernelOut &o, cudaStream_t st, int64_t r0 = 0,
                           int64_t r1 = -1);

// Winograd's form of Strassen's algorithm for a general product X Y^T (one
// level): the digit planes of the seven operand blocks of one side (left:
// X11, X12, X22, S1..S4; right: Y11, Y12, Y22, V1..V4, see k_adds.cu), and
// the seven additions after the products.
struct WinoPlanes {
  Planes q[7];
};
cudaError_t launch_wino_operands(const int32_t *Z, int64_t ldz, int64_t R, int64_t K, const ModP &m,
                                 int b, bool right, const WinoPlanes &o, cudaStream_t st);
cudaError_t launch_wino_combine(const int32_t *W, int64_t ldw, int64_t wstride, int32_t *C,
                                int64_t ldc, int64_t R, int64_t N, const ModP &m,
                                cudaStream_t st);

// Split an int32 residue block into digit planes.
cudaError_t launch_split(const int32_t *X, int64_t ldx, int64_t rows, int64_t cols,
                         const ModP &m, int b, const Planes &P, cudaStream_t st);

// What the SYRK schedule (Table 4) saved of C22 before it received P4^T:
// its strictly lower part transposed into the upper triangle `up` of C11
// (row stride ldc), its diagonal in dg; U5 gains beta times it.
struct SyrkSave {
  const int32_t *up;
  const int32_t *dg;
  MulConst beta;
};

// K6: U4 and U5 of Algorithm 1 from P1 (Low, at P1 with row stride ldp: C11
// in Table 3), P5 (Low, in C12), P3 (in C21) and P4^T (in C22); writes U4
// over C21 and Low(U5) (+ beta Low(C22 before), SYRK) over C22.
cudaError_t launch_postadd(const int32_t *P1, int64_t ldp, int32_t *C12, int32_t *C21,
                           int32_t *C22, int64_t ldc, int64_t h, const ModP &m, cudaStream_t st,
                           const SyrkSave *sv = nullptr);

// Up(C11) <- Low(C22)^T strictly, dg <- diag(C22) (SYRK, Table 4).
cudaError_t launch_save_c22(int32_t *C11, const int32_t *C22, int64_t ldc, int64_t h, int32_t *dg,
                            cudaStream_t st);

// Low(C) <- beta Low(C).
cudaError_t launch_scale_low(int32_t *C, int64_t ldc, int64_t n, MulConst beta, const ModP &m,
                             cudaStream_t st);

// Low(C11) <- Low(C11 + S)   (U3 = P1 + P2)
cudaError_t launch_add_low(int32_t *C11, int64_t ldc, const int32_t *S, int64_t lds, int64_t h,
                           const ModP &m, cudaStream_t st);

// Copy / pad: dst (rows_d x cols_d) <- src (rows x cols) with zeros outside.
cudaError_t launch_pad_copy(const int32_t *src, int64_t lds, int64_t rows, int64_t cols,
                            int32_t *dst, int64_t ldd, int64_t rows_d, int64_t cols_d,
                            cudaStream_t st);
// Low(dst) <- Low(src) for an n x n block.
cudaError_t launch_copy_low(const int32_t *src, int64_t lds, int32_t *dst, int64_t ldd,
                            int64_t n, cudaStream_t st);
cudaError_t launch_zero_upper(int32_t *C, int64_t ldc, int64_t n, cudaStream_t st);
// Quaternion M M^H (Sec. 6.2): the sums U1 = A + B, U2 = C + D, U12 = U1 + U2
// (row stride ldu), and the closing additions from Q1..Q5 (Q_i at
// Q + i qstride, row stride ldq) and Low(Q6) (in H1) to Low(H1..H4).
cudaError_t launch_quat_sums(const int32_t *A, const int32_t *B, const int32_t *C,
                             const int32_t *D, int64_t lda, int64_t n, int64_t k, int32_t *U1,
                             int32_t *U2, int32_t *U12, int64_t ldu, const ModP &m,
                             cudaStream_t st);
cudaError_t launch_quat_combine(const int32_t *Q, int64_t ldq, int64_t qstride, int32_t *H1,
                                int32_t *H2, int32_t *H3, int32_t *H4, int64_t ldh, int64_t n,
                                const ModP &m, cudaStream_t st);

// count balanced residues mod p, element t = SplitMix64 output t of stream
// `seed` mapped to [0, p) by (z >> 32) p >> 32 (synthetic tuning inputs).
cudaError_t launch_fill_residues(int32_t *A, int64_t count, uint32_t p, uint64_t seed,
                                 cudaStream_t st);

// Plain CUDA-core leaf: out <- alpha X Y^T + beta out mod p (lin; lower
// triangle only if `lower`).  Exact int64 arithmetic.
cudaError_t launch_leaf_simt(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                             int64_t M, int64_t N, int64_t K, int32_t *out, int64_t ldo,
                             int lower, const Lin &lin, const ModP &m, cudaStream_t st);

// Warp-level mma.sync leaves (k_leaf_mma.cu): INT8 digits with exact INT32
// accumulation (workspace: leaf_i8_workspace bytes), and FP64 (exact while
// K ((p-1)/2)^2 < 2^53 per chunk).
int i8_digits(uint32_t p);
size_t leaf_i8_workspace(int64_t M, int64_t N, int64_t K, uint32_t p);
cudaError_t launch_leaf_i8(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                           int64_t M, int64_t N, int64_t K, int32_t *out, int64_t ldo, int lower,
                           const Lin &lin, const ModP &m, void *ws, cudaStream_t st);
cudaError_t launch_leaf_f64(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                            int64_t M, int64_t N, int64_t K, int32_t *out, int64_t ldo, int lower,
                            const Lin &lin, const ModP &m, cudaStream_t st);

// Tensor-core leaf: out = sum over digit pairs (i, j) of 2^(b (i + j))
// X_i Y_j^T mod p on tcgen05 (BF16 digits, FP32 accumulation drained to
// int32 before any partial sum can leave the exact range).
struct TcLeafArgs {
  Planes x, y;            // digit planes of X (M x K) and Y (N x K)
  DigitSpec dx, dy;       // their digit specs
  int64_t M, N, K;
  int32_t *out;
  int64_t ldo;
  int lower;              // only tiles/entries with i >= j
  Lin lin;                // out <- alpha product + beta out
  int exact_bits;         // |partial FP32 sums| kept <= 2^exact_bits
  int form;               // kernel form: 0 chosen from the shape, 1 one CTA, 2 CTA pairs
};
cudaError_t launch_leaf_tc(const TcLeafArgs &a, const ModP &m, cudaStream_t st);
// Up to 16 independent leaf products of one modulus and digit base in one
// persistent launch (one tile list over all of them).
cudaError_t launch_leaf_tc_multi(const TcLeafArgs *as, int count, const ModP &m,
                                 cudaStream_t st);
// Whether that one launch is expected to beat one launch per product (the
// idle share of the separate launches' last waves).
bool leaf_tc_fuse_pays(const TcLeafArgs *as, int count);
// Plane products with a non-zero weight mod p that the leaf runs for a
// (only the terms whose planes the operands' plane windows hold); -1 when
// the product does not fit the group table.
int leaf_tc_terms(const TcLeafArgs &a, const ModP &m);
void leaf_tc_release();
// status word of the allocation-free entry point (AAT_OK if it never ran)
int noalloc_status(int reset);

// A batched tensor-core leaf launch: device tables (per-problem tensor maps,
// group tables, one tile list over every problem) built once, then one
// persistent launch over all tiles per call.
struct LeafBatch {
  void *impl = nullptr;
};
cudaError_t leaf_tc_batch_build(const TcLeafArgs *args, const ModP *mods, int count,
                                LeafBatch *out);
cudaError_t leaf_tc_batch_launch(const LeafBatch &lb, cudaStream_t st);
void leaf_tc_batch_free(LeafBatch *lb);

// Batched split: one launch, problem q in blockIdx.y.
struct SplitDesc {
  const int32_t *X;
  int64_t ldx, rows, cols;
  ModP m;
  int b;
  Planes P;
  int first_block;  // first block of this problem in the launch (split_batch_blocks)
  int vec;          // rows start 16-byte aligned and cols % 4 == 0: 4-wide path
};
// Fills first_block / vec of descs (host) and returns the launch's block count.
int split_batch_blocks(SplitDesc *descs, int count);
cudaError_t launch_split_batch(const SplitDesc *descs_dev, int count, int nblocks, double bytes,
                               cudaStream_t st);
void leaf_f32_release();

// Host helpers of the batched plans.
int modp_levels(int64_t n, int64_t k, uint32_t p, uint32_t flags);
Planes planes_layout(const DigitSpec &ds, int64_t rows, int64_t cols);
DigitSpec digits_for_problem(int64_t n, int64_t k, uint32_t p, uint32_t flags);
// One Low(A A^T) mod p with an explicit workspace (dry: only *need).
int modp_run(const int32_t *A, int64_t n, int64_t k, int64_t lda, uint32_t p, int32_t *C,
             int64_t ldc, uint32_t flags, cudaStream_t st, char *ws, bool dry, size_t *need);
// One complex product (method 0: A A^H by 2M, 1: A A^T by 2M, 2: A A^T by
// Algorithm 1) with an explicit workspace (dry: only *need).
int complex_run(int method, const void *A, int64_t n, int64_t k, int64_t lda, void *C,
                int64_t ldc, uint32_t flags, cudaStream_t st, char *ws, bool dry, size_t *need);

// A batch of complex products by Algorithm 2 (2M, A A^H when herm, A A^T
// otherwise) as four launches: one split of every problem, ONE persistent
// FP32 leaf launch over the H and G tiles of all problems, one combine and
// one Hermitian diagonal.  The workspace (cbatch_workspace bytes, caller's)
// holds every problem's planes and products.
struct CBInput {
  const float2 *A;
  int64_t lda, n, k;
  float2 *C;
  int64_t ldc;
  uint32_t flags;  // precision (AAT_C_*)
  int herm;
};
struct CBatch {
  void *impl = nullptr;
};
size_t cbatch_workspace(const CBInput *in, int count);
cudaError_t cbatch_build(const CBInput *in, int count, char *ws, CBatch *out);
cudaError_t cbatch_launch(const CBatch &b, cudaStream_t st);
void cbatch_free(CBatch *b);

// Host helpers shared with the allocation-free entry point (aat_api.cu).
DigitSpec digits_for_prime(uint32_t p);
int check_prime_arg(uint32_t p);
int check_gb300();
int report_error(int code, const char *msg);
// The library's device workspace, grown to at least `bytes`.
int workspace_get(size_t bytes, void **out);

}  // namespace aat
