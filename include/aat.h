/*
 * aat.h -- C ABI of a GB300 (sm_103a) library for the product of a matrix by
 * its adjoint, after Dumas, Pernet and Sedoglavic, "Some fast algorithms
 * multiplying a matrix by its adjoint".
 *
 *   aat_modp    Low(A A^T) mod p by Algorithm 1 (Sec. 3): a 2x2 block
 *               recursion with 5 block products (3 recursive, 2 general)
 *               after block additions that apply a skew-unitary Y with
 *               Y Y^T = -I (Sec. 4: Y = sqrt(-1) I for p = 1 mod 4, else
 *               Y = [[a, b], [-b, a]] (x) I with a^2 + b^2 = -1 from
 *               Algorithm 3).  The result is exact (Theorem 3.1).
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major.  A is n x k with row stride lda (elements);
 *     C is n x n with row stride ldc.
 *   - Device pointers (unless the name ends in _host).  The caller owns A
 *     and C; C must not overlap A.
 *   - Residues: an entry of A may be any int32 congruent to its residue
 *     with |value| < p (canonical [0, p) or balanced (-p/2, p/2)).
 *   - Output: the lower triangle of C, diagonal included, receives the
 *     canonical residues in [0, p).  The strict upper triangle is used as
 *     scratch (Sec. 7, Table 3) and is unspecified on return unless
 *     AAT_ZERO_UPPER is given.
 *   - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream) unless stated.  Internal workspace is owned by the
 *     library, grown on demand and released by aat_shutdown().
 *   - Return codes: AAT_OK or a negative AAT_E*; aat_last_error() gives a
 *     message for the calling thread.  No entry point falls back to the
 *     CPU: without a usable sm_103a GPU they fail with AAT_ECUDA.
 */
#ifndef AAT_H
#define AAT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AAT_API __attribute__((visibility("default")))
#else
#define AAT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define AAT_OK 0
#define AAT_EINVAL (-1)       /* null pointer, bad size or stride, aliasing */
#define AAT_ENOTPRIME (-2)    /* p is not an odd prime */
#define AAT_ERANGE (-3)       /* p >= 2^31, or no exact leaf for (p, k) */
#define AAT_ENOMEM (-4)       /* device workspace allocation failed */
#define AAT_ECUDA (-5)        /* CUDA error (launch, no device, wrong arch) */
#define AAT_ETIMEOUT (-6)     /* a bounded device wait gave up */
#define AAT_EUNSUPPORTED (-7) /* valid request the library does not provide */

/* flags */
#define AAT_IN_BALANCED (1u << 0) /* informational: A holds balanced residues */
#define AAT_ZERO_UPPER (1u << 1)  /* zero the strict upper triangle of C     */
#define AAT_LEAF_TC (0u << 4)     /* leaf products on tcgen05 BF16 digits (default) */
#define AAT_LEAF_SIMT (1u << 4)   /* leaf products by plain CUDA-core int64 (check path) */
#define AAT_LEAF_I8 (2u << 4)     /* INT8 digits on mma.sync, exact INT32 accumulation */
#define AAT_LEAF_F64 (3u << 4)    /* FP64 on mma.sync (DMMA); needs ((p-1)/2)^2 < 2^49 */
#define AAT_LEAF_MASK (0xFu << 4)
/* recursion levels: AAT_LEVELS(0) is the plain lower-triangle product (no
 * recursion); no AAT_LEVELS bits = chosen from (n, k). */
#define AAT_LEVELS(l) ((((uint32_t)(l) + 1u) & 0xFu) << 8)
#define AAT_LEVELS_MASK (0xFu << 8)
/* tensor-core leaf: one product per digit pair (i, j) instead of the
 * pair-sum form that needs L + L(L-1)/2 products (comparison path). */
#define AAT_DIGITS_PLAIN (1u << 12)
/* tensor-core leaf: the two general products P3, P4 of the last recursion
 * level by one level of Winograd's form of Strassen's algorithm (7 products
 * of half the size instead of 8; the MM_omega of Theorem 3.1 and Table 1
 * with omega = log2 7).  Applies where the last level's blocks have even
 * sides; the result is the same. */
#define AAT_WINOGRAD (1u << 13)
/* Low-memory schedule (Sec. 7, Table 3: every S and P block of a level
 * lives in C, with only C12 as temporary storage).  The fast schedule keeps
 * the BF16 digit planes of every leaf operand whole: for p = 2^31 - 1 that
 * is 20 bytes per element of each of seven operand blocks (8.75 GiB of
 * workspace at n = k = 16384).  With this flag the S blocks are int32
 * residues in the blocks of C where Table 3 places them, and each leaf
 * product runs in passes over windows of its operands' plane sequence (a
 * pass splits a window of planes of its two operands and runs the plane
 * products on them, accumulating into the product's block of C).  The
 * window is the widest whose workspace fits under aat_set_workspace_limit's
 * limit, or under A's own size (4 n k bytes) when none is set; one plane per
 * pass (n k / 2 bytes for k <= n with recursion) when none fits.  Measured
 * at n = k = 16384 over F_{2^31-1}: 27.9 ms with 1 GiB (4-plane windows)
 * against 24.9 ms with 8.75 GiB; 37.9 ms with 0.25 GiB (1 plane).  Applies
 * to the tensor-core leaf with the pair-sum digit form (p = 2^31 - 1, 65521,
 * ...); other leaf and digit forms run the fast schedule.  Same result. */
#define AAT_LOW_MEMORY (1u << 14)

/*
 * Low(A A^T) mod p (Algorithm 1, Sec. 3; Low as defined in Sec. 2).
 * p: an odd prime < 2^31.  n, k >= 0.  Odd or non-divisible n, k are
 * zero-padded internally (Sec. 3, "padding or peeling"; Sec. 4.3).
 * Equivalent to aat_modp_ex(A, n, k, k, p, C, n, 0, stream).
 */
AAT_API int aat_modp(const int32_t *A, int64_t n, int64_t k, uint32_t p, int32_t *C,
             void *stream);

/* As aat_modp with explicit strides and flags (AAT_*). lda >= k, ldc >= n. */
AAT_API int aat_modp_ex(const int32_t *A, int64_t n, int64_t k, int64_t lda, uint32_t p,
                int32_t *C, int64_t ldc, uint32_t flags, void *stream);

/*
 * The SYRK form: Low(C) <- alpha Low(A A^T) + beta Low(C) mod p (Sec. 7, the
 * update C <- alpha A A^T + beta C and its schedule of Table 4).  alpha and
 * beta are any uint32 (reduced mod p); A as for aat_modp_ex; C (n x n, row
 * stride ldc) holds on entry residues with |x| < p in its lower triangle
 * (diagonal included) and receives the canonical update there.  Table 4's
 * memory placement: C12, the upper triangle of C11 and one (n/2) x (n/2)
 * temporary of the workspace hold intermediate blocks, so the strict upper
 * triangle of C is unspecified on return (zeroed with AAT_ZERO_UPPER).  With
 * beta = 0 this is alpha times aat_modp_ex.  flags as for aat_modp_ex.
 * Asynchronous on `stream`.
 */
AAT_API int aat_syrk_modp(uint32_t alpha, const int32_t *A, int64_t n, int64_t k, int64_t lda,
                  uint32_t beta, int32_t *C, int64_t ldc, uint32_t p, uint32_t flags,
                  void *stream);

/*
 * Quaternion M M^H mod p (Sec. 6.2): M = A + B i + C j + D k with A, B, C, D
 * n x k over F_p (row stride lda, residues |x| < p), i^2 = j^2 = k^2 = ijk =
 * -1, M^H the conjugate transpose.  Writes H = M M^H = H1 + H2 i + H3 j + H4 k
 * as the lower triangles (diagonal included, canonical) of H1..H4 (n x n,
 * row stride ldh, four distinct buffers not overlapping the inputs); H1 is
 * symmetric and H2..H4 skew-symmetric, so Low(H) determines H.  By the
 * paper's 6-multiplication algorithm: five general products on the exact
 * leaf and one product by its own transpose by Algorithm 1.  The strict
 * upper triangles are unspecified (zeroed with AAT_ZERO_UPPER); other flags
 * as for aat_modp_ex.  Asynchronous on `stream`; uses library workspace of
 * about (3 n k + 5 n^2) int32 plus the leaves' digit planes.
 */
AAT_API int aah_quat_modp(const int32_t *A, const int32_t *B, const int32_t *C, const int32_t *D,
                  int64_t n, int64_t k, int64_t lda, uint32_t p, int32_t *H1, int32_t *H2,
                  int32_t *H3, int32_t *H4, int64_t ldh, uint32_t flags, void *stream);

/*
 * End-to-end form: A_host (n x k, row stride k) and C_host (n x n, row
 * stride n) are HOST buffers (pinned or pageable; pinned buffers let the
 * copies overlap the computation).  The call copies A to the device, runs
 * aat_modp_ex with `flags`, copies the result back and synchronises.  The
 * device buffers are owned by the library.  Only the lower triangle of C is
 * defined (its strict upper triangle is unspecified, as for aat_modp): it is
 * copied back in bands of 512 rows, band [a, b) carrying columns [0, b).
 * When a recursion level runs, A's top-left block A11 is copied first and
 * the product P1 = Low(A11 A11^T) runs while the rest of A arrives, and the
 * rows below n/2 of C go back while the last product still computes.  With
 * AAT_ZERO_UPPER, A is copied whole first and the whole of C (upper
 * triangle zero) after the computation.
 */
AAT_API int aat_modp_host(const int32_t *A_host, int64_t n, int64_t k, uint32_t p,
                  int32_t *C_host, uint32_t flags);

/* Bytes that aat_modp_host copies from the device to the host for size n. */
AAT_API int64_t aat_modp_host_d2h_bytes(int64_t n, uint32_t flags);

/*
 * Autotuning of Low(A A^T) mod p on the tensor-core leaf for one shape.
 * The choices tuned: the recursion depth (the cut-off of Algorithm 1's
 * recursion, Sec. 3; the paper leaves it to the implementation, Sec. 7), the
 * leaf kernel form (form 1: one CTA per 128 x 256 tile; form 2: CTA pairs,
 * 256 x 256 tiles), the digit-product form (plain_digits 1: one product per
 * digit pair) and Winograd's form for the last level's general products
 * (winograd 1, as AAT_WINOGRAD).  aat_tune_modp runs every candidate on
 * synthetic balanced
 * residues of shape n x k on `stream` (one untimed run, then `reps` timed
 * ones; it allocates n k + n^2 int32 of device memory for the duration and
 * synchronises), keeps the fastest in a per-process table and returns it
 * with its time and the untuned choice's time (ms_default).  aat_modp_ex,
 * aat_modp_host and the batched plans take levels, form, digit form and
 * Winograd's form from the table for a (n, k, p) it holds whenever their
 * flags set neither AAT_LEVELS nor AAT_DIGITS_PLAIN.  flags: AAT_LEAF_TC
 * only (others give AAT_EUNSUPPORTED); AAT_LEVELS, AAT_DIGITS_PLAIN,
 * AAT_WINOGRAD and AAT_ZERO_UPPER are ignored.
 * aat_tune_lookup: 1 and *out (may be NULL) if the table holds (n, k, p), else 0.
 * aat_tune_save: writes the table as JSON (with the GPU's name); returns the
 * entry count.  aat_tune_load: adds the entries of such a file, skipping a
 * file written on another kind of GPU (returns 0) and invalid entries;
 * returns the count added.  aat_tune_clear: empties the table.
 */
typedef struct {
  int32_t levels;       /* recursion levels */
  int32_t form;         /* leaf kernel form: 1 one CTA, 2 CTA pairs */
  int32_t plain_digits; /* 1: one plane product per digit pair */
  int32_t winograd;     /* 1: Winograd's form for the last level's P3, P4 */
  double ms;            /* mean time of the chosen configuration */
  double ms_default;    /* mean time of the untuned choice */
} aat_tune_t;
AAT_API int aat_tune_modp(int64_t n, int64_t k, uint32_t p, uint32_t flags, int reps,
                  void *stream, aat_tune_t *out);
AAT_API int aat_tune_lookup(int64_t n, int64_t k, uint32_t p, aat_tune_t *out);
AAT_API int aat_tune_save(const char *path);
AAT_API int aat_tune_load(const char *path);
AAT_API void aat_tune_clear(void);

/*
 * The plain general product C = X Y^T mod p with the same exact leaf
 * kernels and no recursion: all m x n entries are written (canonical).
 * X is m x k (row stride ldx), Y is n x k (row stride ldy).  With X = Y this
 * is the full product A A^T that Algorithm 1 is compared against.
 * flags: AAT_LEAF_TC or AAT_LEAF_SIMT.
 */
AAT_API int aat_gemm_modp(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                  int64_t m, int64_t n, int64_t k, uint32_t p, int32_t *C,
                  int64_t ldc, uint32_t flags, void *stream);

/*
 * aat_gemm_modp without any device allocation.  The paper has no
 * counterpart; this is an interface for callers that cannot allocate device
 * memory when they call the library (a host application that gives all
 * device memory to its own pool and forbids cudaMalloc from plug-ins, code
 * that runs while another component owns the allocator, or a path that
 * cannot afford a first-call allocation or the synchronisation cudaFree
 * implies).  It computes the same C = X Y^T mod p as aat_gemm_modp on the
 * tensor-core leaf, but keeps its scratch (the digit planes of X and Y and
 * the tile list) in a fixed 32 MiB device array inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   - Sizes: needs L * (m + n) * round8(k) * 2 bytes plus 8 bytes per
 *     128 x 256 tile (L = 4 digit planes for p > 2^17, 2 for smaller p);
 *     m = n = k = 1024 with p = 2^31 - 1 uses 16 MiB.  Larger requests are
 *     rejected with AAT_ERANGE and a message giving the bytes needed.
 *   - The first call on a device looks up the device address of the array
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - Every call shares the one array and overwrites it: calls that overlap
 *     on the GPU (other streams, other host threads) race and give wrong
 *     results.  The array keeps the last call's contents; each call rewrites
 *     everything it reads (the tile list is written by a kernel, not copied
 *     from the host) and clears its own status word, which aat_device_status
 *     reports beside the library's (AAT_ETIMEOUT if a bounded wait gave up).
 *   - Calls no cudaMalloc, cudaFree or allocating library routine.
 *     aat_shutdown() makes the next call look the array's address up again.
 * Arguments, layout and return codes as aat_gemm_modp (tensor-core leaf).
 */
AAT_API int aat_gemm_modp_noalloc(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy,
                                  int64_t m, int64_t n, int64_t k, uint32_t p, int32_t *C,
                                  int64_t ldc, void *stream);

/* ------------------------------------------------------------------ C
 * Complex inputs and outputs are complex64, interleaved (re, im) floats,
 * row-major with strides in complex elements.  No product runs in FP32
 * arithmetic: every real product runs on the BF16 tensor cores with the FP32
 * values split into BF16 pieces (x = x0 + x1 + x2, x0 = bf16(x),
 * x1 = bf16(x - x0), ...), piece products of weight >= 2^-16 kept, FP32
 * accumulation.  The precision flags name the accuracy class:
 *   AAT_C_FP32    FP32-accurate: 3 pieces, 6 piece products per real
 *                 product (relative Frobenius error <= 1e-5)
 *   AAT_C_BF16X3  2 pieces, 3 piece products (<= 1e-4)
 *   AAT_C_BF16    plain BF16 (<= 3e-3): one piece per input value; the 2M
 *                 form's sum operand (Ar + Ai or Ar - Ai) keeps 2 pieces (3
 *                 piece products for G), because one piece there would put
 *                 the whole rounding error of G into Re C (3.3e-3 measured).
 *                 Algorithm 1 with recursion levels is refused in this class
 *                 (AAT_EUNSUPPORTED): each level roughly doubles the error.
 * Errors are relative Frobenius errors of Low(C) against FP64 sums, for
 * inputs with i.i.d. N(0, 1) parts.  Only the lower triangle of C (diagonal
 * included) is written.
 */
#define AAT_C_PREC_MASK (3u << 16)
#define AAT_C_FP32 (0u << 16)
#define AAT_C_BF16X3 (1u << 16)
#define AAT_C_BF16 (2u << 16)

/* Low(A A^H) by Algorithm 2 (Sec. 6.1, "2M", eps = i conj(i) = 1): two real
 * products H = Re Im^T and G = Low((Re + Im)(Re + Im)^T), then
 * Re C = G - H - H^T, Im C = H^T - H; the diagonal sum_l |a_il|^2 is summed in
 * FP64 (real, >= 0).  There is no skew-unitary Y for the conjugate
 * transposition over C (Sec. 4), so Algorithm 1 does not apply. */
AAT_API int aah_complex(const void *A, int64_t n, int64_t k, void *C, void *stream);
AAT_API int aah_complex_ex(const void *A, int64_t n, int64_t k, int64_t lda, void *C,
                           int64_t ldc, uint32_t flags, void *stream);
/* Low(A A^T) over C by Algorithm 2 with eps = i i = -1: H = Re Im^T,
 * G = Low((Re + Im)(Re - Im)^T), Re C = G + H - H^T, Im C = H + H^T. */
AAT_API int aat_complex_2m(const void *A, int64_t n, int64_t k, int64_t lda, void *C,
                           int64_t ldc, uint32_t flags, void *stream);

/* Low(A A^T) over C by Algorithm 1 (Sec. 3) with phi the transposition and
 * Y = i I (Sec. 4.1: multiplying by Y swaps real and imaginary parts with one
 * sign flip).  The general products P3, P4 use 3 real products (3M), the
 * recursion ends in Algorithm 2 (eps = -1).  flags: AAT_C_* precision, and
 * AAT_LEVELS(l) (no level bits: one level once n/2 >= 4096, k/2 >= 2048; no
 * level with AAT_C_BF16, which refuses AAT_LEVELS(l >= 1) with
 * AAT_EUNSUPPORTED). */
AAT_API int aat_complex(const void *A, int64_t n, int64_t k, void *C, void *stream);
AAT_API int aat_complex_ex(const void *A, int64_t n, int64_t k, int64_t lda, void *C,
                           int64_t ldc, uint32_t flags, void *stream);

/* ------------------------------------------------------------- batches
 * Many independent products in one plan.  A plan is built once for a fixed
 * list of problems (their pointers, sizes and flags) and executed any number
 * of times; each execution recomputes every C from the current contents of
 * every A.  F_p problems whose recursion depth is 0 share ONE persistent
 * tensor-core leaf launch over all their tiles; complex A A^H problems (2M)
 * share one split, ONE persistent FP32 leaf launch over the tiles of all
 * their products, one combine and one diagonal launch (beside the F_p
 * batch, on a stream of their own); the others run their own launches.
 * Execution is one CUDA graph launch on the given stream (no allocation, no
 * host synchronisation).  The plan owns its workspace.
 */
#define AAT_KIND_MODP 0   /* Low(A A^T) mod p: int32 A and C, field p */
#define AAT_KIND_AAH 1    /* Low(A A^H): complex64 A and C, 2M        */
#define AAT_KIND_AAT_C 2  /* Low(A A^T) over C: complex64, Algorithm 1 */
typedef struct {
  int kind;
  const void *A;
  void *C;
  int64_t n, k, lda, ldc;
  uint32_t p;      /* AAT_KIND_MODP only */
  uint32_t flags;  /* as for the single-problem entry points */
} aat_problem_t;
typedef struct aat_plan aat_plan_t;
AAT_API int aat_plan_create(const aat_problem_t *probs, int count, aat_plan_t **plan);
AAT_API int aat_plan_execute(aat_plan_t *plan, void *stream);
/* problems in the shared (F_p or complex) leaf launches, problems run on
 * their own, workspace bytes */
AAT_API int aat_plan_info(const aat_plan_t *plan, int *batched, int *solo, size_t *workspace);
AAT_API void aat_plan_destroy(aat_plan_t *plan);

/* Bytes of device workspace aat_modp_ex would use for (n, k, p, flags). */
AAT_API size_t aat_workspace_size(int64_t n, int64_t k, uint32_t p, uint32_t flags);

/* Workspace limit of aat_modp_ex and aat_modp_host (per process, all
 * devices): a product whose fast schedule needs more than `bytes` of library
 * workspace runs the low-memory schedule (AAT_LOW_MEMORY) instead.  SIZE_MAX
 * (the default) sets no limit.  Independently of the limit, a product whose
 * fast workspace cannot be allocated (cudaMalloc fails) retries with the
 * low-memory schedule before it reports AAT_ENOMEM. */
AAT_API void aat_set_workspace_limit(size_t bytes);

/* Message for the last error of the calling thread ("" if none). */
AAT_API const char *aat_last_error(void);

/*
 * Synchronises the device and reports the sticky device-side status words
 * that bounded waits in the kernels set when they give up (the library's, and
 * aat_gemm_modp_noalloc's own, on the current device): AAT_OK or
 * AAT_ETIMEOUT.  reset != 0 clears them afterwards.
 */
AAT_API int aat_device_status(int reset);

/*
 * Optional instrumentation.  Between aat_profile_begin() and
 * aat_profile_end(), every kernel launch of the library is bracketed by CUDA
 * events recorded on its own stream; aat_profile_end() synchronises and
 * returns, per kernel class, the launch count, the summed event time and the
 * summed algorithmic work (tensor FLOPs for leaf products: 2 per ring
 * multiply-add and plane product; bytes read + written for the addition
 * kernels).
 */
#define AAT_K_SBLOCKS 0
#define AAT_K_SPLIT 1
#define AAT_K_LEAF_TC 2
#define AAT_K_LEAF_SIMT 3
#define AAT_K_POSTADD 4
#define AAT_K_ADD_LOW 5
#define AAT_K_COPY 6
#define AAT_K_LEAF_F32 7
#define AAT_K_LEAF_MMA 8
#define AAT_K_WINOGRAD 9 /* Winograd operand and combine kernels */
#define AAT_K_NCLASS 10
typedef struct {
  int64_t launches[AAT_K_NCLASS];
  double ms[AAT_K_NCLASS];
  double work[AAT_K_NCLASS];
} aat_profile_t;
AAT_API int aat_profile_begin(void);
AAT_API int aat_profile_end(aat_profile_t *out);

/* Frees every workspace and cache of the library on the current device. */
AAT_API void aat_shutdown(void);

/* Library version, major * 10000 + minor * 100 + patch. */
AAT_API int aat_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AAT_H */
