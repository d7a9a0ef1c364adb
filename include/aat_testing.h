/*
 * aat_testing.h -- C ABI hooks that expose single steps of the library for
 * step-level parity tests and for host-logic tests that need no GPU.
 * Same conventions as aat.h (device pointers, row-major, return codes).
 */
#ifndef AAT_TESTING_H
#define AAT_TESTING_H

#include <stddef.h>
#include <stdint.h>

#include "aat.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- host number theory (no GPU needed) ---- */

/* 1 if p is prime (deterministic Miller-Rabin for p < 2^32), else 0. */
AAT_API int aatx_is_prime(uint64_t p);
/* Square root of a mod the odd prime p (Tonelli-Shanks); -1 if none. */
AAT_API int64_t aatx_sqrt_mod(int64_t a, uint64_t p);
/* Algorithm 3 (Sec. 4.3): a^2 + b^2 == k mod p.  Returns AAT_OK. */
AAT_API int aatx_sos(int64_t k, uint64_t p, uint64_t *a, uint64_t *b);
/* The skew-unitary Y the library uses for p (Sec. 4): kind 1 is Y = a I with
 * a^2 == -1; kind 2 is [[a, b], [-b, a]] (x) I with a^2 + b^2 == -1.  a and b
 * are returned canonical.  Returns AAT_OK or an error code. */
AAT_API int aatx_y_params(uint32_t p, int *kind, uint32_t *a, uint32_t *b);
/* Digit split of balanced residues mod p for the tensor-core leaf: width b
 * bits, L digits, dmax[d] bounds |digit d|.  dmax must hold 8 entries.  The
 * planes also hold the pair sums d_i + d_j (i < j) when the leaf uses the
 * pair-sum form: L(L-1)/2 of them, in the order (0,1), (0,2), ..., (L-2,L-1). */
AAT_API int aatx_digit_spec(uint32_t p, int *b, int *L, int *dmax, int *nsum);

/* Shape of the recursion aat_modp_ex would run (no GPU needed).  Counts are
 * totals over the whole recursion tree. */
typedef struct {
  int levels;             /* recursion levels actually used */
  int64_t n_pad, k_pad;   /* padded sizes */
  int64_t recursive_products; /* P1, P2, P5 calls (all levels) */
  int64_t general_products;   /* P3, P4 leaf products */
  int64_t syrk_leaves;        /* Low(X X^T) leaf products */
  int64_t block_additions;    /* 9 per internal node (Remark 3.3) */
  int64_t half_additions;     /* 3 of them per node on symmetric blocks */
  double ring_macs;           /* sum over leaves: syrk n(n+1)/2 k, gemm m n k */
  size_t workspace_bytes;
} aatx_plan_stats_t;
AAT_API int aatx_plan_stats(int64_t n, int64_t k, uint32_t p, uint32_t flags,
                    aatx_plan_stats_t *out);

/* The groups the tensor-core leaf runs for inner dimension K mod p (host
 * only): per group, in processing order, six int32 (X plane, Y plane, first
 * and one-past-last K block of 64, K blocks per FP32 chunk, Horner ratio mod
 * p applied to the accumulator before the group).  flags may hold
 * AAT_DIGITS_PLAIN.  Returns the group count or a negative error; *nprod
 * receives the number of plane products. */
AAT_API int aatx_leaf_groups(uint32_t p, int64_t K, uint32_t flags, int exact_bits,
                             int32_t *out, int max_groups, int *nprod);

/* ---- single GPU steps (device pointers, asynchronous on stream) ---- */

/* The four additions of Algorithm 1 on A (n x k, even n, k; k/2 even for
 * kind-2 Y), with the library's Y for p.  S1..S4 are h x kappa int32
 * canonical residues with row stride lds. */
AAT_API int aatx_sblocks(const int32_t *A, int64_t n, int64_t k, int64_t lda, uint32_t p,
                 int32_t *S1, int32_t *S2, int32_t *S3, int32_t *S4, int64_t lds,
                 void *stream);

/* Digit planes (then pair-sum planes) of the residue block X (rows x cols)
 * as raw bf16 bits: planes[(d * rows + r) * kstride + c], kstride = cols
 * rounded up to 8. */
AAT_API int aatx_split(const int32_t *X, int64_t rows, int64_t cols, int64_t ldx, uint32_t p,
               uint16_t *planes, void *stream);

/* One leaf product: C = X Y^T mod p (lower != 0: only i >= j written;
 * accumulate != 0: C <- C + X Y^T).  leaf: AAT_LEAF_TC or AAT_LEAF_SIMT,
 * optionally | AAT_DIGITS_PLAIN.  exact_bits: bound 2^exact_bits on |FP32
 * partial sums| (0 = default, 24). */
AAT_API int aatx_leaf(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy, int64_t M,
              int64_t N, int64_t K, uint32_t p, int32_t *C, int64_t ldc, int lower,
              int accumulate, uint32_t leaf, int exact_bits, void *stream);

/* The fused post-additions (U4 over C21, Low(U5) over C22) of one level. */
AAT_API int aatx_postadd(int32_t *C, int64_t ldc, int64_t h, uint32_t p, void *stream);

/* ---- failure paths (no GPU fault: limits and waits that run out) ---- */

/* Workspace requests of more than `bytes` fail with AAT_ENOMEM, as a failed
 * cudaMalloc would, before any CUDA call (SIZE_MAX restores the default: no
 * limit).  Covers the library's shared workspace (aat_modp_ex, aat_syrk_modp,
 * complex products, tuning), not plans. */
AAT_API void aatx_set_alloc_limit(size_t bytes);
/* Grows the shared workspace of the current device to `bytes` (AAT_OK, or
 * AAT_ENOMEM from the limit above or from cudaMalloc). */
AAT_API int aatx_workspace_reserve(size_t bytes);
/* One thread waits, with the bounded mbarrier wait of the leaf kernels and a
 * limit of limit_ns (at most 2 s), for a barrier phase that nothing
 * completes; when the limit runs out it records AAT_ETIMEOUT in the status
 * word that aat_device_status reads: which = 0 the library's word, which = 1
 * the allocation-free entry point's.  No fault, no trap: the kernel returns
 * and the context stays usable.  Asynchronous on stream. */
AAT_API int aatx_wait_probe(int which, int64_t limit_ns, void *stream);

/* ---- instruction peaks (the denominators of the mma.sync leaves) ---- */

/* Launches `blocks` blocks of 8 warps; each warp issues iters x 8
 * independent mma.sync on register operands: kind 0 m16n8k32 s8 (INT8,
 * INT32 accumulation), kind 1 m8n8k4 f64.  *ops receives the operations the
 * launch performs (2 M N K per instruction); divide by its CUDA-event time.
 * sink: device memory of 8 bytes (never written; it keeps the loop alive). */
AAT_API int aatx_mma_peak(int kind, int64_t iters, int blocks, void *sink, double *ops,
                          void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AAT_TESTING_H */
