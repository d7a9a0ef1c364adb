// tc_ptx.cuh -- inline-PTX wrappers of the Blackwell (sm_103a) asynchronous
// machinery used by the tensor-core leaf kernels: mbarriers, TMA tensor
// loads, TMEM allocation and loads, tcgen05.mma and its commit, and a
// bounded mbarrier wait that gives up after kTimeoutNs.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace aat {
namespace tc {

constexpr unsigned long long kTimeoutNs = 4000000000ull;  // 4 s

// ------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The same test with cluster-scope acquire: for barriers that threads of the
// peer CTA of a CTA pair arrive on.
__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Arrive on a barrier given by its shared::cluster address, possibly in the
// peer CTA.  Release at CTA scope only: a cluster-scope release would wait
// for this thread's earlier global stores to become visible to the cluster,
// and the only hazard it guards (TMEM reads before the next MMA) is already
// closed by tcgen05.wait::ld and tcgen05.fence::before_thread_sync.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// shared::cluster address of the variable at shared::cta address `a` in the
// CTA of rank `rank` of this cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t ncluster_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}

// Every thread of both CTAs of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Bounded wait for the phase of parity `parity` of barrier `bar`.  Returns
// false when the limit expires (and raises the CTA abort flag and the device
// status) or when another role of the CTA has aborted.  limit_ns: kTimeoutNs
// in the kernels; the failure-path test probe passes a short one.
template <bool CLUSTER = false>
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          int32_t *status,
                                          unsigned long long limit_ns = kTimeoutNs) {
  auto test = [&]() { return CLUSTER ? mbar_try_cluster(bar, parity) : mbar_try(bar, parity); };
  if (test()) return true;
  const unsigned long long t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (test()) return true;
    if ((it & 63u) == 0) {
      if (*abort_flag) return false;
      if (gtimer() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicExch(status, (int32_t)AAT_ETIMEOUT);
        return false;
      }
    }
  }
}

// Wait with a short limit and no abort check (teardown after an abort).
__device__ __forceinline__ void wait_quiet(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity)) {
    if (gtimer() - t0 > 100000000ull) return;  // 100 ms
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *tm, uint32_t bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// The CTA-pair form: the copy lands in this CTA's shared memory and its
// byte count completes on `cluster_bar`, a barrier of either CTA of the pair.
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap *tm,
                                                 uint32_t cluster_bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(cluster_bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// CTA-pair forms (cta_group::2): one thread of the leader CTA issues the MMA
// for both CTAs (A: 128 rows from each CTA's shared memory, B: half of the N
// rows from each, D: 128 TMEM lanes in each CTA); the commit arrives on the
// barrier at the same offset in every CTA of `mask`.
// One lane of a converged warp (the lowest active one), chosen by
// elect.sync: the warp runs the issuing loop in uniform control flow and the
// elected lane issues the single-thread tcgen05 instructions.
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "elect.sync _|P, 0xffffffff;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(pred));
  return pred != 0;
}

__device__ __forceinline__ void tc_mma_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with
// 128-byte swizzling: rows of 128 bytes, 8-row atoms 1024 bytes apart (SBO),
// descriptor version 1 (bit 46), layout SWIZZLE_128B (2 at bit 61).  The
// start address moves by 32 bytes per K=16 step inside the atom.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// Drain 32 consecutive FP32 columns of this thread's TMEM lane into the
// int32 accumulators acc[B .. B+31]: load, wait, convert (the values are
// exact integers) and add inside one statement, so that the temporaries of
// one load are dead before the next load is issued.
template <int B>
__device__ __forceinline__ void tmem_drain32(uint32_t taddr, int32_t (&acc)[128]) {
  asm volatile(
      "{\n\t.reg .b32 t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15, t16, t17, t18, t19, t20, t21, t22, t23, t24, t25, t26, t27, t28, t29, t30, t31;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15, t16, t17, t18, t19, t20, t21, t22, t23, t24, t25, t26, t27, t28, t29, t30, t31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n\t"
      "cvt.rni.s32.f32 t0, t0;\n\t"
      "add.s32 %0, %0, t0;\n\t"
      "cvt.rni.s32.f32 t1, t1;\n\t"
      "add.s32 %1, %1, t1;\n\t"
      "cvt.rni.s32.f32 t2, t2;\n\t"
      "add.s32 %2, %2, t2;\n\t"
      "cvt.rni.s32.f32 t3, t3;\n\t"
      "add.s32 %3, %3, t3;\n\t"
      "cvt.rni.s32.f32 t4, t4;\n\t"
      "add.s32 %4, %4, t4;\n\t"
      "cvt.rni.s32.f32 t5, t5;\n\t"
      "add.s32 %5, %5, t5;\n\t"
      "cvt.rni.s32.f32 t6, t6;\n\t"
      "add.s32 %6, %6, t6;\n\t"
      "cvt.rni.s32.f32 t7, t7;\n\t"
      "add.s32 %7, %7, t7;\n\t"
      "cvt.rni.s32.f32 t8, t8;\n\t"
      "add.s32 %8, %8, t8;\n\t"
      "cvt.rni.s32.f32 t9, t9;\n\t"
      "add.s32 %9, %9, t9;\n\t"
      "cvt.rni.s32.f32 t10, t10;\n\t"
      "add.s32 %10, %10, t10;\n\t"
      "cvt.rni.s32.f32 t11, t11;\n\t"
      "add.s32 %11, %11, t11;\n\t"
      "cvt.rni.s32.f32 t12, t12;\n\t"
      "add.s32 %12, %12, t12;\n\t"
      "cvt.rni.s32.f32 t13, t13;\n\t"
      "add.s32 %13, %13, t13;\n\t"
      "cvt.rni.s32.f32 t14, t14;\n\t"
      "add.s32 %14, %14, t14;\n\t"
      "cvt.rni.s32.f32 t15, t15;\n\t"
      "add.s32 %15, %15, t15;\n\t"
      "cvt.rni.s32.f32 t16, t16;\n\t"
      "add.s32 %16, %16, t16;\n\t"
      "cvt.rni.s32.f32 t17, t17;\n\t"
      "add.s32 %17, %17, t17;\n\t"
      "cvt.rni.s32.f32 t18, t18;\n\t"
      "add.s32 %18, %18, t18;\n\t"
      "cvt.rni.s32.f32 t19, t19;\n\t"
      "add.s32 %19, %19, t19;\n\t"
      "cvt.rni.s32.f32 t20, t20;\n\t"
      "add.s32 %20, %20, t20;\n\t"
      "cvt.rni.s32.f32 t21, t21;\n\t"
      "add.s32 %21, %21, t21;\n\t"
      "cvt.rni.s32.f32 t22, t22;\n\t"
      "add.s32 %22, %22, t22;\n\t"
      "cvt.rni.s32.f32 t23, t23;\n\t"
      "add.s32 %23, %23, t23;\n\t"
      "cvt.rni.s32.f32 t24, t24;\n\t"
      "add.s32 %24, %24, t24;\n\t"
      "cvt.rni.s32.f32 t25, t25;\n\t"
      "add.s32 %25, %25, t25;\n\t"
      "cvt.rni.s32.f32 t26, t26;\n\t"
      "add.s32 %26, %26, t26;\n\t"
      "cvt.rni.s32.f32 t27, t27;\n\t"
      "add.s32 %27, %27, t27;\n\t"
      "cvt.rni.s32.f32 t28, t28;\n\t"
      "add.s32 %28, %28, t28;\n\t"
      "cvt.rni.s32.f32 t29, t29;\n\t"
      "add.s32 %29, %29, t29;\n\t"
      "cvt.rni.s32.f32 t30, t30;\n\t"
      "add.s32 %30, %30, t30;\n\t"
      "cvt.rni.s32.f32 t31, t31;\n\t"
      "add.s32 %31, %31, t31;\n\t"
      "}"
      : "+r"(acc[B + 0]), "+r"(acc[B + 1]), "+r"(acc[B + 2]), "+r"(acc[B + 3]), "+r"(acc[B + 4]), "+r"(acc[B + 5]), "+r"(acc[B + 6]), "+r"(acc[B + 7]), "+r"(acc[B + 8]), "+r"(acc[B + 9]), "+r"(acc[B + 10]), "+r"(acc[B + 11]), "+r"(acc[B + 12]), "+r"(acc[B + 13]), "+r"(acc[B + 14]), "+r"(acc[B + 15]), "+r"(acc[B + 16]), "+r"(acc[B + 17]), "+r"(acc[B + 18]), "+r"(acc[B + 19]), "+r"(acc[B + 20]), "+r"(acc[B + 21]), "+r"(acc[B + 22]), "+r"(acc[B + 23]), "+r"(acc[B + 24]), "+r"(acc[B + 25]), "+r"(acc[B + 26]), "+r"(acc[B + 27]), "+r"(acc[B + 28]), "+r"(acc[B + 29]), "+r"(acc[B + 30]), "+r"(acc[B + 31])
      : "r"(taddr)
      : "memory");
}



// Drain 16 consecutive FP32 columns of this thread's TMEM lane into the
// int32 accumulators acc[B .. B+15] (load, wait, convert, add in one
// statement); half the temporaries of the 32-column form, so that the
// 128 accumulators and the temporaries fit the epilogue's registers.
template <int B, int N>
__device__ __forceinline__ void tmem_drain16(uint32_t taddr, int32_t (&acc)[N]) {
  asm volatile(
      "{\n\t.reg .b32 t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n\t"
      "cvt.rni.s32.f32 t0, t0;\n\t"
      "add.s32 %0, %0, t0;\n\t"
      "cvt.rni.s32.f32 t1, t1;\n\t"
      "add.s32 %1, %1, t1;\n\t"
      "cvt.rni.s32.f32 t2, t2;\n\t"
      "add.s32 %2, %2, t2;\n\t"
      "cvt.rni.s32.f32 t3, t3;\n\t"
      "add.s32 %3, %3, t3;\n\t"
      "cvt.rni.s32.f32 t4, t4;\n\t"
      "add.s32 %4, %4, t4;\n\t"
      "cvt.rni.s32.f32 t5, t5;\n\t"
      "add.s32 %5, %5, t5;\n\t"
      "cvt.rni.s32.f32 t6, t6;\n\t"
      "add.s32 %6, %6, t6;\n\t"
      "cvt.rni.s32.f32 t7, t7;\n\t"
      "add.s32 %7, %7, t7;\n\t"
      "cvt.rni.s32.f32 t8, t8;\n\t"
      "add.s32 %8, %8, t8;\n\t"
      "cvt.rni.s32.f32 t9, t9;\n\t"
      "add.s32 %9, %9, t9;\n\t"
      "cvt.rni.s32.f32 t10, t10;\n\t"
      "add.s32 %10, %10, t10;\n\t"
      "cvt.rni.s32.f32 t11, t11;\n\t"
      "add.s32 %11, %11, t11;\n\t"
      "cvt.rni.s32.f32 t12, t12;\n\t"
      "add.s32 %12, %12, t12;\n\t"
      "cvt.rni.s32.f32 t13, t13;\n\t"
      "add.s32 %13, %13, t13;\n\t"
      "cvt.rni.s32.f32 t14, t14;\n\t"
      "add.s32 %14, %14, t14;\n\t"
      "cvt.rni.s32.f32 t15, t15;\n\t"
      "add.s32 %15, %15, t15;\n\t"
      "}"
      : "+r"(acc[B + 0]), "+r"(acc[B + 1]), "+r"(acc[B + 2]), "+r"(acc[B + 3]), "+r"(acc[B + 4]), "+r"(acc[B + 5]), "+r"(acc[B + 6]), "+r"(acc[B + 7]), "+r"(acc[B + 8]), "+r"(acc[B + 9]), "+r"(acc[B + 10]), "+r"(acc[B + 11]), "+r"(acc[B + 12]), "+r"(acc[B + 13]), "+r"(acc[B + 14]), "+r"(acc[B + 15])
      : "r"(taddr)
      : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane, waited on in the
// same statement so no register is read before it holds its value.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}


// Add 16 consecutive FP32 TMEM columns of this thread's lane into the FP32
// registers acc[B .. B+15] (round to nearest): load, wait and add in one
// statement (half the temporaries of the 32-column form).
template <int B>
__device__ __forceinline__ void tmem_accum16f(uint32_t taddr, float (&acc)[128]) {
  asm volatile(
      "{\n\t.reg .f32 t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n\t"
      "add.f32 %0, %0, t0;\n\t"
      "add.f32 %1, %1, t1;\n\t"
      "add.f32 %2, %2, t2;\n\t"
      "add.f32 %3, %3, t3;\n\t"
      "add.f32 %4, %4, t4;\n\t"
      "add.f32 %5, %5, t5;\n\t"
      "add.f32 %6, %6, t6;\n\t"
      "add.f32 %7, %7, t7;\n\t"
      "add.f32 %8, %8, t8;\n\t"
      "add.f32 %9, %9, t9;\n\t"
      "add.f32 %10, %10, t10;\n\t"
      "add.f32 %11, %11, t11;\n\t"
      "add.f32 %12, %12, t12;\n\t"
      "add.f32 %13, %13, t13;\n\t"
      "add.f32 %14, %14, t14;\n\t"
      "add.f32 %15, %15, t15;\n\t"
      "}"
      : "+f"(acc[B + 0]), "+f"(acc[B + 1]), "+f"(acc[B + 2]), "+f"(acc[B + 3]), "+f"(acc[B + 4]), "+f"(acc[B + 5]), "+f"(acc[B + 6]), "+f"(acc[B + 7]), "+f"(acc[B + 8]), "+f"(acc[B + 9]), "+f"(acc[B + 10]), "+f"(acc[B + 11]), "+f"(acc[B + 12]), "+f"(acc[B + 13]), "+f"(acc[B + 14]), "+f"(acc[B + 15])
      : "r"(taddr)
      : "memory");
}

// Add 32 consecutive FP32 TMEM columns of this thread's lane into the FP32
// registers acc[B .. B+31] (round to nearest), load, wait and add in one
// statement.
template <int B>
__device__ __forceinline__ void tmem_accum32f(uint32_t taddr, float (&acc)[128]) {
  asm volatile(
      "{\n\t.reg .f32 t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15, t16, t17, t18, t19, t20, t21, t22, t23, t24, t25, t26, t27, t28, t29, t30, t31;\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15, t16, t17, t18, t19, t20, t21, t22, t23, t24, t25, t26, t27, t28, t29, t30, t31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n\t"
      "add.f32 %0, %0, t0;\n\t"
      "add.f32 %1, %1, t1;\n\t"
      "add.f32 %2, %2, t2;\n\t"
      "add.f32 %3, %3, t3;\n\t"
      "add.f32 %4, %4, t4;\n\t"
      "add.f32 %5, %5, t5;\n\t"
      "add.f32 %6, %6, t6;\n\t"
      "add.f32 %7, %7, t7;\n\t"
      "add.f32 %8, %8, t8;\n\t"
      "add.f32 %9, %9, t9;\n\t"
      "add.f32 %10, %10, t10;\n\t"
      "add.f32 %11, %11, t11;\n\t"
      "add.f32 %12, %12, t12;\n\t"
      "add.f32 %13, %13, t13;\n\t"
      "add.f32 %14, %14, t14;\n\t"
      "add.f32 %15, %15, t15;\n\t"
      "add.f32 %16, %16, t16;\n\t"
      "add.f32 %17, %17, t17;\n\t"
      "add.f32 %18, %18, t18;\n\t"
      "add.f32 %19, %19, t19;\n\t"
      "add.f32 %20, %20, t20;\n\t"
      "add.f32 %21, %21, t21;\n\t"
      "add.f32 %22, %22, t22;\n\t"
      "add.f32 %23, %23, t23;\n\t"
      "add.f32 %24, %24, t24;\n\t"
      "add.f32 %25, %25, t25;\n\t"
      "add.f32 %26, %26, t26;\n\t"
      "add.f32 %27, %27, t27;\n\t"
      "add.f32 %28, %28, t28;\n\t"
      "add.f32 %29, %29, t29;\n\t"
      "add.f32 %30, %30, t30;\n\t"
      "add.f32 %31, %31, t31;\n\t"
      "}"
      : "+f"(acc[B + 0]), "+f"(acc[B + 1]), "+f"(acc[B + 2]), "+f"(acc[B + 3]), "+f"(acc[B + 4]), "+f"(acc[B + 5]), "+f"(acc[B + 6]), "+f"(acc[B + 7]), "+f"(acc[B + 8]), "+f"(acc[B + 9]), "+f"(acc[B + 10]), "+f"(acc[B + 11]), "+f"(acc[B + 12]), "+f"(acc[B + 13]), "+f"(acc[B + 14]), "+f"(acc[B + 15]), "+f"(acc[B + 16]), "+f"(acc[B + 17]), "+f"(acc[B + 18]), "+f"(acc[B + 19]), "+f"(acc[B + 20]), "+f"(acc[B + 21]), "+f"(acc[B + 22]), "+f"(acc[B + 23]), "+f"(acc[B + 24]), "+f"(acc[B + 25]), "+f"(acc[B + 26]), "+f"(acc[B + 27]), "+f"(acc[B + 28]), "+f"(acc[B + 29]), "+f"(acc[B + 30]), "+f"(acc[B + 31])
      : "r"(taddr)
      : "memory");
}

}  // namespace tc
}  // namespace aat
