// tc_pair.cuh -- cluster (CTA pair) primitives of the reverse-mode pair
// kernel (mlp_rev2.cu).  Internal to librtn.
#pragma once

#include "tc_common.cuh"

namespace rtn {
namespace {

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// shared::cluster address of `addr` (a shared::cta address) in CTA `rank`
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

// arrival without ordering of earlier stores (tensor-memory release: the
// loads have completed at tcgen05.wait::ld)
__device__ __forceinline__ void arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

// arrival that also announces `bytes` of a bulk copy completing on the barrier
__device__ __forceinline__ void arrive_expect_tx_cluster(uint32_t cluster_addr, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(
                   cluster_addr),
               "r"(bytes)
               : "memory");
}

// the same without ordering earlier stores (announces bytes only)
__device__ __forceinline__ void arrive_expect_tx_cluster_relaxed(uint32_t cluster_addr, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.relaxed.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(
                   cluster_addr),
               "r"(bytes)
               : "memory");
}

// shared::cta -> peer shared memory, complete_tx on a barrier of the peer
__device__ __forceinline__ void bulk_copy_to_peer(uint32_t dst_cl, uint32_t src, uint32_t bytes,
                                                  uint32_t bar_cl) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst_cl),
      "r"(src), "r"(bytes), "r"(bar_cl)
      : "memory");
}


__device__ __forceinline__ uint32_t mbar_try_cl(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok;
}

__device__ __forceinline__ uint32_t mbar_try_cl_sleep(uint32_t bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(ns)
      : "memory");
  return ok;
}

// bounded wait with cluster-scope acquire
__device__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
  if (mbar_try_cl(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_cl_sleep(bar, parity, WAIT_SLEEP_NS)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort_flag = 1;
      atomicExch(err, (int)RTN_E_TIMEOUT);
      return false;
    }
  }
  return true;
}

// the same by every lane of a warp, warp-uniform result
__device__ __forceinline__ bool mbar_wait_cl_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                                  int* err) {
  const bool ok = mbar_try_cl(bar, parity) || mbar_wait_cl(bar, parity, abort_flag, err);
  return __all_sync(0xffffffffu, ok);
}

// weight half of this CTA, completing on the stage barrier of rank 0
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                                 uint32_t bar_cl) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar_cl)
      : "memory");
}

// issued by one elected lane of a converged warp
__device__ __forceinline__ void mma2_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// the four MMAs of one 64-wide K block under one election: accumulate
// into D unless accum0 == 0 for the first (the later three always accumulate)
__device__ __forceinline__ void mma2_bf16_x4(uint32_t d_tmem, const uint64_t (&a)[4], const uint64_t (&b)[4],
                                             uint32_t idesc, uint32_t accum0) {
  asm volatile(
      "{\n\t.reg .pred p, t, e;\n\tsetp.ne.b32 p, %10, 0;\n\tsetp.eq.b32 t, %10, %10;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %9, p;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f16 [%0], %3, %4, %9, t;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f16 [%0], %5, %6, %9, t;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f16 [%0], %7, %8, %9, t;\n\t}" ::"r"(d_tmem),
      "l"(a[0]), "l"(b[0]), "l"(a[1]), "l"(b[1]), "l"(a[2]), "l"(b[2]), "l"(a[3]), "l"(b[3]), "r"(idesc),
      "r"(accum0)
      : "memory");
}

// the six kind::f8f6f4 MMAs of one 64-byte K block (two K steps of 32 e4m3
// elements, each against three B pieces) under one election: accumulate into
// D unless accum0 == 0 for the first
__device__ __forceinline__ void mma2_f8_x6(uint32_t d_tmem, const uint64_t (&a)[2], const uint64_t (&b)[6],
                                           uint32_t idesc, uint32_t accum0) {
  asm volatile(
      "{\n\t.reg .pred p, t, e;\n\tsetp.ne.b32 p, %10, 0;\n\tsetp.eq.b32 t, %10, %10;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %3, %9, p;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %4, %9, t;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %5, %9, t;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %2, %6, %9, t;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %2, %7, %9, t;\n\t"
      "@e tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %2, %8, %9, t;\n\t}" ::"r"(d_tmem),
      "l"(a[0]), "l"(a[1]), "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]), "l"(b[4]), "l"(b[5]), "r"(idesc),
      "r"(accum0)
      : "memory");
}

// arrive on the barrier at this offset in the CTAs of `mask` (bit r = rank r);
// one elected lane of a converged warp
__device__ __forceinline__ void commit2(uint32_t bar, uint16_t mask) {
  asm volatile(
      "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n\t}" ::"r"(
          bar),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

}  // namespace
}  // namespace rtn
