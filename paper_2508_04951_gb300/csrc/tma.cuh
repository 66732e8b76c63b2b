// Bulk asynchronous copies global -> shared (cp.async.bulk, the Blackwell TMA
// engine's unswizzled 1-D form) completed through an mbarrier, with bounded
// waits: a wait that runs out sets the caller's error flag instead of hanging.
#pragma once

#include "common.cuh"

namespace dc {

constexpr int kMbarPollLimit = 1 << 22;

DC_DEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Thread 0 only, then a CTA barrier before use.
DC_DEV void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

DC_DEV void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// dst, src 16-byte aligned; bytes a multiple of 16.
DC_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

DC_DEV bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for phase `parity` with a poll limit; on timeout raise *err = 1 and
// keep polling once more (bounded) for the copy still in flight.
DC_DEV bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity, int* err) {
  for (int i = 0; i < kMbarPollLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicMax(err, 1);
  for (int i = 0; i < kMbarPollLimit; ++i)
    if (mbar_try_wait(bar, parity)) return false;
  return false;
}

// ---------------------------------------------- distributed shared memory
// Address of the same shared-memory location in CTA `rank` of the cluster.
DC_DEV uint32_t dsmem_map(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

// Asynchronous 8-byte store into a peer's shared memory; its arrival is
// counted (8 bytes of transaction) on the peer's mbarrier `rbar`.
DC_DEV void st_async_c64(uint32_t raddr, float2 v, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(
          raddr),
      "f"(v.x), "f"(v.y), "r"(rbar)
      : "memory");
}

// Plain (weak) 8-byte store into a peer's shared memory; a cluster barrier
// (arrive.release, wait.acquire) makes it visible to the peer.  Without the
// per-store transaction count of st.async it moves the same bytes markedly
// faster.
DC_DEV void st_cluster_c64(uint32_t raddr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(raddr), "f"(v.x), "f"(v.y) : "memory");
}

// Cluster-scope acquire wait, for barriers completed by peers' st.async.
DC_DEV bool mbar_try_wait_cluster(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
DC_DEV bool mbar_wait_cluster_bounded(unsigned long long* bar, uint32_t parity, int* err) {
  for (int i = 0; i < kMbarPollLimit; ++i)
    if (mbar_try_wait_cluster(bar, parity)) return true;
  if (err) atomicMax(err, 1);
  for (int i = 0; i < kMbarPollLimit; ++i)
    if (mbar_try_wait_cluster(bar, parity)) return false;
  return false;
}

}  // namespace dc
