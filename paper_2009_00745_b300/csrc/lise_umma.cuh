// lise_umma.cuh -- fifth-generation tensor core (tcgen05) primitives for sm_100-family GPUs:
// tensor-memory allocation, shared-memory matrix descriptors, the bf16 MMA with FP32
// accumulation in tensor memory, completion through an mbarrier, and tensor-memory loads.
//
// Operands are read from shared memory in the canonical no-swizzle "core matrix" layout:
// a core matrix is 8 rows x 16 bytes (8 bf16 values of the contraction index K, rows 16 bytes
// apart, 128 contiguous bytes).  For a K-major operand (rows = M or N, K contiguous within a
// core row) the descriptor's leading byte offset is the distance between core matrices that
// are adjacent along K, the stride byte offset the distance between core matrices adjacent
// along M (or N).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lise {
namespace um {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, leading and stride byte
// offsets (all in 16-byte units, 14 bits each), descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16 with bf16 A and B (both K-major), FP32 accumulator,
// shape M x N (M = 64 or 128, N a multiple of 8 up to 256).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) = A B^T (+ D when acc != 0); issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// Arrive on the mbarrier once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for completion of the mbarrier phase with the given parity; gives up after `limit`
// polls (each poll may suspend the thread for a bounded, hardware-chosen time).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long limit) {
  uint32_t done = 0;
  for (long it = 0; it < limit && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(mbar)), "r"(parity)
        : "memory");
  return done != 0;
}

// The same wait that also gives up once *stop becomes non-zero (another role of the block
// gave up): returns false on timeout or stop.
__device__ __forceinline__ bool mbar_wait_or(uint64_t* mbar, uint32_t parity, long limit, const volatile int* stop) {
  uint32_t done = 0;
  for (long it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(mbar)), "r"(parity)
        : "memory");
    if (!done && *stop) return false;
  }
  return done != 0;
}

// Arrive on an mbarrier (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(mbar)) : "memory");
}

// Named barrier `id` over `count` threads (a multiple of 32; whole warps), and the same with an
// AND over the participating threads' predicates (every participant gets the same result).
__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_and(int id, int count, bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred pi, po;\nsetp.ne.u32 pi, %1, 0;\nbar.red.and.pred po, %2, %3, pi;\nselp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// Tensor-memory allocation (one full warp): ncols columns (a power of 2, >= 32); the base
// address is written to shared memory.
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to the tensor core
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's tensor-memory lane (the warp reads lanes
// 32 (warp % 4) .. + 31; taddr carries the lane base in its upper 16 bits).
__device__ __forceinline__ void ld8(uint32_t r[8], uint32_t taddr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Wait for this thread's tensor-memory loads, then tie every loaded register to a point
// after the wait (the loads' results may only be used once the wait has returned).
template <int L>
__device__ __forceinline__ void wait_ld_deps(uint32_t (&r)[L][8]) {
  wait_ld();
#pragma unroll
  for (int l = 0; l < L; ++l)
    asm volatile("" : "+r"(r[l][0]), "+r"(r[l][1]), "+r"(r[l][2]), "+r"(r[l][3]), "+r"(r[l][4]), "+r"(r[l][5]),
                 "+r"(r[l][6]), "+r"(r[l][7]));
}

// Tensor memory accelerator: arrive on the mbarrier announcing `bytes` of asynchronous
// copies; then box copies of a 4-D tensor map (the map lives in kernel parameter space,
// __grid_constant__) into shared memory (128-byte aligned), completing on that mbarrier.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(mbar))
      : "memory");
}

}  // namespace um
}  // namespace lise
