// Device helpers of the single-pass CG kernels (cg2.cu: one system a launch;
// cg2b.cu: every system of a batch in one launch): ring and vector constants,
// bounded mbarrier waits, the consumer barrier and the global acquire load of
// the grid barriers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tma.cuh"

namespace paro {
namespace {

constexpr int kMaxSlots2 = 6;  // deepest TMA ring (planes in flight)
constexpr int kW2 = 28;      // packed operator weights per node (27 + one pad)
constexpr int kDots = 5;     // (r,z) (r,r) (p,q) (q,z) (q,D^-1 q)
constexpr int kMaxThr2 = 512;

// Slot stride (floats) of one group's [TY+2][TX+2][4] box: rounded up to 128
// bytes, the alignment a TMA destination in shared memory needs.
__host__ __device__ __forceinline__ int box_stride_floats(int HX, int HY) { return (HY * HX * 16 + 127) / 128 * 32; }

__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, unsigned limit) {
  const uint32_t a = smem_u32(bar);
  for (unsigned i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_proxy_async_global2() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void* smem_align8(void* p) {
  return reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(p) + 7) & ~(uintptr_t)7);
}
// Barrier 1 among the nc consumer threads (the producer warp does not take part).
__device__ __forceinline__ void consumer_sync(int nc) { asm volatile("bar.sync 1, %0;" ::"r"(nc) : "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Threads: nthr x G4 consumers (node slot j = tid % nthr, active-group slot
// k = tid / nthr), then one producer warp whose first lane stages the planes by
// TMA into a ring of geo.slots slots: full[s] completes when a slot's copies
// have landed, empty[s] when every consumer warp is done with it.  A node slot
// holds NPT nodes stacked in y (NPT = 2: the two 3 x 3 neighbourhoods share six
// nodes, so a thread forms r, z, p at 12 staged nodes for two outputs instead of
// at 18, and has twice the independent work; up to 384 threads, 170 registers).
constexpr int cg2_max_threads(int npt) { return npt == 1 ? kMaxThr2 : 384; }


}  // namespace
}  // namespace paro
