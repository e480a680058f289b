// grid_sync.cuh -- grid-wide barrier of a cooperative launch, bounded in
// wall-clock time (the persistent kernels: the adjoint's segment kernels and
// the persistent form of the fused step).
#pragma once
#include <cstdint>

#include "tma.cuh"

namespace nlc {

// cumulative arrival counter, zeroed before each launch
struct GridBarrier {
  unsigned arrived;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch.  Thread 0 of each block adds
// its arrival with release semantics and polls the counter with acquire
// semantics until every block of this generation has arrived (the counter
// is cumulative: generation g completes at (g + 1) gridDim.x).  The poll is
// bounded by wait_ns nanoseconds of %globaltimer; returns false in every
// thread of the block if it ran out.
__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned& gen, unsigned* err,
                                          uint64_t wait_ns) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned target = (gen + 1) * gridDim.x;
    red_release_gpu_add(&b->arrived, 1u);
    if (ld_acquire_gpu(&b->arrived) < target) {
      const uint64_t t0 = global_ns();
      while (ld_acquire_gpu(&b->arrived) < target) {
        if (global_ns() - t0 >= wait_ns) {  // wait_ns = 0: give up at once
          ok = 0;
          atomicExch(err, DEV_ERR_GRID_TIMEOUT);
          break;
        }
      }
    }
  }
  gen++;
  return __syncthreads_and(ok) != 0;
}

// orders this thread's earlier generic-proxy global writes (made visible
// by a grid barrier) before later async-proxy (TMA) reads of the same memory
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

}  // namespace nlc
