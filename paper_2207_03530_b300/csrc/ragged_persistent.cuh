// Ragged worlds in one persistent launch (sm_103a): every size class of a
// packed ragged world stepped by one kernel whose warps take work from an
// atomic counter.  The step itself is world_step_body (step_fused.cuh),
// instantiated once per size class.
#pragma once

#include "step_fused.cuh"

namespace vmas {

// Every size class of a packed ragged world in one launch: each warp takes
// work items from an atomic counter (one atomicAdd by lane 0 per item; no
// warp ever waits on another) until the queue is empty.  An item is one
// warp's worth of envs of one class (32 / G of them); items are numbered
// largest class first, so the longest items start first and the short ones
// fill the tail.  The classes' lane layouts are fixed at compile time
// (kPersistLanes, kPersistSlots in params.cuh).
// Each warp owns RaggedQueueParams::slab bytes of shared memory, the most
// any class needs for one warp's envs.
__host__ __device__ inline int persist_slab_bytes() {
  int m = 0;
  for (int c = 0; c < 5; ++c) {
    const int cap = 8 << c, g = c == 0 || c == 1 ? 8 : (c == 2 ? 16 : 32);
    const int b = (32 / g) * fused_env_bytes(cap, g);
    m = b > m ? b : m;
  }
  return m;
}

// MINB: resident CTAs per SM the register budget targets (4: 128 registers,
// no spills to speak of; 5: 96 registers, the largest class spills).
template <int MINB>
__global__ void __launch_bounds__(kFusedWarps * 32, MINB)
    ragged_persistent_kernel(const RaggedQueueParams q) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *slab = smem + warp * q.slab;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(q.queue, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= q.n_items) break;
    // class of the item: items run class 4 (largest) first, class 0 last
    if (item < q.item_end[4]) {
      world_step_body<32, 4, 0, false, true, true>(q.p[4], smem, nullptr, warp, item * 1, slab);
    } else if (item < q.item_end[3]) {
      world_step_body<32, 2, 0, false, true, true>(q.p[3], smem, nullptr, warp,
                                                   (item - q.item_end[4]) * 1, slab);
    } else if (item < q.item_end[2]) {
      world_step_body<16, 2, 0, false, true, true>(q.p[2], smem, nullptr, warp,
                                                   (item - q.item_end[3]) * 2, slab);
    } else if (item < q.item_end[1]) {
      world_step_body<8, 2, 0, false, true, true>(q.p[1], smem, nullptr, warp,
                                                  (item - q.item_end[2]) * 4, slab);
    } else {
      world_step_body<8, 1, 0, false, true, true>(q.p[0], smem, nullptr, warp,
                                                  (item - q.item_end[1]) * 4, slab);
    }
    __syncwarp();
  }
}

}  // namespace vmas
