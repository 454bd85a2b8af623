// Launch parameters of the world-step kernels (plain, tiled, listed, ragged
// and allocation-free forms): plain data only, so that host code which only
// fills them need not compile any kernel.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace vmas {

struct StepParams {
  int E, N, A, S, P;
  float h;      // dt / S
  float damp;   // 1 - zeta
  float gx, gy;
  float ck;     // c * k
  float inv_k;  // 1 / k
  float vmax;   // 0 = no cap
  float skin;   // broad-phase margin of the per-step candidate list
  float *px, *py, *vx, *vy, *th, *om;  // state planes [E * N]
  const float4 *param;                 // {1/m (0 if fixed), 1/I (0 if not rotatable), ha, hb}
  const uint8_t *kind;                 // [E * N]
  const uint16_t *pairs;               // [P] i | j << 8
  const float *actions;                // [E][A][3]
  uint8_t *mask;                       // [E][P], mask kernel only
  int *err;                            // device error word
  unsigned long long *stats;           // optional counters, nullptr = off
  int tile;                            // world steps per launch (actions of step t at + t * act_step)
  size_t act_step;                     // floats per step in the actions array
  size_t EN;                           // entities in the state arrays (bound of every entity index)
  // packed ragged worlds (RAGGED kernels): envs [env_begin, env_end) of one size class
  const int *soff;                     // [E + 1] entity offsets, size-class (sorted) env order
  const int *perm;                     // [E] sorted position -> caller env index
  const int *aoff;                     // [E + 1] action-row offsets, caller env order
  int env_begin, env_end;
  // listed stepping (plain kernels): only envs env_list[0 .. *env_count) are
  // stepped; nullptr = all E envs
  const int *env_list, *env_count;
  // 1: a full CTA of the one-step plain kernel stages its contiguous slice of
  // state, parameters, kinds and actions into shared memory with bulk (TMA)
  // copies; the host sets it only when every copy is 16-byte aligned and the
  // staging fits the CTA's shared memory
  int bulk;
  // test hook: extra transaction bytes the staging mbarrier waits for, which
  // no copy delivers, so that its bounded wait runs out (0 in normal use)
  uint32_t stage_extra_tx;
  // caller-owned buffers of the allocation-free entry point (RAW kernels):
  float *aos_state;                    // [E][N][6] x y vx vy th om, read and written
  const uint8_t *r_shape, *r_flags;    // [E * N]
  const float *r_size_a, *r_size_b, *r_mass, *r_inertia;  // [E * N]
};

// A packed ragged world stepped in one persistent launch: every size class
// (capacities 8, 16, 32, 64, 128) from one atomic work queue.  Lanes per env
// and entities per lane of each class are fixed for this form.
constexpr int kPersistLanes[5] = {8, 8, 16, 32, 32};
constexpr int kPersistSlots[5] = {1, 2, 2, 2, 4};

struct RaggedQueueParams {
  StepParams p[5];  // one per size class: capacity, pair table, env range, actions, tile
  // work items (one warp's envs each) run largest class first: class c owns
  // items [item_end[c + 1], item_end[c]), with item_end[5] = 0 implied
  int item_end[5];
  int n_items;
  int *queue;       // the dequeue counter; must be 0 when the launch starts
  int slab;         // shared-memory bytes per warp
};

// Work items of a class of n_envs envs in the persistent form.
inline int persist_items(int n_envs, int c) {
  const int epw = 32 / kPersistLanes[c];
  return (n_envs + epw - 1) / epw;
}

}  // namespace vmas
