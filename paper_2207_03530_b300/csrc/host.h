// Internal header of the library's host side (not part of the C ABI): the
// world's device layout and the helpers the three host translation units
// share -- vmas.cu (worlds, the step, the allocation-free step, the
// differentiable rollout, LIDAR), ragged.cu (packed ragged worlds) and
// surrogate_host.cu (the learned surrogate).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "params.cuh"
#include "vmas.h"

struct vmas_world {
  int device = 0;
  int E = 0, N = 0, A = 0, S = 0, P = 0;
  float dt = 0, drag = 0, gx = 0, gy = 0, c = 0, k = 0, vmax = 0;
  float skin = 0;  // candidate-list margin
  bool diff_ok = false;  // every entity a sphere, N <= 32 (differentiable rollout)
  bool sur_ok = false;   // a layout the learned surrogate serves (sur_layout != 0)
  int sur_layout = 0;    // 1: 16 agent spheres + 4 walls; 2: 16 agents + 4 boxes + 4 walls
  bool stage_timeout_test = false;  // vmas_debug_stage_timeout
  int tile = 1;          // world steps per launch in vmas_rollout
  float *planes = nullptr;  // 6 * E * N
  float4 *param = nullptr;
  unsigned long long *stats = nullptr;  // optional step counters
  uint8_t *kind = nullptr;
  uint16_t *pairs = nullptr;
  int *err = nullptr;
  float *act = nullptr;
  float *stage = nullptr;
  uint8_t *env_mask = nullptr;
  std::vector<int32_t> pi, pj;
  // host-streaming rollouts (lazy): double-buffered device actions and
  // state staging, an upload and a download stream, and their events
  float *h_act[2] = {nullptr, nullptr};
  float *h_stage[2] = {nullptr, nullptr};
  cudaStream_t s_up = nullptr, s_down = nullptr;
  cudaEvent_t ev_up[2] = {}, ev_used[2] = {}, ev_gathered[2] = {}, ev_down[2] = {};
};

namespace vmas_host {

using vmas::StepParams;

// Record `msg` as this thread's last error and return `code`.
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Launch parameters of the world's plain step (actions left unset).
StepParams make_params(const vmas_world *w);
// Lanes per env the step kernel uses for N entities.
int group_lanes(int N);
// One launch of the plain step over all envs (or the listed ones); tiled =
// p.tile world steps per launch.
int launch_step(const StepParams &p, cudaStream_t st, bool tiled = false);
// One launch of the step kernel over a ragged world's size class.
int launch_ragged_class(const StepParams &p, int G, int slots, int n_envs, cudaStream_t st);
// One persistent launch over every size class of a ragged world (q.slab is
// filled in here); the caller zeroes *q.queue on `st` first.  budget 1: the
// 128-register build (4 CTAs per SM), 2: the 96-register build (5 per SM).
int launch_ragged_persistent(vmas::RaggedQueueParams q, int budget, cudaStream_t st);

}  // namespace vmas_host

#define VMAS_CUDA(call)                                             \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return vmas_host::cuda_fail(e_, #call);  \
  } while (0)
