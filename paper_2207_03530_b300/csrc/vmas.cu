// Host side of the VMAS C ABI (include/vmas.h): world creation, device
// layout, launches and error handling.  The physics lives in step_fused.cuh,
// step.cuh and contact.cuh; the differentiable rollout in diff.cuh, LIDAR in
// lidar.cuh, the learned surrogate in surrogate.cuh (layered GEMM path,
// training) and surrogate_fused.cuh (fused inference).  Sections below: the
// world, the allocation-free step, the differentiable rollout and LIDAR, the
// packed ragged worlds, the surrogate.
//
// Device layout of a world (all library-owned, allocated once at create):
//   state   6 FP32 planes px, py, vx, vy, th, om, each [E * N], env-major
//           (entity i of env e at e * N + i), so a warp reads an env's plane
//           as one contiguous run;
//   param   float4 [E * N] {1/m or 0, 1/I or 0, half size a, half size b}
//           (sphere: r, 0; box: w/2, h/2; line: L/2, 0);
//   kind    uint8  [E * N] shape | flags << 2;
//   pairs   uint16 [P] canonical pair list i | j << 8;
//   err     int32 device error word;
//   act     FP32 [E * A * 3] staging for host actions;
//   stage   FP32 [E * N * 6] staging for host state transfers (lazy);
//   h_act / h_stage  two of each, for host-streaming rollouts (lazy).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "diff.cuh"
#include "lidar.cuh"
#include "step_fused.cuh"
#include "vmas.h"

static_assert(vmas::kStatCount == VMAS_STATS_COUNT, "stats layout");

using vmas::StepParams;

struct vmas_world {
  int device = 0;
  int E = 0, N = 0, A = 0, S = 0, P = 0;
  float dt = 0, drag = 0, gx = 0, gy = 0, c = 0, k = 0, vmax = 0;
  float skin = 0;  // candidate-list margin
  bool diff_ok = false;  // every entity a sphere, N <= 32 (differentiable rollout)
  bool sur_ok = false;   // 16 actuated agent spheres then 4 fixed walls (surrogate)
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

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(VMAS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define VMAS_CUDA(call)                          \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

void free_world(vmas_world *w) {
  if (!w) return;
  cudaFree(w->planes);
  cudaFree(w->param);
  cudaFree(w->stats);
  cudaFree(w->kind);
  cudaFree(w->pairs);
  cudaFree(w->err);
  cudaFree(w->act);
  cudaFree(w->stage);
  cudaFree(w->env_mask);
  for (int b = 0; b < 2; ++b) {
    cudaFree(w->h_act[b]);
    cudaFree(w->h_stage[b]);
    cudaEvent_t evs[4] = {w->ev_up[b], w->ev_used[b], w->ev_gathered[b], w->ev_down[b]};
    for (cudaEvent_t e : evs)
      if (e) cudaEventDestroy(e);
  }
  if (w->s_up) cudaStreamDestroy(w->s_up);
  if (w->s_down) cudaStreamDestroy(w->s_down);
  delete w;
}

StepParams make_params(const vmas_world *w) {
  StepParams p{};
  p.E = w->E;
  p.N = w->N;
  p.A = w->A;
  p.S = w->S;
  p.P = w->P;
  p.h = (float)((double)w->dt / (double)w->S);
  p.damp = (float)(1.0 - (double)w->drag);
  p.gx = w->gx;
  p.gy = w->gy;
  p.ck = (float)((double)w->c * (double)w->k);
  p.inv_k = (float)(1.0 / (double)w->k);
  p.vmax = w->vmax;
  p.skin = w->skin;
  const size_t EN = (size_t)w->E * w->N;
  p.px = w->planes;
  p.py = w->planes + EN;
  p.vx = w->planes + 2 * EN;
  p.vy = w->planes + 3 * EN;
  p.th = w->planes + 4 * EN;
  p.om = w->planes + 5 * EN;
  p.param = w->param;
  p.stats = w->stats;
  p.kind = w->kind;
  p.pairs = w->pairs;
  p.err = w->err;
  p.tile = 1;
  p.act_step = (size_t)w->E * w->A * 3;
  p.EN = EN;
  p.stage_extra_tx = w->stage_timeout_test ? 16u : 0u;
  return p;
}

// One launch of the fused step kernel over `n_envs` environments (for RAGGED
// launches: envs [env_begin, env_begin + n_envs) of one size class).
template <int G, int SLOTS, int NC, bool RAGGED, bool TILED>
int launch_fused(const StepParams &p, int n_envs, cudaStream_t st) {
  if (n_envs <= 0) return VMAS_OK;
  const int smem = vmas::fused_cta_smem_bytes(p.N, p.P, G);
  auto kern = vmas::world_step_kernel<G, SLOTS, NC, false, RAGGED, TILED>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  }
  const int envs_per_cta = vmas::kFusedWarps * (32 / G);
  const int grid = (n_envs + envs_per_cta - 1) / envs_per_cta;
  kern<<<grid, vmas::kFusedWarps * 32, smem, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "world_step_kernel launch");
  return VMAS_OK;
}

// Entity counts with a kernel compiled for exactly that count (fully
// unrolled pair loops); any other count runs the generic kernel.
template <int G, bool TILED>
int launch_step_g(const StepParams &p, cudaStream_t st) {
#ifndef VMAS_NO_SPECIALIZE
  if constexpr (G == 8) {
    if (p.N == 24) return launch_fused<8, 3, 24, false, TILED>(p, p.E, st);
  }
  if constexpr (G == 4) {
    if (p.N == 6) return launch_fused<4, 2, 6, false, TILED>(p, p.E, st);
  }
#endif
  switch ((p.N + G - 1) / G) {
    case 1: return launch_fused<G, 1, 0, false, TILED>(p, p.E, st);
    case 2: return launch_fused<G, 2, 0, false, TILED>(p, p.E, st);
    case 3: return launch_fused<G, 3, 0, false, TILED>(p, p.E, st);
    default: return launch_fused<G, 4, 0, false, TILED>(p, p.E, st);
  }
}

// Ragged size-class launch with a runtime (lanes, slots) choice.
int launch_ragged_class(const StepParams &p, int G, int slots, int n_envs, cudaStream_t st) {
  switch (G * 8 + slots) {
    case 4 * 8 + 2: return launch_fused<4, 2, 0, true, true>(p, n_envs, st);
    case 4 * 8 + 4: return launch_fused<4, 4, 0, true, true>(p, n_envs, st);
    case 8 * 8 + 1: return launch_fused<8, 1, 0, true, true>(p, n_envs, st);
    case 8 * 8 + 2: return launch_fused<8, 2, 0, true, true>(p, n_envs, st);
    case 8 * 8 + 4: return launch_fused<8, 4, 0, true, true>(p, n_envs, st);
    case 16 * 8 + 1: return launch_fused<16, 1, 0, true, true>(p, n_envs, st);
    case 16 * 8 + 2: return launch_fused<16, 2, 0, true, true>(p, n_envs, st);
    case 16 * 8 + 4: return launch_fused<16, 4, 0, true, true>(p, n_envs, st);
    case 32 * 8 + 1: return launch_fused<32, 1, 0, true, true>(p, n_envs, st);
    case 32 * 8 + 2: return launch_fused<32, 2, 0, true, true>(p, n_envs, st);
    case 32 * 8 + 4: return launch_fused<32, 4, 0, true, true>(p, n_envs, st);
    default: return fail(VMAS_EINVAL, "unsupported lanes/slots choice");
  }
}

// Lanes per environment: the smallest group that holds every entity in at
// most 4 slots (N <= 8: 4 lanes, <= 32: 8, <= 64: 16, else 32).
int group_lanes(int N) {
#ifdef VMAS_GROUP_LANES
  const int g = VMAS_GROUP_LANES;  // build-time override for tuning sweeps
  if ((N + g - 1) / g <= 4) return g;
#endif
  return N <= 8 ? 4 : N <= 32 ? 8 : N <= 64 ? 16 : 32;
}

// Whether the one-step kernel may stage a full CTA's inputs with bulk copies:
// every copy a multiple of 16 bytes from a 16-byte aligned address, and the
// staging no larger than the CTA's per-env shared memory it borrows.
bool bulk_staging_ok(const StepParams &p) {
  const int G = group_lanes(p.N), CE = vmas::kFusedWarps * (32 / G);
  const size_t ents = (size_t)CE * p.N;
  if (ents % 16 != 0) return false;  // kind bytes
  auto misaligned = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) != 0; };
  const void *bases[9] = {p.px, p.py, p.vx, p.vy, p.th, p.om, p.param, p.kind, p.actions};
  for (int k = 0; k < 9; ++k)
    if ((k < 8 || p.A > 0) && misaligned(bases[k])) return false;
  const size_t stage = ents * (6 * 4 + 16 + 1) + (size_t)CE * p.A * 12;
  return stage <= (size_t)CE * vmas::fused_env_bytes(p.N, G);
}

int launch_step(const StepParams &p0, cudaStream_t st, bool tiled = false) {
  if (p0.E == 0) return VMAS_OK;
  StepParams p = p0;
  p.bulk = !tiled && !p.env_list && bulk_staging_ok(p) ? 1 : 0;
  switch (group_lanes(p.N)) {
    case 4: return tiled ? launch_step_g<4, true>(p, st) : launch_step_g<4, false>(p, st);
    case 8: return tiled ? launch_step_g<8, true>(p, st) : launch_step_g<8, false>(p, st);
    case 16: return tiled ? launch_step_g<16, true>(p, st) : launch_step_g<16, false>(p, st);
    default: return tiled ? launch_step_g<32, true>(p, st) : launch_step_g<32, false>(p, st);
  }
}

template <int SLOTS>
int launch_mask_s(const StepParams &p, cudaStream_t st) {
  const int smem = vmas::mask_cta_smem_bytes(p.N, p.P);
  auto kern = vmas::pair_mask_kernel<SLOTS>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  }
  const int grid = (p.E + vmas::kWarpsPerCta - 1) / vmas::kWarpsPerCta;
  kern<<<grid, vmas::kWarpsPerCta * 32, smem, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pair_mask_kernel launch");
  return VMAS_OK;
}

int launch_mask(const StepParams &p, cudaStream_t st) {
  if (p.E == 0) return VMAS_OK;
  switch ((p.N + 31) / 32) {
    case 1: return launch_mask_s<1>(p, st);
    case 2: return launch_mask_s<2>(p, st);
    case 3: return launch_mask_s<3>(p, st);
    default: return launch_mask_s<4>(p, st);
  }
}

// [E][N][6] AoS -> planes, for envs whose mask byte is non-zero (or all).
__global__ void scatter_state_kernel(float *planes, const float *aos, const uint8_t *mask,
                                     size_t EN, int N) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= EN) return;
  if (mask && !mask[t / N]) return;
  for (int f = 0; f < 6; ++f) planes[f * EN + t] = aos[t * 6 + f];
}

// planes -> [E][N][6] AoS.
__global__ void gather_state_kernel(float *aos, const float *planes, size_t EN) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= EN) return;
  for (int f = 0; f < 6; ++f) aos[t * 6 + f] = planes[f * EN + t];
}

int ensure_stage(vmas_world *w) {
  if (w->stage) return VMAS_OK;
  const size_t n = (size_t)w->E * w->N * 6;
  VMAS_CUDA(cudaMalloc(&w->stage, n * sizeof(float) + 16));
  return VMAS_OK;
}

int read_err(vmas_world *w, cudaStream_t st, int32_t *bits) {
  int h = 0;
  VMAS_CUDA(cudaMemcpyAsync(&h, w->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  VMAS_CUDA(cudaStreamSynchronize(st));
  if (bits) *bits = h;
  if (h) {
    VMAS_CUDA(cudaMemsetAsync(w->err, 0, sizeof(int), st));
    VMAS_CUDA(cudaStreamSynchronize(st));
    return fail(VMAS_EDEVICE, "device error word set (bits " + std::to_string(h) + ")");
  }
  return VMAS_OK;
}

// ---- allocation-free step (vmas_step_noalloc) -----------------------------
// Its only scratch is this array: the canonical pair table for up to
// VMAS_NOALLOC_MAX_ENTITIES entities (uint16 i | j << 8) followed by a status
// word.  Every device that loads the library holds it until exit; every call
// shares it.
constexpr int kNoallocPairs = VMAS_NOALLOC_MAX_ENTITIES * (VMAS_NOALLOC_MAX_ENTITIES - 1) / 2;
constexpr int kNoallocStatusOffset = ((kNoallocPairs * 2 + 255) / 256) * 256;
constexpr int kNoallocBytes = kNoallocStatusOffset + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[kMaxDevices];  // device address of the array, per device

// Set-up on first use per device (with that device current): the device
// address of the scratch array.  A host-side reference to the array is only a
// stand-in and must never be handed to a kernel.
int noalloc_scratch(unsigned char **out) {
  int dev = 0;
  VMAS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(VMAS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *ptr = nullptr;
    VMAS_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<unsigned char *>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return VMAS_OK;
}

// Canonical pair list (i < j, row-major) for N entities.
__global__ void fill_pairs_kernel(uint16_t *pairs, int N) {
  for (int i = blockIdx.x; i < N - 1; i += gridDim.x) {
    const int row = i * N - i * (i + 1) / 2;
    for (int j = i + 1 + threadIdx.x; j < N; j += blockDim.x)
      pairs[row + (j - i - 1)] = (uint16_t)(i | (j << 8));
  }
}

template <int G, int SLOTS>
int launch_raw_gs(const StepParams &p, cudaStream_t st) {
  const int smem = vmas::fused_cta_smem_bytes(p.N, p.P, G);
  auto kern = vmas::world_step_kernel<G, SLOTS, 0, true>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  }
  const int envs_per_cta = vmas::kFusedWarps * (32 / G);
  const int grid = (p.E + envs_per_cta - 1) / envs_per_cta;
  kern<<<grid, vmas::kFusedWarps * 32, smem, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "world_step_kernel (no-alloc) launch");
  return VMAS_OK;
}

template <int G>
int launch_raw_g(const StepParams &p, cudaStream_t st) {
  switch ((p.N + G - 1) / G) {
    case 1: return launch_raw_gs<G, 1>(p, st);
    case 2: return launch_raw_gs<G, 2>(p, st);
    case 3: return launch_raw_gs<G, 3>(p, st);
    default: return launch_raw_gs<G, 4>(p, st);
  }
}

}  // namespace

extern "C" {

int vmas_step_noalloc(const vmas_step_noalloc_args *a, void *stream) {
  if (!a) return fail(VMAS_EINVAL, "args is NULL");
  if (a->n_envs < 0 || a->n_actuated < 0 || a->substeps < 1)
    return fail(VMAS_EINVAL, "n_envs, n_actuated must be >= 0 and substeps >= 1");
  if (a->n_entities < 1 || a->n_entities > VMAS_NOALLOC_MAX_ENTITIES)
    return fail(VMAS_EINVAL, "n_entities must be 1.." + std::to_string(VMAS_NOALLOC_MAX_ENTITIES) +
                                 ": the allocation-free step keeps its pair table in a fixed "
                                 "scratch array of that size");
  if (!(a->dt > 0) || !std::isfinite(a->dt) || !(a->contact_margin > 0) ||
      !(a->contact_force >= 0) || !(a->max_speed >= 0) || !(a->skin >= 0) ||
      !std::isfinite(a->skin))
    return fail(VMAS_EINVAL, "dt, contact_margin must be > 0; contact_force, max_speed, skin >= 0");
  const size_t EN = (size_t)a->n_envs * a->n_entities;
  if (EN && (!a->state || !a->shape || !a->flags || !a->size_a || !a->size_b || !a->mass ||
             !a->inertia))
    return fail(VMAS_EINVAL, "a device array is NULL");
  if (EN && a->n_actuated && !a->actions) return fail(VMAS_EINVAL, "actions is NULL");
  unsigned char *scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  const int N = a->n_entities;
  uint16_t *pairs = reinterpret_cast<uint16_t *>(scratch);
  int *status = reinterpret_cast<int *>(scratch + kNoallocStatusOffset);
  // the status word must start each call at zero; the pair table is rewritten
  VMAS_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  if (N > 1) {
    fill_pairs_kernel<<<N - 1, 64, 0, st>>>(pairs, N);
    VMAS_CUDA(cudaGetLastError());
  }
  if (!EN) return VMAS_OK;
  StepParams p{};
  p.E = a->n_envs;
  p.N = N;
  p.A = a->n_actuated;
  p.S = a->substeps;
  p.P = N * (N - 1) / 2;
  p.h = (float)((double)a->dt / (double)a->substeps);
  p.damp = (float)(1.0 - (double)a->drag);
  p.gx = a->gx;
  p.gy = a->gy;
  p.ck = (float)((double)a->contact_force * (double)a->contact_margin);
  p.inv_k = (float)(1.0 / (double)a->contact_margin);
  p.vmax = a->max_speed;
  p.skin = a->skin;
  p.tile = 1;
  p.act_step = (size_t)a->n_envs * a->n_actuated * 3;
  p.EN = EN;
  p.pairs = pairs;
  p.actions = a->actions;
  p.err = a->status ? a->status : status;
  p.aos_state = a->state;
  p.r_shape = a->shape;
  p.r_flags = a->flags;
  p.r_size_a = a->size_a;
  p.r_size_b = a->size_b;
  p.r_mass = a->mass;
  p.r_inertia = a->inertia;
  switch (group_lanes(N)) {
    case 4: return launch_raw_g<4>(p, st);
    case 8: return launch_raw_g<8>(p, st);
    case 16: return launch_raw_g<16>(p, st);
    default: return launch_raw_g<32>(p, st);
  }
}


const char *vmas_last_error(void) { return g_last_error.c_str(); }

int vmas_abi_version(void) { return VMAS_ABI_VERSION; }

int vmas_world_create(const vmas_world_desc *d, vmas_world **out) {
  if (!out) return fail(VMAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d) return fail(VMAS_EINVAL, "desc is NULL");
  if (d->n_envs < 0) return fail(VMAS_EINVAL, "n_envs < 0");
  if (d->n_entities < 1 || d->n_entities > VMAS_MAX_ENTITIES)
    return fail(VMAS_EINVAL, "n_entities outside 1.." + std::to_string(VMAS_MAX_ENTITIES));
  if (d->n_actuated < 0) return fail(VMAS_EINVAL, "n_actuated < 0");
  if (d->substeps < 1) return fail(VMAS_EINVAL, "substeps < 1");
  if (!(d->dt > 0) || !std::isfinite(d->dt)) return fail(VMAS_EINVAL, "dt must be > 0");
  if (!std::isfinite(d->drag) || !std::isfinite(d->gx) || !std::isfinite(d->gy))
    return fail(VMAS_EINVAL, "drag / gravity not finite");
  if (!(d->contact_force >= 0) || !std::isfinite(d->contact_force))
    return fail(VMAS_EINVAL, "contact_force must be >= 0");
  if (!(d->contact_margin > 0) || !std::isfinite(d->contact_margin))
    return fail(VMAS_EINVAL, "contact_margin must be > 0");
  if (!(d->max_speed >= 0)) return fail(VMAS_EINVAL, "max_speed must be >= 0");
  const int E = d->n_envs, N = d->n_entities;
  const size_t EN = (size_t)E * N;
  if (EN > 0 && (!d->shape || !d->flags || !d->size_a || !d->size_b || !d->mass ||
                 !d->inertia || !d->init_state))
    return fail(VMAS_EINVAL, "a per-entity array is NULL");

  std::vector<float4> param(EN);
  std::vector<float> bound_r(EN);
  std::vector<uint8_t> kind(EN);
  for (int e = 0; e < E; ++e) {
    int n_act = 0;
    for (int i = 0; i < N; ++i) {
      const size_t t = (size_t)e * N + i;
      const int sh = d->shape[t];
      const int fl = d->flags[t];
      if (sh > 2) return fail(VMAS_EINVAL, "bad shape id at entity " + std::to_string(t));
      if (fl & ~15) return fail(VMAS_EINVAL, "unknown flag bits at entity " + std::to_string(t));
      const double a = d->size_a[t], b = d->size_b[t], m = d->mass[t];
      if (!(a > 0) || !std::isfinite(a))
        return fail(VMAS_EINVAL, "size_a must be > 0 at entity " + std::to_string(t));
      if (sh == VMAS_BOX && (!(b > 0) || !std::isfinite(b)))
        return fail(VMAS_EINVAL, "box size_b must be > 0 at entity " + std::to_string(t));
      if ((fl & VMAS_MOVABLE) && (!(m > 0) || !std::isfinite(m)))
        return fail(VMAS_EINVAL, "movable entity needs mass > 0 at " + std::to_string(t));
      double I = d->inertia[t];
      if (I == 0) {
        if (sh == VMAS_BOX) I = m * (a * a + b * b) / 12.0;
        else if (sh == VMAS_LINE) I = m * a * a / 12.0;
        else I = 0.5 * m * a * a;
      }
      if ((fl & VMAS_ROTATABLE) && (!(I > 0) || !std::isfinite(I)))
        return fail(VMAS_EINVAL, "rotatable entity needs inertia > 0 at " + std::to_string(t));
      if (fl & VMAS_ACTUATED) ++n_act;
      double ha, hb;
      if (sh == VMAS_SPHERE) { ha = a; hb = 0; }
      else if (sh == VMAS_BOX) { ha = 0.5 * a; hb = 0.5 * b; }
      else { ha = 0.5 * a; hb = 0; }
      param[t] = make_float4((fl & VMAS_MOVABLE) ? (float)(1.0 / m) : 0.f,
                             (fl & VMAS_ROTATABLE) ? (float)(1.0 / I) : 0.f, (float)ha, (float)hb);
      bound_r[t] = (float)std::sqrt(ha * ha + hb * hb);
      kind[t] = (uint8_t)(sh | (fl << 2));
    }
    if (n_act > d->n_actuated)
      return fail(VMAS_EINVAL, "env " + std::to_string(e) + " has more actuated entities (" +
                                   std::to_string(n_act) + ") than n_actuated");
  }
  for (size_t t = 0; t < EN * 6; ++t)
    if (!std::isfinite(d->init_state[t])) return fail(VMAS_EINVAL, "init_state not finite");

  vmas_world *w = new vmas_world();
  cudaGetDevice(&w->device);
  w->E = E;
  w->N = N;
  w->A = d->n_actuated;
  w->S = d->substeps;
  w->P = N * (N - 1) / 2;
  w->dt = d->dt;
  w->drag = d->drag;
  w->gx = d->gx;
  w->gy = d->gy;
  w->c = d->contact_force;
  w->k = d->contact_margin;
  w->vmax = d->max_speed;
  {
    bool spheres = N <= 32;
    for (size_t t = 0; t < EN && spheres; ++t) spheres = d->shape[t] == VMAS_SPHERE;
    w->diff_ok = spheres;
  }
  {
    // layout the learned surrogate is trained for: per env 16 movable,
    // actuated, non-rotating agent spheres (action rows 0..15), then 4 fixed
    // lines (the walls), at least 16 action rows
    bool ok = N == 20 && w->A >= 16;
    for (int e = 0; e < E && ok; ++e)
      for (int i = 0; i < N && ok; ++i) {
        const size_t t = (size_t)e * N + i;
        const int fl = d->flags[t];
        if (i < 16)
          ok = d->shape[t] == VMAS_SPHERE && (fl & VMAS_MOVABLE) && (fl & VMAS_ACTUATED) &&
               !(fl & VMAS_ROTATABLE);
        else
          ok = d->shape[t] == VMAS_LINE && !(fl & (VMAS_MOVABLE | VMAS_ACTUATED));
      }
    w->sur_ok = ok;
  }
  {
    // candidate-list margin: half the median bounding radius of the movable
    // entities (any value >= 0 gives the same results; this one balances
    // list length against rebuilds)
    std::vector<float> r;
    for (size_t t = 0; t < EN; ++t)
      if (d->flags[t] & VMAS_MOVABLE) r.push_back(bound_r[t]);
    float med = 0.05f;
    if (!r.empty()) {
      std::nth_element(r.begin(), r.begin() + r.size() / 2, r.end());
      med = r[r.size() / 2];
    }
    w->skin = 0.5f * med;
  }
  std::vector<uint16_t> pairs(w->P > 0 ? w->P : 1);
  w->pi.resize(w->P);
  w->pj.resize(w->P);
  {
    int q = 0;
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j, ++q) {
        pairs[q] = (uint16_t)(i | (j << 8));
        w->pi[q] = i;
        w->pj[q] = j;
      }
  }
  std::vector<float> planes(EN * 6);
  for (size_t t = 0; t < EN; ++t)
    for (int f = 0; f < 6; ++f) planes[f * EN + t] = d->init_state[t * 6 + f];

  auto alloc = [&](void **ptr, size_t bytes) -> bool {
    return cudaMalloc(ptr, bytes > 0 ? bytes : 16) == cudaSuccess;
  };
  bool ok = alloc((void **)&w->planes, EN * 6 * sizeof(float)) &&
            alloc((void **)&w->param, EN * sizeof(float4)) &&
            alloc((void **)&w->kind, EN) &&
            alloc((void **)&w->pairs, pairs.size() * sizeof(uint16_t)) &&
            alloc((void **)&w->err, 4 * sizeof(int)) &&
            alloc((void **)&w->act, (size_t)E * w->A * 3 * sizeof(float)) &&
            alloc((void **)&w->env_mask, (size_t)E);
  if (!ok) {
    cudaGetLastError();
    free_world(w);
    return fail(VMAS_ENOMEM, "cudaMalloc failed while creating the world");
  }
  cudaError_t e = cudaSuccess;
  if (EN) {
    if (e == cudaSuccess) e = cudaMemcpy(w->planes, planes.data(), EN * 6 * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->param, param.data(), EN * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->kind, kind.data(), EN, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(w->pairs, pairs.data(), pairs.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(w->err, 0, 4 * sizeof(int));
  if (e != cudaSuccess) {
    free_world(w);
    return cuda_fail(e, "world upload");
  }
  *out = w;
  return VMAS_OK;
}

int vmas_world_destroy(vmas_world *w) {
  if (!w) return VMAS_OK;
  cudaDeviceSynchronize();
  free_world(w);
  return VMAS_OK;
}

int vmas_world_set_skin(vmas_world *w, float skin) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (!(skin >= 0) || !std::isfinite(skin)) return fail(VMAS_EINVAL, "skin must be >= 0");
  w->skin = skin;
  return VMAS_OK;
}

int vmas_world_get_skin(const vmas_world *w, float *skin) {
  if (!w || !skin) return fail(VMAS_EINVAL, "NULL argument");
  *skin = w->skin;
  return VMAS_OK;
}

int vmas_world_set_stats(vmas_world *w, int32_t enable) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (!enable) {
    cudaFree(w->stats);
    w->stats = nullptr;
    return VMAS_OK;
  }
  if (!w->stats) {
    VMAS_CUDA(cudaMalloc(&w->stats, VMAS_STATS_COUNT * sizeof(unsigned long long)));
    VMAS_CUDA(cudaMemset(w->stats, 0, VMAS_STATS_COUNT * sizeof(unsigned long long)));
  }
  return VMAS_OK;
}

int vmas_world_get_stats(vmas_world *w, uint64_t *out, int32_t reset, void *stream) {
  if (!w || !out) return fail(VMAS_EINVAL, "NULL argument");
  if (!w->stats) return fail(VMAS_EINVAL, "stats are not enabled");
  cudaStream_t st = as_stream(stream);
  VMAS_CUDA(cudaMemcpyAsync(out, w->stats, VMAS_STATS_COUNT * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
  if (reset)
    VMAS_CUDA(cudaMemsetAsync(w->stats, 0, VMAS_STATS_COUNT * sizeof(unsigned long long), st));
  VMAS_CUDA(cudaStreamSynchronize(st));
  return VMAS_OK;
}

int vmas_world_info(const vmas_world *w, int32_t *n_envs, int32_t *n_entities,
                    int32_t *n_actuated, int32_t *substeps, int32_t *n_pairs) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (n_envs) *n_envs = w->E;
  if (n_entities) *n_entities = w->N;
  if (n_actuated) *n_actuated = w->A;
  if (substeps) *substeps = w->S;
  if (n_pairs) *n_pairs = w->P;
  return VMAS_OK;
}

int vmas_step(vmas_world *w, const float *d_actions, void *stream) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (w->A > 0 && w->E > 0 && !d_actions) return fail(VMAS_EINVAL, "d_actions is NULL");
  StepParams p = make_params(w);
  p.actions = d_actions;
  return launch_step(p, as_stream(stream));
}

int vmas_step_host(vmas_world *w, const float *h_actions, void *stream) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  const size_t bytes = (size_t)w->E * w->A * 3 * sizeof(float);
  if (bytes) {
    if (!h_actions) return fail(VMAS_EINVAL, "h_actions is NULL");
    VMAS_CUDA(cudaMemcpyAsync(w->act, h_actions, bytes, cudaMemcpyHostToDevice, as_stream(stream)));
  }
  return vmas_step(w, w->act, stream);
}

int vmas_rollout(vmas_world *w, const float *d_actions, int32_t n_steps, void *stream) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (n_steps < 0) return fail(VMAS_EINVAL, "n_steps < 0");
  if (w->A > 0 && w->E > 0 && n_steps > 0 && !d_actions) return fail(VMAS_EINVAL, "d_actions is NULL");
  const size_t per = (size_t)w->E * w->A * 3;
  if (w->tile <= 1) {
    for (int t = 0; t < n_steps; ++t) {
      const int rc = vmas_step(w, d_actions ? d_actions + per * t : nullptr, stream);
      if (rc) return rc;
    }
    return VMAS_OK;
  }
  // w->tile steps per launch: state and candidate lists stay on chip
  for (int t = 0; t < n_steps; t += w->tile) {
    StepParams p = make_params(w);
    p.actions = d_actions ? d_actions + per * t : nullptr;
    p.tile = std::min(w->tile, n_steps - t);
    const int rc = launch_step(p, as_stream(stream), true);
    if (rc) return rc;
  }
  return VMAS_OK;
}

static int ensure_streaming(vmas_world *w) {
  if (w->s_down) return VMAS_OK;
  const size_t act = (size_t)w->E * w->A * 3, st = (size_t)w->E * w->N * 6;
  for (int b = 0; b < 2; ++b) {
    VMAS_CUDA(cudaMalloc(&w->h_act[b], (act > 0 ? act : 1) * sizeof(float)));
    VMAS_CUDA(cudaMalloc(&w->h_stage[b], (st > 0 ? st : 1) * sizeof(float)));
    VMAS_CUDA(cudaEventCreateWithFlags(&w->ev_up[b], cudaEventDisableTiming));
    VMAS_CUDA(cudaEventCreateWithFlags(&w->ev_used[b], cudaEventDisableTiming));
    VMAS_CUDA(cudaEventCreateWithFlags(&w->ev_gathered[b], cudaEventDisableTiming));
    VMAS_CUDA(cudaEventCreateWithFlags(&w->ev_down[b], cudaEventDisableTiming));
  }
  VMAS_CUDA(cudaStreamCreateWithFlags(&w->s_up, cudaStreamNonBlocking));
  VMAS_CUDA(cudaStreamCreateWithFlags(&w->s_down, cudaStreamNonBlocking));
  return VMAS_OK;
}

int vmas_rollout_host(vmas_world *w, const float *h_actions, int32_t n_steps, float *h_states,
                      void *stream) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (n_steps < 0) return fail(VMAS_EINVAL, "n_steps < 0");
  const size_t per_act = (size_t)w->E * w->A * 3, per_st = (size_t)w->E * w->N * 6;
  if (n_steps == 0 || per_st == 0) return VMAS_OK;
  if (per_act > 0 && !h_actions) return fail(VMAS_EINVAL, "h_actions is NULL");
  if (!h_states) return fail(VMAS_EINVAL, "h_states is NULL");
  int rc = ensure_streaming(w);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  // the upload and download streams start after the work already on `stream`
  VMAS_CUDA(cudaEventRecord(w->ev_used[0], st));
  VMAS_CUDA(cudaStreamWaitEvent(w->s_up, w->ev_used[0], 0));
  VMAS_CUDA(cudaStreamWaitEvent(w->s_down, w->ev_used[0], 0));
  VMAS_CUDA(cudaEventRecord(w->ev_used[1], st));
  VMAS_CUDA(cudaEventRecord(w->ev_down[0], st));
  VMAS_CUDA(cudaEventRecord(w->ev_down[1], st));
  for (int t = 0; t < n_steps; ++t) {
    const int b = t & 1;
    // upload step t's actions once step t - 2 has consumed buffer b
    if (per_act > 0) {
      VMAS_CUDA(cudaStreamWaitEvent(w->s_up, w->ev_used[b], 0));
      VMAS_CUDA(cudaMemcpyAsync(w->h_act[b], h_actions + per_act * t, per_act * sizeof(float),
                                cudaMemcpyHostToDevice, w->s_up));
      VMAS_CUDA(cudaEventRecord(w->ev_up[b], w->s_up));
      VMAS_CUDA(cudaStreamWaitEvent(st, w->ev_up[b], 0));
    }
    StepParams p = make_params(w);
    p.actions = w->h_act[b];
    if ((rc = launch_step(p, st))) return rc;
    VMAS_CUDA(cudaEventRecord(w->ev_used[b], st));
    // stage the new state once the download of step t - 2 has left buffer b
    VMAS_CUDA(cudaStreamWaitEvent(st, w->ev_down[b], 0));
    gather_state_kernel<<<(unsigned)((per_st / 6 + 255) / 256), 256, 0, st>>>(
        w->h_stage[b], w->planes, per_st / 6);
    VMAS_CUDA(cudaGetLastError());
    VMAS_CUDA(cudaEventRecord(w->ev_gathered[b], st));
    VMAS_CUDA(cudaStreamWaitEvent(w->s_down, w->ev_gathered[b], 0));
    VMAS_CUDA(cudaMemcpyAsync(h_states + per_st * t, w->h_stage[b], per_st * sizeof(float),
                              cudaMemcpyDeviceToHost, w->s_down));
    VMAS_CUDA(cudaEventRecord(w->ev_down[b], w->s_down));
  }
  VMAS_CUDA(cudaStreamSynchronize(w->s_down));
  VMAS_CUDA(cudaStreamSynchronize(w->s_up));
  return read_err(w, st, nullptr);
}

int vmas_world_set_rollout_tile(vmas_world *w, int32_t steps_per_launch) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (steps_per_launch < 1 || steps_per_launch > 1024)
    return fail(VMAS_EINVAL, "steps_per_launch must be 1..1024");
  w->tile = steps_per_launch;
  return VMAS_OK;
}

int vmas_state(vmas_world *w, float *out, int32_t out_is_device, void *stream) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  const size_t EN = (size_t)w->E * w->N;
  if (EN && !out) return fail(VMAS_EINVAL, "out is NULL");
  cudaStream_t st = as_stream(stream);
  if (EN) {
    float *dst = out;
    if (!out_is_device) {
      const int rc = ensure_stage(w);
      if (rc) return rc;
      dst = w->stage;
    }
    gather_state_kernel<<<(unsigned)((EN + 255) / 256), 256, 0, st>>>(dst, w->planes, EN);
    VMAS_CUDA(cudaGetLastError());
    if (!out_is_device)
      VMAS_CUDA(cudaMemcpyAsync(out, w->stage, EN * 6 * sizeof(float), cudaMemcpyDeviceToHost, st));
  }
  if (!out_is_device) return read_err(w, st, nullptr);
  return VMAS_OK;
}

int vmas_set_state(vmas_world *w, const float *state, int32_t state_is_device,
                   const uint8_t *env_mask, void *stream) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  const size_t EN = (size_t)w->E * w->N;
  if (!EN) return VMAS_OK;
  if (!state) return fail(VMAS_EINVAL, "state is NULL");
  cudaStream_t st = as_stream(stream);
  const float *src = state;
  if (!state_is_device) {
    const int rc = ensure_stage(w);
    if (rc) return rc;
    VMAS_CUDA(cudaMemcpyAsync(w->stage, state, EN * 6 * sizeof(float), cudaMemcpyHostToDevice, st));
    src = w->stage;
  }
  const uint8_t *dmask = nullptr;
  if (env_mask) {
    VMAS_CUDA(cudaMemcpyAsync(w->env_mask, env_mask, (size_t)w->E, cudaMemcpyHostToDevice, st));
    dmask = w->env_mask;
  }
  scatter_state_kernel<<<(unsigned)((EN + 255) / 256), 256, 0, st>>>(w->planes, src, dmask, EN, w->N);
  VMAS_CUDA(cudaGetLastError());
  // host inputs are consumed before returning
  if (!state_is_device || env_mask) VMAS_CUDA(cudaStreamSynchronize(st));
  return VMAS_OK;
}

int vmas_debug_pairs(vmas_world *w, uint8_t *d_mask, void *stream) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if ((size_t)w->E * w->P && !d_mask) return fail(VMAS_EINVAL, "d_mask is NULL");
  if (w->P == 0) return VMAS_OK;
  StepParams p = make_params(w);
  p.mask = d_mask;
  return launch_mask(p, as_stream(stream));
}

int vmas_pair_table(const vmas_world *w, int32_t *pair_i, int32_t *pair_j) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (w->P && (!pair_i || !pair_j)) return fail(VMAS_EINVAL, "output is NULL");
  if (w->P) {
    std::memcpy(pair_i, w->pi.data(), w->P * sizeof(int32_t));
    std::memcpy(pair_j, w->pj.data(), w->P * sizeof(int32_t));
  }
  return VMAS_OK;
}

#ifdef VMAS_CHECKED
// Self-checking build only: the error words {bits, first bad index, limit}.
int vmas_debug_err_words(vmas_world *w, int32_t *out) {
  if (!w || !out) return VMAS_EINVAL;
  cudaDeviceSynchronize();
  return cudaMemcpy(out, w->err, 3 * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : VMAS_ECUDA;
}
#endif

// Lanes per env of the differentiable rollout kernels: the smallest power
// of two that holds the env's entities.
static int diff_group_lanes(int N) { return N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32; }

static int diff_setup(vmas_world *w, int32_t T, int32_t K, vmas::DiffParams *p) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (!w->diff_ok)
    return fail(VMAS_EINVAL, "the differentiable rollout needs a world of spheres with at most 32 entities");
  if (w->vmax > 0) return fail(VMAS_EINVAL, "the differentiable rollout does not support a speed cap");
  if (T < 0 || K < 1) return fail(VMAS_EINVAL, "n_steps must be >= 0 and ckpt_every >= 1");
  *p = vmas::DiffParams{};
  p->E = w->E;
  p->N = w->N;
  p->A = w->A;
  p->S = w->S;
  p->T = T;
  p->K = K;
  p->h = (float)((double)w->dt / (double)w->S);
  p->damp = (float)(1.0 - (double)w->drag);
  p->gx = w->gx;
  p->gy = w->gy;
  p->ck = (float)((double)w->c * (double)w->k);
  p->inv_k = (float)(1.0 / (double)w->k);
  p->c = w->c;
  const size_t EN = (size_t)w->E * w->N;
  p->px = w->planes;
  p->py = w->planes + EN;
  p->vx = w->planes + 2 * EN;
  p->vy = w->planes + 3 * EN;
  p->param = w->param;
  p->kind = w->kind;
  return VMAS_OK;
}

int vmas_diff_rollout(vmas_world *w, const float *d_actions, int32_t n_steps,
                      const float *d_goals, int32_t ckpt_every, float *d_ckpt, float *d_loss,
                      void *stream) {
  vmas::DiffParams p;
  int rc = diff_setup(w, n_steps, ckpt_every, &p);
  if (rc) return rc;
  if (w->E == 0) return VMAS_OK;
  if (!d_loss || (w->A && (!d_goals || (n_steps && !d_actions))) || (n_steps && !d_ckpt))
    return fail(VMAS_EINVAL, "NULL buffer");
  p.actions = d_actions;
  p.goals = d_goals;
  p.ckpt = d_ckpt;
  p.loss = d_loss;
  const int G = diff_group_lanes(w->N), per_cta = vmas::kDiffWarps * (32 / G);
  const int grid = (w->E + per_cta - 1) / per_cta;
  cudaStream_t st = as_stream(stream);
  switch (G) {
    case 4: vmas::diff_forward_kernel<4><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    case 8: vmas::diff_forward_kernel<8><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    case 16: vmas::diff_forward_kernel<16><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    default: vmas::diff_forward_kernel<32><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
  }
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

int vmas_diff_backward(vmas_world *w, const float *d_actions, int32_t n_steps,
                       const float *d_goals, int32_t ckpt_every, const float *d_ckpt,
                       const float *d_dloss, float *d_grad, void *stream) {
  vmas::DiffParams p;
  int rc = diff_setup(w, n_steps, ckpt_every, &p);
  if (rc) return rc;
  const size_t ng = (size_t)n_steps * w->E * w->A * 3;
  if (ng == 0) return VMAS_OK;
  if (!d_actions || !d_goals || !d_ckpt || !d_dloss || !d_grad)
    return fail(VMAS_EINVAL, "NULL buffer");
  const size_t per_warp = vmas::diff_traj_bytes(ckpt_every, w->S);
  const size_t smem = per_warp * vmas::kDiffWarps;
  if (smem > 220 * 1024)
    return fail(VMAS_EINVAL, "ckpt_every * substeps too large for on-chip segment replay; "
                             "use a shorter checkpoint interval");
  const int G = diff_group_lanes(w->N), per_cta = vmas::kDiffWarps * (32 / G);
  auto kern = G == 4 ? vmas::diff_backward_kernel<4>
                     : G == 8 ? vmas::diff_backward_kernel<8>
                              : G == 16 ? vmas::diff_backward_kernel<16>
                                        : vmas::diff_backward_kernel<32>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  }
  cudaStream_t st = as_stream(stream);
  vmas::diff_zero_grad_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(d_grad, ng);
  VMAS_CUDA(cudaGetLastError());
  p.actions = d_actions;
  p.goals = d_goals;
  p.ckpt = const_cast<float *>(d_ckpt);
  p.dloss = d_dloss;
  p.grad = d_grad;
  const int grid = (w->E + per_cta - 1) / per_cta;
  kern<<<grid, vmas::kDiffWarps * 32, smem, st>>>(p);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

int vmas_lidar(vmas_world *w, int32_t n_rays, float max_range, float *d_out, void *stream) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (n_rays < 1 || !(max_range >= 0) || !std::isfinite(max_range))
    return fail(VMAS_EINVAL, "n_rays must be >= 1 and max_range >= 0");
  if ((size_t)w->E * w->A == 0) return VMAS_OK;
  if (!d_out) return fail(VMAS_EINVAL, "d_out is NULL");
  vmas::LidarParams p{};
  p.E = w->E;
  p.N = w->N;
  p.A = w->A;
  p.R = n_rays;
  p.range = max_range;
  const size_t EN = (size_t)w->E * w->N;
  p.px = w->planes;
  p.py = w->planes + EN;
  p.th = w->planes + 4 * EN;
  p.param = w->param;
  p.kind = w->kind;
  p.out = d_out;
  const size_t smem = (size_t)w->N * (16 + 8 + 1) + 16;
  vmas::lidar_kernel<<<w->E, 128, smem, as_stream(stream)>>>(p);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

int vmas_debug_stage_timeout(vmas_world *w, int32_t on) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  w->stage_timeout_test = on != 0;
  return VMAS_OK;
}

int vmas_debug_body_axes(const float *d_theta, float *d_cos_sin, int32_t n, void *stream) {
  if (n < 0 || (n > 0 && (!d_theta || !d_cos_sin))) return fail(VMAS_EINVAL, "bad arguments");
  if (n == 0) return VMAS_OK;
  vmas::body_axes_kernel<<<(n + 255) / 256, 256, 0, as_stream(stream)>>>(d_theta, d_cos_sin, n);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

int vmas_check(vmas_world *w, void *stream, int32_t *bits) {
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  return read_err(w, as_stream(stream), bits);
}

}  // extern "C"

// ============================================================================
// Packed ragged worlds: environments with different entity counts.
//
// Entities of all envs are packed without padding.  Envs are sorted into size
// classes of capacity 8, 16, 32, 64, 128 entities (smallest class that holds
// the env); each class is stepped by the fused kernel compiled for its (lanes
// per env, entities per lane) choice, which the autotuner picks by timing, as
// it picks the number of world steps per launch of a rollout.  Rollouts are
// captured into a CUDA graph (one node per class per tile of steps) and
// replayed.
// ============================================================================

struct vmas_ragged {
  static constexpr int kClasses = 5;
  int device = 0;
  int E = 0, S = 0;
  size_t total = 0, total_act = 0;
  float dt = 0, drag = 0, gx = 0, gy = 0, c = 0, k = 0, vmax = 0, skin = 0;
  int cap[kClasses] = {8, 16, 32, 64, 128};
  int cls_begin[kClasses + 1] = {};  // sorted env ranges per class
  int lanes[kClasses] = {};          // chosen lanes per env
  int slots[kClasses] = {};          // chosen entities per lane
  int tile = 1;                      // steps per launch in rollouts
  float *planes = nullptr;           // 6 planes x total, sorted order
  float4 *param = nullptr;
  uint8_t *kind = nullptr;
  uint16_t *pairs[kClasses] = {};    // canonical pair table per class capacity
  int *soff = nullptr, *perm = nullptr, *aoff = nullptr;
  int *to_sorted = nullptr;          // caller entity index -> sorted entity index
  int *err = nullptr;
  float *stage = nullptr;            // [total][6]
  float *backup = nullptr;           // autotuner's copy of the planes
  std::vector<int> h_aoff;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const float *graph_actions = nullptr;
  int graph_T = -1, graph_version = -1;
  int version = 0;                   // bumps whenever the tuning changes
};

namespace {

void free_ragged(vmas_ragged *r) {
  if (!r) return;
  if (r->gexec) cudaGraphExecDestroy(r->gexec);
  if (r->graph) cudaGraphDestroy(r->graph);
  cudaFree(r->planes);
  cudaFree(r->param);
  cudaFree(r->kind);
  for (auto *q : r->pairs) cudaFree(q);
  cudaFree(r->soff);
  cudaFree(r->perm);
  cudaFree(r->aoff);
  cudaFree(r->to_sorted);
  cudaFree(r->err);
  cudaFree(r->stage);
  cudaFree(r->backup);
  delete r;
}

StepParams ragged_params(const vmas_ragged *r, int c) {
  StepParams p{};
  p.E = r->E;
  p.N = r->cap[c];
  p.P = r->cap[c] * (r->cap[c] - 1) / 2;
  p.A = 0;
  p.S = r->S;
  p.h = (float)((double)r->dt / (double)r->S);
  p.damp = (float)(1.0 - (double)r->drag);
  p.gx = r->gx;
  p.gy = r->gy;
  p.ck = (float)((double)r->c * (double)r->k);
  p.inv_k = (float)(1.0 / (double)r->k);
  p.vmax = r->vmax;
  p.skin = r->skin;
  const size_t T = r->total;
  p.px = r->planes;
  p.py = r->planes + T;
  p.vx = r->planes + 2 * T;
  p.vy = r->planes + 3 * T;
  p.th = r->planes + 4 * T;
  p.om = r->planes + 5 * T;
  p.param = r->param;
  p.kind = r->kind;
  p.pairs = r->pairs[c];
  p.err = r->err;
  p.tile = 1;
  p.act_step = r->total_act * 3;
  p.EN = T;
  p.soff = r->soff;
  p.perm = r->perm;
  p.aoff = r->aoff;
  p.env_begin = r->cls_begin[c];
  p.env_end = r->cls_begin[c + 1];
  return p;
}

// One tile of `tile` steps for every class, actions of the tile's first step
// at d_actions.
int ragged_launch_tile(vmas_ragged *r, const float *d_actions, int tile, cudaStream_t st) {
  for (int c = 0; c < vmas_ragged::kClasses; ++c) {
    const int n = r->cls_begin[c + 1] - r->cls_begin[c];
    if (n == 0) continue;
    StepParams p = ragged_params(r, c);
    p.actions = d_actions;
    p.tile = tile;
    const int rc = launch_ragged_class(p, r->lanes[c], r->slots[c], n, st);
    if (rc) return rc;
  }
  return VMAS_OK;
}

__global__ void ragged_gather_kernel(float *aos, const float *planes, const int *to_sorted,
                                     size_t total) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const size_t s = (size_t)to_sorted[t];
  for (int f = 0; f < 6; ++f) aos[t * 6 + f] = planes[f * total + s];
}

__global__ void ragged_scatter_kernel(float *planes, const float *aos, const int *to_sorted,
                                      size_t total) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const size_t s = (size_t)to_sorted[t];
  for (int f = 0; f < 6; ++f) planes[f * total + s] = aos[t * 6 + f];
}

}  // namespace

extern "C" {

int vmas_ragged_create(const vmas_ragged_desc *d, vmas_ragged **out) {
  if (!out) return fail(VMAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d || !d->env_offsets) return fail(VMAS_EINVAL, "desc or env_offsets is NULL");
  if (d->n_envs < 0 || d->substeps < 1) return fail(VMAS_EINVAL, "n_envs >= 0 and substeps >= 1");
  if (!(d->dt > 0) || !(d->contact_margin > 0) || !(d->contact_force >= 0) || !(d->max_speed >= 0))
    return fail(VMAS_EINVAL, "dt, contact_margin must be > 0; contact_force, max_speed >= 0");
  const int E = d->n_envs;
  if (d->env_offsets[0] != 0) return fail(VMAS_EINVAL, "env_offsets[0] must be 0");
  std::vector<int> cnt(E), cls(E);
  for (int e = 0; e < E; ++e) {
    cnt[e] = d->env_offsets[e + 1] - d->env_offsets[e];
    if (cnt[e] < 1 || cnt[e] > VMAS_MAX_ENTITIES)
      return fail(VMAS_EINVAL, "env " + std::to_string(e) + " has " + std::to_string(cnt[e]) +
                                   " entities (1.." + std::to_string(VMAS_MAX_ENTITIES) + " allowed)");
  }
  const size_t total = E ? (size_t)d->env_offsets[E] : 0;
  if (total && (!d->shape || !d->flags || !d->size_a || !d->size_b || !d->mass || !d->inertia ||
                !d->init_state))
    return fail(VMAS_EINVAL, "a per-entity array is NULL");
  vmas_ragged *r = new vmas_ragged();
  cudaGetDevice(&r->device);
  r->E = E;
  r->S = d->substeps;
  r->total = total;
  r->dt = d->dt;
  r->drag = d->drag;
  r->gx = d->gx;
  r->gy = d->gy;
  r->c = d->contact_force;
  r->k = d->contact_margin;
  r->vmax = d->max_speed;
  // classes, sorted order (stable by class)
  for (int e = 0; e < E; ++e) {
    int c = 0;
    while (r->cap[c] < cnt[e]) ++c;
    cls[e] = c;
  }
  std::vector<int> perm;
  for (int c = 0; c < vmas_ragged::kClasses; ++c) {
    r->cls_begin[c] = (int)perm.size();
    for (int e = 0; e < E; ++e)
      if (cls[e] == c) perm.push_back(e);
    // default: fewest lanes that keep 4 entities or fewer per lane
    r->lanes[c] = std::max(4, r->cap[c] / 4);
    r->slots[c] = r->cap[c] / r->lanes[c];
  }
  r->cls_begin[vmas_ragged::kClasses] = (int)perm.size();
  // packed parameters in sorted order; action offsets in caller order
  std::vector<int> soff(E + 1, 0), to_sorted(total);
  r->h_aoff.assign(E + 1, 0);
  std::vector<float4> param(total);
  std::vector<uint8_t> kind(total);
  std::vector<float> planes(total * 6);
  std::vector<float> bound;
  for (int e = 0; e < E; ++e) {
    int na = 0;
    for (int i = d->env_offsets[e]; i < d->env_offsets[e + 1]; ++i)
      if (d->flags[i] & VMAS_ACTUATED) ++na;
    r->h_aoff[e + 1] = r->h_aoff[e] + na;
  }
  r->total_act = (size_t)r->h_aoff[E];
  size_t pos = 0;
  for (int s = 0; s < E; ++s) {
    const int e = perm[s];
    soff[s] = (int)pos;
    for (int i = d->env_offsets[e]; i < d->env_offsets[e + 1]; ++i, ++pos) {
      const int sh = d->shape[i], fl = d->flags[i];
      const double a = d->size_a[i], b = d->size_b[i], m = d->mass[i];
      if (sh > 2 || (fl & ~15) || !(a > 0) || (sh == VMAS_BOX && !(b > 0)) ||
          ((fl & VMAS_MOVABLE) && !(m > 0))) {
        free_ragged(r);
        return fail(VMAS_EINVAL, "invalid entity " + std::to_string(i));
      }
      double I = d->inertia[i];
      if (I == 0)
        I = sh == VMAS_BOX ? m * (a * a + b * b) / 12.0 : (sh == VMAS_LINE ? m * a * a / 12.0 : 0.5 * m * a * a);
      if ((fl & VMAS_ROTATABLE) && !(I > 0)) {
        free_ragged(r);
        return fail(VMAS_EINVAL, "rotatable entity needs inertia > 0 at " + std::to_string(i));
      }
      const double ha = sh == VMAS_SPHERE ? a : 0.5 * a, hb = sh == VMAS_BOX ? 0.5 * b : 0.0;
      param[pos] = make_float4((fl & VMAS_MOVABLE) ? (float)(1.0 / m) : 0.f,
                               (fl & VMAS_ROTATABLE) ? (float)(1.0 / I) : 0.f, (float)ha, (float)hb);
      kind[pos] = (uint8_t)(sh | (fl << 2));
      to_sorted[i] = (int)pos;
      for (int f = 0; f < 6; ++f) planes[f * total + pos] = d->init_state[(size_t)i * 6 + f];
      if (fl & VMAS_MOVABLE) bound.push_back((float)std::sqrt(ha * ha + hb * hb));
    }
  }
  soff[E] = (int)pos;
  float med = 0.05f;
  if (!bound.empty()) {
    std::nth_element(bound.begin(), bound.begin() + bound.size() / 2, bound.end());
    med = bound[bound.size() / 2];
  }
  r->skin = 0.5f * med;
  auto up = [&](void **dst, const void *src, size_t bytes) -> bool {
    if (cudaMalloc(dst, bytes ? bytes : 16) != cudaSuccess) return false;
    return !bytes || cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  bool ok = up((void **)&r->planes, planes.data(), planes.size() * sizeof(float)) &&
            up((void **)&r->param, param.data(), param.size() * sizeof(float4)) &&
            up((void **)&r->kind, kind.data(), kind.size()) &&
            up((void **)&r->soff, soff.data(), soff.size() * sizeof(int)) &&
            up((void **)&r->perm, perm.data(), perm.size() * sizeof(int)) &&
            up((void **)&r->aoff, r->h_aoff.data(), r->h_aoff.size() * sizeof(int)) &&
            up((void **)&r->to_sorted, to_sorted.data(), to_sorted.size() * sizeof(int)) &&
            cudaMalloc((void **)&r->err, 4 * sizeof(int)) == cudaSuccess &&
            cudaMemset(r->err, 0, 4 * sizeof(int)) == cudaSuccess;
  for (int c = 0; c < vmas_ragged::kClasses && ok; ++c) {
    std::vector<uint16_t> pt;
    for (int i = 0; i < r->cap[c]; ++i)
      for (int j = i + 1; j < r->cap[c]; ++j) pt.push_back((uint16_t)(i | (j << 8)));
    ok = up((void **)&r->pairs[c], pt.data(), pt.size() * sizeof(uint16_t));
  }
  if (!ok) {
    cudaGetLastError();
    free_ragged(r);
    return fail(VMAS_ENOMEM, "allocation or upload failed while creating the ragged world");
  }
  *out = r;
  return VMAS_OK;
}

int vmas_ragged_destroy(vmas_ragged *r) {
  if (!r) return VMAS_OK;
  cudaDeviceSynchronize();
  free_ragged(r);
  return VMAS_OK;
}

int vmas_ragged_info(const vmas_ragged *r, int32_t *n_envs, int64_t *n_entities,
                     int64_t *n_action_rows, int32_t *class_envs) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (n_envs) *n_envs = r->E;
  if (n_entities) *n_entities = (int64_t)r->total;
  if (n_action_rows) *n_action_rows = (int64_t)r->total_act;
  if (class_envs)
    for (int c = 0; c < vmas_ragged::kClasses; ++c) class_envs[c] = r->cls_begin[c + 1] - r->cls_begin[c];
  return VMAS_OK;
}

int vmas_ragged_action_offsets(const vmas_ragged *r, int32_t *out) {
  if (!r || !out) return fail(VMAS_EINVAL, "NULL argument");
  std::memcpy(out, r->h_aoff.data(), r->h_aoff.size() * sizeof(int32_t));
  return VMAS_OK;
}

int vmas_ragged_step(vmas_ragged *r, const float *d_actions, void *stream) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (r->total_act && !d_actions) return fail(VMAS_EINVAL, "d_actions is NULL");
  return ragged_launch_tile(r, d_actions, 1, as_stream(stream));
}

int vmas_ragged_rollout(vmas_ragged *r, const float *d_actions, int32_t n_steps, void *stream) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (n_steps < 0) return fail(VMAS_EINVAL, "n_steps < 0");
  if (n_steps == 0 || r->E == 0) return VMAS_OK;
  if (r->total_act && !d_actions) return fail(VMAS_EINVAL, "d_actions is NULL");
  cudaStream_t st = as_stream(stream);
  if (!(r->gexec && r->graph_actions == d_actions && r->graph_T == n_steps &&
        r->graph_version == r->version)) {
    if (r->gexec) cudaGraphExecDestroy(r->gexec);
    if (r->graph) cudaGraphDestroy(r->graph);
    r->gexec = nullptr;
    r->graph = nullptr;
    // The size classes touch disjoint envs, so each class's chain of tiles
    // is its own branch of the graph (forked from and joined back into the
    // capture stream): a class with few, slow envs no longer holds the GPU
    // while the others wait.
    constexpr int C = vmas_ragged::kClasses;
    cudaStream_t cap = nullptr, cs[C] = {};
    cudaEvent_t fork = nullptr, join[C] = {};
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    for (int c = 0; c < C && e == cudaSuccess; ++c) {
      e = cudaStreamCreateWithFlags(&cs[c], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    int rc = VMAS_OK;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = cudaEventRecord(fork, cap);
      for (int c = 0; c < C && e == cudaSuccess; ++c) {
        const int n = r->cls_begin[c + 1] - r->cls_begin[c];
        e = cudaStreamWaitEvent(cs[c], fork, 0);
        for (int t = 0; n > 0 && t < n_steps && rc == VMAS_OK && e == cudaSuccess; t += r->tile) {
          StepParams p = ragged_params(r, c);
          p.actions = d_actions + (size_t)t * r->total_act * 3;
          p.tile = std::min(r->tile, n_steps - t);
          rc = launch_ragged_class(p, r->lanes[c], r->slots[c], n, cs[c]);
        }
        if (e == cudaSuccess) e = cudaEventRecord(join[c], cs[c]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, join[c], 0);
      }
      cudaError_t e2 = cudaStreamEndCapture(cap, &r->graph);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && rc == VMAS_OK) e = cudaGraphInstantiate(&r->gexec, r->graph, 0);
    for (int c = 0; c < C; ++c) {
      if (join[c]) cudaEventDestroy(join[c]);
      if (cs[c]) cudaStreamDestroy(cs[c]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    if (rc) {
      cudaGetLastError();
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "rollout graph capture");
    r->graph_actions = d_actions;
    r->graph_T = n_steps;
    r->graph_version = r->version;
  }
  VMAS_CUDA(cudaGraphLaunch(r->gexec, st));
  return VMAS_OK;
}

int vmas_ragged_state(vmas_ragged *r, float *out, int32_t out_is_device, void *stream) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (!r->total) return VMAS_OK;
  if (!out) return fail(VMAS_EINVAL, "out is NULL");
  cudaStream_t st = as_stream(stream);
  float *dst = out;
  if (!out_is_device) {
    if (!r->stage) VMAS_CUDA(cudaMalloc(&r->stage, r->total * 6 * sizeof(float)));
    dst = r->stage;
  }
  ragged_gather_kernel<<<(unsigned)((r->total + 255) / 256), 256, 0, st>>>(dst, r->planes,
                                                                          r->to_sorted, r->total);
  VMAS_CUDA(cudaGetLastError());
  if (!out_is_device) {
    VMAS_CUDA(cudaMemcpyAsync(out, r->stage, r->total * 6 * sizeof(float), cudaMemcpyDeviceToHost, st));
    int h = 0;
    VMAS_CUDA(cudaMemcpyAsync(&h, r->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VMAS_CUDA(cudaStreamSynchronize(st));
    if (h) {
      cudaMemset(r->err, 0, sizeof(int));
      return fail(VMAS_EDEVICE, "device error word set (bits " + std::to_string(h) + ")");
    }
  }
  return VMAS_OK;
}

int vmas_ragged_set_state(vmas_ragged *r, const float *d_state, void *stream) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (!r->total) return VMAS_OK;
  if (!d_state) return fail(VMAS_EINVAL, "d_state is NULL");
  ragged_scatter_kernel<<<(unsigned)((r->total + 255) / 256), 256, 0, as_stream(stream)>>>(
      r->planes, d_state, r->to_sorted, r->total);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

int vmas_ragged_set_tuning(vmas_ragged *r, const int32_t *lanes, int32_t steps_per_launch) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (steps_per_launch < 1 || steps_per_launch > 1024)
    return fail(VMAS_EINVAL, "steps_per_launch must be 1..1024");
  if (lanes) {
    for (int c = 0; c < vmas_ragged::kClasses; ++c) {
      const int g = lanes[c], sl = r->cap[c] / g;
      const bool ok = (g == 4 || g == 8 || g == 16 || g == 32) && g * sl == r->cap[c] && sl >= 1 &&
                      sl <= 4 && sl != 3;
      if (!ok) return fail(VMAS_EINVAL, "lanes for class " + std::to_string(c) + " invalid");
    }
    for (int c = 0; c < vmas_ragged::kClasses; ++c) {
      r->lanes[c] = lanes[c];
      r->slots[c] = r->cap[c] / lanes[c];
    }
  }
  r->tile = steps_per_launch;
  ++r->version;
  return VMAS_OK;
}

int vmas_ragged_get_tuning(const vmas_ragged *r, int32_t *lanes, int32_t *steps_per_launch) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (lanes)
    for (int c = 0; c < vmas_ragged::kClasses; ++c) lanes[c] = r->lanes[c];
  if (steps_per_launch) *steps_per_launch = r->tile;
  return VMAS_OK;
}

int vmas_ragged_autotune(vmas_ragged *r, const float *d_actions, int32_t n_steps, void *stream) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (n_steps < 1) return fail(VMAS_EINVAL, "n_steps must be >= 1");
  if (r->total_act && !d_actions) return fail(VMAS_EINVAL, "d_actions is NULL");
  cudaStream_t st = as_stream(stream);
  const size_t bytes = r->total * 6 * sizeof(float);
  if (!r->backup) VMAS_CUDA(cudaMalloc(&r->backup, bytes ? bytes : 16));
  VMAS_CUDA(cudaMemcpyAsync(r->backup, r->planes, bytes, cudaMemcpyDeviceToDevice, st));
  cudaEvent_t a, b;
  VMAS_CUDA(cudaEventCreate(&a));
  VMAS_CUDA(cudaEventCreate(&b));
  const int tiles[] = {1, 2, 4, 8, 16};
  int rc = VMAS_OK;
  for (int c = 0; c < vmas_ragged::kClasses && rc == VMAS_OK; ++c) {
    const int n = r->cls_begin[c + 1] - r->cls_begin[c];
    if (n == 0) continue;
    float best = 3.4e38f;
    int best_g = r->lanes[c];
    for (int g = 4; g <= 32 && rc == VMAS_OK; g *= 2) {
      const int sl = r->cap[c] / g;
      if (sl < 1 || sl > 4 || sl == 3 || g * sl != r->cap[c]) continue;
      StepParams p = ragged_params(r, c);
      float ms = 0;
      for (int rep = 0; rep < 2 && rc == VMAS_OK; ++rep) {  // first pass warms up
        cudaEventRecord(a, st);
        for (int t = 0; t < n_steps && rc == VMAS_OK; ++t) {
          p.actions = d_actions + (size_t)t * r->total_act * 3;
          rc = launch_ragged_class(p, g, sl, n, st);
        }
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
      }
      if (ms < best) { best = ms; best_g = g; }
    }
    r->lanes[c] = best_g;
    r->slots[c] = r->cap[c] / best_g;
  }
  // steps per launch, all classes together
  float best = 3.4e38f;
  int best_tile = 1;
  for (int ti = 0; ti < 5 && rc == VMAS_OK; ++ti) {
    const int tile = tiles[ti];
    if (tile > n_steps) break;
    float ms = 0;
    for (int rep = 0; rep < 2 && rc == VMAS_OK; ++rep) {
      cudaEventRecord(a, st);
      for (int t = 0; t + tile <= n_steps && rc == VMAS_OK; t += tile)
        rc = ragged_launch_tile(r, d_actions + (size_t)t * r->total_act * 3, tile, st);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms, a, b);
    }
    const float per_step = ms / (float)((n_steps / tile) * tile);
    if (per_step < best) { best = per_step; best_tile = tile; }
  }
  r->tile = best_tile;
  ++r->version;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaError_t e = cudaMemcpyAsync(r->planes, r->backup, bytes, cudaMemcpyDeviceToDevice, st);
  if (rc == VMAS_OK && e != cudaSuccess) rc = cuda_fail(e, "restore after autotune");
  if (rc == VMAS_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "autotune");
  }
  return rc;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Learned surrogate (surrogate.cuh): a per-agent message-passing network
// that predicts a whole world step of the 16-agent walled sphere world, with
// the plain step as the fallback for envs whose prediction overlaps.

#include "surrogate_fused.cuh"

namespace {

using vmas::sur::bf16;
namespace sur = vmas::sur;

using namespace vmas::sur;  // parameter offsets kOff*
constexpr int kSurParams = vmas::sur::kParams;
constexpr int kSplitCap = 256;  // split-K / column-sum partial blocks

}  // namespace

struct vmas_surrogate {
  int device = 0;
  int cap = 0;  // envs
  int mode = VMAS_SUR_FUSED;
  int n_sm = 0;
  bool fused_ready = false;  // shared-memory opt-in of the fused kernel done
  int adam_t = 0;
  float *p32 = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  bf16 *pbf = nullptr;
  // forward
  bf16 *node = nullptr, *edge = nullptr, *he = nullptr, *zin = nullptr, *h1 = nullptr,
       *h2 = nullptr;
  float *mask = nullptr, *ze2 = nullptr, *out = nullptr;
  // training (allocated on first use)
  float *ze1 = nullptr, *z1 = nullptr, *z2 = nullptr;
  float *d_out = nullptr, *g128 = nullptr, *d_zin = nullptr, *ge = nullptr;
  bf16 *d_outbf = nullptr, *g128bf = nullptr, *gebf = nullptr;
  float *part = nullptr, *loss_part = nullptr, *save = nullptr, *target = nullptr;
  int *list = nullptr, *list_len = nullptr;
};

namespace {

void free_sur(vmas_surrogate *s) {
  if (!s) return;
  void *ptrs[] = {s->p32,   s->grad,  s->adam_m, s->adam_v, s->pbf,    s->node,   s->edge,
                  s->he,    s->zin,   s->h1,     s->h2,     s->mask,   s->ze2,    s->out,
                  s->ze1,   s->z1,    s->z2,     s->d_out,  s->g128,   s->d_zin,  s->ge,
                  s->d_outbf, s->g128bf, s->gebf, s->part,  s->loss_part, s->save, s->target,
                  s->list,  s->list_len};
  for (void *q : ptrs) cudaFree(q);
  delete s;
}

template <typename T>
bool dalloc(T **ptr, size_t count) {
  return cudaMalloc((void **)ptr, (count > 0 ? count : 1) * sizeof(T)) == cudaSuccess;
}

int ensure_training(vmas_surrogate *s) {
  if (s->ze1) return VMAS_OK;
  const size_t R = (size_t)s->cap * sur::kAgents, RK = R * sur::kK;
  const bool ok = dalloc(&s->ze1, RK * 64) && dalloc(&s->z1, R * 128) && dalloc(&s->z2, R * 128) &&
                  dalloc(&s->d_out, R * 8) && dalloc(&s->d_outbf, R * 8) &&
                  dalloc(&s->g128, R * 128) && dalloc(&s->g128bf, R * 128) &&
                  dalloc(&s->d_zin, R * 80) && dalloc(&s->ge, RK * 64) &&
                  dalloc(&s->gebf, RK * 64) && dalloc(&s->save, R * 4) &&
                  dalloc(&s->target, R * 4);
  if (!ok) {
    cudaGetLastError();
    return fail(VMAS_ENOMEM, "cudaMalloc failed for the surrogate's training buffers");
  }
  return VMAS_OK;
}

unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// C = A B (+ bias, GELU) through gemm_bf16_kernel; `splits` > 1 sums K in
// chunks into part, reduced into out_f32 (then no bias / bf16 output).
int gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, const bf16 *A, int lda,
         const bf16 *B, int ldb, const float *bias, int act, float *out_f32, int ldc_f,
         bf16 *out_bf, int ldc_b, float *part = nullptr, int splits = 1) {
  if (M == 0 || N == 0) return VMAS_OK;
  sur::GemmArgs g{};
  g.M = M; g.N = N; g.K = K; g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
  g.bias = bias; g.act = act;
  g.ldc_f = ldc_f; g.out_bf = out_bf; g.ldc_b = ldc_b;
  if (splits > 1 && K > 0) {
    int chunk = (K + splits - 1) / splits;
    chunk = (chunk + sur::kBK - 1) / sur::kBK * sur::kBK;
    splits = (K + chunk - 1) / chunk;
    g.kchunk = chunk;
    g.out_f32 = part;
    g.ldc_f = N;
  } else {
    splits = 1;
    g.kchunk = K > 0 ? K : 1;
    g.out_f32 = out_f32;
  }
  const dim3 grid(blocks_for((size_t)M, sur::kBM), blocks_for((size_t)N, sur::kBN), splits);
  if (!ta && !tb) sur::gemm_bf16_kernel<false, false><<<grid, 128, 0, st>>>(g);
  else if (!ta && tb) sur::gemm_bf16_kernel<false, true><<<grid, 128, 0, st>>>(g);
  else if (ta && !tb) sur::gemm_bf16_kernel<true, false><<<grid, 128, 0, st>>>(g);
  else sur::gemm_bf16_kernel<true, true><<<grid, 128, 0, st>>>(g);
  VMAS_CUDA(cudaGetLastError());
  if (g.out_f32 == part && part) {
    const size_t MN = (size_t)M * N;
    sur::sum_partials_kernel<<<blocks_for(MN, 256), 256, 0, st>>>(out_f32, part, splits, MN);
    VMAS_CUDA(cudaGetLastError());
  }
  return VMAS_OK;
}

// Column sums of x [M][N] (N <= 128) into out [N]: up to 4,096 row chunks
// summed in parallel, then the chunk sums per column (two stages).
int col_sum(cudaStream_t st, float *out, const float *x, int M, int N, float *part) {
  const int chunks = std::max(1, std::min(4096, (M + 255) / 256));
  const int chunk = (M + chunks - 1) / chunks;
  sur::col_sum_kernel<<<chunks, 128, 0, st>>>(part, x, M, N, chunk > 0 ? chunk : 1);
  VMAS_CUDA(cudaGetLastError());
  // second stage: 64 groups of chunks, then the groups
  const int groups = std::min(64, chunks), per = (chunks + groups - 1) / groups;
  float *part2 = part + (size_t)chunks * N;
  sur::col_sum_kernel<<<groups, 128, 0, st>>>(part2, part, chunks, N, per);
  VMAS_CUDA(cudaGetLastError());
  sur::sum_partials_kernel<<<1, 128, 0, st>>>(out, part2, groups, (size_t)N);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

int sur_check(vmas_surrogate *s, vmas_world *w, const float *d_actions) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (!w->sur_ok)
    return fail(VMAS_EINVAL, "world layout is not 16 actuated agent spheres then 4 fixed lines");
  if (w->E > s->cap)
    return fail(VMAS_EINVAL, "world has " + std::to_string(w->E) + " envs, surrogate capacity " +
                                 std::to_string(s->cap));
  if (w->E > 0 && !d_actions) return fail(VMAS_EINVAL, "d_actions is NULL");
  return VMAS_OK;
}

// Features of the world's current state, then the network; train = true also
// keeps the FP32 pre-activations the backward needs.
int sur_forward(vmas_surrogate *s, vmas_world *w, const float *d_actions, bool train,
                cudaStream_t st) {
  const int E = w->E;
  const int R = E * sur::kAgents, RK = R * sur::kK;
  if (E == 0) return VMAS_OK;
  sur::FeatureArgs f{};
  const size_t EN = (size_t)E * w->N;
  f.E = E; f.N = w->N; f.A = w->A;
  f.px = w->planes; f.py = w->planes + EN; f.vx = w->planes + 2 * EN; f.vy = w->planes + 3 * EN;
  f.param = w->param; f.actions = d_actions;
  f.node = s->node; f.edge = s->edge; f.mask = s->mask;
  sur::features_kernel<<<blocks_for(R, 128), 128, 0, st>>>(f);
  VMAS_CUDA(cudaGetLastError());
  const bf16 *W = s->pbf;
  const float *P = s->p32;
  int rc;
  // edge MLP
  if ((rc = gemm(st, false, true, RK, 64, 16, s->edge, 16, W + kOffWe1, 16, P + kOffbe1, 1,
                 train ? s->ze1 : nullptr, 64, s->he, 64)))
    return rc;
  if ((rc = gemm(st, false, true, RK, 64, 64, s->he, 64, W + kOffWe2, 64, P + kOffbe2, 0, s->ze2,
                 64, nullptr, 0)))
    return rc;
  sur::aggregate_kernel<<<blocks_for((size_t)R * 80, 256), 256, 0, st>>>(R, s->ze2, s->mask,
                                                                          s->node, s->zin);
  VMAS_CUDA(cudaGetLastError());
  // node MLP
  if ((rc = gemm(st, false, true, R, 128, 80, s->zin, 80, W + kOffW1, 80, P + kOffb1, 1,
                 train ? s->z1 : nullptr, 128, s->h1, 128)))
    return rc;
  if ((rc = gemm(st, false, true, R, 128, 128, s->h1, 128, W + kOffW2, 128, P + kOffb2, 1,
                 train ? s->z2 : nullptr, 128, s->h2, 128)))
    return rc;
  return gemm(st, false, true, R, 8, 128, s->h2, 128, W + kOffW3, 128, P + kOffb3, 0, s->out, 8,
              nullptr, 0);
}

// Loss against target [R][4] and the gradient into s->grad (after sur_forward
// with train = true).
int sur_backward(vmas_surrogate *s, int E, const float *target, float *d_loss, cudaStream_t st) {
  const int R = E * sur::kAgents, RK = R * sur::kK;
  float *G = s->grad;
  const bf16 *W = s->pbf;
  VMAS_CUDA(cudaMemsetAsync(G, 0, kSurParams * sizeof(float), st));
  if (E == 0) {
    if (d_loss) VMAS_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), st));
    return VMAS_OK;
  }
  const int lb = (int)blocks_for((size_t)R * 8, 256);
  sur::loss_kernel<<<lb, 256, 0, st>>>(R, s->out, target, s->d_out, s->d_outbf, s->loss_part);
  VMAS_CUDA(cudaGetLastError());
  if (d_loss) {
    sur::finish_loss_kernel<<<1, 256, 0, st>>>(s->loss_part, lb, R, d_loss);
    VMAS_CUDA(cudaGetLastError());
  }
  int rc;
  const int sp = kSplitCap;
  // output layer
  if ((rc = gemm(st, true, false, 8, 128, R, s->d_outbf, 8, s->h2, 128, nullptr, 0, G + kOffW3,
                 128, nullptr, 0, s->part, sp)))
    return rc;
  if ((rc = col_sum(st, G + kOffb3, s->d_out, R, 8, s->part))) return rc;
  if ((rc = gemm(st, false, false, R, 128, 8, s->d_outbf, 8, W + kOffW3, 128, nullptr, 0, s->g128,
                 128, nullptr, 0)))
    return rc;
  // node layer 2
  sur::gelu_back_kernel<<<blocks_for((size_t)R * 128, 256), 256, 0, st>>>((size_t)R * 128, s->g128,
                                                                           s->z2, s->g128, s->g128bf);
  VMAS_CUDA(cudaGetLastError());
  if ((rc = gemm(st, true, false, 128, 128, R, s->g128bf, 128, s->h1, 128, nullptr, 0, G + kOffW2,
                 128, nullptr, 0, s->part, sp)))
    return rc;
  if ((rc = col_sum(st, G + kOffb2, s->g128, R, 128, s->part))) return rc;
  if ((rc = gemm(st, false, false, R, 128, 128, s->g128bf, 128, W + kOffW2, 128, nullptr, 0,
                 s->g128, 128, nullptr, 0)))
    return rc;
  // node layer 1
  sur::gelu_back_kernel<<<blocks_for((size_t)R * 128, 256), 256, 0, st>>>((size_t)R * 128, s->g128,
                                                                           s->z1, s->g128, s->g128bf);
  VMAS_CUDA(cudaGetLastError());
  if ((rc = gemm(st, true, false, 128, 80, R, s->g128bf, 128, s->zin, 80, nullptr, 0, G + kOffW1, 80,
                 nullptr, 0, s->part, sp)))
    return rc;
  if ((rc = col_sum(st, G + kOffb1, s->g128, R, 128, s->part))) return rc;
  if ((rc = gemm(st, false, false, R, 80, 128, s->g128bf, 128, W + kOffW1, 80, nullptr, 0, s->d_zin,
                 80, nullptr, 0)))
    return rc;
  // edge layer 2 (through the masked sum)
  sur::edge_back_kernel<<<blocks_for((size_t)RK * 64, 256), 256, 0, st>>>(R, s->d_zin, s->mask,
                                                                           s->ze2, s->ge, s->gebf);
  VMAS_CUDA(cudaGetLastError());
  if ((rc = gemm(st, true, false, 64, 64, RK, s->gebf, 64, s->he, 64, nullptr, 0, G + kOffWe2, 64,
                 nullptr, 0, s->part, sp)))
    return rc;
  if ((rc = col_sum(st, G + kOffbe2, s->ge, RK, 64, s->part))) return rc;
  if ((rc = gemm(st, false, false, RK, 64, 64, s->gebf, 64, W + kOffWe2, 64, nullptr, 0, s->ge, 64,
                 nullptr, 0)))
    return rc;
  // edge layer 1
  sur::gelu_back_kernel<<<blocks_for((size_t)RK * 64, 256), 256, 0, st>>>((size_t)RK * 64, s->ge,
                                                                          s->ze1, s->ge, s->gebf);
  VMAS_CUDA(cudaGetLastError());
  if ((rc = gemm(st, true, false, 64, 16, RK, s->gebf, 64, s->edge, 16, nullptr, 0, G + kOffWe1, 16,
                 nullptr, 0, s->part, sp)))
    return rc;
  return col_sum(st, G + kOffbe1, s->ge, RK, 64, s->part);
}

int sur_adam(vmas_surrogate *s, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  ++s->adam_t;
  const float c1 = (float)(1.0 - std::pow((double)b1, s->adam_t));
  const float c2 = (float)(1.0 - std::pow((double)b2, s->adam_t));
  sur::adam_kernel<<<blocks_for(kSurParams, 256), 256, 0, st>>>(
      kSurParams, s->p32, s->grad, s->adam_m, s->adam_v, s->pbf, lr, b1, b2, eps, c1, c2);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

// The fused inference kernel over the world's envs: network output into
// out (may be NULL); apply = true also applies the prediction and lists the
// fallback envs.
int sur_fused(vmas_surrogate *s, vmas_world *w, const float *d_actions, float *out, bool apply,
              float limit, cudaStream_t st) {
  const int E = w->E;
  if (E == 0) return VMAS_OK;
  const size_t smem = sur::fused_smem_bytes();
  if (!s->fused_ready) {  // > 48 KB of dynamic shared memory needs an opt-in
    VMAS_CUDA(cudaFuncSetAttribute(sur::sur_fused_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    s->fused_ready = true;
  }
  sur::FusedArgs a{};
  const size_t EN = (size_t)E * w->N;
  a.E = E; a.N = w->N; a.A = w->A;
  a.px = w->planes; a.py = w->planes + EN; a.vx = w->planes + 2 * EN; a.vy = w->planes + 3 * EN;
  a.param = w->param; a.actions = d_actions;
  a.w = s->pbf; a.p = s->p32;
  a.out = out; a.apply = apply ? 1 : 0; a.limit = limit;
  a.list = s->list; a.list_len = s->list_len;
  const int need = (E + sur::kFusedWarpsPerCta - 1) / sur::kFusedWarpsPerCta;
  const int grid = std::max(1, std::min(need, s->n_sm));
  sur::sur_fused_kernel<<<grid, sur::kFusedWarpsPerCta * 32, smem, st>>>(a);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

__global__ void f32_to_bf16_kernel(const float *x, bf16 *y, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = __float2bfloat16_rn(x[t]);
}

}  // namespace

extern "C" {

int vmas_sur_param_count(void) { return kSurParams; }

int vmas_sur_create(int32_t max_envs, vmas_surrogate **out) {
  if (!out) return fail(VMAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_envs < 0 || max_envs > (1 << 22))
    return fail(VMAS_EINVAL, "max_envs must be 0.." + std::to_string(1 << 22));
  vmas_surrogate *s = new vmas_surrogate();
  cudaGetDevice(&s->device);
  if (cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
      s->n_sm < 1) {
    cudaGetLastError();
    s->n_sm = 1;
  }
  s->cap = max_envs;
  const size_t R = (size_t)max_envs * sur::kAgents, RK = R * sur::kK;
  const bool ok =
      dalloc(&s->p32, kSurParams) && dalloc(&s->grad, kSurParams) && dalloc(&s->adam_m, kSurParams) &&
      dalloc(&s->adam_v, kSurParams) && dalloc(&s->pbf, kSurParams) && dalloc(&s->node, R * 16) &&
      dalloc(&s->edge, RK * 16) && dalloc(&s->he, RK * 64) && dalloc(&s->zin, R * 80) &&
      dalloc(&s->h1, R * 128) && dalloc(&s->h2, R * 128) && dalloc(&s->mask, RK) &&
      dalloc(&s->ze2, RK * 64) && dalloc(&s->out, R * 8) &&
      dalloc(&s->part, (size_t)kSplitCap * 128 * 128) && dalloc(&s->loss_part, R * 8 / 256 + 1) &&
      dalloc(&s->list, (size_t)max_envs) && dalloc(&s->list_len, 1);
  if (!ok) {
    cudaGetLastError();
    free_sur(s);
    return fail(VMAS_ENOMEM, "cudaMalloc failed while creating the surrogate");
  }
  cudaError_t e = cudaMemset(s->p32, 0, kSurParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->pbf, 0, kSurParams * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMemset(s->adam_m, 0, kSurParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->adam_v, 0, kSurParams * sizeof(float));
  if (e != cudaSuccess) {
    free_sur(s);
    return cuda_fail(e, "surrogate init");
  }
  *out = s;
  return VMAS_OK;
}

int vmas_sur_destroy(vmas_surrogate *s) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  free_sur(s);
  return VMAS_OK;
}

int vmas_sur_set_params(vmas_surrogate *s, const float *h_params) {
  if (!s || !h_params) return fail(VMAS_EINVAL, "surrogate or h_params is NULL");
  for (int q = 0; q < kSurParams; ++q)
    if (!std::isfinite(h_params[q])) return fail(VMAS_EINVAL, "a parameter is not finite");
  VMAS_CUDA(cudaMemcpy(s->p32, h_params, kSurParams * sizeof(float), cudaMemcpyHostToDevice));
  f32_to_bf16_kernel<<<blocks_for(kSurParams, 256), 256>>>(s->p32, s->pbf, kSurParams);
  VMAS_CUDA(cudaGetLastError());
  VMAS_CUDA(cudaMemset(s->adam_m, 0, kSurParams * sizeof(float)));
  VMAS_CUDA(cudaMemset(s->adam_v, 0, kSurParams * sizeof(float)));
  VMAS_CUDA(cudaDeviceSynchronize());
  s->adam_t = 0;
  return VMAS_OK;
}

int vmas_sur_get_params(vmas_surrogate *s, float *h_params) {
  if (!s || !h_params) return fail(VMAS_EINVAL, "surrogate or h_params is NULL");
  VMAS_CUDA(cudaDeviceSynchronize());
  VMAS_CUDA(cudaMemcpy(h_params, s->p32, kSurParams * sizeof(float), cudaMemcpyDeviceToHost));
  return VMAS_OK;
}

int vmas_sur_set_mode(vmas_surrogate *s, int32_t mode) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  if (mode != VMAS_SUR_FUSED && mode != VMAS_SUR_LAYERED) return fail(VMAS_EINVAL, "unknown mode");
  s->mode = mode;
  return VMAS_OK;
}

int vmas_sur_forward(vmas_surrogate *s, vmas_world *w, const float *d_actions, float *d_out,
                     void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  if (s->mode == VMAS_SUR_FUSED)
    return sur_fused(s, w, d_actions, d_out ? d_out : s->out, false, 0.f, st);
  if ((rc = sur_forward(s, w, d_actions, false, st))) return rc;
  if (d_out && w->E)
    VMAS_CUDA(cudaMemcpyAsync(d_out, s->out, (size_t)w->E * sur::kAgents * 8 * sizeof(float),
                              cudaMemcpyDeviceToDevice, st));
  return VMAS_OK;
}

int vmas_sur_loss_grad(vmas_surrogate *s, vmas_world *w, const float *d_actions,
                       const float *d_target, float *d_loss, float *d_grad, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  if (w->E > 0 && !d_target) return fail(VMAS_EINVAL, "d_target is NULL");
  if ((rc = ensure_training(s))) return rc;
  cudaStream_t st = as_stream(stream);
  if ((rc = sur_forward(s, w, d_actions, true, st))) return rc;
  if ((rc = sur_backward(s, w->E, d_target, d_loss, st))) return rc;
  if (d_grad)
    VMAS_CUDA(cudaMemcpyAsync(d_grad, s->grad, kSurParams * sizeof(float), cudaMemcpyDeviceToDevice,
                              st));
  return VMAS_OK;
}

int vmas_sur_adam(vmas_surrogate *s, float lr, const float *d_grad, void *stream) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  if (!(lr >= 0) || !std::isfinite(lr)) return fail(VMAS_EINVAL, "lr must be >= 0");
  cudaStream_t st = as_stream(stream);
  if (d_grad && d_grad != s->grad)
    VMAS_CUDA(cudaMemcpyAsync(s->grad, d_grad, kSurParams * sizeof(float), cudaMemcpyDeviceToDevice,
                              st));
  return sur_adam(s, lr, st);
}

// Forward on the world's current state, the plain step (the world advances)
// as the target, loss and gradient into s->grad.
static int sur_train_grad(vmas_surrogate *s, vmas_world *w, const float *d_actions,
                          float *d_loss, cudaStream_t st) {
  int rc = ensure_training(s);
  if (rc) return rc;
  const int E = w->E, R = E * sur::kAgents;
  if (E == 0) {
    VMAS_CUDA(cudaMemsetAsync(s->grad, 0, kSurParams * sizeof(float), st));
    if (d_loss) VMAS_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), st));
    return VMAS_OK;
  }
  const size_t EN = (size_t)E * w->N;
  float *px = w->planes, *py = px + EN, *vx = px + 2 * EN, *vy = px + 3 * EN;
  if ((rc = sur_forward(s, w, d_actions, true, st))) return rc;
  sur::save_agents_kernel<<<blocks_for(R, 256), 256, 0, st>>>(E, w->N, px, py, vx, vy, s->save);
  VMAS_CUDA(cudaGetLastError());
  StepParams p = make_params(w);
  p.actions = d_actions;
  if ((rc = launch_step(p, st))) return rc;
  sur::targets_kernel<<<blocks_for(R, 256), 256, 0, st>>>(E, w->N, px, py, vx, vy, s->save,
                                                           s->target);
  VMAS_CUDA(cudaGetLastError());
  return sur_backward(s, E, s->target, d_loss, st);
}

int vmas_sur_train_grad(vmas_surrogate *s, vmas_world *w, const float *d_actions, float *d_loss,
                        float *d_grad, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  if ((rc = sur_train_grad(s, w, d_actions, d_loss, st))) return rc;
  if (d_grad)
    VMAS_CUDA(cudaMemcpyAsync(d_grad, s->grad, kSurParams * sizeof(float), cudaMemcpyDeviceToDevice,
                              st));
  return VMAS_OK;
}

int vmas_sur_train_step(vmas_surrogate *s, vmas_world *w, const float *d_actions, float lr,
                        float *d_loss, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  if (!(lr >= 0) || !std::isfinite(lr)) return fail(VMAS_EINVAL, "lr must be >= 0");
  cudaStream_t st = as_stream(stream);
  if ((rc = sur_train_grad(s, w, d_actions, d_loss, st))) return rc;
  if (w->E == 0) return VMAS_OK;
  return sur_adam(s, lr, st);
}

int vmas_sur_step(vmas_surrogate *s, vmas_world *w, const float *d_actions, float limit,
                  int32_t *d_n_fallback, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  if (!(limit >= 0) || !std::isfinite(limit)) return fail(VMAS_EINVAL, "limit must be >= 0");
  cudaStream_t st = as_stream(stream);
  const int E = w->E;
  if (E == 0) {
    if (d_n_fallback) VMAS_CUDA(cudaMemsetAsync(d_n_fallback, 0, sizeof(int32_t), st));
    return VMAS_OK;
  }
  VMAS_CUDA(cudaMemsetAsync(s->list_len, 0, sizeof(int), st));
  if (s->mode == VMAS_SUR_FUSED) {
    if ((rc = sur_fused(s, w, d_actions, nullptr, true, limit, st))) return rc;
  } else {
    if ((rc = sur_forward(s, w, d_actions, false, st))) return rc;
    sur::PredictArgs a{};
    const size_t EN = (size_t)E * w->N;
    a.E = E; a.N = w->N;
    a.px = w->planes; a.py = w->planes + EN; a.vx = w->planes + 2 * EN; a.vy = w->planes + 3 * EN;
    a.param = w->param; a.out = s->out; a.limit = limit;
    a.list = s->list; a.list_len = s->list_len;
    sur::predict_kernel<<<blocks_for(E, 128), 128, 0, st>>>(a);
    VMAS_CUDA(cudaGetLastError());
  }
  // the plain step for the listed envs (grid sized for all; blocks past the
  // device-side count return at once)
  StepParams p = make_params(w);
  p.actions = d_actions;
  p.env_list = s->list;
  p.env_count = s->list_len;
  if ((rc = launch_step(p, st))) return rc;
  if (d_n_fallback)
    VMAS_CUDA(cudaMemcpyAsync(d_n_fallback, s->list_len, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return VMAS_OK;
}

int vmas_sur_debug_features(vmas_surrogate *s, vmas_world *w, const float *d_actions,
                            uint16_t *d_node, uint16_t *d_edge, float *d_mask, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  if ((rc = sur_forward(s, w, d_actions, false, st))) return rc;
  const size_t R = (size_t)w->E * sur::kAgents, RK = R * sur::kK;
  if (!R) return VMAS_OK;
  if (d_node) VMAS_CUDA(cudaMemcpyAsync(d_node, s->node, R * 16 * 2, cudaMemcpyDeviceToDevice, st));
  if (d_edge) VMAS_CUDA(cudaMemcpyAsync(d_edge, s->edge, RK * 16 * 2, cudaMemcpyDeviceToDevice, st));
  if (d_mask) VMAS_CUDA(cudaMemcpyAsync(d_mask, s->mask, RK * 4, cudaMemcpyDeviceToDevice, st));
  return VMAS_OK;
}

int vmas_debug_gemm_bf16(int32_t trans_a, int32_t trans_b, int32_t M, int32_t N, int32_t K,
                         const uint16_t *d_a, int32_t lda, const uint16_t *d_b, int32_t ldb,
                         const float *d_bias, int32_t gelu, float *d_out_f32, uint16_t *d_out_bf16,
                         int32_t splits, void *stream) {
  if (M < 0 || N < 0 || K < 0 || splits < 1 || splits > kSplitCap)
    return fail(VMAS_EINVAL, "bad GEMM sizes");
  if (splits > 1 && (d_bias || d_out_bf16 || gelu))
    return fail(VMAS_EINVAL, "split-K GEMMs take no bias, GELU or bfloat16 output");
  if ((size_t)M * N == 0) return VMAS_OK;
  if ((K > 0 && (!d_a || !d_b)) || (!d_out_f32 && !d_out_bf16))
    return fail(VMAS_EINVAL, "NULL buffer");
  if (lda < (trans_a ? M : K) || ldb < (trans_b ? K : N))
    return fail(VMAS_EINVAL, "leading dimension too small");
  cudaStream_t st = as_stream(stream);
  float *part = nullptr;
  if (splits > 1) VMAS_CUDA(cudaMalloc(&part, (size_t)splits * M * N * sizeof(float)));
  const int rc = gemm(st, trans_a, trans_b, M, N, K, reinterpret_cast<const bf16 *>(d_a), lda,
                      reinterpret_cast<const bf16 *>(d_b), ldb, d_bias, gelu ? 1 : 0, d_out_f32, N,
                      reinterpret_cast<bf16 *>(d_out_bf16), N, part, splits);
  if (part) {
    cudaStreamSynchronize(st);
    cudaFree(part);
  }
  return rc;
}

}  // extern "C"
