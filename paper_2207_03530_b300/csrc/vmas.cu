// Host side of the VMAS C ABI (include/vmas.h): world creation, device
// layout, launches and error handling.  The physics lives in step_fused.cuh,
// step.cuh and contact.cuh; the differentiable rollout in diff.cuh, LIDAR in
// lidar.cuh, the learned surrogate in surrogate.cuh (layered GEMM path,
// training) and surrogate_fused.cuh (fused inference).  This file: the world,
// the allocation-free step, the differentiable rollout and LIDAR.
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
//
// The packed ragged worlds live in ragged.cu, the surrogate's host side in
// surrogate_host.cu; host.h holds what the three share.
#include "diff.cuh"
#include "host.h"
#include "lidar.cuh"
#include "ragged_persistent.cuh"
#include "step_fused.cuh"

static_assert(vmas::kStatCount == VMAS_STATS_COUNT, "stats layout");

namespace vmas_host {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(VMAS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

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
  // the largest shared-memory carveout: measured 0.6 % faster per step at
  // 30,000 envs when other kernels (an L2 flush) run between the steps
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
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

template <int MINB>
int launch_ragged_persistent_b(vmas::RaggedQueueParams q, cudaStream_t st) {
  q.slab = vmas::persist_slab_bytes();
  const int smem = vmas::kFusedWarps * q.slab;
  // resident CTAs per SM and SM count, found once per process (thread-safe
  // initialisation; the process is assumed to use one GPU model)
  struct Occ { cudaError_t err; int resident, sms; };
  static const Occ occ = [smem]() {
    Occ o{cudaSuccess, 1, 1};
    int dev = 0;
    if (smem > 48 * 1024)
      o.err = cudaFuncSetAttribute(vmas::ragged_persistent_kernel<MINB>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (o.err == cudaSuccess) o.err = cudaGetDevice(&dev);
    if (o.err == cudaSuccess) o.err = cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
    if (o.err == cudaSuccess)
      o.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &o.resident, vmas::ragged_persistent_kernel<MINB>, vmas::kFusedWarps * 32, smem);
    if (o.resident < 1) o.resident = 1;
    return o;
  }();
  if (occ.err != cudaSuccess) return cuda_fail(occ.err, "ragged_persistent_kernel set-up");
  // one wave of resident CTAs, fewer when there are fewer items than warps
  const int need = (q.n_items + vmas::kFusedWarps - 1) / vmas::kFusedWarps;
  const int grid = std::min(need, occ.sms * occ.resident);
  vmas::ragged_persistent_kernel<MINB><<<grid, vmas::kFusedWarps * 32, smem, st>>>(q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ragged_persistent_kernel launch");
  return VMAS_OK;
}

int launch_ragged_persistent(vmas::RaggedQueueParams q, int budget, cudaStream_t st) {
  if (q.n_items <= 0) return VMAS_OK;
  return budget == 2 ? launch_ragged_persistent_b<5>(q, st) : launch_ragged_persistent_b<4>(q, st);
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

int launch_step(const StepParams &p0, cudaStream_t st, bool tiled) {
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
  int h[3] = {0, 0, 0};  // bits; bounds-checked builds: site << 20 | index, bound
  VMAS_CUDA(cudaMemcpyAsync(h, w->err, sizeof(h), cudaMemcpyDeviceToHost, st));
  VMAS_CUDA(cudaStreamSynchronize(st));
  if (bits) *bits = h[0];
  if (h[0]) {
    VMAS_CUDA(cudaMemsetAsync(w->err, 0, sizeof(h), st));
    VMAS_CUDA(cudaStreamSynchronize(st));
    std::string msg = "device error word set (bits " + std::to_string(h[0]) + ")";
    if (h[0] & VMAS_DEVERR_INDEX)
      msg += "; first index out of range: site " + std::to_string(h[1] >> 20) + ", index " +
             std::to_string(h[1] & 0xfffff) + ", bound " + std::to_string(h[2]);
    return fail(VMAS_EDEVICE, msg);
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
#ifdef VMAS_CHECKED
__global__ void or_status_kernel(int *dst, const int *src) { atomicOr(dst, src[0]); }
#endif

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

}  // namespace vmas_host

using namespace vmas_host;

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
  if (!std::isfinite(a->drag) || !std::isfinite(a->gx) || !std::isfinite(a->gy) ||
      !std::isfinite(a->contact_margin) || !std::isfinite(a->contact_force) ||
      !std::isfinite(a->max_speed))
    return fail(VMAS_EINVAL, "drag, gravity and the contact and speed parameters must be finite");
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
  // the status words must start each call at zero; the pair table is rewritten
  VMAS_CUDA(cudaMemsetAsync(status, 0, 3 * sizeof(int), st));
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
#ifdef VMAS_CHECKED
  // a bounds-checked kernel also writes the two words after the bits, so it
  // gets the library's own three; their bits are ORed into the caller's word
  p.err = status;
#else
  p.err = a->status ? a->status : status;
#endif
  p.aos_state = a->state;
  p.r_shape = a->shape;
  p.r_flags = a->flags;
  p.r_size_a = a->size_a;
  p.r_size_b = a->size_b;
  p.r_mass = a->mass;
  p.r_inertia = a->inertia;
  switch (group_lanes(N)) {
    case 4: rc = launch_raw_g<4>(p, st); break;
    case 8: rc = launch_raw_g<8>(p, st); break;
    case 16: rc = launch_raw_g<16>(p, st); break;
    default: rc = launch_raw_g<32>(p, st); break;
  }
#ifdef VMAS_CHECKED
  if (rc == VMAS_OK && a->status) {
    or_status_kernel<<<1, 1, 0, st>>>(a->status, status);
    VMAS_CUDA(cudaGetLastError());
  }
#endif
  return rc;
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
    // the box world (the paper-scale layout): 16 such agents (rows 0..15),
    // 4 movable, rotatable, actuated boxes (rows 16..19), 4 fixed lines
    bool ok2 = N == 24 && w->A >= 20;
    for (int e = 0; e < E && ok2; ++e)
      for (int i = 0; i < N && ok2; ++i) {
        const size_t t = (size_t)e * N + i;
        const int fl = d->flags[t];
        if (i < 16)
          ok2 = d->shape[t] == VMAS_SPHERE && (fl & VMAS_MOVABLE) && (fl & VMAS_ACTUATED) &&
                !(fl & VMAS_ROTATABLE);
        else if (i < 20)
          ok2 = d->shape[t] == VMAS_BOX && (fl & VMAS_MOVABLE) && (fl & VMAS_ROTATABLE) &&
                (fl & VMAS_ACTUATED);
        else
          ok2 = d->shape[t] == VMAS_LINE && !(fl & (VMAS_MOVABLE | VMAS_ACTUATED));
      }
    w->sur_layout = ok ? 1 : (ok2 ? 2 : 0);
    w->sur_ok = w->sur_layout != 0;
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


// Lanes per env of the differentiable rollout kernels: the smallest power
// of two that holds the env's entities.
static int diff_group_lanes(int N) { return N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32; }

// Half-groups per env in the differentiable rollout: 1 by default; 2 (each
// env's pair loops split over two half-groups of lanes, where two groups fit
// a warp) when vmas_debug_diff_split chose it.  Process-wide.  The split
// fills more warps but not more envs, and costs the second half-group's copy
// of the integration: measured 546 against 507 us for the 4,096-env
// backward, so it stays off.
static int g_diff_split = 0;  // 0: automatic (1)
static int diff_split(int G) {
  if (G >= 32) return 1;
  return g_diff_split ? g_diff_split : 1;
}

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
  // candidate masks of the pair sums: 4 x the step's list margin (the mask
  // build is a pass over all N partners, cheaper than the step's list build,
  // so a wider margin with fewer rebuilds pays; 2 x to 8 x measured within
  // 1 % of each other on 4,096 envs of 8 agents + 2 landmarks, 1 x 16 %
  // slower)
  p->skin = 4.f * w->skin;
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
  const int G = diff_group_lanes(w->N), spl = diff_split(G);
  const int per_cta = vmas::kDiffWarps * (32 / (G * spl));
  const int grid = (w->E + per_cta - 1) / per_cta;
  cudaStream_t st = as_stream(stream);
  switch (G * 4 + spl) {
    case 4 * 4 + 1: vmas::diff_forward_kernel<4, 1><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    case 4 * 4 + 2: vmas::diff_forward_kernel<4, 2><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    case 8 * 4 + 1: vmas::diff_forward_kernel<8, 1><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    case 8 * 4 + 2: vmas::diff_forward_kernel<8, 2><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    case 16 * 4 + 1: vmas::diff_forward_kernel<16, 1><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    case 16 * 4 + 2: vmas::diff_forward_kernel<16, 2><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
    default: vmas::diff_forward_kernel<32, 1><<<grid, vmas::kDiffWarps * 32, 0, st>>>(p); break;
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
  const int G = diff_group_lanes(w->N), spl = diff_split(G);
  const int per_cta = vmas::kDiffWarps * (32 / (G * spl));
  auto kern = vmas::diff_backward_kernel<32, 1>;
  switch (G * 4 + spl) {
    case 4 * 4 + 1: kern = vmas::diff_backward_kernel<4, 1>; break;
    case 4 * 4 + 2: kern = vmas::diff_backward_kernel<4, 2>; break;
    case 8 * 4 + 1: kern = vmas::diff_backward_kernel<8, 1>; break;
    case 8 * 4 + 2: kern = vmas::diff_backward_kernel<8, 2>; break;
    case 16 * 4 + 1: kern = vmas::diff_backward_kernel<16, 1>; break;
    case 16 * 4 + 2: kern = vmas::diff_backward_kernel<16, 2>; break;
    default: break;
  }
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

int vmas_debug_diff_split(int32_t split) {
  if (split < 0 || split > 2) return fail(VMAS_EINVAL, "split must be 0, 1 or 2");
  g_diff_split = split;
  return VMAS_OK;
}

// culled LIDAR kernel unless a comparison switched it off
static bool g_lidar_cull = true;

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
  // the culled kernel where its shared arrays fit the default 48 KB
  if (g_lidar_cull && (int64_t)w->A * n_rays <= vmas::kLidarCullMaxRays &&
      vmas::lidar_cull_smem_bytes(w->N, w->A, n_rays) <= 48 * 1024) {
    const size_t smem = (size_t)vmas::lidar_cull_smem_bytes(w->N, w->A, n_rays);
    vmas::lidar_cull_kernel<<<w->E, 128, smem, as_stream(stream)>>>(p);
  } else {
    const size_t smem = (size_t)vmas::lidar_smem_bytes(w->N);
    vmas::lidar_kernel<<<w->E, 128, smem, as_stream(stream)>>>(p);
  }
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

int vmas_debug_lidar_cull(int32_t on) {
  g_lidar_cull = on != 0;
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
