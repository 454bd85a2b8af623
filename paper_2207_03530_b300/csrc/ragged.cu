// Host side of the packed ragged worlds (include/vmas.h, vmas_ragged_*):
// environments with different entity counts.
//
// Entities of all envs are packed without padding.  Envs are sorted into size
// classes of capacity 8, 16, 32, 64, 128 entities (smallest class that holds
// the env); each class is stepped by the fused kernel compiled for its (lanes
// per env, entities per lane) choice, which the autotuner picks by timing, as
// it picks the number of world steps per launch of a rollout.  Rollouts are
// captured into a CUDA graph (one node per class per tile of steps) and
// replayed.  The persistent schedule instead steps every class in one launch
// per tile: warps take one warp's worth of envs at a time from an atomic
// work queue, largest class first, with fixed lanes per class.  The
// autotuner times both schedules.  The step kernels themselves are
// instantiated in vmas.cu and reached through launch_ragged_class and
// launch_ragged_persistent.

#include "host.h"

using namespace vmas_host;
using vmas::StepParams;

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
  int persistent = 0;                // 1, 2: one persistent launch per tile for all classes
                                     // (128- or 96-register build)
  int *queue = nullptr;              // work-queue counters, one per launch of a rollout
  int queue_cap = 0;
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
  cudaFree(r->queue);
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

// At least n work-queue counters.
int ragged_queue_reserve(vmas_ragged *r, int n) {
  if (r->queue_cap >= n) return VMAS_OK;
  cudaFree(r->queue);
  r->queue = nullptr;
  r->queue_cap = 0;
  VMAS_CUDA(cudaMalloc(&r->queue, (size_t)n * sizeof(int)));
  r->queue_cap = n;
  return VMAS_OK;
}

// The persistent launch of one tile: every class, counter `counter` (zeroed
// by the caller on the same stream).
int ragged_persist_tile(vmas_ragged *r, const float *d_actions, int tile, int *counter,
                        cudaStream_t st) {
  vmas::RaggedQueueParams q{};
  int end = 0;
  for (int c = vmas_ragged::kClasses - 1; c >= 0; --c) {
    q.p[c] = ragged_params(r, c);
    q.p[c].actions = d_actions;
    q.p[c].tile = tile;
    end += vmas::persist_items(r->cls_begin[c + 1] - r->cls_begin[c], c);
    q.item_end[c] = end;
  }
  q.n_items = end;
  q.queue = counter;
  return launch_ragged_persistent(q, r->persistent, st);
}

// One tile of `tile` steps for every class, actions of the tile's first step
// at d_actions.
int ragged_launch_tile(vmas_ragged *r, const float *d_actions, int tile, cudaStream_t st) {
  if (r->persistent) {
    int rc = ragged_queue_reserve(r, 1);
    if (rc) return rc;
    VMAS_CUDA(cudaMemsetAsync(r->queue, 0, sizeof(int), st));
    return ragged_persist_tile(r, d_actions, tile, r->queue, st);
  }
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
    const int n_tiles = (n_steps + r->tile - 1) / r->tile;
    if (r->persistent) {
      rc = ragged_queue_reserve(r, n_tiles);
      if (rc) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess && r->persistent) {
      // one memset of every tile's counter, then the tiles in order
      e = cudaMemsetAsync(r->queue, 0, (size_t)n_tiles * sizeof(int), cap);
      for (int k = 0; k < n_tiles && rc == VMAS_OK && e == cudaSuccess; ++k) {
        const int t = k * r->tile;
        rc = ragged_persist_tile(r, d_actions + (size_t)t * r->total_act * 3,
                                 std::min(r->tile, n_steps - t), r->queue + k, cap);
      }
      cudaError_t e2 = cudaStreamEndCapture(cap, &r->graph);
      if (e == cudaSuccess) e = e2;
    } else if (e == cudaSuccess) {
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

}  // extern "C"

namespace {
// Wait for `st`, then report (and clear) the device error word.
int ragged_read_err(vmas_ragged *r, cudaStream_t st, int32_t *bits) {
  int h[3] = {0, 0, 0};  // bits; bounds-checked builds: site << 20 | index, bound
  VMAS_CUDA(cudaMemcpyAsync(h, r->err, sizeof(h), cudaMemcpyDeviceToHost, st));
  VMAS_CUDA(cudaStreamSynchronize(st));
  if (bits) *bits = h[0];
  if (h[0]) {
    VMAS_CUDA(cudaMemsetAsync(r->err, 0, sizeof(h), st));
    VMAS_CUDA(cudaStreamSynchronize(st));
    std::string msg = "device error word set (bits " + std::to_string(h[0]) + ")";
    if (h[0] & VMAS_DEVERR_INDEX)
      msg += "; first index out of range: site " + std::to_string(h[1] >> 20) + ", index " +
             std::to_string(h[1] & 0xfffff) + ", bound " + std::to_string(h[2]);
    return fail(VMAS_EDEVICE, msg);
  }
  return VMAS_OK;
}
}  // namespace

extern "C" {

int vmas_ragged_check(vmas_ragged *r, void *stream, int32_t *bits) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  return ragged_read_err(r, as_stream(stream), bits);
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
    return ragged_read_err(r, st, nullptr);
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

int vmas_ragged_set_schedule(vmas_ragged *r, int32_t persistent) {
  if (!r) return fail(VMAS_EINVAL, "world is NULL");
  if (persistent < 0 || persistent > 2) return fail(VMAS_EINVAL, "schedule must be 0, 1 or 2");
  r->persistent = persistent;
  ++r->version;
  return VMAS_OK;
}

int vmas_ragged_get_schedule(const vmas_ragged *r, int32_t *persistent) {
  if (!r || !persistent) return fail(VMAS_EINVAL, "NULL argument");
  *persistent = r->persistent;
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
  // every candidate starts from the caller's state: a state evolved by the
  // earlier candidates' steps (more contacts, say) would bias the choice
  auto restore = [&]() {
    return cudaMemcpyAsync(r->planes, r->backup, bytes, cudaMemcpyDeviceToDevice, st);
  };
  const int tiles[] = {1, 2, 4, 8, 16, 32, 64};
  constexpr int kTiles = (int)(sizeof(tiles) / sizeof(tiles[0]));
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
        restore();
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
  // steps per launch and schedule, all classes together, each timed as the
  // graph-captured rollout it will run as (the per-class launches are graph
  // branches that run side by side; a stream of direct launches would
  // serialise them)
  float best = 3.4e38f;
  int best_tile = 1, best_sched = 0;
  for (int sched = 0; sched < 3 && rc == VMAS_OK; ++sched) {
    for (int ti = 0; ti < kTiles && rc == VMAS_OK; ++ti) {
      const int tile = tiles[ti];
      if (tile > n_steps) break;
      r->persistent = sched;
      r->tile = tile;
      ++r->version;
      restore();
      rc = vmas_ragged_rollout(r, d_actions, n_steps, stream);  // capture + warm-up
      float ms = 0;
      if (rc == VMAS_OK) {
        restore();
        cudaEventRecord(a, st);
        rc = vmas_ragged_rollout(r, d_actions, n_steps, stream);  // replay
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
      }
      if (rc == VMAS_OK && ms < best) { best = ms; best_tile = tile; best_sched = sched; }
    }
  }
  r->tile = best_tile;
  r->persistent = best_sched;
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
