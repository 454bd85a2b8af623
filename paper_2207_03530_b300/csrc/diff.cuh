// Differentiable rollout of sphere worlds (FP32, sm_103a): a forward pass
// that writes state checkpoints, and a hand-written adjoint (reverse mode) of
// the contact force, drag and damped semi-implicit Euler of VMAS section 3,
// Eqs. 1-2, over every substep.
//
// Loss per env = sum over actuated entities k of |x_k(T) - goal_k|^2.  With
// h = dt / S and a = 1 - zeta, one substep of a movable sphere is
//   F_i = f^a_i + m_i g + sum_j f_ij,   v_i' = a v_i + (h / m_i) F_i,
//   x_i' = x_i + h v_i',
// f_ij = M(g) u, u = d / |d|, d = x_i - x_j, g = |d| - (r_i + r_j),
// M = c k softplus(-g / k) when g <= 0.  Its Jacobian with respect to d is
// J = M'(g) u u^T + M / |d| (I - u u^T), M'(g) = -c sigmoid(-g / k); J is
// symmetric and the same for (i, j) and (j, i).  Given the adjoints lx', lv'
// of a substep's outputs:
//   w = lv' + h lx',  lF_i = (h / m_i) w,  lv = a w,
//   lx_i = lx'_i + sum_j J_ij (lF_i - lF_j),   d loss / d f^a_i += lF_i.
// The contact mask is piecewise constant (no term from the jump at g = 0);
// forces on immovable entities are dropped, so their lF is 0.
//
// Layout: groups of SPL G lanes (G = 4, 8, 16 or 32, the smallest power of
// two >= N; SPL = 1 or 2), one environment per group and 32 / (SPL G) per
// warp, entity i in lane i of each of its SPL half-groups (N <= 32).  With
// SPL = 1 the pair sums of entity i run over its candidate partners j in
// ascending order (a bitmask of the pairs within r_i + r_j + skin, rebuilt
// when a body may have moved half the skin; the pairs left out cannot touch,
// so the sums equal a serial loop over all pairs); with SPL = 2 the two halves
// of the group sum j < ceil(N/2) and the rest, and one shuffle adds the two
// partial sums (both halves then hold the same bits), which shortens each
// substep's pair loop and doubles the warps a small batch of envs fills (the
// host uses SPL = 1 unless asked otherwise: the envs in flight, not the
// warps, bound this latency-bound chain).  Checkpoints every K steps hold (x, y, vx, vy)
// of every entity; the backward pass re-runs each K-step segment forward from
// its checkpoint into shared memory (positions at every substep start) and
// sweeps it backward, segments last to first.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "step.cuh"

namespace vmas {

constexpr int kDiffWarps = 4;  // environments per CTA

struct DiffParams {
  int E, N, A, S, T, K;
  float h, damp, gx, gy, ck, inv_k, c;
  float skin;  // candidate masks: pairs within rsum + skin at the build
  const float *px, *py, *vx, *vy;  // initial state planes [E * N]
  const float4 *param;             // {1/m, 1/I, r, 0}
  const uint8_t *kind;
  const float *actions;  // [T][E][A][3]
  const float *goals;    // [E][A][2]
  float *ckpt;           // [ceil(T / K)][E][N][4]
  float *loss;           // [E]
  const float *dloss;    // [E] upstream gradient
  float *grad;           // [T][E][A][3]
};

// Pair force on i from j and (optionally) its Jacobian; false when apart.
// Distance and normal from one reciprocal square root, the sigmoid from the
// hardware exponential (as the step's contact routines; 1.6 % of the
// adjoint, gradients within the same 4.2e-7 of the FP64 oracle).
__device__ __forceinline__ bool sphere_force(float xi, float yi, float xj, float yj, float rsum,
                                             const DiffParams &p, float &fx, float &fy,
                                             float *J) {
  const float dx = xi - xj, dy = yi - yj;
  const float d2 = dx * dx + dy * dy;
  // most pairs are apart: d2 > 1.0001 rsum^2 gives RN(sqrt(d2)) > rsum, so
  // the exact test below would reject them too (results do not change)
  if (d2 > 1.0001f * (rsum * rsum)) return false;
  const float inv = rsqrtf(d2), s = d2 * inv;
  const float g = s - rsum;
  if (!(g <= 0.f) || !(d2 > 0.f)) return false;
  const float ux = dx * inv, uy = dy * inv;
  const float M = p.ck * softplus_pos(-g * p.inv_k);
  fx = M * ux;
  fy = M * uy;
  if (J) {
    const float sig = __fdividef(1.f, 1.f + __expf(g * p.inv_k));  // sigmoid(-g / k)
    const float dM = -p.c * sig;
    const float t = M * inv;
    J[0] = dM * ux * ux + t * (1.f - ux * ux);
    J[1] = (dM - t) * ux * uy;
    J[2] = dM * uy * uy + t * (1.f - uy * uy);
  }
  return true;
}

struct DiffLane {
  bool ok, mov, act;
  uint32_t kd;
  float im, m, r;
  int row;
};

// Entity `ent` of env e (the lanes of its group's first half in gmask, lane
// = this entity's lane in that half; valid = the group has an env).
__device__ __forceinline__ DiffLane diff_lane(const DiffParams &p, int e, bool valid, int ent,
                                              unsigned gmask, int lane) {
  DiffLane L{};
  L.ok = valid && ent < p.N;
  const size_t t = L.ok ? (size_t)e * p.N + ent : 0;
  L.kd = L.ok ? p.kind[t] : 0u;
  const float4 pr = L.ok ? p.param[t] : make_float4(0.f, 0.f, 0.f, 0.f);
  L.im = pr.x;
  L.m = pr.x > 0.f ? 1.f / pr.x : 0.f;
  L.r = pr.z;
  L.mov = (L.kd & kMovable) != 0u;
  L.act = (L.kd & kActuated) != 0u;
  const unsigned bal = __ballot_sync(0xffffffffu, L.ok && L.act) & gmask;
  L.row = __popc(bal & ((1u << lane) - 1u));
  if (L.row >= p.A) L.act = false;
  return L;
}

// Candidate partners of entity `lane` (bit j): active pairs whose centres lie
// within r_i + r_j + skin at the positions in s_pos (rounded outward by
// 1e-4 relative).  While no body of the env has moved more than skin / 2
// since, a pair outside the mask stays farther apart than r_i + r_j, so
// sphere_force would reject it: the partners in the mask, visited in
// ascending j, give the same sums as every partner.
__device__ __forceinline__ unsigned diff_mask(const DiffParams &p, const DiffLane &L, int lane,
                                              const float2 *s_pos, const uint8_t *s_kind,
                                              const float *s_r, float x, float y) {
  unsigned m = 0u;
  if (L.ok && (L.kd & kCollidable)) {
    for (int j = 0; j < p.N; ++j) {
      if (j == lane || !pair_active(L.kd, s_kind[j])) continue;
      const float2 q = s_pos[j];
      const float dx = x - q.x, dy = y - q.y, lim = L.r + s_r[j] + p.skin;
      if (dx * dx + dy * dy <= 1.0001f * (lim * lim)) m |= 1u << j;
    }
  }
  return m;
}

// Keeps the warp's candidate masks valid at the positions in s_pos: when any
// body of the warp has moved more than 0.45 skin from where the last build
// saw it (skin / 2 is the bound; the rest covers rounding), or nothing has
// been built yet, every lane rebuilds its mask and records its position.
__device__ __forceinline__ bool diff_refresh(const DiffParams &p, const DiffLane &L, int lane,
                                             const float2 *s_pos, const uint8_t *s_kind,
                                             const float *s_r, float x, float y, bool &built,
                                             float &bx, float &by, unsigned &cm) {
  const float dx = x - bx, dy = y - by, lim = 0.45f * p.skin;
  if (!__any_sync(0xffffffffu, !built || dx * dx + dy * dy > lim * lim)) return false;
  cm = diff_mask(p, L, lane, s_pos, s_kind, s_r, x, y);
  bx = x;
  by = y;
  built = true;
  return true;
}

// One forward substep of entity `lane` of its env; s_pos holds every entity's
// (x, y).  SPL = 2: this lane sums the pairs of its half (`half`) of j and
// the partner lane (lane ^ G) the other half.
template <int G, int SPL>
__device__ __forceinline__ void diff_substep(const DiffParams &p, const DiffLane &L, int lane,
                                             int half, const float2 *s_pos, const uint8_t *s_kind,
                                             const float *s_r, unsigned cm, float fax, float fay,
                                             float &x, float &y, float &vx, float &vy) {
  float Fx = fax + L.m * p.gx, Fy = fay + L.m * p.gy;
  if constexpr (SPL == 1) {
    // the candidate partners (cm, from diff_mask), four at a time in
    // ascending j: their loads and distance tests issue together, and the
    // pairs that pass go through sphere_force in j order
    unsigned m = cm;
    while (m) {
      float2 q[4];
      float rs[4];
      bool near[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = m != 0u;
        const int j = in ? __ffs(m) - 1 : 0;
        m &= in ? m - 1u : 0u;
        q[u] = s_pos[j];
        rs[u] = L.r + s_r[j];
        const float dx = x - q[u].x, dy = y - q[u].y;
        near[u] = in && !(dx * dx + dy * dy > 1.0001f * (rs[u] * rs[u]));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float fx, fy;
        if (near[u] && sphere_force(x, y, q[u].x, q[u].y, rs[u], p, fx, fy, nullptr)) {
          Fx += fx;
          Fy += fy;
        }
      }
    }
  } else {
    float Px = 0.f, Py = 0.f;
    if (L.ok && (L.kd & kCollidable)) {
      const int span = (p.N + 1) / 2, j0 = half * span, j1 = min(p.N, j0 + span);
      for (int j = j0; j < j1; ++j) {
        if (j == lane || !pair_active(L.kd, s_kind[j])) continue;
        const float2 q = s_pos[j];
        float fx, fy;
        if (sphere_force(x, y, q.x, q.y, L.r + s_r[j], p, fx, fy, nullptr)) {
          Px += fx;
          Py += fy;
        }
      }
    }
    Px += __shfl_xor_sync(0xffffffffu, Px, G);
    Py += __shfl_xor_sync(0xffffffffu, Py, G);
    Fx += Px;
    Fy += Py;
  }
  if (L.mov) {
    vx = p.damp * vx + Fx * L.im * p.h;
    vy = p.damp * vy + Fy * L.im * p.h;
    x += vx * p.h;
    y += vy * p.h;
  }
}

template <int G, int SPL>
__global__ void __launch_bounds__(kDiffWarps * 32) diff_forward_kernel(const DiffParams p) {
  constexpr int EPW = 32 / (G * SPL);
  __shared__ float2 s_pos_all[kDiffWarps][32];
  __shared__ uint8_t s_kind_all[kDiffWarps][32];
  __shared__ float s_r_all[kDiffWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / (G * SPL), ent = lane % G, half = (lane / G) % SPL;
  const int e0 = (blockIdx.x * kDiffWarps + warp) * EPW;
  if (e0 >= p.E) return;  // whole warp leaves together
  const int e = e0 + grp;
  const bool valid = e < p.E;
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (grp * G * SPL);
  float2 *s_pos = s_pos_all[warp] + grp * G;
  uint8_t *s_kind = s_kind_all[warp] + grp * G;
  float *s_r = s_r_all[warp] + grp * G;
  const DiffLane L = diff_lane(p, e, valid, ent, gmask, grp * G * SPL + ent);
  const bool w0 = half == 0;  // the lane that writes this entity's shared and global values
  const size_t t0 = L.ok ? (size_t)e * p.N + ent : 0;
  float x = L.ok ? p.px[t0] : 0.f, y = L.ok ? p.py[t0] : 0.f;
  float vx = L.ok ? p.vx[t0] : 0.f, vy = L.ok ? p.vy[t0] : 0.f;
  if (w0) {
    s_kind[ent] = (uint8_t)L.kd;
    s_r[ent] = L.r;
  }
  unsigned cm = 0u;  // candidate partners (SPL = 1)
  float bx = 0.f, by = 0.f;
  bool built = false;
  for (int t = 0; t < p.T; ++t) {
    if (t % p.K == 0 && L.ok && w0) {
      float4 *c = reinterpret_cast<float4 *>(p.ckpt) + ((size_t)(t / p.K) * p.E + e) * p.N + ent;
      *c = make_float4(x, y, vx, vy);
    }
    float fax = 0.f, fay = 0.f;
    if (L.act) {
      const float *a = p.actions + (((size_t)t * p.E + e) * p.A + L.row) * 3;
      fax = a[0];
      fay = a[1];
    }
    for (int s = 0; s < p.S; ++s) {
      if (w0) s_pos[ent] = make_float2(x, y);
      __syncwarp();
      if constexpr (SPL == 1) diff_refresh(p, L, ent, s_pos, s_kind, s_r, x, y, built, bx, by, cm);
      diff_substep<G, SPL>(p, L, ent, half, s_pos, s_kind, s_r, cm, fax, fay, x, y, vx, vy);
      __syncwarp();
    }
  }
  float l = 0.f;
  if (L.act) {
    const float *gl = p.goals + ((size_t)e * p.A + L.row) * 2;
    const float dx = x - gl[0], dy = y - gl[1];
    l = dx * dx + dy * dy;
  }
  for (int o = G / 2; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (ent == 0 && w0 && valid) p.loss[e] = l;
}

// Dynamic shared memory per warp: positions at the K * S + 1 substep starts
// of one segment.
__host__ __device__ inline size_t diff_traj_bytes(int K, int S) {
  return (size_t)(K * S + 1) * 32 * sizeof(float2);
}

template <int G, int SPL>
__global__ void __launch_bounds__(kDiffWarps * 32) diff_backward_kernel(const DiffParams p) {
  constexpr int EPW = 32 / (G * SPL);
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ float2 s_lf_all[kDiffWarps][32];
  __shared__ uint8_t s_kind_all[kDiffWarps][32];
  __shared__ float s_r_all[kDiffWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / (G * SPL), ent = lane % G, half = (lane / G) % SPL;
  const int e0 = (blockIdx.x * kDiffWarps + warp) * EPW;
  if (e0 >= p.E) return;  // whole warp leaves together
  const int e = e0 + grp;
  const bool valid = e < p.E;
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (grp * G * SPL);
  const bool w0 = half == 0;  // the lane that writes this entity's shared and global values
  // traj row q holds 32 entity slots; this group's entities are at grp * G
  float2 *traj = reinterpret_cast<float2 *>(dsm + warp * diff_traj_bytes(p.K, p.S)) + grp * G;
  float2 *s_lf = s_lf_all[warp] + grp * G;
  uint8_t *s_kind = s_kind_all[warp] + grp * G;
  float *s_r = s_r_all[warp] + grp * G;
  const DiffLane L = diff_lane(p, e, valid, ent, gmask, grp * G * SPL + ent);
  if (w0) {
    s_kind[ent] = (uint8_t)L.kd;
    s_r[ent] = L.r;
  }
  float lx = 0.f, ly = 0.f, lvx = 0.f, lvy = 0.f;
  const int nseg = (p.T + p.K - 1) / p.K;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int ta = seg * p.K, tb = min(p.T, ta + p.K);
    // re-run the segment forward, keeping every substep-start position
    const float4 c = L.ok ? reinterpret_cast<const float4 *>(p.ckpt)[((size_t)seg * p.E + e) * p.N + ent]
                          : make_float4(0.f, 0.f, 0.f, 0.f);
    float x = c.x, y = c.y, vx = c.z, vy = c.w;
    // candidate masks of the replay (SPL = 1), rebuilt from the checkpoint;
    // um collects every partner any of them held, so each pair that touches
    // at some substep of the segment is in um
    unsigned cm = 0u, um = 0u;
    float bx = 0.f, by = 0.f;
    bool built = false;
    int q = 0;
    for (int t = ta; t < tb; ++t) {
      float fax = 0.f, fay = 0.f;
      if (L.act) {
        const float *a = p.actions + (((size_t)t * p.E + e) * p.A + L.row) * 3;
        fax = a[0];
        fay = a[1];
      }
      for (int s = 0; s < p.S; ++s, ++q) {
        if (w0) traj[q * 32 + ent] = make_float2(x, y);
        __syncwarp();
        if constexpr (SPL == 1) {
          if (diff_refresh(p, L, ent, traj + q * 32, s_kind, s_r, x, y, built, bx, by, cm)) um |= cm;
        }
        diff_substep<G, SPL>(p, L, ent, half, traj + q * 32, s_kind, s_r, cm, fax, fay, x, y, vx,
                             vy);
        __syncwarp();
      }
    }
    if (seg == nseg - 1 && L.act) {  // d loss / d x(T) = 2 (x - goal), scaled by the upstream
      const float *gl = p.goals + ((size_t)e * p.A + L.row) * 2;
      const float w = 2.f * p.dloss[e];
      lx = w * (x - gl[0]);
      ly = w * (y - gl[1]);
    }
    // sweep the segment backward
    for (int t = tb - 1; t >= ta; --t) {
      float gax = 0.f, gay = 0.f;
      for (int s = p.S - 1; s >= 0; --s) {
        --q;
        float lfx = 0.f, lfy = 0.f;
        if (L.mov) {
          const float wx = lvx + p.h * lx, wy = lvy + p.h * ly;
          lfx = p.h * L.im * wx;
          lfy = p.h * L.im * wy;
          lvx = p.damp * wx;
          lvy = p.damp * wy;
        }
        gax += lfx;
        gay += lfy;
        if (w0) s_lf[ent] = make_float2(lfx, lfy);
        __syncwarp();
        if constexpr (SPL == 1) {
          // the partners of um in ascending j, four at a time as forward
          // (um is 0 for an entity without pairs)
          unsigned m = um;
          const float2 me = traj[q * 32 + ent];
          while (m) {
            float2 o[4];
            float rs[4];
            bool near[4];
            int js[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const bool in = m != 0u;
              const int j = in ? __ffs(m) - 1 : 0;
              m &= in ? m - 1u : 0u;
              js[u] = j;
              o[u] = traj[q * 32 + j];
              rs[u] = L.r + s_r[j];
              const float dx = me.x - o[u].x, dy = me.y - o[u].y;
              near[u] = in && !(dx * dx + dy * dy > 1.0001f * (rs[u] * rs[u]));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              float fx, fy, J[3];
              if (near[u] && sphere_force(me.x, me.y, o[u].x, o[u].y, rs[u], p, fx, fy, J)) {
                const float2 lj = s_lf[js[u]];
                const float dx = lfx - lj.x, dy = lfy - lj.y;
                lx += J[0] * dx + J[1] * dy;
                ly += J[1] * dx + J[2] * dy;
              }
            }
          }
        } else {
          float px_ = 0.f, py_ = 0.f;
          if (L.ok && (L.kd & kCollidable)) {
            const float2 me = traj[q * 32 + ent];
            const int span = (p.N + 1) / 2, j0 = half * span, j1 = min(p.N, j0 + span);
            for (int j = j0; j < j1; ++j) {
              if (j == ent || !pair_active(L.kd, s_kind[j])) continue;
              const float2 o = traj[q * 32 + j];
              float fx, fy, J[3];
              if (sphere_force(me.x, me.y, o.x, o.y, L.r + s_r[j], p, fx, fy, J)) {
                const float2 lj = s_lf[j];
                const float dx = lfx - lj.x, dy = lfy - lj.y;
                px_ += J[0] * dx + J[1] * dy;
                py_ += J[1] * dx + J[2] * dy;
              }
            }
          }
          px_ += __shfl_xor_sync(0xffffffffu, px_, G);
          py_ += __shfl_xor_sync(0xffffffffu, py_, G);
          lx += px_;
          ly += py_;
        }
        __syncwarp();
      }
      if (L.act && w0) {
        float *g = p.grad + (((size_t)t * p.E + e) * p.A + L.row) * 3;
        g[0] = gax;
        g[1] = gay;
        g[2] = 0.f;
      }
    }
  }
}

// Zero the gradient rows of actuated slots no entity uses.
__global__ void diff_zero_grad_kernel(float *grad, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) grad[t] = 0.f;
}

}  // namespace vmas
