// Fused VMAS world step kernel (sm_103a, FP32 CUDA cores).
//
// One warp steps one environment through all S substeps of one world step
// (VMAS section 3, Eqs. 1-3); state stays in registers and shared memory
// between substeps and touches HBM once on the way in and once on the way
// out.
//
//   lanes own entities   : entity i lives in lane i % 32, slot i / 32
//   lanes own pairs      : pair q (canonical i < j, row-major) in lane q % 32
//   contact sums         : hits are appended, in pair order, to a per-warp
//                          shared buffer (ballot + popc), then every lane
//                          adds the records that touch its entities in that
//                          order -- the same summation order as a serial loop
//                          over pairs, with no atomics.
//
// Broad phase: a pair is skipped when the bounding circles (inflated by a
// rounding allowance) are apart, or when a line's infinite carrier is
// farther from the other body's centre than that body's bounding radius.
// Both tests only skip pairs the narrow phase would reject, so results do
// not depend on them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "contact.cuh"

namespace vmas {

constexpr int kWarpsPerCta = 8;  // environments per CTA
constexpr int kCap = 64;         // buffered contact records per warp

// kind byte = shape | flags << 2
enum : uint32_t {
  kMovable = 1u << 2,
  kRotatable = 2u << 2,
  kCollidable = 4u << 2,
  kActuated = 8u << 2
};

struct StepParams {
  int E, N, A, S, P;
  float h;      // dt / S
  float damp;   // 1 - zeta
  float gx, gy;
  float ck;     // c * k
  float inv_k;  // 1 / k
  float vmax;   // 0 = no cap
  float *px, *py, *vx, *vy, *th, *om;  // state planes [E * N]
  const float4 *phys;                  // {m, 1/m (0 if fixed), 1/I (0 if not rotatable), 0}
  const float4 *geom;                  // {ha, hb, bounding radius, 0}
  const uint8_t *kind;                 // [E * N]
  const uint16_t *pairs;               // [P] i | j << 8
  const float *actions;                // [E][A][3]
  uint8_t *mask;                       // [E][P], mask kernel only
  int *err;                            // device error word
};

__host__ __device__ inline int align16(int b) { return (b + 15) & ~15; }
__host__ __device__ inline int warp_smem_bytes(int N) {
  return 2 * N * 16 + kCap * 16 + kCap * 4;
}
__host__ __device__ inline int cta_smem_bytes(int N, int P) {
  return align16(2 * P) + kWarpsPerCta * warp_smem_bytes(N);
}

__device__ __forceinline__ bool pair_active(uint32_t ki, uint32_t kj) {
  return (ki & kCollidable) && (kj & kCollidable) && ((ki | kj) & (kMovable | kRotatable));
}

// softplus(z) = log(1 + e^z) for z >= 0 without overflow.
__device__ __forceinline__ float softplus_pos(float z) { return z + log1pf(expf(-z)); }

// Narrow phase for the ordered pair (i, j); bi/bj = {x, y, inflated R, kind}.
__device__ __forceinline__ bool pair_hit(const float4 bi, const float4 bj, uint32_t ki,
                                         uint32_t kj, const float4 *s_ng, int i, int j,
                                         Hit &h) {
  const float dx = bi.x - bj.x, dy = bi.y - bj.y;
  const float lim = bi.z + bj.z;
  if (dx * dx + dy * dy > lim * lim) return false;
  const uint32_t si = ki & 3u, sj = kj & 3u;
  if (si == kSphere && sj == kSphere) {
    const float ri = s_ng[i].z, rj = s_ng[j].z;
    return hit_sphere_sphere(bi.x, bi.y, ri, bj.x, bj.y, rj, h);
  }
  const float4 gi = s_ng[i], gj = s_ng[j];  // {cos, sin, ha, hb}
  // slab test against a line's carrier
  if (sj == kLine && fabsf(dx * gj.y - dy * gj.x) > bi.z + 1e-5f * (fabsf(bj.x) + fabsf(bj.y)))
    return false;
  if (si == kLine && fabsf(dx * gi.y - dy * gi.x) > bj.z + 1e-5f * (fabsf(bi.x) + fabsf(bi.y)))
    return false;
  if (si == kSphere) {
    if (sj == kLine) return hit_sphere_line(bi.x, bi.y, gi.z, bj.x, bj.y, gj.x, gj.y, gj.z, h);
    return hit_sphere_box(bi.x, bi.y, gi.z, bj.x, bj.y, gj.x, gj.y, gj.z, gj.w, h);
  }
  if (sj == kSphere) {
    bool ok;
    if (si == kLine) ok = hit_sphere_line(bj.x, bj.y, gj.z, bi.x, bi.y, gi.x, gi.y, gi.z, h);
    else ok = hit_sphere_box(bj.x, bj.y, gj.z, bi.x, bi.y, gi.x, gi.y, gi.z, gi.w, h);
    if (ok) {  // computed for (j, i): flip the normal, swap the levers
      h.nx = -h.nx;
      h.ny = -h.ny;
      const float t = h.tj;
      h.tj = 0.f;
      h.ti = -t;
    }
    return ok;
  }
  const Poly A{bi.x, bi.y, gi.x, gi.y, gi.z, gi.w, si == kBox};
  const Poly B{bj.x, bj.y, gj.x, gj.y, gj.z, gj.w, sj == kBox};
  return hit_poly_poly(A, B, h);
}

template <int SLOTS, bool MASK_ONLY>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    world_step_kernel(const StepParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = p.N, P = p.P;
  uint16_t *s_pairs = reinterpret_cast<uint16_t *>(smem);
  for (int q = threadIdx.x; q < P; q += blockDim.x) s_pairs[q] = p.pairs[q];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *wb = smem + align16(2 * P) + warp * warp_smem_bytes(N);
  float4 *s_bp = reinterpret_cast<float4 *>(wb);  // {x, y, inflated R, kind}
  float4 *s_ng = s_bp + N;                         // {cos, sin, ha, hb}
  float4 *s_rec = s_ng + N;                        // {fx, fy, ti, tj}
  uint32_t *s_rij = reinterpret_cast<uint32_t *>(s_rec + kCap);
  __syncthreads();

  const int e = blockIdx.x * kWarpsPerCta + warp;
  if (e >= p.E) return;
  const size_t eb = (size_t)e * N;
  const unsigned lt = (1u << lane) - 1u;

  float x[SLOTS], y[SLOTS], vx[SLOTS], vy[SLOTS], th[SLOTS], om[SLOTS];
  float fax[SLOTS], fay[SLOTS], tau[SLOTS], ms[SLOTS], im[SLOTS], iI[SLOTS], ha[SLOTS],
      hb[SLOTS], rb[SLOTS];
  uint32_t kd[SLOTS];
  int act_base = 0;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int i = lane + 32 * s;
    const bool ok = i < N;
    kd[s] = ok ? p.kind[eb + i] : 0u;
    x[s] = ok ? p.px[eb + i] : 0.f;
    y[s] = ok ? p.py[eb + i] : 0.f;
    vx[s] = ok ? p.vx[eb + i] : 0.f;
    vy[s] = ok ? p.vy[eb + i] : 0.f;
    th[s] = ok ? p.th[eb + i] : 0.f;
    om[s] = ok ? p.om[eb + i] : 0.f;
    const float4 ph = ok ? p.phys[eb + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 ge = ok ? p.geom[eb + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    ms[s] = ph.x;
    im[s] = ph.y;
    iI[s] = ph.z;
    ha[s] = ge.x;
    hb[s] = ge.y;
    rb[s] = ge.z;
    const bool actuated = ok && (kd[s] & kActuated);
    const unsigned bal = __ballot_sync(0xffffffffu, actuated);
    const int slot = act_base + __popc(bal & lt);
    act_base += __popc(bal);
    fax[s] = fay[s] = tau[s] = 0.f;
    if (!MASK_ONLY && actuated && slot < p.A) {
      const float *a = p.actions + ((size_t)e * p.A + slot) * 3;
      fax[s] = a[0];
      fay[s] = a[1];
      tau[s] = (kd[s] & kRotatable) ? a[2] : 0.f;
    }
  }

  const int n_sub = MASK_ONLY ? 1 : p.S;
  for (int sub = 0; sub < n_sub; ++sub) {
    // publish the substep-start pose
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int i = lane + 32 * s;
      if (i < N) {
        const float infl = rb[s] + 1e-5f * (rb[s] + fabsf(x[s]) + fabsf(y[s]));
        s_bp[i] = make_float4(x[s], y[s], infl, __uint_as_float(kd[s]));
        float sn = 0.f, cs = 1.f;
        if ((kd[s] & 3u) != kSphere) sincosf(th[s], &sn, &cs);
        s_ng[i] = make_float4(cs, sn, ha[s], hb[s]);
      }
    }
    __syncwarp();

    // Eq. 1: action + gravity; Eq. 3: action torque
    float Fx[SLOTS], Fy[SLOTS], T[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      Fx[s] = fax[s] + ms[s] * p.gx;
      Fy[s] = fay[s] + ms[s] * p.gy;
      T[s] = tau[s];
    }

    int count = 0;
    auto drain = [&](int n) {
      for (int c = 0; c < n; ++c) {
        const float4 r = s_rec[c];
        const uint32_t ij = s_rij[c];
        const int ci = (int)(ij & 0xffffu), cj = (int)(ij >> 16);
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          const int me = lane + 32 * s;
          if (me == ci) { Fx[s] += r.x; Fy[s] += r.y; T[s] += r.z; }
          if (me == cj) { Fx[s] -= r.x; Fy[s] -= r.y; T[s] += r.w; }
        }
      }
    };

    for (int q0 = 0; q0 < P; q0 += 32) {
      const int q = q0 + lane;
      bool hit = false;
      Hit hh;
      int i = 0, j = 0;
      if (q < P) {
        const uint32_t ij = s_pairs[q];
        i = (int)(ij & 0xffu);
        j = (int)(ij >> 8);
        const float4 bi = s_bp[i], bj = s_bp[j];
        const uint32_t ki = __float_as_uint(bi.w), kj = __float_as_uint(bj.w);
        if (pair_active(ki, kj)) hit = pair_hit(bi, bj, ki, kj, s_ng, i, j, hh);
        if (MASK_ONLY) p.mask[(size_t)e * P + q] = hit ? 1 : 0;
      }
      if (!MASK_ONLY) {
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        const int nh = __popc(bal);
        if (count + nh > kCap) {  // warp-uniform
          __syncwarp();
          drain(count);
          __syncwarp();
          count = 0;
        }
        if (hit) {
          // Eq. 2 magnitude c k log(1 + exp(-g / k)), g <= 0
          const float mag = p.ck * softplus_pos(-hh.g * p.inv_k);
          const int slot = count + __popc(bal & lt);
          s_rec[slot] = make_float4(mag * hh.nx, mag * hh.ny, mag * hh.ti, -mag * hh.tj);
          s_rij[slot] = (uint32_t)i | ((uint32_t)j << 16);
        }
        count += nh;
      }
    }
    if (MASK_ONLY) return;
    __syncwarp();
    drain(count);
    __syncwarp();

    // Eqs. 1 and 3: damped semi-implicit Euler
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      if (kd[s] & kMovable) {
        vx[s] = p.damp * vx[s] + Fx[s] * im[s] * p.h;
        vy[s] = p.damp * vy[s] + Fy[s] * im[s] * p.h;
        if (p.vmax > 0.f) {
          const float sp = sqrtf(vx[s] * vx[s] + vy[s] * vy[s]);
          if (sp > p.vmax) {
            const float sc = p.vmax / sp;
            vx[s] *= sc;
            vy[s] *= sc;
          }
        }
        x[s] += vx[s] * p.h;
        y[s] += vy[s] * p.h;
      }
      if (kd[s] & kRotatable) {
        om[s] = p.damp * om[s] + T[s] * iI[s] * p.h;
        th[s] += om[s] * p.h;
      }
    }
  }

  bool bad = false;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int i = lane + 32 * s;
    if (i < N) {
      p.px[eb + i] = x[s];
      p.py[eb + i] = y[s];
      p.vx[eb + i] = vx[s];
      p.vy[eb + i] = vy[s];
      p.th[eb + i] = th[s];
      p.om[eb + i] = om[s];
      bad |= !(isfinite(x[s]) && isfinite(y[s]) && isfinite(vx[s]) && isfinite(vy[s]) &&
               isfinite(th[s]) && isfinite(om[s]));
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(p.err, 1);
}

}  // namespace vmas
