// LIDAR ray casts (VMAS section 3: agents can carry LIDAR sensors), FP32.
//
// Every actuated entity casts n_rays rays from its centre at angles
// th + 2 pi k / n_rays; a ray reports the smallest distance t in
// [0, range] at which it meets another collidable entity (0 when its origin
// lies inside one), or `range` when it meets none.  Spheres are discs, boxes
// filled rectangles, lines segments (a ray exactly parallel to a segment
// misses it).  One CTA per environment: its collidable bodies are staged in
// shared memory grouped by shape, so that every loop tests one shape, and
// threads take (agent, ray) items, an agent's rays in consecutive lanes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "step.cuh"

namespace vmas {

struct LidarParams {
  int E, N, A, R;
  float range;
  const float *px, *py, *th;
  const float4 *param;  // {1/m, 1/I, ha, hb}
  const uint8_t *kind;
  float *out;           // [E][A][R]
};

// Entry distance of the ray o + t d (|d| = 1) into one body: 0 when o lies
// inside it, +inf on a miss.  Written without branches: a warp's lanes cast
// different rays at the same body, and every select costs less than a
// divergent early exit.
// Distances are absolute (at most the range), so the nearer root is taken
// as -b - sqrt(disc): its cancellation costs relative, not absolute, accuracy.
// Divides use the fast reciprocal (within 2 ulp) and the square root the
// hardware reciprocal square root (disc * rsqrt(disc)): both err by about
// 1e-7 of a unit-range distance.
__device__ __forceinline__ float ray_sphere(float ox, float oy, float dx, float dy, float4 b) {
  // b = {x, y, r, -}
  const float inf = __int_as_float(0x7f800000);
  const float px = ox - b.x, py = oy - b.y;
  const float cq = px * px + py * py - b.z * b.z;
  const float bb = px * dx + py * dy;
  const float disc = bb * bb - cq;
  const float t = -bb - (disc > 0.f ? disc * rsqrtf(disc) : 0.f);
  return cq <= 0.f ? 0.f : ((bb >= 0.f || disc < 0.f) ? inf : t);  // inside; away or past
}

// b = {x, y, cos, sin}, h = half sizes: slab test in the box frame.
__device__ __forceinline__ float ray_box(float ox, float oy, float dx, float dy, float4 b,
                                         float2 h) {
  const float inf = __int_as_float(0x7f800000);
  const float px = ox - b.x, py = oy - b.y;
  const float lx = b.z * px + b.w * py, ly = -b.w * px + b.z * py;
  const float ldx = b.z * dx + b.w * dy, ldy = -b.w * dx + b.z * dy;
  const float ix = __fdividef(1.f, ldx), iy = __fdividef(1.f, ldy);
  const float ax = (-h.x - lx) * ix, bx = (h.x - lx) * ix;
  const float ay = (-h.y - ly) * iy, by = (h.y - ly) * iy;
  // a ray parallel to a slab misses when it starts outside it, else that
  // slab does not bound t
  const float txa = ldx == 0.f ? -inf : fminf(ax, bx);
  const float txb = ldx == 0.f ? (fabsf(lx) > h.x ? -inf : inf) : fmaxf(ax, bx);
  const float tya = ldy == 0.f ? -inf : fminf(ay, by);
  const float tyb = ldy == 0.f ? (fabsf(ly) > h.y ? -inf : inf) : fmaxf(ay, by);
  const float tmin = fmaxf(txa, tya), tmax = fminf(txb, tyb);
  const bool inside = fabsf(lx) <= h.x && fabsf(ly) <= h.y;
  return inside ? 0.f : ((tmin > tmax || tmax < 0.f) ? inf : fmaxf(tmin, 0.f));
}

// b = {x, y, cos, sin}, half length hl; a ray exactly parallel misses.
__device__ __forceinline__ float ray_line(float ox, float oy, float dx, float dy, float4 b,
                                          float hl) {
  const float inf = __int_as_float(0x7f800000);
  const float px = ox - b.x, py = oy - b.y;
  const float lx = b.z * px + b.w * py, ly = -b.w * px + b.z * py;
  const float ldx = b.z * dx + b.w * dy, ldy = -b.w * dx + b.z * dy;
  const float t = __fdividef(-ly, ldy);
  return (ldy != 0.f && t >= 0.f && fabsf(lx + t * ldx) <= hl) ? t : inf;
}

// Bytes of dynamic shared memory per CTA for N entities.
__host__ __device__ inline int lidar_smem_bytes(int N) { return N * (16 + 8 + 1); }

// Shared setup of both LIDAR kernels, for env `e`: the kinds, the
// collidable bodies grouped by shape (s_ent / s_slot, list starts in
// s_start[0..3]), the casters (s_agent, s_nact) and each body's pose and
// half sizes by list slot.  Ends with a barrier.
__device__ __forceinline__ void lidar_setup(const LidarParams &p, int e, float4 *s_pose,
                                            float2 *s_half, uint8_t *s_kind, int *s_ent,
                                            int *s_slot, int *s_agent, int *s_start, int *s_nact) {
  const size_t eb = (size_t)e * p.N;
  for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
    s_kind[i] = p.kind[eb + i];
    s_slot[i] = -1;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // the collidable bodies, grouped by shape (each group in entity order),
    // and the casters, compacted with warp votes
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    int n = 0;
    for (int sh = 0; sh < 3; ++sh) {
      if (lane == 0) s_start[sh] = n;
      for (int c0 = 0; c0 < p.N; c0 += 32) {
        const int i = c0 + lane;
        const uint32_t kd = i < p.N ? s_kind[i] : 0u;
        const bool in = i < p.N && (kd & 3u) == (uint32_t)sh && (kd & kCollidable);
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
          s_ent[n + __popc(m & lt)] = i;
          s_slot[i] = n + __popc(m & lt);
        }
        n += __popc(m);
      }
    }
    int na = 0;
    for (int c0 = 0; c0 < p.N; c0 += 32) {
      const int i = c0 + lane;
      const bool act = i < p.N && (s_kind[i] & kActuated);
      const unsigned m = __ballot_sync(0xffffffffu, act);
      const int k = na + __popc(m & lt);
      if (act && k < p.A) s_agent[k] = i;
      na += __popc(m);
    }
    if (lane == 0) {
      s_start[3] = n;
      *s_nact = na < p.A ? na : p.A;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < s_start[3]; q += blockDim.x) {
    const int i = s_ent[q];
    const float4 pr = p.param[eb + i];
    float c = 1.f, s = 0.f;
    if ((s_kind[i] & 3u) != kSphere) body_axes(p.th[eb + i], c, s);
    const bool sphere = (s_kind[i] & 3u) == kSphere;
    // a sphere's slot holds {x, y, r, -}: one load per test
    s_pose[q] = make_float4(p.px[eb + i], p.py[eb + i], sphere ? pr.z : c, sphere ? 0.f : s);
    s_half[q] = make_float2(pr.z, pr.w);
  }
  __syncthreads();
}

// Direction of ray r of a caster with frame (c0, s0): the frame rotated by
// r * step, whose cos and sin (cr, sr) come from body_axes(r * step).  The
// rounding is pinned (explicit fma and products), so both kernels cast the
// same rays, and the ray angles follow the caster's frame exactly whatever
// the size of its angle.
__device__ __forceinline__ void lidar_ray_rot(float step, int r, float &cr, float &sr) {
  body_axes(__fmul_rn(step, (float)r), cr, sr);
}
__device__ __forceinline__ void lidar_ray_dir(float c0, float s0, float cr, float sr, float &dx,
                                              float &dy) {
  dx = __fmaf_rn(c0, cr, -__fmul_rn(s0, sr));
  dy = __fmaf_rn(s0, cr, __fmul_rn(c0, sr));
}

__global__ void __launch_bounds__(128) lidar_kernel(const LidarParams p) {
  extern __shared__ __align__(16) unsigned char lsm[];
  float4 *s_pose = reinterpret_cast<float4 *>(lsm);            // [N] by list slot
  float2 *s_half = reinterpret_cast<float2 *>(s_pose + p.N);   // [N] by list slot
  uint8_t *s_kind = reinterpret_cast<uint8_t *>(s_half + p.N);  // [N] by entity
  __shared__ int s_ent[VMAS_LIDAR_MAX_ENTITIES];    // entity of each list slot
  __shared__ int s_slot[VMAS_LIDAR_MAX_ENTITIES];   // list slot of each entity (-1: none)
  __shared__ int s_agent[VMAS_LIDAR_MAX_ENTITIES];  // k-th actuated entity
  __shared__ int s_start[4];                        // list starts: spheres, boxes, lines, end
  __shared__ int s_nact;
  const int e = blockIdx.x;
  const size_t eb = (size_t)e * p.N;
  lidar_setup(p, e, s_pose, s_half, s_kind, s_ent, s_slot, s_agent, s_start, &s_nact);
  const int nact = s_nact, b0 = s_start[1], l0 = s_start[2], end = s_start[3];
  const float inf = __int_as_float(0x7f800000);
  const float step = 6.283185307179586f / (float)p.R;
  for (int it = threadIdx.x; it < p.A * p.R; it += blockDim.x) {
    const int k = it / p.R, r = it - k * p.R;
    float best = p.range;
    if (k < nact) {
      const int i = s_agent[k];
      const int self = s_slot[i];  // the caster's own slot is skipped
      const float ox = p.px[eb + i], oy = p.py[eb + i];
      float c0, s0, cr, sr, dx, dy;
      body_axes(p.th[eb + i], c0, s0);
      lidar_ray_rot(step, r, cr, sr);
      lidar_ray_dir(c0, s0, cr, sr, dx, dy);
#pragma unroll 4
      for (int q = 0; q < b0; ++q) {
        const float4 b = s_pose[q];
        const float t = ray_sphere(ox, oy, dx, dy, b);
        best = fminf(best, q == self ? inf : t);
      }
#pragma unroll 2
      for (int q = b0; q < l0; ++q) {
        const float t = ray_box(ox, oy, dx, dy, s_pose[q], s_half[q]);
        best = fminf(best, q == self ? inf : t);
      }
#pragma unroll 2
      for (int q = l0; q < end; ++q) {
        const float t = ray_line(ox, oy, dx, dy, s_pose[q], s_half[q].x);
        best = fminf(best, q == self ? inf : t);
      }
    }
    p.out[((size_t)e * p.A + k) * p.R + r] = best;
  }
}

// ---- Culled LIDAR -------------------------------------------------------
// The same readings as lidar_kernel -- per ray the least entry distance over
// the same bodies, computed by the same ray_* routines on the same ray
// directions -- but each (body, caster) pair tests only the rays whose
// direction can meet the body.  From an origin outside a convex body the
// directions that meet it form one arc: spheres and boxes take the arc of
// their bounding circle, centre direction +- an upper bound of asin(R / d),
// segments the arc between their endpoints.  The arc is widened by the
// angle errors (an arctangent within 0.0016 rad, the tests' own rounding at
// a grazing ray, the caster's frame and the rounding of its ray directions,
// which are the caster's frame rotated by 2 pi r / R), and a pair tests the
// rays inside it.  A pair whose body lies beyond the range, by its bounding
// circle or its closest point, is skipped (every entry distance exceeds the
// range, which the reading keeps); an origin inside a sphere or a box reads
// 0 on every ray, as there.  A pair tests every ray when the origin lies
// inside the bounding circle or when a segment's arc approaches pi.
// Minima are taken with atomicMin on order-preserving keys in shared
// memory, so the reading is the minimum whatever the order.

constexpr int kLidarCullMaxRays = 3072;  // n_actuated x n_rays held in shared memory

__host__ __device__ inline int lidar_cull_smem_bytes(int N, int A, int R) {
  return align16(lidar_smem_bytes(N)) + A * R * 12 + R * 8;  // + directions, rotations, keys
}

// Order-preserving keys of floats: a < b exactly when key(a) < key(b)
// (NaN aside).
__device__ __forceinline__ uint32_t lidar_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float lidar_unkey(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// atan2 within 0.0016 rad: atan z ~ (pi/4) z - z (|z| - 1)(0.2447 + 0.0663 |z|)
// on |z| <= 1 (Rajan et al., IEEE Signal Processing Magazine 2006), octants by
// symmetry.
__device__ __forceinline__ float lidar_atan2_approx(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const bool swap = ay > ax;
  const float z = __fdividef(swap ? ax : ay, fmaxf(swap ? ay : ax, 1e-30f));
  float a = z * (0.78539816f - (z - 1.f) * (0.2447f + 0.0663f * z));
  a = swap ? 1.57079633f - a : a;
  a = x < 0.f ? 3.14159265f - a : a;
  return y < 0.f ? -a : a;
}

// Ray range [r_lo, r_hi] (indices taken modulo R) of the arc centre phi,
// half width half, for a caster whose ray 0 points at phi0; false when the
// arc covers every ray.
__device__ __forceinline__ bool lidar_arc(float phi, float half, float phi0, float inv_step,
                                          int R, int &r_lo, int &r_hi) {
  // |phi0| <= pi, |phi| <= 3 pi / 2 (a segment's arc centre may pass -pi or
  // pi), so u lies in (-3 R / 2, 3 R / 2); reduce it modulo R into [0, R]
  float u = (phi - phi0) * inv_step;
  u -= (float)R * floorf(u * (1.f / (float)R));
  u = fminf(fmaxf(u, 0.f), (float)R);  // rounding; NaN becomes 0 (w then decides)
  // the rays whose angle lies within the arc widened by the angle errors:
  // 0.0016 rad from the arctangent at each edge, 1e-5 rad for the tests'
  // own rounding at a grazing ray, and 1 % of a spacing for the rounding
  // of the ray directions (about 2e-7 rad)
  const float w = half * inv_step + 0.0025f * inv_step + 0.01f;
  if (!(w < 0.5f * (float)R)) return false;  // wide, or not a number: every ray
  r_lo = (int)ceilf(u - w);   // in (-R / 2, R]
  r_hi = (int)floorf(u + w);  // in [0, 3 R / 2)
  return r_hi - r_lo + 1 < R;
}

// 16 CTAs per SM (32 registers): the kernel is issue-bound and wants every warp
__global__ void __launch_bounds__(128, 16) lidar_cull_kernel(const LidarParams p) {
  extern __shared__ __align__(16) unsigned char lsm[];
  float4 *s_pose = reinterpret_cast<float4 *>(lsm);            // [N] by list slot
  float2 *s_half = reinterpret_cast<float2 *>(s_pose + p.N);   // [N] by list slot
  uint8_t *s_kind = reinterpret_cast<uint8_t *>(s_half + p.N);  // [N] by entity
  const int AR = p.A * p.R;
  // 8-byte arrays first, then the 4-byte ones (every start stays aligned)
  float2 *s_dir = reinterpret_cast<float2 *>(lsm + align16(lidar_smem_bytes(p.N)));  // [A][R]
  float2 *s_rot = s_dir + AR;                                                          // [R]
  uint32_t *s_key = reinterpret_cast<uint32_t *>(s_rot + p.R);                         // [A][R]
  __shared__ int s_ent[VMAS_LIDAR_MAX_ENTITIES];
  __shared__ int s_slot[VMAS_LIDAR_MAX_ENTITIES];
  __shared__ int s_agent[VMAS_LIDAR_MAX_ENTITIES];
  __shared__ int s_start[4];
  __shared__ int s_nact;
  __shared__ float s_ox[VMAS_LIDAR_MAX_ENTITIES], s_oy[VMAS_LIDAR_MAX_ENTITIES];
  __shared__ float s_phi0[VMAS_LIDAR_MAX_ENTITIES];  // direction of the caster's ray 0
  __shared__ float2 s_frame[VMAS_LIDAR_MAX_ENTITIES];  // the caster's (cos, sin)
  const int e = blockIdx.x;
  const size_t eb = (size_t)e * p.N;
  lidar_setup(p, e, s_pose, s_half, s_kind, s_ent, s_slot, s_agent, s_start, &s_nact);
  const int nact = s_nact, b0 = s_start[1], l0 = s_start[2], nb = s_start[3];
  const float step = 6.283185307179586f / (float)p.R, inv_step = (float)p.R / 6.283185307179586f;
  for (int k = threadIdx.x; k < nact; k += blockDim.x) {
    const int i = s_agent[k];
    const float th = p.th[eb + i];
    float c, sn;
    body_axes(th, c, sn);
    s_ox[k] = p.px[eb + i];
    s_oy[k] = p.py[eb + i];
    s_phi0[k] = atan2f(sn, c);
    s_frame[k] = make_float2(c, sn);
  }
  for (int r = threadIdx.x; r < p.R; r += blockDim.x) {
    float cr, sr;
    lidar_ray_rot(step, r, cr, sr);
    s_rot[r] = make_float2(cr, sr);
  }
  __syncthreads();
  // a warp per caster, its rays across the lanes (no division per item)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int k = warp; k < p.A; k += nwarps) {
    const float2 fr = k < nact ? s_frame[k] : make_float2(1.f, 0.f);
    for (int r = lane; r < p.R; r += 32) {
      float dx = 1.f, dy = 0.f;
      const float2 ro = s_rot[r];
      if (k < nact) lidar_ray_dir(fr.x, fr.y, ro.x, ro.y, dx, dy);
      s_dir[k * p.R + r] = make_float2(dx, dy);
      s_key[k * p.R + r] = lidar_key(p.range);
    }
  }
  __syncthreads();
  // (body, caster) pairs, body-major: a warp takes one body (one shape)
  // against consecutive casters
  const float cut = p.range * 1.0001f + 1e-5f;  // every entry beyond it exceeds the range
  // item it = q * nact + k advanced by the block size without a division
  const int dq = nact > 0 ? (int)blockDim.x / nact : 0, dk = (int)blockDim.x - dq * nact;
  int q = nact > 0 ? (int)threadIdx.x / nact : nb, k = (int)threadIdx.x - q * nact;
  for (; q < nb; q += dq, k += dk, q += k >= nact ? 1 : 0, k -= k >= nact ? nact : 0) {
    if (q == s_slot[s_agent[k]]) continue;  // the caster's own slot
    const float ox = s_ox[k], oy = s_oy[k];
    const float4 b = s_pose[q];
    const float2 hs = s_half[q];
    const int shape = q < b0 ? 0 : (q < l0 ? 1 : 2);
    const float px = b.x - ox, py = b.y - oy;  // centre seen from the origin
    bool every = false;
    float phi, half;
    if (shape == 2) {
      // segment: its closest point against the range, its endpoints for the arc
      const float sc = fminf(fmaxf(-(px * b.z + py * b.w), -hs.x), hs.x);
      const float cx = px + sc * b.z, cy = py + sc * b.w;
      if (cx * cx + cy * cy > cut * cut) continue;
      const float p1 = lidar_atan2_approx(py - hs.x * b.w, px - hs.x * b.z);
      const float p2 = lidar_atan2_approx(py + hs.x * b.w, px + hs.x * b.z);
      float dl = p2 - p1;
      if (dl > 3.14159265f) dl -= 6.28318531f;
      if (dl < -3.14159265f) dl += 6.28318531f;
      every = every || fabsf(dl) > 3.1f;  // an origin on (or by) the carrier
      phi = p1 + 0.5f * dl;
      half = 0.5f * fabsf(dl);
    } else {
      // sphere or box: its bounding circle
      const float rb = shape == 0 ? b.z : sqrtf(hs.x * hs.x + hs.y * hs.y);
      const float d = sqrtf(px * px + py * py);
      if (d - rb > cut) continue;
      every = every || d <= rb * 1.0001f + 1e-6f;  // the origin may lie inside
      phi = lidar_atan2_approx(py, px);
      const float xr = __fdividef(rb, d);  // asin x <= 1.0473 x (x <= 1/2), <= (pi/2) x
      half = every ? 0.f : xr * (xr <= 0.5f ? 1.0473f : 1.5708f);
    }
    int r0 = 0, r1 = p.R - 1;
    if (!every && !lidar_arc(phi, half, s_phi0[k], inv_step, p.R, r0, r1)) {
      r0 = 0;
      r1 = p.R - 1;
    }
    uint32_t *key = s_key + k * p.R;
    const float2 *dir = s_dir + k * p.R;
    int idx = r0 < 0 ? r0 + p.R : (r0 >= p.R ? r0 - p.R : r0);  // r0 in (-R, R]: idx in [0, R)
    // one loop per shape: a select between the three routines would run all three
    auto cast = [&](auto test) {
      for (int r = r0; r <= r1; ++r) {
        const float2 dv = dir[idx];
        const float t = test(dv);
        if (t < p.range) atomicMin(key + idx, lidar_key(t));
        idx = idx + 1 == p.R ? 0 : idx + 1;
      }
    };
    if (shape == 0)
      cast([&](float2 dv) { return ray_sphere(ox, oy, dv.x, dv.y, b); });
    else if (shape == 1)
      cast([&](float2 dv) { return ray_box(ox, oy, dv.x, dv.y, b, hs); });
    else
      cast([&](float2 dv) { return ray_line(ox, oy, dv.x, dv.y, b, hs.x); });
  }
  __syncthreads();
  for (int it = threadIdx.x; it < AR; it += blockDim.x)
    p.out[(size_t)e * AR + it] = lidar_unkey(s_key[it]);
}

}  // namespace vmas
