// LIDAR ray casts (VMAS section 3: agents can carry LIDAR sensors), FP32.
//
// Every actuated entity casts n_rays rays from its centre at angles
// th + 2 pi k / n_rays; a ray reports the smallest distance t in
// [0, range] at which it meets another collidable entity (0 when its origin
// lies inside one), or `range` when it meets none.  Spheres are discs, boxes
// filled rectangles, lines segments (a ray exactly parallel to a segment
// misses it).  One CTA per environment: its bodies are staged in shared
// memory, threads take (agent, ray) items.
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

// Entry distance of the ray o + t d (|d| = 1) into body b, or +inf.
// pose = {x, y, cos, sin}, geo = {ha, hb, shape}.
__device__ __forceinline__ float ray_hit(float ox, float oy, float dx, float dy, float4 pose,
                                         float2 half, uint32_t shape) {
  const float inf = __int_as_float(0x7f800000);
  const float px = ox - pose.x, py = oy - pose.y;
  if (shape == kSphere) {
    const float cq = px * px + py * py - half.x * half.x;
    if (cq <= 0.f) return 0.f;
    const float b = px * dx + py * dy;
    if (b >= 0.f) return inf;  // outside and pointing away
    const float disc = b * b - cq;
    if (disc < 0.f) return inf;
    return cq / (-b + sqrtf(disc));  // the nearer root, free of cancellation
  }
  const float c = pose.z, s = pose.w;
  const float lx = c * px + s * py, ly = -s * px + c * py;   // body frame
  const float ldx = c * dx + s * dy, ldy = -s * dx + c * dy;
  if (shape == kBox) {
    const float hw = half.x, hh = half.y;
    if (fabsf(lx) <= hw && fabsf(ly) <= hh) return 0.f;
    float tmin = -inf, tmax = inf;
    if (ldx == 0.f) {
      if (fabsf(lx) > hw) return inf;
    } else {
      float t1 = (-hw - lx) / ldx, t2 = (hw - lx) / ldx;
      tmin = fmaxf(tmin, fminf(t1, t2));
      tmax = fminf(tmax, fmaxf(t1, t2));
    }
    if (ldy == 0.f) {
      if (fabsf(ly) > hh) return inf;
    } else {
      float t1 = (-hh - ly) / ldy, t2 = (hh - ly) / ldy;
      tmin = fmaxf(tmin, fminf(t1, t2));
      tmax = fminf(tmax, fmaxf(t1, t2));
    }
    if (tmin > tmax || tmax < 0.f) return inf;
    return fmaxf(tmin, 0.f);
  }
  if (ldy == 0.f) return inf;  // segment along the body x axis
  const float t = -ly / ldy;
  if (t < 0.f || fabsf(lx + t * ldx) > half.x) return inf;
  return t;
}

__global__ void __launch_bounds__(128) lidar_kernel(const LidarParams p) {
  extern __shared__ __align__(16) unsigned char lsm[];
  float4 *s_pose = reinterpret_cast<float4 *>(lsm);   // [N] {x, y, cos, sin}
  float2 *s_half = reinterpret_cast<float2 *>(s_pose + p.N);  // [N]
  uint8_t *s_kind = reinterpret_cast<uint8_t *>(s_half + p.N);  // [N]
  __shared__ int s_agent[VMAS_LIDAR_MAX_ENTITIES];
  __shared__ int s_nact;
  const int e = blockIdx.x;
  const size_t eb = (size_t)e * p.N;
  for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
    const uint32_t kd = p.kind[eb + i];
    const float4 pr = p.param[eb + i];
    float c = 1.f, s = 0.f;
    body_axes(p.th[eb + i], c, s);
    s_pose[i] = make_float4(p.px[eb + i], p.py[eb + i], c, s);
    s_half[i] = make_float2(pr.z, pr.w);
    s_kind[i] = (uint8_t)kd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // k-th actuated entity, in entity order
    int n = 0;
    for (int i = 0; i < p.N; ++i)
      if ((s_kind[i] & kActuated) && n < p.A) s_agent[n++] = i;
    s_nact = n;
  }
  __syncthreads();
  const int nact = s_nact;
  const float step = 6.283185307179586f / (float)p.R;
  for (int it = threadIdx.x; it < p.A * p.R; it += blockDim.x) {
    const int k = it / p.R, r = it - k * p.R;
    float best = p.range;
    if (k < nact) {
      const int i = s_agent[k];
      const float4 me = s_pose[i];
      float dx, dy;
      body_axes(p.th[eb + i] + step * (float)r, dx, dy);
      for (int j = 0; j < p.N; ++j) {
        const uint32_t kj = s_kind[j];
        if (j == i || !(kj & kCollidable)) continue;
        best = fminf(best, ray_hit(me.x, me.y, dx, dy, s_pose[j], s_half[j], kj & 3u));
      }
    }
    p.out[((size_t)e * p.A + k) * p.R + r] = best;
  }
}

}  // namespace vmas
