// Shared pieces of the world step (sm_103a, FP32 CUDA cores): parameters,
// the pair activity rule, the Eq. 2 magnitude, the exact narrow-phase
// dispatch, and the first-substep contact-mask kernel (debug path).
//
// Exact rejection inside pair_hit: a pair is skipped when the bounding
// circles (radii inflated by a rounding allowance of 1e-5 (R + |x| + |y|))
// are apart, or when a line's infinite carrier is farther from the other
// body's centre than that body's inflated radius.  Both tests only skip
// pairs the narrow phase would reject, so results do not depend on them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "contact.cuh"
#include "mbar.cuh"
#include "params.cuh"
#include "vmas.h"

#define VMAS_LIDAR_MAX_ENTITIES VMAS_MAX_ENTITIES

namespace vmas {

constexpr int kWarpsPerCta = 8;  // environments per CTA of the mask kernel

// kind byte = shape | flags << 2
enum : uint32_t {
  kMovable = 1u << 2,
  kRotatable = 2u << 2,
  kCollidable = 4u << 2,
  kActuated = 8u << 2
};

__host__ __device__ inline int align16(int b) { return (b + 15) & ~15; }

// Self-checking build (compiled with -DVMAS_CHECKED only): every shared and
// global index goes through VIDX, which records the first index outside
// [0, lim) in the error words (bit 2 of word 0; word 1 = code << 20 | index,
// word 2 = lim) and clamps it to 0 so the access stays inside the buffer.
#ifdef VMAS_CHECKED
__device__ __forceinline__ int vmas_checked_index(int idx, int lim, int code, int *err) {
  if ((unsigned)idx < (unsigned)lim) return idx;
  atomicOr(err, 2);
  atomicCAS(err + 1, 0, (code << 20) | (idx & 0xfffff));
  atomicCAS(err + 2, 0, lim);
  return 0;
}
#define VIDX(idx, lim, code) vmas_checked_index((int)(idx), (int)(lim), (code), p.err)
#else
#define VIDX(idx, lim, code) (idx)
#endif

__device__ __forceinline__ bool pair_active(uint32_t ki, uint32_t kj) {
  return (ki & kCollidable) && (kj & kCollidable) && ((ki | kj) & (kMovable | kRotatable));
}

// cos and sin of a body angle, written out (no library call): Cody-Waite
// reduction r = th - k pi/2 with a fused multiply-add, then the Taylor series
// of sin to r^9 and cos to r^10 and the quadrant k mod 4.  pi/2 is split in
// two floats, P1 = fl(pi/2) and P2 = fl(pi/2 - P1).  The fma forms k P1
// exactly, and th - k P1 is then a multiple of 2^-23 (of 2^-24 when
// |th| < 1) below 2 (below 1) in magnitude, so the first step is exact
// while k is within one of th's quadrant; the split's error, |k| * 3e-15,
// and the second step's rounding
// stay below 1e-8 for |th| up to about 2e6 rad.  Over that range k, rounded
// from th * fl(2/pi), is off the nearest quadrant by at most 0.15, so
// |r| <= 0.97, where the series truncate below 2e-8.  Absolute error about
// 1e-7 up to 2e6 rad; beyond it grows with |th|.  r is clamped to [-1, 1],
// so for any input (huge, inf or NaN angles included) the result stays a
// unit vector to that accuracy.  Shared by every kernel that needs a body
// frame.
__device__ __forceinline__ void body_axes(float th, float &c, float &s) {
  const float k = rintf(th * 0.63661977236758134f);  // 2 / pi
  float r = fmaf(-k, 1.57079637050628662109375f, th);   // P1 = 0x1.921fb6p+0
  r = fmaf(-k, -4.37113882867379300296306610107421875e-8f, r);  // P2 = -0x1.777a5cp-25
  r = fminf(fmaxf(r, -1.f), 1.f);  // NaN becomes -1
  const int q = __float2int_rz(k) & 3;  // saturating conversion: defined for every k
  const float z = r * r;
  const float ps = fmaf(fmaf(fmaf(2.7557319223985891e-6f, z, -1.9841269841269841e-4f), z,
                             8.3333333333333333e-3f), z, -1.6666666666666667e-1f);
  const float sr = fmaf(r * z, ps, r);
  const float pc = fmaf(fmaf(fmaf(fmaf(-2.7557319223985891e-7f, z, 2.4801587301587302e-5f), z,
                                  -1.3888888888888889e-3f), z, 4.1666666666666667e-2f), z, -0.5f);
  const float cr = fmaf(z, pc, 1.0f);
  c = q == 0 ? cr : (q == 1 ? -sr : (q == 2 ? -cr : sr));
  s = q == 0 ? sr : (q == 1 ? cr : (q == 2 ? -sr : -cr));
}

// Diagnostic kernel: body_axes of n angles (for the accuracy test).
__global__ void body_axes_kernel(const float *th, float *cs, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) body_axes(th[t], cs[2 * t], cs[2 * t + 1]);
}

// softplus(z) = log(1 + e^z) for z >= 0 without overflow, as z + ln(1 + e^-z)
// with the hardware exp2/log2 approximations (__expf, __logf).  The second
// term lies in (0, ln 2]: __logf on [1, 2] is within 3.6e-7 absolute, the
// __expf error (2 + 1.2 z ulp of e^-z) adds at most 1.2e-7 and the rounding
// of 1 + e^-z 6e-8, so the term is within 5.5e-7 of ln(1 + e^-z), and the
// result, at least ln 2, within 8e-7 relative.  The accurate library pair
// cost 3 % of the step at 262,144 envs.
__device__ __forceinline__ float softplus_pos(float z) { return z + __logf(1.f + __expf(-z)); }

// Narrow phase for the ordered pair (i, j); bi/bj = {x, y, inflated R, kind},
// gi/gj = {cos, sin, ha, hb} (a sphere's radius in ha), loaded by the caller
// beside the poses so both shared-memory reads overlap.
__device__ __forceinline__ bool pair_hit(const float4 bi, const float4 bj, uint32_t ki,
                                         uint32_t kj, const float4 gi, const float4 gj,
                                         Hit &h) {
  const float dx = bi.x - bj.x, dy = bi.y - bj.y;
  const float lim = bi.z + bj.z;
  if (dx * dx + dy * dy > lim * lim) return false;
  const uint32_t si = ki & 3u, sj = kj & 3u;
  if (si == kSphere && sj == kSphere) return hit_sphere_sphere(bi.x, bi.y, gi.z, bj.x, bj.y, gj.z, h);
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

// First-substep contact mask (debug path): one warp per environment, lanes
// own pairs; writes 1 where the pair is active and its gap is <= 0 with a
// defined normal, using the same narrow phase as the step kernel.
template <int SLOTS>
__global__ void __launch_bounds__(kWarpsPerCta * 32) pair_mask_kernel(const StepParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = p.N, P = p.P;
  uint16_t *s_pairs = reinterpret_cast<uint16_t *>(smem);
  for (int q = threadIdx.x; q < P; q += blockDim.x) s_pairs[q] = p.pairs[q];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4 *s_bp = reinterpret_cast<float4 *>(smem + align16(2 * P) + warp * 32 * N);
  float4 *s_ng = s_bp + N;
  __syncthreads();
  const int e = blockIdx.x * kWarpsPerCta + warp;
  if (e >= p.E) return;
  const size_t eb = (size_t)e * N;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int i = lane + 32 * s;
    if (i < N) {
      const uint32_t kd = p.kind[eb + i];
      const float x = p.px[eb + i], y = p.py[eb + i], th = p.th[eb + i];
      const float4 pr = p.param[eb + i];
      const float R = (kd & 3u) == kBox ? sqrtf(pr.z * pr.z + pr.w * pr.w) : pr.z;
      const float infl = R + 1e-5f * (R + fabsf(x) + fabsf(y));
      s_bp[i] = make_float4(x, y, infl, __uint_as_float(kd));
      float sn = 0.f, cs = 1.f;
      if ((kd & 3u) != kSphere) body_axes(th, cs, sn);
      s_ng[i] = make_float4(cs, sn, pr.z, pr.w);
    }
  }
  __syncwarp();
  for (int q = lane; q < P; q += 32) {
    const uint32_t ij = s_pairs[q];
    const int i = (int)(ij & 0xffu), j = (int)(ij >> 8);
    const float4 bi = s_bp[i], bj = s_bp[j];
    const uint32_t ki = __float_as_uint(bi.w), kj = __float_as_uint(bj.w);
    Hit h;
    const bool hit = pair_active(ki, kj) && pair_hit(bi, bj, ki, kj, s_ng[i], s_ng[j], h);
    p.mask[(size_t)e * P + q] = hit ? 1 : 0;
  }
}

__host__ __device__ inline int mask_cta_smem_bytes(int N, int P) {
  return align16(2 * P) + kWarpsPerCta * 32 * N;
}

}  // namespace vmas
