// Closest points and penetration of one entity pair, FP32, device side.
//
// VMAS section 3, Eq. 2: the contact force acts along x_ij, the offset that
// joins the two entities' closest surface points, when |x_ij| <= d_min.  Each routine returns the signed gap
// g = |x_ij| - d_min, the unit normal n pointing from j towards i and the
// lever terms ti = (p_i - x_i) x n, tj = (p_j - x_j) x n of the contact
// points p_i, p_j (Eq. 3 torque, read as the signed 2D cross product).
//
// Shapes (section 3, "Core"): sphere of radius r; box of half extents
// (hw, hh) along its axes e1 = (cos th, sin th), e2 = (-sin th, cos th);
// line = zero-thickness segment of half length hl along e1.
//   sphere-sphere: centre offset, d_min = r_i + r_j;
//   sphere-line / sphere-box: distance from the centre to the segment / box
//     boundary, d_min = r; a centre inside a box leaves through the face of
//     least depth (faces +e1, -e1, +e2, -e2, first minimum wins);
//   box / line pairs: least separating-axis overlap (axes of i, then of j;
//     box e1, e2; line e2; first minimum wins), the axis owner is the
//     reference body, the contact point lies on the other body's incident
//     edge clipped to the reference face, its clipped ends weighted by their
//     depth beneath that face.
// A pair whose normal is undefined (coincident closest points) exerts no
// force.  The sphere routines take the distance and the unit normal from one
// hardware reciprocal square root (rsqrtf, within 2 ulp): the IEEE square
// root and divide cost 2.5 % of the step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vmas {

enum : uint32_t { kSphere = 0, kBox = 1, kLine = 2 };

struct Hit {
  float g;       // signed gap (<= 0 when the force acts)
  float nx, ny;  // unit normal from j towards i
  float ti, tj;  // (p_i - x_i) x n and (p_j - x_j) x n
};

// Sphere i against sphere j.
__device__ __forceinline__ bool hit_sphere_sphere(float xi, float yi, float ri, float xj,
                                                  float yj, float rj, Hit &h) {
  const float dx = xi - xj, dy = yi - yj;
  const float d2 = dx * dx + dy * dy;
  const float inv = rsqrtf(d2), dist = d2 * inv;
  const float g = dist - (ri + rj);
  if (!(g <= 0.f) || !(d2 > 0.f)) return false;
  h.g = g;
  h.nx = dx * inv;
  h.ny = dy * inv;
  h.ti = 0.f;  // p_i - x_i = -r_i n is parallel to n
  h.tj = 0.f;
  return true;
}

// Sphere (sx, sy, r) against the segment centred at (lx, ly) along (c, s)
// with half length hl.  Returned for the order (sphere, line); the lever of
// the line is t (e1 x n) where t is the clamped abscissa of the closest point.
__device__ __forceinline__ bool hit_sphere_line(float sx, float sy, float r, float lx, float ly,
                                                float c, float s, float hl, Hit &h) {
  const float ex = sx - lx, ey = sy - ly;
  const float t = fminf(fmaxf(ex * c + ey * s, -hl), hl);
  const float dx = ex - t * c, dy = ey - t * s;
  const float d2 = dx * dx + dy * dy;
  const float inv = rsqrtf(d2), dist = d2 * inv;
  const float g = dist - r;
  if (!(g <= 0.f) || !(d2 > 0.f)) return false;
  h.g = g;
  h.nx = dx * inv;
  h.ny = dy * inv;
  h.ti = 0.f;
  h.tj = t * (c * h.ny - s * h.nx);
  return true;
}

// Sphere (sx, sy, r) against the box centred at (bx, by), axes (c, s),
// half extents (hw, hh).  Returned for the order (sphere, box).
__device__ __forceinline__ bool hit_sphere_box(float sx, float sy, float r, float bx, float by,
                                               float c, float s, float hw, float hh, Hit &h) {
  const float ex = sx - bx, ey = sy - by;
  const float lx = c * ex + s * ey;  // box frame
  const float ly = -s * ex + c * ey;
  float nlx, nly, qx, qy, g;
  if (fabsf(lx) <= hw && fabsf(ly) <= hh) {
    // centre inside: leave through the face of least depth
    const float d0 = hw - lx, d1 = hw + lx, d2 = hh - ly, d3 = hh + ly;
    float best = d0;
    nlx = 1.f; nly = 0.f; qx = hw; qy = ly;
    if (d1 < best) { best = d1; nlx = -1.f; nly = 0.f; qx = -hw; qy = ly; }
    if (d2 < best) { best = d2; nlx = 0.f; nly = 1.f; qx = lx; qy = hh; }
    if (d3 < best) { best = d3; nlx = 0.f; nly = -1.f; qx = lx; qy = -hh; }
    g = -best - r;
  } else {
    qx = fminf(fmaxf(lx, -hw), hw);
    qy = fminf(fmaxf(ly, -hh), hh);
    const float dx = lx - qx, dy = ly - qy;
    const float d2 = dx * dx + dy * dy;
    const float inv = rsqrtf(d2), dist = d2 * inv;
    g = dist - r;
    if (!(g <= 0.f) || !(d2 > 0.f)) return false;
    nlx = dx * inv;
    nly = dy * inv;
  }
  h.g = g;
  h.nx = c * nlx - s * nly;
  h.ny = s * nlx + c * nly;
  h.ti = 0.f;
  h.tj = qx * nly - qy * nlx;  // (q - centre) x n, rotation invariant
  return true;
}

// A box or a line as a polygon: centre, e1, half extents (hb = 0 for lines).
struct Poly {
  float cx, cy, ux, uy, ha, hb;
  bool box;
};

__device__ __forceinline__ float half_extent(const Poly &p, float ax, float ay) {
  return p.ha * fabsf(ax * p.ux + ay * p.uy) + p.hb * fabsf(ay * p.ux - ax * p.uy);
}

// Corner k of a box, counter-clockwise from (-hw, -hh) in the box frame.
__device__ __forceinline__ void box_corner(const Poly &p, int k, float &vx, float &vy) {
  const float a = (k == 1 || k == 2) ? p.ha : -p.ha;
  const float b = (k >= 2) ? p.hb : -p.hb;
  vx = p.cx + a * p.ux - b * p.uy;
  vy = p.cy + a * p.uy + b * p.ux;
}

// Edge k of a box runs from corner k to corner k+1 (outward normals -e2,
// +e1, +e2, -e1); a line's only edge runs from -hl to +hl along e1.
__device__ __forceinline__ void poly_edge(const Poly &p, int k, float &ax, float &ay, float &bx,
                                          float &by) {
  if (p.box) {
    box_corner(p, k, ax, ay);
    box_corner(p, (k + 1) & 3, bx, by);
  } else {
    ax = p.cx - p.ha * p.ux;
    ay = p.cy - p.ha * p.uy;
    bx = p.cx + p.ha * p.ux;
    by = p.cy + p.ha * p.uy;
  }
}

// Box/line i against box/line j.  Inlined: as an out-of-line call its
// by-value arguments went through the stack and the call site cost the step
// kernel its spill-free register allocation (4 % of the step).
__device__ __forceinline__ bool hit_poly_poly(const Poly A, const Poly B, Hit &h) {
  // candidate axes in fixed slots, tried in order: A's first (box e1 | line
  // e2), A's e2 (boxes), B's first, B's e2 (boxes), and for two exactly
  // parallel lines A's e1 (their normals coincide); held in registers
  const float ax0 = A.box ? A.ux : -A.uy, ay0 = A.box ? A.uy : A.ux;
  const float ax2 = B.box ? B.ux : -B.uy, ay2 = B.box ? B.uy : B.ux;
  const bool ok4 = !A.box && !B.box && A.ux * B.uy - A.uy * B.ux == 0.f;
  const float dcx = A.cx - B.cx, dcy = A.cy - B.cy;
  float best = __int_as_float(0x7f800000);
  float bax = 0.f, bay = 0.f;
  int bq = 0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const bool ok = q == 0 || q == 2 || (q == 1 && A.box) || (q == 3 && B.box) || (q == 4 && ok4);
    if (ok) {
      const float axq = q == 0 ? ax0 : q == 1 ? -A.uy : q == 2 ? ax2 : q == 3 ? -B.uy : A.ux;
      const float ayq = q == 0 ? ay0 : q == 1 ? A.ux : q == 2 ? ay2 : q == 3 ? B.ux : A.uy;
      const float d = dcx * axq + dcy * ayq;
      const float depth = half_extent(A, axq, ayq) + half_extent(B, axq, ayq) - fabsf(d);
      if (depth < 0.f) return false;  // separating axis
      if (depth < best) { best = depth; bax = axq; bay = ayq; bq = q; }
    }
  }
  float ux = bax, uy = bay;
  if (dcx * ux + dcy * uy < 0.f) { ux = -ux; uy = -uy; }
  const float g = -best;
  const bool ref_i = bq < 2;
  const Poly R = ref_i ? A : B;
  const Poly Q = ref_i ? B : A;
  const float nrx = ref_i ? -ux : ux, nry = ref_i ? -uy : uy;  // R's outward normal
  const int kr = bq == 4 ? 1 : (bq & 1);  // the parallel-lines axis has no face

  bool have_face = true;
  float fax = 0.f, fay = 0.f, fbx = 0.f, fby = 0.f;
  if (R.box) {
    const float dn = nrx * bax + nry * bay;
    const int e = (kr == 0) ? (dn > 0.f ? 1 : 3) : (dn > 0.f ? 2 : 0);
    poly_edge(R, e, fax, fay, fbx, fby);
  } else if (kr == 0) {
    poly_edge(R, 0, fax, fay, fbx, fby);
  } else {
    have_face = false;
  }
  // incident edge: outward normal most opposed to nR (edges in order)
  int ie = 0;
  if (Q.box) {
    const float d1 = Q.ux * nrx + Q.uy * nry;   // +e1 . nR
    const float d2 = Q.ux * nry - Q.uy * nrx;   // +e2 . nR
    float bd = -d2;                             // edge 0: -e2
    if (d1 < bd) { bd = d1; ie = 1; }
    if (d2 < bd) { bd = d2; ie = 2; }
    if (-d1 < bd) { bd = -d1; ie = 3; }
  }
  float i0x, i0y, i1x, i1y;
  poly_edge(Q, ie, i0x, i0y, i1x, i1y);

  bool have_point = false;
  float qx = 0.f, qy = 0.f;
  if (have_face) {
    float tx = fbx - fax, ty = fby - fay;
    const float flen = sqrtf(tx * tx + ty * ty);
    if (flen > 0.f) {
      tx /= flen;
      ty /= flen;
      const float s0 = (i0x - fax) * tx + (i0y - fay) * ty;
      const float s1 = (i1x - fax) * tx + (i1y - fay) * ty;
      float lo, hi;
      bool nonempty;
      if (s1 == s0) {
        lo = 0.f;
        hi = 1.f;
        nonempty = s0 >= 0.f && s0 <= flen;
      } else {
        const float la = (0.f - s0) / (s1 - s0), lb = (flen - s0) / (s1 - s0);
        lo = fmaxf(fminf(la, lb), 0.f);
        hi = fminf(fmaxf(la, lb), 1.f);
        nonempty = lo <= hi;
      }
      if (nonempty) {
        const float c0x = i0x + lo * (i1x - i0x), c0y = i0y + lo * (i1y - i0y);
        const float c1x = i0x + hi * (i1x - i0x), c1y = i0y + hi * (i1y - i0y);
        const float w0 = fmaxf(-((c0x - fax) * nrx + (c0y - fay) * nry), 0.f);
        const float w1 = fmaxf(-((c1x - fax) * nrx + (c1y - fay) * nry), 0.f);
        if (w0 + w1 > 0.f) {
          const float iw = 1.f / (w0 + w1);
          qx = (w0 * c0x + w1 * c1x) * iw;
          qy = (w0 * c0y + w1 * c1y) * iw;
        } else {
          qx = 0.5f * (c0x + c1x);
          qy = 0.5f * (c0y + c1y);
        }
        have_point = true;
      }
    }
  }
  if (!have_point) {
    // Q's deepest vertex along -nR, vertices in order
    const int nv = Q.box ? 4 : 2;
    float bp = __int_as_float(0x7f800000);
    for (int k = 0; k < nv; ++k) {
      float vx, vy;
      if (Q.box) {
        box_corner(Q, k, vx, vy);
      } else {
        const float sg = k == 0 ? -1.f : 1.f;
        vx = Q.cx + sg * Q.ha * Q.ux;
        vy = Q.cy + sg * Q.ha * Q.uy;
      }
      const float pr = vx * nrx + vy * nry;
      if (pr < bp) { bp = pr; qx = vx; qy = vy; }
    }
  }
  float pix, piy, pjx, pjy;
  if (ref_i) {
    pjx = qx; pjy = qy;
    pix = qx + g * ux; piy = qy + g * uy;
  } else {
    pix = qx; piy = qy;
    pjx = qx - g * ux; pjy = qy - g * uy;
  }
  h.g = g;
  h.nx = ux;
  h.ny = uy;
  h.ti = (pix - A.cx) * uy - (piy - A.cy) * ux;
  h.tj = (pjx - B.cx) * uy - (pjy - B.cy) * ux;
  return true;
}

}  // namespace vmas
