/*
 * FP64 CPU oracle of the VMAS batched world step.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this file; the CUDA product path never
 * does.  It shares no code, header, table or helper with the CUDA path.
 *
 * Source: Bettini et al., "VMAS: A Vectorized Multi-Agent Simulator for
 * Collective Robot Learning", section 3 ("Core"):
 *
 *   Eq. 1   f_i   = f^a_i + m_i g + sum_{j != i} f^e_ij
 *           xdot_i <- (1 - zeta) xdot_i + f_i / m_i * dt
 *           x_i    <- x_i + xdot_i * dt                (semi-implicit Euler)
 *   Eq. 2   f^e_ij = c * x_ij / |x_ij| * k * log(1 + exp(-(|x_ij| - d_min)/k))
 *                    if |x_ij| <= d_min, else 0
 *   Eq. 3   tau_i  = sum_j r_ij x f^e_ij
 *           thdot_i <- (1 - zeta) thdot_i + tau_i / I_i * dt
 *           th_i    <- th_i + thdot_i * dt
 *
 * Entities are spheres, boxes and lines (section 3, "Core"), with state
 * (x, xdot, theta, thetadot), a mass, an optional maximum speed and the
 * movable / rotatable / collidable switches.
 *
 * Readings taken where the paper is silent (each is marked "Reading Rn" at
 * the code that takes it):
 *   R1  c and k are world parameters (no values are printed).
 *   R2  the contact cut-off is inclusive: the force acts when gap <= 0.
 *   R3  the torque of Eq. 3 is the signed 2D cross product r x f, not its
 *       norm (a norm would spin every body the same way).
 *   R4  I_i is an input; 0 selects box m(w^2+h^2)/12, line m L^2/12,
 *       sphere m r^2/2.
 *   R5  substeps: each is one full Eq. 1-3 application with dt/S, the same
 *       zeta, actions held over the step, contacts recomputed per substep.
 *   R6  forces on immovable entities are dropped (their state never moves).
 *   R7  the maximum speed clamps |xdot| after the velocity update.
 *   R8  an undefined normal (coincident closest points) gives no force.
 *   R9  ties: strict "<" over fixed candidate orders (first minimum wins).
 *   R15 a pair acts when both entities are collidable and at least one of
 *       them can move or rotate.
 *   R16 closest points of two polygons (box/line pairs): separating-axis
 *       depth; contact point from the incident edge clipped to the
 *       reference face, weighted by each clipped end's penetration.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OW_SPHERE 0
#define OW_BOX 1
#define OW_LINE 2

#define OW_MOVABLE 1
#define OW_ROTATABLE 2
#define OW_COLLIDABLE 4
#define OW_ACTUATED 8

/* World description: every per-entity array is [n_envs * n_entities]. */
typedef struct {
  int32_t n_envs, n_entities, n_actuated, substeps;
  double dt, drag, gx, gy, c, k, max_speed;
  const uint8_t *shape;
  const uint8_t *flags;
  const double *size_a; /* sphere radius | box width | line length */
  const double *size_b; /* box height (unused otherwise)           */
  const double *mass;
  const double *inertia; /* 0 => default of Reading R4 */
} ow_world;

/* Pose and shape of one entity. */
typedef struct {
  int shape;
  double x, y, th, a, b;
} ow_body;

/* Result of the closest-points computation for an ordered pair (i, j). */
typedef struct {
  double g;        /* signed gap |x_ij| - d_min: > 0 apart, <= 0 touching */
  double nx, ny;   /* unit normal pointing from j towards i              */
  double pix, piy; /* closest / contact point on i                        */
  double pjx, pjy; /* closest / contact point on j                        */
  int has_normal;  /* 0 when the normal is undefined (Reading R8)         */
  /* Decision margin (Reading R9): how far the nearest discrete choice the
   * geometry made for this pair (face, axis, incident edge, clip, normal
   * orientation) is from switching to another candidate, in world units
   * (dot products of unit normals for the incident-edge choice); INFINITY
   * where the result is continuous.  Used only to certify near ties. */
  double margin;
} ow_contact;

static double clampd(double v, double lo, double hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

/* softplus(z) = log(1 + e^z), written so that it neither overflows for large
 * z nor loses the small result for very negative z. */
static double softplus(double z) {
  if (z > 0) return z + log1p(exp(-z));
  return log1p(exp(z));
}

/* ---- closest points, sphere cases (Eq. 2: x_ij between closest points) --- */

/* Sphere i - sphere j: x_ij is the centre offset and d_min = r_i + r_j. */
static ow_contact sphere_sphere(const ow_body *bi, const ow_body *bj) {
  ow_contact r;
  memset(&r, 0, sizeof r);
  r.margin = INFINITY;
  double dx = bi->x - bj->x, dy = bi->y - bj->y;
  double dist = sqrt(dx * dx + dy * dy);
  r.g = dist - (bi->a + bj->a);
  if (dist > 0) {
    r.nx = dx / dist;
    r.ny = dy / dist;
    r.has_normal = 1;
  }
  r.pix = bi->x - bi->a * r.nx;
  r.piy = bi->y - bi->a * r.ny;
  r.pjx = bj->x + bj->a * r.nx;
  r.pjy = bj->y + bj->a * r.ny;
  return r;
}

/* Sphere s - line l (a zero-thickness segment of length a centred at (x,y)
 * along angle th): closest point q of the segment, d_min = r. */
static ow_contact sphere_line(const ow_body *s, const ow_body *l) {
  ow_contact r;
  memset(&r, 0, sizeof r);
  r.margin = INFINITY;
  double ux = cos(l->th), uy = sin(l->th);
  double ax = l->x - 0.5 * l->a * ux, ay = l->y - 0.5 * l->a * uy;
  double bx = l->x + 0.5 * l->a * ux, by = l->y + 0.5 * l->a * uy;
  double ex = bx - ax, ey = by - ay;
  double len2 = ex * ex + ey * ey;
  double t = 0.5;
  if (len2 > 0) t = ((s->x - ax) * ex + (s->y - ay) * ey) / len2;
  t = clampd(t, 0.0, 1.0);
  double qx = ax + t * ex, qy = ay + t * ey;
  double dx = s->x - qx, dy = s->y - qy;
  double dist = sqrt(dx * dx + dy * dy);
  r.g = dist - s->a;
  if (dist > 0) {
    r.nx = dx / dist;
    r.ny = dy / dist;
    r.has_normal = 1;
  }
  r.pix = s->x - s->a * r.nx;
  r.piy = s->y - s->a * r.ny;
  r.pjx = qx;
  r.pjy = qy;
  return r;
}

/* Sphere s - box b (width a, height b, rotated by th).  Outside: clamp the
 * centre into the box in box coordinates.  Centre inside (or on the edge):
 * push out through the face of least depth, faces ordered +x, -x, +y, -y
 * (Reading R9), with the gap negative by that depth. */
static ow_contact sphere_box(const ow_body *s, const ow_body *b) {
  ow_contact r;
  memset(&r, 0, sizeof r);
  r.margin = INFINITY;
  double c = cos(b->th), sn = sin(b->th);
  double dx = s->x - b->x, dy = s->y - b->y;
  double lx = c * dx + sn * dy;  /* box-local coordinates: R(-th) d */
  double ly = -sn * dx + c * dy;
  double hw = 0.5 * b->a, hh = 0.5 * b->b;
  double qx, qy, nlx, nly;
  if (fabs(lx) <= hw && fabs(ly) <= hh) {
    double depth[4] = {hw - lx, hw + lx, hh - ly, hh + ly};
    int f = 0;
    for (int q = 1; q < 4; ++q)
      if (depth[q] < depth[f]) f = q;
    for (int q = 0; q < 4; ++q) /* runner-up face */
      if (q != f && depth[q] - depth[f] < r.margin) r.margin = depth[q] - depth[f];
    if (f == 0) { nlx = 1; nly = 0; qx = hw; qy = ly; }
    else if (f == 1) { nlx = -1; nly = 0; qx = -hw; qy = ly; }
    else if (f == 2) { nlx = 0; nly = 1; qx = lx; qy = hh; }
    else { nlx = 0; nly = -1; qx = lx; qy = -hh; }
    r.g = -depth[f] - s->a;
    r.has_normal = 1;
  } else {
    qx = clampd(lx, -hw, hw);
    qy = clampd(ly, -hh, hh);
    double ex = lx - qx, ey = ly - qy;
    double dist = sqrt(ex * ex + ey * ey);
    nlx = ex / dist;
    nly = ey / dist;
    r.g = dist - s->a;
    r.has_normal = 1;
  }
  r.nx = c * nlx - sn * nly; /* back to world: R(th) n_local */
  r.ny = sn * nlx + c * nly;
  r.pjx = b->x + c * qx - sn * qy;
  r.pjy = b->y + sn * qx + c * qy;
  r.pix = s->x - s->a * r.nx;
  r.piy = s->y - s->a * r.ny;
  return r;
}

/* ---- closest points, polygon cases (box-box, box-line, line-line) --------
 * A box is the polygon of its 4 corners, counter-clockwise from the local
 * (-w/2, -h/2) corner; its edge k runs from corner k to corner k+1 (edge 0
 * faces local -y, 1 faces +x, 2 faces +y, 3 faces -x).  A line is the
 * 2-vertex polygon (centre -/+ L/2 along its direction) with one edge. */
typedef struct {
  int nv, ne;
  double vx[4], vy[4];
  double enx[4], eny[4]; /* outward edge normals (boxes only) */
} ow_poly;

static void make_poly(const ow_body *b, ow_poly *p) {
  double c = cos(b->th), s = sin(b->th);
  if (b->shape == OW_BOX) {
    double hw = 0.5 * b->a, hh = 0.5 * b->b;
    double lx[4] = {-hw, hw, hw, -hw}, ly[4] = {-hh, -hh, hh, hh};
    double nlx[4] = {0, 1, 0, -1}, nly[4] = {-1, 0, 1, 0};
    p->nv = 4;
    p->ne = 4;
    for (int q = 0; q < 4; ++q) {
      p->vx[q] = b->x + c * lx[q] - s * ly[q];
      p->vy[q] = b->y + s * lx[q] + c * ly[q];
      p->enx[q] = c * nlx[q] - s * nly[q];
      p->eny[q] = s * nlx[q] + c * nly[q];
    }
  } else {
    double h = 0.5 * b->a;
    p->nv = 2;
    p->ne = 1;
    p->vx[0] = b->x - h * c;
    p->vy[0] = b->y - h * s;
    p->vx[1] = b->x + h * c;
    p->vy[1] = b->y + h * s;
    p->enx[0] = -s; /* one of the two normals; only used for boxes */
    p->eny[0] = c;
  }
}

static void edge_of(const ow_poly *p, int e, double *ax, double *ay,
                    double *bx, double *by) {
  int e1 = (e + 1) % p->nv;
  *ax = p->vx[e];
  *ay = p->vy[e];
  *bx = p->vx[e1];
  *by = p->vy[e1];
}

/* Half-extent of a box or line along the unit direction (ux, uy). */
static double half_extent(const ow_body *b, double ux, double uy) {
  double c = cos(b->th), s = sin(b->th);
  double along = ux * c + uy * s;   /* u . e1 (direction of width / length) */
  double across = -ux * s + uy * c; /* u . e2                                */
  if (b->shape == OW_BOX) return 0.5 * b->a * fabs(along) + 0.5 * b->b * fabs(across);
  return 0.5 * b->a * fabs(along);
}

/* Separating-axis candidates of one body: box -> its two axes, line -> its
 * normal. */
static int body_axes(const ow_body *b, double *ax, double *ay) {
  double c = cos(b->th), s = sin(b->th);
  if (b->shape == OW_BOX) {
    ax[0] = c; ay[0] = s;
    ax[1] = -s; ay[1] = c;
    return 2;
  }
  ax[0] = -s; ay[0] = c;
  return 1;
}

/* Closest point of segment [a, b] to point p (the textbook projection). */
static void closest_on_segment(double px, double py, double ax, double ay,
                               double bx, double by, double *qx, double *qy) {
  double ex = bx - ax, ey = by - ay;
  double len2 = ex * ex + ey * ey;
  double t = 0.0;
  if (len2 > 0) t = clampd(((px - ax) * ex + (py - ay) * ey) / len2, 0.0, 1.0);
  *qx = ax + t * ex;
  *qy = ay + t * ey;
}

static ow_contact poly_poly(const ow_body *bi, const ow_body *bj) {
  ow_contact r;
  memset(&r, 0, sizeof r);
  r.margin = INFINITY;
  double depth_all[5];
  double ax[5], ay[5];
  int nai = body_axes(bi, ax, ay);
  int naj = body_axes(bj, ax + nai, ay + nai);
  int na = nai + naj;
  /* Two exactly parallel lines: their normals coincide and miss the axis
   * along the lines, so add line i's direction. */
  if (bi->shape == OW_LINE && bj->shape == OW_LINE) {
    double ci = cos(bi->th), si = sin(bi->th), cj = cos(bj->th), sj = sin(bj->th);
    r.margin = fabs(ci * sj - si * cj);
    if (ci * sj - si * cj == 0) {
      ax[na] = ci;
      ay[na] = si;
      ++na;
    }
  }
  double best = INFINITY;
  int bk = -1;
  for (int q = 0; q < na; ++q) {
    double delta = (bi->x - bj->x) * ax[q] + (bi->y - bj->y) * ay[q];
    double depth = half_extent(bi, ax[q], ay[q]) + half_extent(bj, ax[q], ay[q]) - fabs(delta);
    depth_all[q] = depth;
    if (depth < best) {
      best = depth;
      bk = q;
    }
  }
  ow_poly pi, pj;
  make_poly(bi, &pi);
  make_poly(bj, &pj);

  if (best < 0) {
    /* Separated: the distance of two convex polygons is the least
     * vertex-to-edge distance, taken both ways (vertices of i against edges
     * of j first, then vertices of j against edges of i). */
    double dbest = INFINITY;
    for (int v = 0; v < pi.nv; ++v)
      for (int e = 0; e < pj.ne; ++e) {
        double a0, a1, b0, b1, qx, qy;
        edge_of(&pj, e, &a0, &a1, &b0, &b1);
        closest_on_segment(pi.vx[v], pi.vy[v], a0, a1, b0, b1, &qx, &qy);
        double d = sqrt((pi.vx[v] - qx) * (pi.vx[v] - qx) + (pi.vy[v] - qy) * (pi.vy[v] - qy));
        if (d < dbest) {
          dbest = d;
          r.pix = pi.vx[v]; r.piy = pi.vy[v];
          r.pjx = qx; r.pjy = qy;
        }
      }
    for (int v = 0; v < pj.nv; ++v)
      for (int e = 0; e < pi.ne; ++e) {
        double a0, a1, b0, b1, qx, qy;
        edge_of(&pi, e, &a0, &a1, &b0, &b1);
        closest_on_segment(pj.vx[v], pj.vy[v], a0, a1, b0, b1, &qx, &qy);
        double d = sqrt((pj.vx[v] - qx) * (pj.vx[v] - qx) + (pj.vy[v] - qy) * (pj.vy[v] - qy));
        if (d < dbest) {
          dbest = d;
          r.pix = qx; r.piy = qy;
          r.pjx = pj.vx[v]; r.pjy = pj.vy[v];
        }
      }
    r.g = dbest;
    if (dbest > 0) {
      r.nx = (r.pix - r.pjx) / dbest;
      r.ny = (r.piy - r.pjy) / dbest;
      r.has_normal = 1;
    }
    return r;
  }

  /* Overlapping (or touching): gap = -(least depth), normal = that axis
   * turned to point from j towards i. */
  double ux = ax[bk], uy = ay[bk];
  double delta = (bi->x - bj->x) * ux + (bi->y - bj->y) * uy;
  for (int q = 0; q < na; ++q) /* runner-up separating axis */
    if (q != bk && depth_all[q] - best < r.margin) r.margin = depth_all[q] - best;
  if (fabs(delta) < r.margin) r.margin = fabs(delta); /* orientation of the normal */
  if (delta < 0) { ux = -ux; uy = -uy; }
  r.g = -best;
  r.nx = ux;
  r.ny = uy;
  r.has_normal = 1;

  /* Reading R16: the body owning the axis is the reference R, the other the
   * incident Q.  nR is R's outward normal towards Q. */
  int ref_is_i = bk < nai;
  const ow_body *bR = ref_is_i ? bi : bj;
  const ow_poly *pR = ref_is_i ? &pi : &pj;
  const ow_poly *pQ = ref_is_i ? &pj : &pi;
  double nRx = ref_is_i ? -ux : ux, nRy = ref_is_i ? -uy : uy;
  int kR = ref_is_i ? bk : bk - nai; /* which axis of R */

  /* Reference face [fa, fb]. */
  int have_face = 1;
  double fax = 0, fay = 0, fbx = 0, fby = 0;
  if (bR->shape == OW_BOX) {
    /* axis 0 is e1 (faces +x: edge 1, -x: edge 3), axis 1 is e2 (+y: edge 2,
     * -y: edge 0); the sign of nR along the axis picks the face. */
    double dotn = nRx * ax[bk] + nRy * ay[bk];
    int e;
    if (kR == 0) e = dotn > 0 ? 1 : 3;
    else e = dotn > 0 ? 2 : 0;
    edge_of(pR, e, &fax, &fay, &fbx, &fby);
  } else if (kR == 0) {
    edge_of(pR, 0, &fax, &fay, &fbx, &fby);
  } else {
    have_face = 0; /* the extra along-line axis of two parallel lines */
  }

  /* Incident edge of Q: the one whose outward normal is most opposed to nR
   * (edges in order, strict "<"); a line's only edge is itself. */
  double i0x, i0y, i1x, i1y;
  if (pQ->nv == 4) {
    int e = 0;
    double bestdot = INFINITY;
    for (int q = 0; q < 4; ++q) {
      double d = pQ->enx[q] * nRx + pQ->eny[q] * nRy;
      if (d < bestdot) { bestdot = d; e = q; }
    }
    for (int q = 0; q < 4; ++q) { /* runner-up incident edge */
      double d = pQ->enx[q] * nRx + pQ->eny[q] * nRy;
      if (q != e && d - bestdot < r.margin) r.margin = d - bestdot;
    }
    edge_of(pQ, e, &i0x, &i0y, &i1x, &i1y);
  } else {
    edge_of(pQ, 0, &i0x, &i0y, &i1x, &i1y);
  }

  /* Clip the incident edge to the span of the reference face, then weight
   * the clipped ends by how far each lies beneath the face. */
  int have_point = 0;
  double qx = 0, qy = 0;
  if (have_face) {
    double tx = fbx - fax, ty = fby - fay;
    double flen = sqrt(tx * tx + ty * ty);
    if (flen > 0) {
      tx /= flen;
      ty /= flen;
      double s0 = (i0x - fax) * tx + (i0y - fay) * ty;
      double s1 = (i1x - fax) * tx + (i1y - fay) * ty;
      double lo, hi;
      int nonempty;
      double ilen = sqrt((i1x - i0x) * (i1x - i0x) + (i1y - i0y) * (i1y - i0y));
      if (s1 == s0) {
        lo = 0.0;
        hi = 1.0;
        nonempty = (s0 >= 0 && s0 <= flen);
        double mc = fmin(fabs(s0), fabs(flen - s0)); /* span test */
        if (mc < r.margin) r.margin = mc;
      } else {
        double la = (0.0 - s0) / (s1 - s0), lb = (flen - s0) / (s1 - s0);
        lo = la < lb ? la : lb;
        hi = la < lb ? lb : la;
        if (lo < 0) lo = 0;
        if (hi > 1) hi = 1;
        nonempty = lo <= hi;
        double mc = fabs(hi - lo) * ilen; /* clipped length (or gap) */
        if (mc < r.margin) r.margin = mc;
      }
      if (nonempty) {
        double c0x = i0x + lo * (i1x - i0x), c0y = i0y + lo * (i1y - i0y);
        double c1x = i0x + hi * (i1x - i0x), c1y = i0y + hi * (i1y - i0y);
        double d0 = -((c0x - fax) * nRx + (c0y - fay) * nRy);
        double d1 = -((c1x - fax) * nRx + (c1y - fay) * nRy);
        double w0 = d0 > 0 ? d0 : 0, w1 = d1 > 0 ? d1 : 0;
        if (fabs(fmax(d0, d1)) < r.margin) r.margin = fabs(fmax(d0, d1)); /* midpoint rule */
        if (w0 + w1 > 0) {
          qx = (w0 * c0x + w1 * c1x) / (w0 + w1);
          qy = (w0 * c0y + w1 * c1y) / (w0 + w1);
        } else {
          qx = 0.5 * (c0x + c1x);
          qy = 0.5 * (c0y + c1y);
        }
        have_point = 1;
      }
    }
  }
  if (!have_point) {
    /* Fallback: Q's deepest vertex along -nR (vertices in order). */
    int v = 0;
    double bestp = INFINITY;
    for (int q = 0; q < pQ->nv; ++q) {
      double p = pQ->vx[q] * nRx + pQ->vy[q] * nRy;
      if (p < bestp) { bestp = p; v = q; }
    }
    for (int q = 0; q < pQ->nv; ++q) { /* runner-up deepest vertex */
      double p = pQ->vx[q] * nRx + pQ->vy[q] * nRy;
      if (q != v && p - bestp < r.margin) r.margin = p - bestp;
    }
    qx = pQ->vx[v];
    qy = pQ->vy[v];
  }
  if (ref_is_i) {
    r.pjx = qx; r.pjy = qy;
    r.pix = qx + r.g * r.nx;
    r.piy = qy + r.g * r.ny;
  } else {
    r.pix = qx; r.piy = qy;
    r.pjx = qx - r.g * r.nx;
    r.pjy = qy - r.g * r.ny;
  }
  return r;
}

/* Swap the roles of a contact computed for (j, i) so it reads for (i, j). */
static ow_contact swap_contact(ow_contact c) {
  ow_contact r = c;
  r.nx = -c.nx;
  r.ny = -c.ny;
  r.pix = c.pjx; r.piy = c.pjy;
  r.pjx = c.pix; r.pjy = c.piy;
  return r;
}

/* Closest points and signed gap of the ordered pair (i, j). */
static ow_contact pair_geometry(const ow_body *bi, const ow_body *bj) {
  int si = bi->shape, sj = bj->shape;
  if (si == OW_SPHERE && sj == OW_SPHERE) return sphere_sphere(bi, bj);
  if (si == OW_SPHERE && sj == OW_LINE) return sphere_line(bi, bj);
  if (si == OW_LINE && sj == OW_SPHERE) return swap_contact(sphere_line(bj, bi));
  if (si == OW_SPHERE && sj == OW_BOX) return sphere_box(bi, bj);
  if (si == OW_BOX && sj == OW_SPHERE) return swap_contact(sphere_box(bj, bi));
  return poly_poly(bi, bj);
}

/* Reading R4: default moment of inertia when the input is 0. */
static double inertia_of(int shape, double m, double a, double b, double given) {
  if (given != 0) return given;
  if (shape == OW_BOX) return m * (a * a + b * b) / 12.0;
  if (shape == OW_LINE) return m * a * a / 12.0;
  return 0.5 * m * a * a;
}

/* Reading R15. */
static int pair_active(uint8_t fi, uint8_t fj) {
  if (!(fi & OW_COLLIDABLE) || !(fj & OW_COLLIDABLE)) return 0;
  return ((fi | fj) & (OW_MOVABLE | OW_ROTATABLE)) != 0;
}

/* Eq. 2 with Reading R2: force magnitude c*k*softplus(-gap/k) when the gap
 * is <= 0, along the unit normal. */
static double contact_magnitude(double c, double k, double gap) {
  return c * k * softplus(-gap / k);
}

static void load_body(const ow_world *w, const double *st, size_t base, int i,
                      ow_body *b) {
  b->shape = w->shape[base + i];
  b->x = st[6 * i + 0];
  b->y = st[6 * i + 1];
  b->th = st[6 * i + 4];
  b->a = w->size_a[base + i];
  b->b = w->size_b[base + i];
}

/* One call = one world step of one environment: S substeps of Eqs. 1-3.
 * st points at that env's [n_entities][6] state (x, y, vx, vy, th, om);
 * act at its [n_actuated][3] actions (fx, fy, torque). */
static void step_env(const ow_world *w, int e, double *st, const double *act,
                     double *F, double *T, double *margin) {
  int N = w->n_entities;
  size_t base = (size_t)e * N;
  double h = w->dt / w->substeps; /* Reading R5 */
  for (int s = 0; s < w->substeps; ++s) {
    /* Eq. 1, first line, action and gravity terms. */
    int a = 0;
    for (int i = 0; i < N; ++i) {
      uint8_t f = w->flags[base + i];
      F[2 * i] = 0;
      F[2 * i + 1] = 0;
      T[i] = 0;
      if (f & OW_ACTUATED) {
        F[2 * i] = act[3 * a + 0];
        F[2 * i + 1] = act[3 * a + 1];
        T[i] = act[3 * a + 2];
        ++a;
      }
      double m = w->mass[base + i];
      F[2 * i] += m * w->gx;
      F[2 * i + 1] += m * w->gy;
    }
    /* Eq. 1 sum and Eq. 3 torque: every pair i < j in canonical order. */
    for (int i = 0; i < N; ++i) {
      for (int j = i + 1; j < N; ++j) {
        if (!pair_active(w->flags[base + i], w->flags[base + j])) continue;
        ow_body bi, bj;
        load_body(w, st, base, i, &bi);
        load_body(w, st, base, j, &bj);
        ow_contact c = pair_geometry(&bi, &bj);
        if (margin) { /* Reading R9: the contact decision g <= 0, and the choices behind a contact */
          double m = fabs(c.g);
          if (c.g <= 0 && c.has_normal && c.margin < m) m = c.margin;
          if (m < *margin) *margin = m;
        }
        if (!(c.g <= 0) || !c.has_normal) continue; /* Readings R2, R8 */
        double mag = contact_magnitude(w->c, w->k, c.g);
        double fx = mag * c.nx, fy = mag * c.ny;
        F[2 * i] += fx;
        F[2 * i + 1] += fy;
        F[2 * j] -= fx;
        F[2 * j + 1] -= fy;
        /* Reading R3: signed cross product r x f. */
        T[i] += (c.pix - bi.x) * fy - (c.piy - bi.y) * fx;
        T[j] += (c.pjx - bj.x) * (-fy) - (c.pjy - bj.y) * (-fx);
      }
    }
    /* Eq. 1 (lines 2-3) and Eq. 3 (lines 2-3): damped semi-implicit Euler. */
    for (int i = 0; i < N; ++i) {
      uint8_t f = w->flags[base + i];
      double *x = st + 6 * i;
      if (f & OW_MOVABLE) { /* Reading R6 */
        double m = w->mass[base + i];
        x[2] = (1.0 - w->drag) * x[2] + F[2 * i] / m * h;
        x[3] = (1.0 - w->drag) * x[3] + F[2 * i + 1] / m * h;
        if (w->max_speed > 0) { /* Reading R7 */
          double sp = sqrt(x[2] * x[2] + x[3] * x[3]);
          if (sp > w->max_speed) {
            x[2] = x[2] * (w->max_speed / sp);
            x[3] = x[3] * (w->max_speed / sp);
          }
        }
        x[0] = x[0] + x[2] * h;
        x[1] = x[1] + x[3] * h;
      }
      if (f & OW_ROTATABLE) {
        double I = inertia_of(w->shape[base + i], w->mass[base + i], w->size_a[base + i],
                              w->size_b[base + i], w->inertia[base + i]);
        x[5] = (1.0 - w->drag) * x[5] + T[i] / I * h;
        x[4] = x[4] + x[5] * h;
      }
    }
  }
}

/* ---------------------------------------------------------------- exports */

static int ow_threads(int t) {
#ifdef _OPENMP
  return t > 0 ? t : omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}

/* Advance every environment by n_steps world steps.
 * state   : [n_envs][n_entities][6], updated in place.
 * actions : [n_steps][n_envs][n_actuated][3]; the k-th actuated entity of an
 *           env (in entity order) reads row k.
 * threads : OpenMP threads over environments (<= 0: library default). */
static int step_all(const ow_world *w, double *state, const double *actions, int n_steps,
                    int threads, double *margin) {
  int E = w->n_envs, N = w->n_entities, A = w->n_actuated;
  if (E < 0 || N < 0 || A < 0 || w->substeps < 1 || n_steps < 0) return -1;
  if (margin)
    for (int e = 0; e < E; ++e) margin[e] = INFINITY;
  int nt = ow_threads(threads);
  (void)nt;
#pragma omp parallel num_threads(nt)
  {
    double *F = (double *)malloc(sizeof(double) * 2 * (N > 0 ? N : 1));
    double *T = (double *)malloc(sizeof(double) * (N > 0 ? N : 1));
    for (int t = 0; t < n_steps; ++t) {
#pragma omp for schedule(static)
      for (int e = 0; e < E; ++e)
        step_env(w, e, state + (size_t)e * N * 6,
                 actions + ((size_t)t * E + e) * A * 3, F, T, margin ? margin + e : NULL);
    }
    free(F);
    free(T);
  }
  return 0;
}

int ow_step(const ow_world *w, double *state, const double *actions, int n_steps,
            int threads) {
  return step_all(w, state, actions, n_steps, threads, NULL);
}

/* As ow_step, and margin [n_envs] receives, per env, the smallest decision
 * margin met over all substeps (Reading R9): the least |gap| of any active
 * pair (the case split of Eq. 2) and, for pairs in contact, the margin of
 * the geometry's discrete choices (see ow_contact.margin).  A result that
 * differs between two correct implementations in different precisions
 * (FP32 against FP64) can only come from a choice whose margin is within
 * their rounding difference. */
int ow_step_margin(const ow_world *w, double *state, const double *actions, int n_steps,
                   int threads, double *margin) {
  return step_all(w, state, actions, n_steps, threads, margin);
}

/* Canonical unordered pair list: (i, j), i < j, row-major. */
int ow_pair_list(int n, int32_t *pi, int32_t *pj) {
  int p = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      pi[p] = i;
      pj[p] = j;
      ++p;
    }
  return p;
}

/* First-substep contact mask and gap for every pair of every env, from the
 * given state: mask = pair active (Reading R15) and gap <= 0 with a defined
 * normal; gap is reported for every active pair (INFINITY for the others). */
int ow_pairs(const ow_world *w, const double *state, uint8_t *mask, double *gap) {
  int E = w->n_envs, N = w->n_entities;
  size_t P = (size_t)N * (N - 1) / 2;
  for (int e = 0; e < E; ++e) {
    size_t base = (size_t)e * N;
    const double *st = state + base * 6;
    size_t p = 0;
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j, ++p) {
        uint8_t fi = w->flags[base + i], fj = w->flags[base + j];
        if (!pair_active(fi, fj)) {
          mask[e * P + p] = 0;
          gap[e * P + p] = INFINITY;
          continue;
        }
        ow_body bi, bj;
        load_body(w, st, base, i, &bi);
        load_body(w, st, base, j, &bj);
        ow_contact c = pair_geometry(&bi, &bj);
        gap[e * P + p] = c.g;
        mask[e * P + p] = (uint8_t)(c.g <= 0 && c.has_normal);
      }
  }
  return 0;
}

/* Closest points of one ordered pair.  body = {shape, x, y, th, a, b};
 * out = {g, nx, ny, pix, piy, pjx, pjy}; returns has_normal. */
int ow_pair_geometry(const double *body_i, const double *body_j, double *out) {
  ow_body bi = {(int)body_i[0], body_i[1], body_i[2], body_i[3], body_i[4], body_i[5]};
  ow_body bj = {(int)body_j[0], body_j[1], body_j[2], body_j[3], body_j[4], body_j[5]};
  ow_contact c = pair_geometry(&bi, &bj);
  out[0] = c.g;
  out[1] = c.nx;
  out[2] = c.ny;
  out[3] = c.pix;
  out[4] = c.piy;
  out[5] = c.pjx;
  out[6] = c.pjy;
  return c.has_normal;
}

/* Eq. 2 magnitude, exported for the tests of Reading R1/R2. */
double ow_contact_magnitude(double c, double k, double gap) {
  return contact_magnitude(c, k, gap);
}

/* Reading R4, exported for tests. */
double ow_inertia(int shape, double m, double a, double b, double given) {
  return inertia_of(shape, m, a, b, given);
}

int ow_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- adjoint
 * Gradient of a differentiable rollout (sphere worlds), FP64.
 *
 * Forward: T world steps of Eqs. 1-3 from `state` with actions
 * [T][E][A][3]; loss per env = sum over actuated entities k of
 * |x_k(T) - goal_k|^2.  Backward: reverse-mode through every substep.  With
 * a = 1 - zeta and h = dt / S, one substep of a movable sphere is
 *   F_i = f^a_i + m_i g + sum_j f_ij,   v_i' = a v_i + (h / m_i) F_i,
 *   x_i' = x_i + h v_i',
 * and the pair force f_ij = M(g) u, u = d / |d|, d = x_i - x_j,
 * g = |d| - (r_i + r_j), M(g) = c k softplus(-g / k) (g <= 0, Eq. 2), whose
 * Jacobian is J = dM/dg u u^T + M / |d| (I - u u^T), dM/dg = -c sigmoid(-g/k).
 * The contact mask is treated as piecewise constant (Reading R2: no term
 * from the jump at g = 0).  Adjoints, given lx', lv' of a substep's outputs:
 *   lv'' = lv' + h lx',  lx = lx' + sum over pairs of J (lF_i - lF_j) terms,
 *   lv = a lv'',  lF_i = (h / m_i) lv''_i,  d loss / d f^a_i += lF_i.
 * Forces on immovable entities are dropped (Reading R6), so their lF is 0. */

static void sphere_pair_force(const double *xi, const double *xj, double ri, double rj,
                              double c, double k, int *hit, double f[2], double J[4]) {
  double dx = xi[0] - xj[0], dy = xi[1] - xj[1];
  double s = sqrt(dx * dx + dy * dy);
  double g = s - (ri + rj);
  *hit = (g <= 0 && s > 0);
  if (!*hit) return;
  double ux = dx / s, uy = dy / s;
  double M = contact_magnitude(c, k, g);
  double sig = 1.0 / (1.0 + exp(g / k)); /* sigmoid(-g/k) */
  double dM = -c * sig;
  f[0] = M * ux;
  f[1] = M * uy;
  double t = M / s;
  J[0] = dM * ux * ux + t * (1 - ux * ux);
  J[1] = dM * ux * uy - t * ux * uy;
  J[2] = J[1];
  J[3] = dM * uy * uy + t * (1 - uy * uy);
}

/* Forward of one env through T steps, recording (x, y, vx, vy) at every
 * substep start into traj [(T*S + 1)][N][4]; returns the final loss. */
static double rollout_env(const ow_world *w, int e, const double *st0, const double *act_all,
                          int T, const double *goals, double *traj) {
  int N = w->n_entities, A = w->n_actuated, S = w->substeps, E = w->n_envs;
  size_t base = (size_t)e * N;
  double h = w->dt / S;
  double *F = (double *)malloc(sizeof(double) * 2 * N);
  double *cur = (double *)malloc(sizeof(double) * 4 * N);
  for (int i = 0; i < N; ++i) {
    cur[4 * i + 0] = st0[6 * i + 0];
    cur[4 * i + 1] = st0[6 * i + 1];
    cur[4 * i + 2] = st0[6 * i + 2];
    cur[4 * i + 3] = st0[6 * i + 3];
  }
  int q = 0;
  memcpy(traj, cur, sizeof(double) * 4 * N);
  for (int t = 0; t < T; ++t) {
    const double *act = act_all + ((size_t)t * E + e) * A * 3;
    for (int s = 0; s < S; ++s) {
      int a = 0;
      for (int i = 0; i < N; ++i) {
        uint8_t fl = w->flags[base + i];
        double m = w->mass[base + i];
        F[2 * i] = m * w->gx;
        F[2 * i + 1] = m * w->gy;
        if (fl & OW_ACTUATED) {
          F[2 * i] += act[3 * a];
          F[2 * i + 1] += act[3 * a + 1];
          ++a;
        }
      }
      for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
          if (!pair_active(w->flags[base + i], w->flags[base + j])) continue;
          int hit;
          double f[2], J[4];
          sphere_pair_force(cur + 4 * i, cur + 4 * j, w->size_a[base + i], w->size_a[base + j],
                            w->c, w->k, &hit, f, J);
          if (!hit) continue;
          F[2 * i] += f[0];
          F[2 * i + 1] += f[1];
          F[2 * j] -= f[0];
          F[2 * j + 1] -= f[1];
        }
      for (int i = 0; i < N; ++i) {
        if (!(w->flags[base + i] & OW_MOVABLE)) continue;
        double m = w->mass[base + i];
        cur[4 * i + 2] = (1.0 - w->drag) * cur[4 * i + 2] + F[2 * i] / m * h;
        cur[4 * i + 3] = (1.0 - w->drag) * cur[4 * i + 3] + F[2 * i + 1] / m * h;
        cur[4 * i + 0] += cur[4 * i + 2] * h;
        cur[4 * i + 1] += cur[4 * i + 3] * h;
      }
      ++q;
      memcpy(traj + (size_t)q * 4 * N, cur, sizeof(double) * 4 * N);
    }
  }
  double loss = 0;
  int a = 0;
  for (int i = 0; i < N; ++i)
    if (w->flags[base + i] & OW_ACTUATED) {
      double dx = cur[4 * i] - goals[((size_t)e * A + a) * 2];
      double dy = cur[4 * i + 1] - goals[((size_t)e * A + a) * 2 + 1];
      loss += dx * dx + dy * dy;
      ++a;
    }
  free(F);
  free(cur);
  return loss;
}

/* Differentiable rollout of sphere worlds.  state [E][N][6] (only x, y, vx,
 * vy are used), actions [T][E][A][3], goals [E][A][2].  loss [E] receives
 * each env's loss; grad (if not NULL) [T][E][A][3] receives d loss_e /
 * d action (torque component 0).  Returns -1 if a non-sphere entity or a
 * speed cap is present. */
int ow_rollout_grad(const ow_world *w, const double *state, const double *actions, int T,
                    const double *goals, double *loss, double *grad) {
  int E = w->n_envs, N = w->n_entities, A = w->n_actuated, S = w->substeps;
  if (w->max_speed > 0) return -1;
  for (size_t t = 0; t < (size_t)E * N; ++t)
    if (w->shape[t] != OW_SPHERE) return -1;
  double h = w->dt / S, a_drag = 1.0 - w->drag;
  size_t Q = (size_t)T * S + 1;
  double *traj = (double *)malloc(sizeof(double) * Q * 4 * N);
  double *lx = (double *)malloc(sizeof(double) * 2 * N);
  double *lv = (double *)malloc(sizeof(double) * 2 * N);
  double *lF = (double *)malloc(sizeof(double) * 2 * N);
  for (int e = 0; e < E; ++e) {
    size_t base = (size_t)e * N;
    loss[e] = rollout_env(w, e, state + base * 6, actions, T, goals, traj);
    if (!grad) continue;
    /* d loss / d x(T) = 2 (x - goal); d loss / d v(T) = 0 */
    const double *fin = traj + (Q - 1) * 4 * N;
    int a = 0;
    for (int i = 0; i < N; ++i) {
      lx[2 * i] = lx[2 * i + 1] = 0;
      lv[2 * i] = lv[2 * i + 1] = 0;
      if (w->flags[base + i] & OW_ACTUATED) {
        lx[2 * i] = 2 * (fin[4 * i] - goals[((size_t)e * A + a) * 2]);
        lx[2 * i + 1] = 2 * (fin[4 * i + 1] - goals[((size_t)e * A + a) * 2 + 1]);
        ++a;
      }
    }
    for (int t = T - 1; t >= 0; --t) {
      double *gact = grad + ((size_t)t * E + e) * A * 3;
      for (int q = 0; q < A * 3; ++q) gact[q] = 0;
      for (int s = S - 1; s >= 0; --s) {
        const double *cur = traj + ((size_t)t * S + s) * 4 * N; /* substep start */
        /* through x' = x + h v' and v' = a v + (h/m) F */
        for (int i = 0; i < N; ++i) {
          lF[2 * i] = lF[2 * i + 1] = 0;
          if (!(w->flags[base + i] & OW_MOVABLE)) continue;
          double m = w->mass[base + i];
          double lvx = lv[2 * i] + h * lx[2 * i], lvy = lv[2 * i + 1] + h * lx[2 * i + 1];
          lF[2 * i] = h / m * lvx;
          lF[2 * i + 1] = h / m * lvy;
          lv[2 * i] = a_drag * lvx;
          lv[2 * i + 1] = a_drag * lvy;
        }
        /* actions feed F directly */
        int k = 0;
        for (int i = 0; i < N; ++i)
          if (w->flags[base + i] & OW_ACTUATED) {
            gact[3 * k] += lF[2 * i];
            gact[3 * k + 1] += lF[2 * i + 1];
            ++k;
          }
        /* contact forces depend on positions at the substep start */
        for (int i = 0; i < N; ++i)
          for (int j = i + 1; j < N; ++j) {
            if (!pair_active(w->flags[base + i], w->flags[base + j])) continue;
            int hit;
            double f[2], J[4];
            sphere_pair_force(cur + 4 * i, cur + 4 * j, w->size_a[base + i],
                              w->size_a[base + j], w->c, w->k, &hit, f, J);
            if (!hit) continue;
            double dx = lF[2 * i] - lF[2 * j], dy = lF[2 * i + 1] - lF[2 * j + 1];
            double gx = J[0] * dx + J[1] * dy, gy = J[2] * dx + J[3] * dy;
            lx[2 * i] += gx;
            lx[2 * i + 1] += gy;
            lx[2 * j] -= gx;
            lx[2 * j + 1] -= gy;
          }
      }
    }
  }
  free(traj);
  free(lx);
  free(lv);
  free(lF);
  return 0;
}

/* ------------------------------------------------------------------ LIDAR
 * Ray casts (section 3: agents can carry LIDAR sensors).  Every actuated
 * entity casts n_rays rays from its centre at angles th + 2 pi k / n_rays
 * (k = 0 .. n_rays-1); a ray reports the smallest distance t in [0, range]
 * at which it meets another collidable entity (0 when its origin is inside
 * one), or `range` when it meets none.  The caster itself is excluded.
 * Shapes: sphere = disc of radius r, box = filled rectangle, line = segment
 * (a ray exactly parallel to a segment does not meet it). */

/* Smallest t >= 0 at which o + t d enters the shape, or INFINITY. */
static double ray_shape(double ox, double oy, double dx, double dy, const ow_body *b) {
  if (b->shape == OW_SPHERE) {
    double px = ox - b->x, py = oy - b->y;
    double c = px * px + py * py - b->a * b->a;
    if (c <= 0) return 0.0; /* origin inside */
    double bq = px * dx + py * dy;
    double disc = bq * bq - c;
    if (disc < 0) return INFINITY;
    double t = -bq - sqrt(disc);
    return t >= 0 ? t : INFINITY;
  }
  double cs = cos(b->th), sn = sin(b->th);
  /* ray in the body frame */
  double lx = cs * (ox - b->x) + sn * (oy - b->y), ly = -sn * (ox - b->x) + cs * (oy - b->y);
  double ldx = cs * dx + sn * dy, ldy = -sn * dx + cs * dy;
  if (b->shape == OW_BOX) {
    double hw = 0.5 * b->a, hh = 0.5 * b->b;
    if (fabs(lx) <= hw && fabs(ly) <= hh) return 0.0;
    /* slabs */
    double tmin = -INFINITY, tmax = INFINITY;
    double o[2] = {lx, ly}, d[2] = {ldx, ldy}, h[2] = {hw, hh};
    for (int q = 0; q < 2; ++q) {
      if (d[q] == 0) {
        if (fabs(o[q]) > h[q]) return INFINITY;
      } else {
        double t1 = (-h[q] - o[q]) / d[q], t2 = (h[q] - o[q]) / d[q];
        if (t1 > t2) { double tt = t1; t1 = t2; t2 = tt; }
        if (t1 > tmin) tmin = t1;
        if (t2 < tmax) tmax = t2;
      }
    }
    if (tmin > tmax || tmax < 0) return INFINITY;
    return tmin >= 0 ? tmin : 0.0;
  }
  /* line: segment from (-L/2, 0) to (L/2, 0) in the body frame */
  if (ldy == 0) return INFINITY;
  double t = -ly / ldy;
  if (t < 0) return INFINITY;
  double xh = lx + t * ldx;
  if (fabs(xh) > 0.5 * b->a) return INFINITY;
  return t;
}

/* out [E][A][n_rays]; rows of actuated slots an env does not use stay at
 * `range`. */
int ow_lidar(const ow_world *w, const double *state, int n_rays, double range, double *out) {
  int E = w->n_envs, N = w->n_entities, A = w->n_actuated;
  const double two_pi = 6.283185307179586476925286766559;
  for (size_t q = 0; q < (size_t)E * A * n_rays; ++q) out[q] = range;
  for (int e = 0; e < E; ++e) {
    size_t base = (size_t)e * N;
    const double *st = state + base * 6;
    int a = 0;
    for (int i = 0; i < N; ++i) {
      if (!(w->flags[base + i] & OW_ACTUATED)) continue;
      if (a >= A) break;
      for (int k = 0; k < n_rays; ++k) {
        double ang = st[6 * i + 4] + two_pi * k / n_rays;
        double dx = cos(ang), dy = sin(ang);
        double best = range;
        for (int j = 0; j < N; ++j) {
          if (j == i || !(w->flags[base + j] & OW_COLLIDABLE)) continue;
          ow_body bj;
          load_body(w, st, base, j, &bj);
          double t = ray_shape(st[6 * i], st[6 * i + 1], dx, dy, &bj);
          if (t < best) best = t;
        }
        out[((size_t)e * A + a) * n_rays + k] = best;
      }
      ++a;
    }
  }
  return 0;
}
