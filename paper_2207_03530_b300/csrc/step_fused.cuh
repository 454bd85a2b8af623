// Fused VMAS world step kernel (sm_103a, FP32 CUDA cores).
//
// One group of G lanes steps one environment through all S substeps of one
// world step (VMAS section 3, Eqs. 1-3); state stays in registers and shared
// memory between substeps and touches HBM once on the way in and once on the
// way out.  32 / G environments share a warp.
//
//   entities   entity a lives in lane a % G of its group, slot a / G; its
//              pose and velocity in registers, its inverse mass and inertia,
//              bounding radius and the step's action + gravity force and
//              torque in the lane's own shared-memory entries (read once per
//              substep: cheaper there than in registers the narrow phase
//              needs)
//   candidates once per step (and again only if some body may have moved
//              more than half the skin since: a per-lane bound adds
//              (|vx| + |vy|) h of its fastest body every substep) every lane
//              tests the pairs
//              {a, a + d mod N}, d = 1 .. N/2, of its entities -- each
//              unordered pair exactly once, the same count for every lane --
//              against bounding circles grown by the skin (and, for a line
//              that cannot rotate, its carrier grown by the skin).  Survivors
//              are compacted, in (lane, slot, d) order, into one list per
//              environment.  A pair left out is farther apart than its
//              bounding circles for the rest of the list's life, so the list
//              never changes results, and the list order does not depend on
//              the skin.  Where a lane's (slot, offset) pairs fit 64 bits,
//              the bounding tests run without branches into a bit mask first.
//   contacts   per substep the group walks its list G pairs at a time through
//              the exact narrow phase; hits are appended to a per-env buffer
//              in list order (ballot + popc) and every lane adds the records
//              touching its entities in that order: deterministic sums, no
//              atomics.
//   fallback   if a lane's list overflows, that environment scans all pairs
//              in canonical order every substep until the next rebuild.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "step.cuh"

namespace vmas {

#ifndef VMAS_FUSED_WARPS
#define VMAS_FUSED_WARPS 4
#endif
constexpr int kFusedWarps = VMAS_FUSED_WARPS;  // warps per CTA
// Resident CTAs per SM the register budget targets: 5 (96 registers) for up
// to 3 entities per lane measured fastest on B300 at 24 entities per env; 4
// slots need more registers.  A build may override it for tuning sweeps.
#ifdef VMAS_MIN_BLOCKS
template <int SLOTS>
constexpr int min_blocks() { return VMAS_MIN_BLOCKS; }
#else
template <int SLOTS>
constexpr int min_blocks() { return SLOTS <= 3 ? 5 : 3; }
#endif
constexpr int kLaneCand = 16;    // candidate slots per lane
constexpr int kRecCap = 32;      // buffered contact records per environment
constexpr int kTypes = 6;        // SS SB SL BB BL LL

// Stats counters (only when StepParams::stats != nullptr).
enum {
  kStatEnvSteps = 0,
  kStatRebuilds = 1,
  kStatCandidates = 2,
  kStatEval = 3,   // + type, narrow-phase evaluations
  kStatHits = 9,   // + type, contacts
  kStatFullScan = 15,
  kStatCount = 16
};

// Per-environment shared memory: poses, body frames, the lane-private
// constants of the step (inverse mass and inertia, bounding radius, base force
// and torque: 24 B per entity, kept here rather than in registers), contact
// records (whose area also holds the per-lane candidate lists while the list
// is built) and the compacted candidate list.
__host__ __device__ inline int fused_rec_bytes(int G) {
  return kRecCap * 20 > align16(2 * G * kLaneCand) ? kRecCap * 20 : align16(2 * G * kLaneCand);
}
__host__ __device__ inline int fused_env_bytes(int N, int G) {
  return align16(56 * N) + fused_rec_bytes(G) + align16(2 * G * kLaneCand);
}
__host__ __device__ inline int fused_cta_smem_bytes(int N, int P, int G) {
  (void)P;  // the pair table stays in global memory (read only by full scans)
  return kFusedWarps * (32 / G) * fused_env_bytes(N, G);
}

// Shape-pair class of two shape ids: SS 0, SB 1, SL 2, BB 3, BL 4, LL 5.
__device__ __forceinline__ int pair_type(uint32_t sa, uint32_t sb) {
  const uint32_t lo = sa < sb ? sa : sb, hi = sa < sb ? sb : sa;
  return lo == 0u ? (int)hi : (lo == 1u ? 2 + (int)hi : 5);
}

// G lanes per environment, SLOTS = ceil(N / G) entities per lane; NC > 0
// compiles the kernel for exactly NC entities (fully unrolled pair loops),
// NC == 0 takes N from the parameters.
// RAW = true is the allocation-free variant: it reads the caller's raw
// entity arrays and [E][N][6] state and packs the per-entity parameters on
// the fly instead of reading the library's packed planes.  RAGGED = true
// steps envs [env_begin, env_end) of a packed ragged world, each with its own
// entity count (at most p.N, the layout capacity) at its own offset.  TILED
// kernels run p.tile consecutive world steps per launch (others run one);
// the state and the candidate list stay on chip between them.
//
// The body steps the 32 / G environments of one warp: env slots slot0 +
// group (of the size class's range, for RAGGED kernels), per-env shared
// memory from `wsmem` on.  `smem`, `warp` (the warp's index in its CTA),
// `blk` (the CTA's block of envs) and `phase` (the parity the staging
// mbarrier, initialised by the caller, completes next) serve the CTA-wide
// bulk staging of the one-step plain kernel only, the one form that
// synchronises its CTA; every other form is warp-local, which lets a
// persistent kernel run different size classes in the warps of one CTA.
// Returns false if the staging copies did not arrive in time (the envs are
// left unchanged and the error word flagged).
template <int G, int SLOTS, int NC, bool RAW, bool RAGGED, bool TILED>
__device__ __forceinline__ bool world_step_body(const StepParams &p, unsigned char *smem,
                                                unsigned long long *mbar, int warp, int slot0,
                                                unsigned char *wsmem, int blk = 0,
                                                uint32_t phase = 0) {
  constexpr int EPW = 32 / G;
  constexpr unsigned FULL = 0xffffffffu;
  const int NL = NC > 0 ? NC : p.N;  // layout capacity per env
  const int P = NC > 0 ? NC * (NC - 1) / 2 : p.P;
  // Bulk staging (one-step plain kernels, full CTAs): the CTA's envs are
  // contiguous in every plane, so one thread issues a bulk copy per plane,
  // for the parameters, the actions and the kinds into the per-env area
  // (which is free until the poses are published), counted on one mbarrier.
  constexpr int CE = kFusedWarps * EPW;  // envs per CTA
  constexpr bool kCanStage = !RAW && !RAGGED && !TILED;
  unsigned long long &s_mbar = *mbar;
  bool bulk = false;
  if constexpr (kCanStage)
    bulk = p.bulk && !p.env_list && (blk + 1) * CE <= p.E;
  unsigned char *stage = smem;
  const uint32_t plane_b = (uint32_t)(CE * NL * 4), param_b = 4 * plane_b;
  const uint32_t act_b = (uint32_t)(CE * p.A * 12), kind_b = (uint32_t)(CE * NL);
  if (bulk && threadIdx.x == 0) {
    const uint32_t bar = smem_u32(&s_mbar);
    mbar_expect_tx(bar, 6 * plane_b + param_b + act_b + kind_b + p.stage_extra_tx);
    const size_t e0 = (size_t)blk * CE * NL;
    const float *planes[6] = {p.px, p.py, p.vx, p.vy, p.th, p.om};
    for (int f = 0; f < 6; ++f) bulk_g2s(smem_u32(stage + f * plane_b), planes[f] + e0, plane_b, bar);
    bulk_g2s(smem_u32(stage + 6 * plane_b), p.param + e0, param_b, bar);
    if (act_b)
      bulk_g2s(smem_u32(stage + 6 * plane_b + param_b),
               p.actions + (size_t)blk * CE * p.A * 3, act_b, bar);
    bulk_g2s(smem_u32(stage + 6 * plane_b + param_b + act_b), p.kind + e0, kind_b, bar);
  }
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, lg = lane % G;
  const int LC = G * kLaneCand;  // candidate capacity per env
  (void)LC;
  const unsigned gbits = (G == 32) ? FULL : (((1u << G) - 1u) << (grp * G));
  const unsigned lt = (1u << lane) - 1u;
  unsigned char *es = wsmem + grp * fused_env_bytes(NL, G);
  float4 *s_bp = reinterpret_cast<float4 *>(es);  // [NL] {x, y, inflated R, kind}
  float4 *s_ng = s_bp + NL;                        // [NL] {cos, sin, ha, hb}
  float4 *s_mi = s_ng + NL;                        // [NL] {1/m, 1/I, R, action torque}
  float2 *s_fb = reinterpret_cast<float2 *>(s_mi + NL);  // [NL] action + gravity force
  float4 *s_rec = reinterpret_cast<float4 *>(es + align16(56 * NL));  // {fx, fy, ti, tj}
  uint32_t *s_rij = reinterpret_cast<uint32_t *>(s_rec + kRecCap);
  // per-lane lists [G][kLaneCand]: only live while the list is built, before
  // any contact record of the substep is written
  uint16_t *s_lc = reinterpret_cast<uint16_t *>(s_rec);
  uint16_t *s_cand = reinterpret_cast<uint16_t *>(reinterpret_cast<unsigned char *>(s_rec) +
                                                  fused_rec_bytes(G));  // compact list
  // the staging mbarrier is initialised before any thread waits on it
  if constexpr (kCanStage) __syncthreads();

  // this group's environment: index, entity base and count, action rows
  int e, N, A_e;
  size_t eb, arow0;
  bool valid;
  if constexpr (RAGGED) {
    e = p.env_begin + slot0 + grp;
    valid = e < p.env_end;
    const int s0 = valid ? p.soff[e] : 0, s1 = valid ? p.soff[e + 1] : 0;
    eb = (size_t)s0;
    N = s1 - s0;
    const int oe = valid ? p.perm[e] : 0;
    arow0 = valid ? (size_t)p.aoff[oe] : 0;
    A_e = valid ? p.aoff[oe + 1] - p.aoff[oe] : 0;
  } else {
    const int slot = slot0 + grp;
    if (!RAW && p.env_list) {
      valid = slot < *p.env_count;
      e = valid ? p.env_list[slot] : 0;
      valid = valid && e >= 0 && e < p.E;
    } else {
      e = slot;
      valid = e < p.E;
    }
    N = NL;
    eb = (size_t)e * NL;
    arow0 = (size_t)e * p.A;
    A_e = p.A;
  }
  unsigned long long *const stats = p.stats;

  float x[SLOTS], y[SLOTS], vx[SLOTS], vy[SLOTS], th[SLOTS], om[SLOTS];
  float fbx[SLOTS], fby[SLOTS], tau[SLOTS];  // live only until stored to s_fb / s_mi
  uint32_t kd[SLOTS];  // kind byte; bits 8.. hold 1 + the entity's action row (0: none)
  float4 prs[SLOTS];
  const int le = warp * EPW + grp;  // this env's index within the CTA
  if (bulk) {
    // bounded wait for the staging copies; a CTA whose copies did not arrive
    // flags the error, waits once more for them (bounded) and leaves its
    // envs unchanged
    const bool late = !mbar_wait(smem_u32(&s_mbar), phase, 1 << 20);  // about 1 s
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        atomicOr(p.err, 8);  // VMAS_DEVERR_TIMEOUT
        mbar_wait(smem_u32(&s_mbar), phase, 1 << 20);
      }
      __syncthreads();
      return false;
    }
    const float *sp = reinterpret_cast<const float *>(stage);
    const float4 *sq = reinterpret_cast<const float4 *>(stage + 6 * plane_b);
    const unsigned char *sk = stage + 6 * plane_b + param_b + act_b;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int a = lg + G * s;
      const bool ok = a < N;
      const int q = le * NL + (ok ? a : 0);
      kd[s] = ok ? sk[q] : 0u;
      x[s] = ok ? sp[q] : 0.f;
      y[s] = ok ? sp[CE * NL + q] : 0.f;
      vx[s] = ok ? sp[2 * CE * NL + q] : 0.f;
      vy[s] = ok ? sp[3 * CE * NL + q] : 0.f;
      th[s] = ok ? sp[4 * CE * NL + q] : 0.f;
      om[s] = ok ? sp[5 * CE * NL + q] : 0.f;
      prs[s] = ok ? sq[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else if constexpr (!RAW) {
    // every slot's loads first, so that they are in flight together (the
    // processing below synchronises the warp once per slot)
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int a = lg + G * s;
      const bool ok = valid && a < N;
      const size_t ga_ = ok ? VIDX(eb + a, p.EN, 1) : 0;
      kd[s] = ok ? p.kind[ga_] : 0u;
      x[s] = ok ? p.px[ga_] : 0.f;
      y[s] = ok ? p.py[ga_] : 0.f;
      vx[s] = ok ? p.vx[ga_] : 0.f;
      vy[s] = ok ? p.vy[ga_] : 0.f;
      th[s] = ok ? p.th[ga_] : 0.f;
      om[s] = ok ? p.om[ga_] : 0.f;
      prs[s] = ok ? p.param[ga_] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // the action rows are read once the kind bytes give each entity its
    // row: pull them towards L2 meanwhile
    if (valid && A_e > 0 && p.actions) {
      const char *a0 = reinterpret_cast<const char *>(p.actions + arow0 * 3);
      for (int off = lg * 128; off < A_e * 12; off += G * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a0 + off));
    }
  }
  // the k-th actuated entity of the env (entity order = slot-major) reads row k
  int act_base = 0;
  auto assign_rows = [&]() {
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const bool ok = valid && lg + G * s < N;
      const bool actuated = ok && (kd[s] & kActuated);
      const unsigned gb = __ballot_sync(FULL, actuated) & gbits;
      const int r = act_base + __popc(gb & lt);
      act_base += __popc(gb);
      if (actuated && r < A_e) kd[s] |= (uint32_t)(r + 1) << 8;
    }
  };
  // Eq. 1: action + gravity, constant over a step (only movable bodies
  // integrate, so only their mass matters); a staged step reads its actions
  // from shared memory.  store_fb moves them to the lane's own entries.
  auto load_actions = [&](int t) {
    const float *base = (bulk && t == 0)
                            ? reinterpret_cast<const float *>(stage + 6 * plane_b + param_b) +
                                  (size_t)le * p.A * 3
                            : p.actions + (size_t)t * p.act_step + arow0 * 3;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      float fax = 0.f, fay = 0.f;
      tau[s] = 0.f;
      if (kd[s] >> 8) {
        const float *ap = base + ((kd[s] >> 8) - 1) * 3;
        fax = ap[0];
        fay = ap[1];
        tau[s] = (kd[s] & kRotatable) ? ap[2] : 0.f;
      }
      const float m = prs[s].x > 0.f ? 1.f / prs[s].x : 0.f;
      fbx[s] = fax + m * p.gx;
      fby[s] = fay + m * p.gy;
    }
  };
  auto store_fb = [&]() {
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int a = lg + G * s;
      if (valid && a < N) {
        s_fb[a] = make_float2(fbx[s], fby[s]);
        s_mi[a].w = tau[s];
      }
    }
  };
  if constexpr (!RAW) {
    assign_rows();
    load_actions(0);
    if (bulk) __syncthreads();  // staging read: the per-env area may now be written
  }
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int a = lg + G * s;
    const bool ok = valid && a < N;
    float4 pr;
    if constexpr (RAW) {
      const size_t ga_ = ok ? VIDX(eb + a, p.EN, 1) : 0;
      pr = make_float4(0.f, 0.f, 0.f, 0.f);
      kd[s] = 0u;
      x[s] = y[s] = vx[s] = vy[s] = th[s] = om[s] = 0.f;
      if (ok) {
        const float *st = p.aos_state + ga_ * 6;
        x[s] = st[0]; y[s] = st[1]; vx[s] = st[2]; vy[s] = st[3]; th[s] = st[4]; om[s] = st[5];
        const uint32_t sh = p.r_shape[ga_], fl = p.r_flags[ga_];
        const float sa = p.r_size_a[ga_], sb = p.r_size_b[ga_], m = p.r_mass[ga_];
        float I = p.r_inertia[ga_];
        if (I == 0.f)
          I = sh == kBox ? m * (sa * sa + sb * sb) / 12.f
                         : (sh == kLine ? m * sa * sa / 12.f : 0.5f * m * sa * sa);
        const bool bad = sh > 2u || (fl & ~15u) || !(sa > 0.f) || (sh == kBox && !(sb > 0.f)) ||
                         ((fl & 1u) && !(m > 0.f)) || ((fl & 2u) && !(I > 0.f));
        if (bad) {
          atomicOr(p.err, 4);  // VMAS_DEVERR_BAD_ENTITY: the entity is left inert
        } else {
          kd[s] = sh | (fl << 2);
          pr = make_float4((fl & 1u) ? 1.f / m : 0.f, (fl & 2u) ? 1.f / I : 0.f,
                           sh == kSphere ? sa : 0.5f * sa, sh == kBox ? 0.5f * sb : 0.f);
        }
      }
      prs[s] = pr;
    } else {
      pr = prs[s];
    }
    const uint32_t sh = kd[s] & 3u;
    const float rb = sh == kBox ? sqrtf(pr.z * pr.z + pr.w * pr.w) : pr.z;
    if (ok) {
      float c = 1.f, sn = 0.f;
      if (sh != kSphere) body_axes(th[s], c, sn);
      s_ng[VIDX(a, N, 2)] = make_float4(c, sn, pr.z, pr.w);  // {cos, sin, ha, hb}
      // immovable bodies are published once here
      const float infl = rb + 1e-5f * (rb + fabsf(x[s]) + fabsf(y[s]));
      s_bp[VIDX(a, N, 5)] = make_float4(x[s], y[s], infl, __uint_as_float(kd[s]));
      s_mi[VIDX(a, N, 6)] = make_float4(pr.x, pr.y, rb, 0.f);
    }
  }
  if constexpr (RAW) {
    assign_rows();
    load_actions(0);
  }
  store_fb();  // after the frames: the torque shares their float4

  const float move_limit = 0.499f * p.skin;
  bool full = false;    // group scans all pairs (list overflow)
  int ncand = 0;        // list length (group-uniform)
  bool rebuild = true;  // warp-uniform
  float moved = 0.f;    // bound on how far this lane's bodies moved since the build

  const int tile = TILED ? p.tile : 1;
  for (int t = 0; t < tile; ++t) {
  if (t > 0) {
    load_actions(t);
    store_fb();
  }
  for (int sub = 0; sub < p.S; ++sub) {
    // publish the substep-start pose of bodies that move or turn
    if (t > 0 || sub > 0) {
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int a = lg + G * s;
        if (valid && a < N) {
          if ((kd[s] & kRotatable) && (kd[s] & 3u) != kSphere) {
            float c, sn;
            body_axes(th[s], c, sn);
            *reinterpret_cast<float2 *>(&s_ng[VIDX(a, N, 4)]) = make_float2(c, sn);
          }
          if (kd[s] & kMovable) {
            const float rb = s_mi[VIDX(a, N, 3)].z;
            const float infl = rb + 1e-5f * (rb + fabsf(x[s]) + fabsf(y[s]));
            s_bp[VIDX(a, N, 5)] = make_float4(x[s], y[s], infl, __uint_as_float(kd[s]));
          }
        }
      }
    }

    if (rebuild) {
      __syncwarp();
      // candidate list: pairs {a, a + d mod N}, each unordered pair once
      int n = 0;
      bool over = false;
      // The bounding tests run without branches into 64-bit masks of
      // (slot, offset) pairs -- offsets up to N / 2, where N is the compiled
      // count or at most the layout's G * SLOTS -- whose set bits are then
      // walked in (slot, offset) order.  One mask holds all slots where they
      // fit; ragged kernels (whose envs hold no padding) use one mask per
      // slot otherwise; the remaining kernels walk the offsets with a branch
      // per test, which leaves a padded world's many inert partners early.
      constexpr int D = NC > 0 ? NC / 2 : (G * SLOTS) / 2;  // at most 64
      constexpr bool kOneMask = SLOTS * D <= 64;
      constexpr bool kMask = kOneMask || RAGGED;
      // Kernels that build masks test axis-aligned bounding boxes instead of
      // circles.  A fixed wall's bounding circle covers most of the world, so
      // with circles nearly every (body, wall) pair reached the bit walk,
      // where only the exact carrier test removed it; a box is tight around
      // a body that cannot turn.  Each entity publishes {x, y, half width,
      // half height}: a rotatable body the square around its bounding circle
      // (any angle it takes before the next build fits), a body that cannot
      // turn its own box from its frame, each grown by the rounding allowance
      // of the circle test; the half height is negative for a body that
      // neither moves nor turns (two such bodies never interact) and the half
      // width -1e30 for a body that does not collide.  A pair is kept when
      // the boxes grown by the skin overlap: that holds for every pair that
      // can touch before the next build, so the list keeps every pair the
      // circles kept that can touch, in the same order, and the contacts and
      // results are bitwise the same.  A kernel compiled for a fixed count
      // keeps the boxes in the record area beside the lane lists and wraps
      // partner a + d modulo N (the compiler resolves the wrap for a known
      // N); one with a runtime count writes them twice, at a and at a + N,
      // so the partner needs no wrap (4 % on the ragged rollout, 1 % slower
      // for the fixed count), filling the record and compact-list areas,
      // which the lane lists and the compaction only write after every mask
      // is built.
      // Kernels with one mask per slot (ragged classes of 3 or 4 slots of 16
      // or 32 lanes) keep a single copy there when two do not fit, and build
      // every slot's mask before the first lane list is written.
      constexpr int kCap = NC > 0 ? NC : G * SLOTS;
      constexpr int kLcBytes = (2 * G * kLaneCand + 15) & ~15;  // lane lists; compact list
      constexpr int kRecBytes = kRecCap * 20 > kLcBytes ? kRecCap * 20 : kLcBytes;
      constexpr bool kBeside = NC > 0 && kLcBytes + 16 * kCap <= kRecBytes;  // after the lane lists
      constexpr bool kTwice = !kBeside && 32 * kCap <= kRecBytes + kLcBytes;
      constexpr bool kOnce = !kBeside && !kTwice && 16 * kCap <= kRecBytes + kLcBytes;
      constexpr bool kAabb = kMask && (kBeside || kTwice || kOnce);
      float4 *s_ab = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(s_rec) +
                                                (kBeside ? kLcBytes : 0));  // [N] or [2 N]
      [[maybe_unused]] const int NB = kTwice ? 2 * N : N;  // bound of the checked build
      if constexpr (kAabb) {
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          const int a = lg + G * s;
          if (valid && a < N) {
            const uint32_t ka = kd[s];
            float4 ab = make_float4(x[s], y[s], -1e30f, 0.f);
            if (ka & kCollidable) {
              const float rb = s_mi[VIDX(a, N, 29)].z;
              const float eps = 1e-5f * (rb + fabsf(x[s]) + fabsf(y[s]));
              float hx = rb, hy = rb;
              if (!(ka & kRotatable) && (ka & 3u) != kSphere) {
                const float4 g = s_ng[VIDX(a, N, 30)];  // {cos, sin, ha, hb}
                hx = g.z * fabsf(g.x) + g.w * fabsf(g.y);
                hy = g.z * fabsf(g.y) + g.w * fabsf(g.x);
              }
              ab.z = hx + eps;
              ab.w = (ka & (kMovable | kRotatable)) ? hy + eps : -(hy + eps);
            }
            s_ab[VIDX(a, NB, 31)] = ab;
            if constexpr (kTwice) s_ab[VIDX(a + N, NB, 34)] = ab;
          }
        }
        __syncwarp();
      }
      if constexpr (kMask) {
        const int dmax = (N - 1) / 2;
        auto pass1 = [&](int s) {
          unsigned long long m = 0ull;
          const int a = lg + G * s;
          const uint32_t ka = kd[s];
          if (a >= N || !(ka & kCollidable)) return m;
          const float ax_ = x[s], ay_ = y[s];
          const float rb = s_mi[VIDX(a, N, 11)].z;
          const float infl_a = rb + 1e-5f * (rb + fabsf(ax_) + fabsf(ay_));
          const float ra = infl_a + p.skin;
          const bool a_moves = (ka & (kMovable | kRotatable)) != 0u;
          const int dlast = dmax + ((N % 2 == 0 && a < N / 2) ? 1 : 0);
          auto circle = [&](int d) {
            const int b = a + d >= N ? a + d - N : a + d;
            const float4 bb = s_bp[VIDX(b, N, 8)];
            const uint32_t kb = __float_as_uint(bb.w);
            const float dx = ax_ - bb.x, dy = ay_ - bb.y;
            const float lim = ra + bb.z;
            return (kb & kCollidable) && (a_moves || (kb & (kMovable | kRotatable))) &&
                   !(dx * dx + dy * dy > lim * lim);
          };
          if constexpr (kAabb) {
            const float4 aa = s_ab[VIDX(a, NB, 32)];
            const float hxa = aa.z + p.skin, hya = fabsf(aa.w) + p.skin;
            const bool fixed_a = aa.w < 0.f;
            auto boxes = [&](int d) {
              const int b = kTwice || a + d < N ? a + d : a + d - N;  // (a + d) mod N
              const float4 bb = s_ab[VIDX(b, NB, 33)];
              return (fabsf(aa.x - bb.x) <= hxa + bb.z) & (fabsf(aa.y - bb.y) <= hya + fabsf(bb.w)) &
                     !(fixed_a & (bb.w < 0.f));
            };
            if constexpr (NC > 0) {
#pragma unroll
              for (int d = 1; d <= D; ++d)
                m |= (unsigned long long)(d <= dlast && boxes(d)) << (d - 1);
            } else {
#pragma unroll 4
              for (int d = 1; d <= dlast; ++d) m |= (unsigned long long)boxes(d) << (d - 1);
            }
          } else if constexpr (NC > 0) {
#pragma unroll
            for (int d = 1; d <= D; ++d)
              m |= (unsigned long long)(d <= dlast && circle(d)) << (d - 1);
          } else {
#pragma unroll 4
            for (int d = 1; d <= dlast; ++d) m |= (unsigned long long)circle(d) << (d - 1);
          }
          return m;
        };
        // the exact line tests and the appends, in mask order; the published
        // pose of a is its current position and inflated radius
        auto walk = [&](unsigned long long m, int s0) {
          while (m) {
            const int bit = __ffsll((long long)m) - 1;
            m &= m - 1ull;
            const int s = kOneMask ? bit / D : s0;
            const int d = kOneMask ? bit - s * D + 1 : bit + 1;
            const int a = lg + G * s;
            const int b = a + d >= N ? a + d - N : a + d;
            const float4 ba = s_bp[VIDX(a, N, 27)], bb = s_bp[VIDX(b, N, 28)];
            const uint32_t ka = __float_as_uint(ba.w), kb = __float_as_uint(bb.w);
            const float dx = ba.x - bb.x, dy = ba.y - bb.y;
            if ((kb & 3u) == kLine && !(kb & kRotatable)) {
              const float4 gb4 = s_ng[VIDX(b, N, 9)];
              if (fabsf(dx * gb4.y - dy * gb4.x) >
                  ba.z + p.skin + 1e-5f * (fabsf(bb.x) + fabsf(bb.y)))
                continue;
            }
            if ((ka & 3u) == kLine && !(ka & kRotatable)) {
              const float4 ga = s_ng[VIDX(a, N, 7)];
              if (fabsf(dx * ga.y - dy * ga.x) >
                  bb.z + p.skin + 1e-5f * (fabsf(ba.x) + fabsf(ba.y)))
                continue;
            }
            if (n < kLaneCand) {
              const int lo = a < b ? a : b, hi = a < b ? b : a;
              s_lc[VIDX(lg * kLaneCand + n, LC, 10)] = (uint16_t)(lo | (hi << 8));
            } else {
              over = true;
            }
            ++n;
          }
        };
        if constexpr (kOneMask) {
          unsigned long long m = 0ull;
          if (valid) {
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) m |= pass1(s) << (s * D);
          }
          if constexpr (kAabb && !kBeside) __syncwarp();  // every box read: lane lists may overwrite them
          if (valid) walk(m, 0);
        } else if constexpr (kAabb) {
          unsigned long long ms[SLOTS];
#pragma unroll
          for (int s = 0; s < SLOTS; ++s) ms[s] = valid ? pass1(s) : 0ull;
          __syncwarp();  // every box read: lane lists may overwrite them
          if (valid) {
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) walk(ms[s], s);
          }
        } else if (valid) {
#pragma unroll
          for (int s = 0; s < SLOTS; ++s) walk(pass1(s), s);
        }
      } else if (valid) {
        const int dmax = (N - 1) / 2;
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          const int a = lg + G * s;
          if (a >= N) continue;
          const uint32_t ka = kd[s];
          if (!(ka & kCollidable)) continue;
          const float ax_ = x[s], ay_ = y[s];
          const float rb = s_mi[VIDX(a, N, 11)].z;
          const float infl_a = rb + 1e-5f * (rb + fabsf(ax_) + fabsf(ay_));
          const float ra = infl_a + p.skin;  // grown by the skin on both sides
          const bool a_line = (ka & 3u) == kLine && !(ka & kRotatable);
          const float4 ga = s_ng[VIDX(a, N, 7)];
          const bool a_moves = (ka & (kMovable | kRotatable)) != 0u;
          const int dlast = dmax + ((N % 2 == 0 && a < N / 2) ? 1 : 0);
          auto test_partner = [&](int d) {
            const int b = a + d >= N ? a + d - N : a + d;
            const float4 bb = s_bp[VIDX(b, N, 8)];
            const uint32_t kb = __float_as_uint(bb.w);
            if (!(kb & kCollidable) || !(a_moves || (kb & (kMovable | kRotatable)))) return;
            const float dx = ax_ - bb.x, dy = ay_ - bb.y;
            const float lim = ra + bb.z;
            if (dx * dx + dy * dy > lim * lim) return;
            if ((kb & 3u) == kLine && !(kb & kRotatable)) {
              const float4 gb4 = s_ng[VIDX(b, N, 9)];
              if (fabsf(dx * gb4.y - dy * gb4.x) >
                  infl_a + p.skin + 1e-5f * (fabsf(bb.x) + fabsf(bb.y)))
                return;
            }
            if (a_line && fabsf(dx * ga.y - dy * ga.x) >
                              bb.z + p.skin + 1e-5f * (fabsf(ax_) + fabsf(ay_)))
              return;
            if (n < kLaneCand) {
              const int lo = a < b ? a : b, hi = a < b ? b : a;
              s_lc[VIDX(lg * kLaneCand + n, LC, 10)] = (uint16_t)(lo | (hi << 8));
            } else {
              over = true;
            }
            ++n;
          };
          if (NC > 0) {
#pragma unroll
            for (int d = 1; d <= (NC > 0 ? NC / 2 : 1); ++d)
              if (d <= dlast) test_partner(d);
          } else {
            for (int d = 1; d <= dlast; ++d) test_partner(d);
          }
        }
      }
      // compact the lane lists in lane order
      const int cnt = n < kLaneCand ? n : kLaneCand;
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o, G);
        if (lg >= o) incl += v;
      }
      const int total = __shfl_sync(FULL, incl, G - 1, G);
      for (int k = 0, off = incl - cnt; k < cnt; ++k)
        s_cand[VIDX(off + k, LC, 15)] = s_lc[VIDX(lg * kLaneCand + k, LC, 12)];
      // every lane votes (a warp-wide vote skipped by some lanes is undefined)
      const unsigned over_bits = __ballot_sync(FULL, over);
      full = valid && (over_bits & gbits) != 0u;
      ncand = valid ? (full ? P : total) : 0;
      moved = 0.f;
      if (stats && valid && lg == 0) {
        atomicAdd(stats + kStatRebuilds, 1ull);
        atomicAdd(stats + kStatCandidates, (unsigned long long)total);
      }
    }
    __syncwarp();

    // Eq. 1: action + gravity; Eq. 3: action torque
    float Fx[SLOTS], Fy[SLOTS], T[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int a = lg + G * s;
      const bool ok = valid && a < N;
      const float2 f0 = ok ? s_fb[VIDX(a, N, 13)] : make_float2(0.f, 0.f);
      Fx[s] = f0.x;
      Fy[s] = f0.y;
      T[s] = ok ? s_mi[VIDX(a, N, 14)].w : 0.f;
    }
    auto drain = [&](int n) {
      const int nmax = (int)__reduce_max_sync(FULL, (unsigned)n);
      for (int c = 0; c < nmax; ++c) {
        if (c < n) {
          const float4 r = s_rec[VIDX(c, kRecCap, 16)];
          const uint32_t ij = s_rij[VIDX(c, kRecCap, 17)];
          const int ci = (int)(ij & 0xffffu), cj = (int)(ij >> 16);
#pragma unroll
          for (int s = 0; s < SLOTS; ++s) {
            const int me = lg + G * s;
            if (me == ci) { Fx[s] += r.x; Fy[s] += r.y; T[s] += r.z; }
            if (me == cj) { Fx[s] -= r.x; Fy[s] -= r.y; T[s] += r.w; }
          }
        }
      }
    };

    int count = 0;
    const int iters = (int)__reduce_max_sync(FULL, (unsigned)((ncand + G - 1) / G));
    if (stats && lg == 0 && full) atomicAdd(stats + kStatFullScan, 1ull);
    for (int k = 0; k < iters; ++k) {
      const int c = k * G + lg;
      bool hit = false;
      Hit hh;
      int i = 0, j = 0;
      if (c < ncand) {
        // a full scan (after a list overflow, rare) reads the canonical
        // pair table from global memory, where it stays L2-resident
        const uint32_t ij = full ? p.pairs[VIDX(c, P, 21)] : s_cand[VIDX(c, LC, 20)];
        i = VIDX((int)(ij & 0xffu), NL, 22);
        j = VIDX((int)(ij >> 8), NL, 23);
        const bool in_env = !RAGGED || j < N;  // a full scan covers the layout capacity
        const float4 bi = s_bp[in_env ? i : 0], bj = s_bp[in_env ? j : 0];
        const float4 gi = s_ng[in_env ? i : 0], gj = s_ng[in_env ? j : 0];  // {cos, sin, ha, hb}
        const uint32_t ki = __float_as_uint(bi.w), kj = __float_as_uint(bj.w);
        if (in_env && pair_active(ki, kj)) {
          hit = pair_hit(bi, bj, ki, kj, gi, gj, hh);
          if (stats) {
            const int t = pair_type(ki & 3u, kj & 3u);
            atomicAdd(stats + kStatEval + t, 1ull);
            if (hit) atomicAdd(stats + kStatHits + t, 1ull);
          }
        }
      }
      const unsigned gb = __ballot_sync(FULL, hit) & gbits;
      const int nh = __popc(gb);
      if (__any_sync(FULL, count + nh > kRecCap)) {
        __syncwarp();
        drain(count);
        __syncwarp();
        count = 0;
      }
      if (hit) {
        // Eq. 2 magnitude c k log(1 + exp(-g / k)), g <= 0
        const float mag = p.ck * softplus_pos(-hh.g * p.inv_k);
        const int slot = count + __popc(gb & lt);
        s_rec[VIDX(slot, kRecCap, 24)] = make_float4(mag * hh.nx, mag * hh.ny, mag * hh.ti, -mag * hh.tj);
        s_rij[VIDX(slot, kRecCap, 25)] = (uint32_t)i | ((uint32_t)j << 16);
      }
      count += nh;
    }
    __syncwarp();
    drain(count);
    __syncwarp();

    // Eqs. 1 and 3: damped semi-implicit Euler
    float fastest = 0.f;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      float im = 0.f, iI = 0.f;  // kind bits are set only for this env's entities
      if (kd[s] & (kMovable | kRotatable)) {
        const float4 mi = s_mi[VIDX(lg + G * s, N, 18)];
        im = mi.x;
        iI = mi.y;
      }
      if (kd[s] & kMovable) {
        vx[s] = p.damp * vx[s] + Fx[s] * im * p.h;
        vy[s] = p.damp * vy[s] + Fy[s] * im * p.h;
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
        fastest = fmaxf(fastest, fabsf(vx[s]) + fabsf(vy[s]));
      }
      if (kd[s] & kRotatable) {
        om[s] = p.damp * om[s] + T[s] * iI * p.h;
        th[s] += om[s] * p.h;
      }
    }
    // |displacement| <= (|vx| + |vy|) h per substep
    moved = fmaf(fastest, p.h, moved);
    rebuild = __any_sync(FULL, moved > move_limit);
    __syncwarp();
  }
  }

  bool bad = false;
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int a = lg + G * s;
    if (valid && a < N) {
      const size_t go_ = VIDX(eb + a, p.EN, 26);
      if constexpr (RAW) {
        float *st = p.aos_state + go_ * 6;
        st[0] = x[s]; st[1] = y[s]; st[2] = vx[s]; st[3] = vy[s]; st[4] = th[s]; st[5] = om[s];
      } else {
        p.px[go_] = x[s];
        p.py[go_] = y[s];
        p.vx[go_] = vx[s];
        p.vy[go_] = vy[s];
        p.th[go_] = th[s];
        p.om[go_] = om[s];
      }
      bad |= !(isfinite(x[s]) && isfinite(y[s]) && isfinite(vx[s]) && isfinite(vy[s]) &&
               isfinite(th[s]) && isfinite(om[s]));
    }
  }
  if (stats && valid && lg == 0) atomicAdd(stats + kStatEnvSteps, (unsigned long long)tile);
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(p.err, 1);  // VMAS_DEVERR_NONFINITE
  return true;
}

// One launch steps a grid of CTAs of kFusedWarps warps, 32 / G envs per warp.
template <int G, int SLOTS, int NC, bool RAW = false, bool RAGGED = false, bool TILED = false>
__global__ void __launch_bounds__(kFusedWarps * 32, min_blocks<SLOTS>())
    world_step_kernel(const StepParams p) {
  constexpr int EPW = 32 / G;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long s_mbar;
  if constexpr (!RAGGED && !RAW) {
    // listed stepping: a block past the end of the list has nothing to do
    // (uniform over the block, before its first barrier)
    if (p.env_list && (int)(blockIdx.x * kFusedWarps * EPW) >= *p.env_count) return;
  }
  const int warp = threadIdx.x >> 5;
  const int NL = NC > 0 ? NC : p.N;
  if constexpr (!RAW && !RAGGED && !TILED)
    if (threadIdx.x == 0) mbar_init(smem_u32(&s_mbar), 1);  // staging; the body's barrier orders it
  world_step_body<G, SLOTS, NC, RAW, RAGGED, TILED>(
      p, smem, &s_mbar, warp, (blockIdx.x * kFusedWarps + warp) * EPW,
      smem + warp * EPW * fused_env_bytes(NL, G), blockIdx.x, 0u);
}

}  // namespace vmas
