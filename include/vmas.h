/*
 * vmas.h -- C ABI of the B300-native VMAS world step.
 *
 * The library steps many independent 2D worlds ("environments") at once on
 * one CUDA device.  Each world holds n_entities bodies (spheres, boxes,
 * lines) with state (x, y, vx, vy, theta, omega); one world step applies the
 * VMAS core of Bettini et al. (section 3, "Core"):
 *
 *   Eq. 1  f_i = f^a_i + m_i g + sum_j f^e_ij,   v <- (1-zeta) v + f/m dt,
 *          x <- x + v dt                           (semi-implicit Euler)
 *   Eq. 2  f^e_ij = c k log(1 + exp(-gap/k)) n_ij  when gap <= 0, else 0,
 *          gap = |x_ij| - d_min between the closest points of i and j
 *   Eq. 3  tau_i = sum_j r_ij x f^e_ij,  omega <- (1-zeta) omega + tau/I dt,
 *          theta <- theta + omega dt
 *
 * repeated `substeps` times per call with dt / substeps (actions held).
 * The torque of Eq. 3 is the signed 2D cross product; a box or line pair's
 * closest points come from its separating-axis penetration, with the
 * contact point on the incident edge clipped to the reference face.
 *
 * Conventions for every entry point:
 *  - Return 0 (VMAS_OK) on success or a negative VMAS_E* code; the message
 *    of the last failure on the calling thread is vmas_last_error().
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it and the call returns without waiting unless stated.
 *  - Device pointers are borrowed: they must stay valid until the work
 *    enqueued on `stream` has finished.  Host pointers are read or written
 *    before the call returns unless stated.
 *  - All floating-point data is FP32, little-endian, C order.
 *  - A world is not thread-safe: serialise calls on one world.
 *  - A world lives on the device that is current when it is created; make
 *    that device current for every later call on it, and pass streams of
 *    that device (the Python binding creates its tensors there).
 */
#ifndef VMAS_H_
#define VMAS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VMAS_ABI_VERSION 1

/* Entity shapes (section 3, Core: every entity is a sphere, a box or a line). */
enum { VMAS_SPHERE = 0, VMAS_BOX = 1, VMAS_LINE = 2 };

/* Entity flags (section 3: movable, rotatable, collidable; actuated = takes an
 * action row).  An entity with none of the bits set is inert padding. */
enum {
  VMAS_MOVABLE = 1,
  VMAS_ROTATABLE = 2,
  VMAS_COLLIDABLE = 4,
  VMAS_ACTUATED = 8
};

/* Status codes. */
enum {
  VMAS_OK = 0,
  VMAS_EINVAL = -1,  /* bad argument or world description              */
  VMAS_ENOMEM = -2,  /* device or host allocation failed                */
  VMAS_ECUDA = -3,   /* a CUDA runtime call failed                      */
  VMAS_EDEVICE = -4  /* a kernel raised its device error word (see below) */
};

/* Bits of the device error word reported through VMAS_EDEVICE. */
enum {
  VMAS_DEVERR_NONFINITE = 1, /* a state value became NaN or Inf */
  VMAS_DEVERR_INDEX = 2,     /* bounds-checked builds (-DVMAS_CHECKED) only: an index was out
                                of range and was not used; vmas_last_error() names the first
                                one (site code, index, bound) */
  VMAS_DEVERR_BAD_ENTITY = 4, /* vmas_step_noalloc met an invalid entity and left it inert */
  VMAS_DEVERR_TIMEOUT = 8     /* a step's staging copies did not arrive in time; its CTA
                                 left its envs unchanged */
};

/* Largest supported entity count per environment. */
#define VMAS_MAX_ENTITIES 128

typedef struct vmas_world vmas_world; /* opaque, owned by the library */

/* World description, read by vmas_world_create and not kept.
 * Per-entity arrays are host arrays of n_envs * n_entities elements, entity
 * index fastest.  The k-th actuated entity of an env (in entity order) reads
 * action row k; an env may have fewer actuated entities than n_actuated,
 * never more. */
typedef struct {
  int32_t n_envs;      /* >= 0                                            */
  int32_t n_entities;  /* 1 .. VMAS_MAX_ENTITIES                          */
  int32_t n_actuated;  /* action rows per env, >= 0                       */
  int32_t substeps;    /* >= 1                                            */
  float dt;            /* step length delta t (> 0)                       */
  float drag;          /* velocity damping zeta, applied every substep     */
  float gx, gy;        /* gravity g                                        */
  float contact_force; /* c of Eq. 2 (>= 0)                                */
  float contact_margin;/* k of Eq. 2 (> 0)                                 */
  float max_speed;     /* |v| cap applied after the velocity update; 0 = off */
  const uint8_t *shape;   /* VMAS_SPHERE / VMAS_BOX / VMAS_LINE            */
  const uint8_t *flags;   /* VMAS_MOVABLE | ...                            */
  const float *size_a;    /* sphere radius | box width | line length (> 0) */
  const float *size_b;    /* box height (> 0 for boxes, ignored otherwise) */
  const float *mass;      /* > 0 for movable entities                      */
  const float *inertia;   /* moment of inertia; 0 selects box m(w^2+h^2)/12,
                             line m L^2/12, sphere m r^2/2                 */
  const float *init_state;/* [n_envs][n_entities][6]: x y vx vy theta omega */
} vmas_world_desc;

/* Create a world on the current CUDA device (the scenario's make_world of
 * section 3, "Scenario": it creates the entities and spawns them; the
 * entity attributes are those of section 3, "Core": shape, mass, movable /
 * rotatable / collidable, maximum speed, and the world's delta t, damping
 * zeta and gravity g).  Validates the description, allocates the device
 * state and parameter planes and copies them in (synchronously).  On failure
 * *out is NULL and nothing is leaked. */
int vmas_world_create(const vmas_world_desc *desc, vmas_world **out);

/* Free a world and its device memory (waits for the device).  NULL is a
 * no-op. */
int vmas_world_destroy(vmas_world *world);

/* Sizes of a world; any pointer may be NULL.  n_pairs = N (N - 1) / 2. */
int vmas_world_info(const vmas_world *world, int32_t *n_envs, int32_t *n_entities,
                    int32_t *n_actuated, int32_t *substeps, int32_t *n_pairs);

/* Margin of the per-step contact-candidate list (world units, >= 0).  The
 * step keeps, for each environment, the pairs whose bounding circles are
 * within `skin` of touching and rebuilds the list whenever a body has moved
 * more than skin / 2 since; pairs left out cannot touch, so results do not
 * depend on the value, only speed does.  Default at create: half the median
 * bounding radius of the movable entities. */
int vmas_world_set_skin(vmas_world *world, float skin);
int vmas_world_get_skin(const vmas_world *world, float *skin);

/* vmas_rollout launches `steps_per_launch` world steps per kernel (default
 * 1): the state and the contact-candidate lists stay on chip between them.
 * Results are bitwise the same for any value. */
int vmas_world_set_rollout_tile(vmas_world *world, int32_t steps_per_launch);

/* Optional step counters, for tuning (they cost a few atomics per env per
 * substep while enabled).  vmas_world_get_stats waits for `stream` and
 * copies VMAS_STATS_COUNT counters into `out`, zeroing them if `reset`:
 *   [0] env-steps  [1] candidate-list builds  [2] candidates listed
 *   [3..8] narrow-phase evaluations of sphere-sphere, sphere-box,
 *          sphere-line, box-box, box-line, line-line candidates
 *   [9..14] contacts found, same order   [15] env-substeps in full scan */
#define VMAS_STATS_COUNT 16
int vmas_world_set_stats(vmas_world *world, int32_t enable);
int vmas_world_get_stats(vmas_world *world, uint64_t *out, int32_t reset, void *stream);

/* One world step of every environment (section 3, Eqs. 1-3, substeps fused
 * on chip).  d_actions: device [n_envs][n_actuated][3] (fx, fy, torque); the
 * torque is applied to rotatable actuated entities only.  May be NULL when
 * n_actuated == 0.  Enqueues one kernel on `stream`. */
int vmas_step(vmas_world *world, const float *d_actions, void *stream);

/* As vmas_step with a HOST action array of the same layout: the actions are
 * copied into a library-owned device buffer on `stream` first.  The host
 * array must stay valid until that copy has run (pinned memory makes the
 * copy asynchronous; pageable memory makes it synchronous). */
int vmas_step_host(vmas_world *world, const float *h_actions, void *stream);

/* T consecutive world steps: d_actions is device [T][n_envs][n_actuated][3].
 * Enqueues T kernels on `stream`. */
int vmas_rollout(vmas_world *world, const float *d_actions, int32_t n_steps, void *stream);

/* n_steps world steps between HOST buffers: h_actions [T][n_envs][n_actuated]
 * [3] in, every step's state h_states [T][n_envs][n_entities][6] (as
 * vmas_state) out.  Uploads, steps and downloads overlap: step t + 1's
 * actions go up and step t's state comes down on the library's own copy
 * streams while the steps run in order on `stream`, through two device
 * buffers each way.  Pinned host memory makes the copies asynchronous.
 * Returns when every state has arrived (it waits for `stream`), with
 * VMAS_EDEVICE if a kernel raised the device error word. */
int vmas_rollout_host(vmas_world *world, const float *h_actions, int32_t n_steps, float *h_states,
                      void *stream);

/* Read the state into caller memory as [n_envs][n_entities][6]
 * (x y vx vy theta omega): the vectorized state (x_i, xdot_i, theta_i,
 * thetadot_i) of every entity in every environment (section 3, "Core"),
 * returned as one batched tensor as section 3's "Interface" returns its
 * outputs for all environments.  out_is_device != 0: `out` is device memory and
 * the copy is enqueued on `stream`.  out_is_device == 0: `out` is host
 * memory; the call waits for `stream` and then returns VMAS_EDEVICE if a
 * kernel has raised the device error word since the last check. */
int vmas_state(vmas_world *world, float *out, int32_t out_is_device, void *stream);

/* Overwrite the state of the environments selected by env_mask (the reset of
 * section 3's scenario interface, reset_world_at).  state: [n_envs]
 * [n_entities][6], device if state_is_device else host.  env_mask: HOST
 * uint8 [n_envs] (non-zero = reset this env) or NULL for all envs.  Host
 * inputs are consumed before the call returns. */
int vmas_set_state(vmas_world *world, const float *state, int32_t state_is_device,
                   const uint8_t *env_mask, void *stream);

/* First-substep contact mask of the current state: the case split of Eq. 2
 * (section 3), i.e. which pairs have |x_ij| <= d_min and so a non-zero
 * environmental force f^e_ij.  d_mask is device uint8 [n_envs][n_pairs],
 * pairs (i < j) in row-major order; 1 where the pair is active (both
 * collidable, one movable or rotatable) and gap <= 0 with a defined normal.
 * Does not change the state. */
int vmas_debug_pairs(vmas_world *world, uint8_t *d_mask, void *stream);

/* The canonical pair list into host arrays of n_pairs elements: the pairs
 * (i, j), i < j, row-major, over which Eq. 1's sum over j in N \ {i} runs
 * (each unordered pair once, its force applied to both with opposite signs). */
int vmas_pair_table(const vmas_world *world, int32_t *pair_i, int32_t *pair_j);

/* Wait for `stream` and return VMAS_EDEVICE (clearing the word) if a kernel
 * has raised the device error word since the last check; *bits (may be NULL)
 * receives the VMAS_DEVERR_* bits seen. */
int vmas_check(vmas_world *world, void *stream, int32_t *bits);

/* ---- Packed ragged worlds ----------------------------------------------
 * Environments with different entity counts (1 .. VMAS_MAX_ENTITIES each),
 * packed without padding.  env_offsets [n_envs + 1] (host) gives env e the
 * entities [env_offsets[e], env_offsets[e + 1]) of every per-entity array
 * (host, as in vmas_world_desc) and of init_state [total][6].  Actions are
 * packed the same way: env e owns the action rows
 * [aoff[e], aoff[e + 1]) of a [n_action_rows][3] array, aoff given by
 * vmas_ragged_action_offsets (the k-th actuated entity of env e reads row
 * aoff[e] + k).
 *
 * The library sorts the envs into size classes of capacity 8, 16, 32, 64
 * and 128 entities (Table 1 of the paper lists VMAS for "< 100 agents" per
 * world; section 3's vectorized interface steps any number of worlds in one
 * batch).  Two schedules step them:
 *  - per class (schedule 0): each class by the fused kernel compiled for its
 *    choice of lanes per environment (4, 8, 16 or 32), the classes' launches
 *    side by side;
 *  - persistent (schedules 1 and 2): every class in ONE launch, whose warps
 *    take one warp's worth of envs at a time from an atomic work queue,
 *    largest class first, with fixed lanes per class (8, 8, 16, 32, 32).  No
 *    warp ever waits on another: a warp takes its next item with one atomic
 *    add.  Schedule 1 is the kernel built for 128 registers (4 CTAs per SM),
 *    schedule 2 the same kernel built for 96 (5 CTAs per SM; the largest
 *    class spills registers).
 * Rollouts run steps_per_launch world steps per launch and are captured once
 * into a CUDA graph per (actions buffer, n_steps, tuning, schedule), then
 * replayed.  vmas_ragged_autotune times the lanes per class, then every
 * steps_per_launch under every schedule as a graph-captured rollout of
 * n_steps steps, on the caller's actions (the world state is restored
 * afterwards), and keeps the fastest.  Every schedule gives bitwise the same
 * result for the same lanes per class. */
typedef struct vmas_ragged vmas_ragged;
typedef struct {
  int32_t n_envs, substeps;
  float dt, drag, gx, gy, contact_force, contact_margin, max_speed;
  const int32_t *env_offsets;
  const uint8_t *shape, *flags;
  const float *size_a, *size_b, *mass, *inertia;
  const float *init_state;
} vmas_ragged_desc;
int vmas_ragged_create(const vmas_ragged_desc *desc, vmas_ragged **out);
int vmas_ragged_destroy(vmas_ragged *world);
/* class_envs [5]: envs per size class (8, 16, 32, 64, 128). */
int vmas_ragged_info(const vmas_ragged *world, int32_t *n_envs, int64_t *n_entities,
                     int64_t *n_action_rows, int32_t *class_envs);
int vmas_ragged_action_offsets(const vmas_ragged *world, int32_t *aoff);
/* One world step: d_actions [n_action_rows][3] (device). */
int vmas_ragged_step(vmas_ragged *world, const float *d_actions, void *stream);
/* n_steps world steps: d_actions [n_steps][n_action_rows][3] (device). */
int vmas_ragged_rollout(vmas_ragged *world, const float *d_actions, int32_t n_steps, void *stream);
/* State [total][6] in the caller's entity order (see vmas_state). */
int vmas_ragged_state(vmas_ragged *world, float *out, int32_t out_is_device, void *stream);
int vmas_ragged_set_state(vmas_ragged *world, const float *d_state, void *stream);
/* As vmas_check, for a ragged world's device error word. */
int vmas_ragged_check(vmas_ragged *world, void *stream, int32_t *bits);
/* lanes [5] per size class (NULL keeps them); steps_per_launch 1..1024. */
int vmas_ragged_set_tuning(vmas_ragged *world, const int32_t *lanes, int32_t steps_per_launch);
int vmas_ragged_get_tuning(const vmas_ragged *world, int32_t *lanes, int32_t *steps_per_launch);
int vmas_ragged_autotune(vmas_ragged *world, const float *d_actions, int32_t n_steps, void *stream);
/* Schedule: 0 = per-class launches (default at create), 1 or 2 = one
 * persistent launch with an atomic work queue (128- or 96-register build).
 * VMAS_EINVAL for other values. */
int vmas_ragged_set_schedule(vmas_ragged *world, int32_t schedule);
int vmas_ragged_get_schedule(const vmas_ragged *world, int32_t *schedule);

/* LIDAR (section 3: agents can carry LIDAR sensors).  Every actuated
 * entity of every env casts n_rays rays from its centre at angles
 * theta + 2 pi k / n_rays (k = 0 .. n_rays-1) against the other collidable
 * entities of its env, from the current state; d_out [n_envs][n_actuated]
 * [n_rays] (device) receives the distance to the first entry into a sphere,
 * box or line segment, 0 when the ray starts inside one, max_range when it
 * meets none (also for action rows an env does not use).  A ray exactly
 * parallel to a segment misses it.  Distances are FP32 within about 1e-7 of
 * a unit range (fast reciprocal and reciprocal square root); a ray that
 * grazes a body within that margin may read hit or miss.  Enqueues one
 * kernel on `stream`. */
int vmas_lidar(vmas_world *world, int32_t n_rays, float max_range, float *d_out, void *stream);

/* Diagnostic: which LIDAR kernel vmas_lidar runs (process-wide).  on != 0
 * (the default): the culled kernel, where n_actuated x n_rays <= 3072
 * and its shared arrays fit 48 KB --
 * each (body, caster) pair tests only the rays within the body's angular arc
 * (bounding circle or segment endpoints, one ray of slack each side), with
 * the same per-ray routines, so the readings are the same minima.  on == 0:
 * every ray against every body.  Always VMAS_OK. */
int vmas_debug_lidar_cull(int32_t on);

/* ---- Differentiable rollout (sphere worlds) -----------------------------
 * Loss per env = sum over its actuated entities k of |x_k(T) - goal_k|^2
 * after n_steps world steps from the world's current state (which is left
 * unchanged), and its gradient with respect to every action by a
 * hand-written adjoint of the contact force (Eq. 2), drag and damped
 * semi-implicit Euler (Eq. 1) over all substeps; the contact mask is held
 * piecewise constant (no term from the force jump at gap 0).  Requires every
 * entity to be a sphere, n_entities <= 32 and no speed cap (VMAS_EINVAL
 * otherwise).  Each entity's pair sums visit its candidate partners (pairs
 * within 4 x the world's skin of touching, rebuilt when a body may have moved
 * half of that) in ascending order, so the loss and gradient do not depend
 * on the skin, only speed does.
 *   d_actions [n_steps][n_envs][n_actuated][3], d_goals [n_envs][n_actuated][2];
 *   d_ckpt    [ceil(n_steps / ckpt_every)][n_envs][n_entities][4] (x y vx vy at
 *             steps 0, ckpt_every, ...), written by vmas_diff_rollout and read
 *             by vmas_diff_backward, which replays each segment on chip;
 *   d_loss    [n_envs] (written);  d_dloss [n_envs] = d L / d loss_e;
 *   d_grad    [n_steps][n_envs][n_actuated][3] (written; torque entries 0).
 * All device memory, enqueued on `stream`.  ckpt_every * substeps is limited by
 * shared memory (VMAS_EINVAL beyond about 200 substeps per segment). */
int vmas_diff_rollout(vmas_world *world, const float *d_actions, int32_t n_steps,
                      const float *d_goals, int32_t ckpt_every, float *d_ckpt, float *d_loss,
                      void *stream);
int vmas_diff_backward(vmas_world *world, const float *d_actions, int32_t n_steps,
                       const float *d_goals, int32_t ckpt_every, const float *d_ckpt,
                       const float *d_dloss, float *d_grad, void *stream);

/* Diagnostic: lanes per env of the differentiable rollout, process-wide:
 * 1 = one group of G lanes per env (G the smallest power of two >= n_entities),
 * 2 = two such groups per env where two fit a warp, each summing half of
 * every entity's pairs; 0 = the default (1).  Both give the gradient to
 * rounding; split 2 fills twice the warps with the same envs. */
int vmas_debug_diff_split(int32_t split);

/* Test hook for failure detection without a GPU fault: while `on` is set,
 * every CTA of vmas_step that stages its inputs with bulk copies waits for 16
 * transaction bytes that no copy delivers, so its bounded wait runs out (in
 * a few seconds); the CTA then sets VMAS_DEVERR_TIMEOUT and leaves its envs
 * unchanged, and the context stays usable.  Off by default. */
int vmas_debug_stage_timeout(vmas_world *world, int32_t on);

/* Diagnostic: the cosine and sine the step uses for a body angle, for n
 * device angles d_theta into device d_cos_sin [n][2] (cos, sin); the
 * library's own range reduction and series, absolute error about 1e-7 for
 * |theta| up to 2e6 rad (beyond that the error grows with |theta|).  For
 * any input, huge, inf or NaN angles included, the result is a unit vector
 * (to that accuracy); far beyond the range it bears no relation to theta. */
int vmas_debug_body_axes(const float *d_theta, float *d_cos_sin, int32_t n, void *stream);

/* ---- Allocation-free step --------------------------------------------
 * Not part of the method: the paper has no counterpart.  Some callers cannot
 * let a library call cudaMalloc: code that owns all device memory through
 * its own allocator (a framework's memory pool, an arena reserved up front),
 * loops that must not stall on the device synchronisation that cudaMalloc and
 * cudaFree can cause, and code running under stream capture, where those
 * calls are not allowed.  vmas_step_noalloc is one world step (the same
 * kernel as vmas_step) over buffers the caller owns; it allocates nothing.
 *
 * Its only scratch is a fixed 16,640-byte array in the library's device
 * memory (a 16,384-byte pair table for up to VMAS_NOALLOC_MAX_ENTITIES
 * entities plus a 256-byte status block), present on every device that
 * loads the library until the process exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array and rewrites it, so calls that can overlap on
 * the GPU (on different streams) race: serialise them.
 *
 * Arguments: every pointer is device memory, entity arrays [n_envs *
 * n_entities] as in vmas_world_desc, state [n_envs][n_entities][6] read and
 * overwritten in place, actions [n_envs][n_actuated][3] (NULL when
 * n_actuated == 0).  skin >= 0 is the candidate-list margin (see
 * vmas_world_set_skin; 0 rebuilds the list every substep, always valid).
 * status (optional, device int32): the call ORs VMAS_DEVERR_* bits into it;
 * the caller clears it.  Entities are checked on the device: an invalid one
 * is left inert and raises VMAS_DEVERR_BAD_ENTITY.  Returns VMAS_EINVAL
 * (before enqueuing anything) when n_entities > VMAS_NOALLOC_MAX_ENTITIES or a
 * world parameter is out of range or not finite. */
#define VMAS_NOALLOC_MAX_ENTITIES 128
typedef struct {
  int32_t n_envs, n_entities, n_actuated, substeps;
  float dt, drag, gx, gy, contact_force, contact_margin, max_speed, skin;
  const uint8_t *shape, *flags;
  const float *size_a, *size_b, *mass, *inertia;
  float *state;
  const float *actions;
  int32_t *status;
} vmas_step_noalloc_args;
int vmas_step_noalloc(const vmas_step_noalloc_args *args, void *stream);

/* ---- Learned surrogate of the world step --------------------------------
 * Not part of the paper's method: a network trained on the transitions that
 * the step of section 3 (Eqs. 1-3, all substeps) produces, standing in for
 * it on two world layouts (walls at x = +-1 and y = +-1):
 *  - the sphere world: per env 16 movable, actuated, non-rotating agent
 *    spheres (action rows 0..15), then 4 fixed lines;
 *  - the box world (the paper-scale layout): the same 16 agents, then 4
 *    movable, rotatable, actuated boxes (action rows 16..19, torque used),
 *    then 4 fixed lines.
 * Worlds of any other layout give VMAS_EINVAL.  The network has one row
 * ("node") per agent and per box: nodes = 16 or 20 per env.
 *
 * Network, per node: node features (10 vx, 10 vy, f/m, 10 R, 1/m and the 4
 * wall gaps min(gap, 0.3)/0.3 of its bounding circle of radius R; a box adds
 * a flag, cos theta, sin theta, 0.1 omega, 0.01 torque / I); edge features
 * for up to 6 nearest other nodes within 0.3 (relative position / 0.3, 10
 * relative velocity, 10 R_j, bounding-circle gap / 0.3, 1; a box neighbour
 * adds a flag, cos theta_j, sin theta_j, 0.1 omega_j); edge MLP 16 -> 64 ->
 * 64 (GELU) summed over the edges; node MLP 80 -> 128 -> 128 -> 8 (GELU);
 * prediction x' = x + 0.01 out[0:2], v' = v + 0.1 out[2:4], and for a box
 * theta' = theta + 0.1 out[4], omega' = omega + out[5].  Weights and
 * activations bfloat16, accumulation FP32 (tensor cores: tcgen05 for the
 * layered path's large GEMMs, warp-level mma elsewhere), biases FP32.
 *
 * Parameters: vmas_sur_param_count() FP32 values in the order We1 [64][16],
 * be1 [64], We2 [64][64], be2 [64], W1 [128][80], b1 [128], W2 [128][128],
 * b2 [128], W3 [8][128], b3 [8] (weights [out][in]); the library keeps an
 * FP32 master copy and rounds the weights to bfloat16 for the GEMMs.
 * Training minimises the mean of (out - target)^2 over the outputs each node
 * uses (4 for an agent, 6 for a box), the target being the plain step's
 * deltas of (x, y, vx, vy[, theta, omega]) over (0.01, 0.01, 0.1, 0.1[, 0.1,
 * 1]), with Adam (beta 0.9 / 0.999, eps 1e-8).
 *
 * A surrogate is created for at most max_envs envs (its activations are
 * sized for them) and serves any world of that layout and size; d_actions
 * is the world's [n_envs][n_actuated][3] device action array.  Calls on one
 * surrogate must be serialised; all work is enqueued on `stream` except in
 * set_params / get_params, which synchronise the device. */
typedef struct vmas_surrogate vmas_surrogate;
int vmas_sur_param_count(void);
int vmas_sur_create(int32_t max_envs, vmas_surrogate **out);
int vmas_sur_destroy(vmas_surrogate *sur);
/* h_params / out: host [vmas_sur_param_count()]; set_params resets Adam. */
int vmas_sur_set_params(vmas_surrogate *sur, const float *h_params);
int vmas_sur_get_params(vmas_surrogate *sur, float *h_params);
/* Inference kernels of vmas_sur_forward and vmas_sur_step:
 * VMAS_SUR_FUSED (the default): one kernel, one warp per env, everything on
 * chip (sphere world only; box worlds always take the layered path);
 * VMAS_SUR_LAYERED: one GEMM launch per layer over all envs, with the
 * activations in device memory (the path training uses).  Both round at the
 * same points.  The layered path runs the edge MLP on the neighbour slots in
 * use only (compacted in slot order on the device); it reads their count
 * back to size the edge GEMMs, so each layered forward (inference or
 * training) synchronises `stream` once. */
enum { VMAS_SUR_FUSED = 0, VMAS_SUR_LAYERED = 1 };
int vmas_sur_set_mode(vmas_surrogate *sur, int32_t mode);
/* The network on the world's current state: d_out [n_envs * nodes][8]
 * (device, may be NULL), row e * nodes + i for node i of env e. */
int vmas_sur_forward(vmas_surrogate *sur, vmas_world *world, const float *d_actions,
                     float *d_out, void *stream);
/* Loss against d_target [n_envs * nodes][tw] (tw = 4: x y vx vy; 6 in the
 * box world: also theta omega) into d_loss [1] (may be NULL) and
 * its gradient, kept for vmas_sur_adam and copied to d_grad
 * [vmas_sur_param_count()] (may be NULL).  The world is not changed. */
int vmas_sur_loss_grad(vmas_surrogate *sur, vmas_world *world, const float *d_actions,
                       const float *d_target, float *d_loss, float *d_grad, void *stream);
/* One Adam update with the gradient d_grad [vmas_sur_param_count()] (device;
 * NULL = the gradient of the last loss_grad / train_grad / train_step), e.g.
 * one averaged over data-parallel ranks. */
int vmas_sur_adam(vmas_surrogate *sur, float lr, const float *d_grad, void *stream);
/* The gradient half of a training step on a fresh transition: the network on
 * the current state, then the plain step (vmas_step) advances the world and
 * its result is the target; loss into d_loss [1] and the gradient, kept for
 * vmas_sur_adam and copied to d_grad (both device, may be NULL). */
int vmas_sur_train_grad(vmas_surrogate *sur, vmas_world *world, const float *d_actions,
                        float *d_loss, float *d_grad, void *stream);
/* vmas_sur_train_grad then one Adam update. */
int vmas_sur_train_step(vmas_surrogate *sur, vmas_world *world, const float *d_actions, float lr,
                        float *d_loss, void *stream);
/* One world step by the surrogate.  Envs whose predicted bodies overlap one
 * another, or a wall, by more than `limit` world units (sphere-box and box-box
 * by the step's narrow phase; or whose prediction is not finite) are stepped
 * by the plain step instead; the other envs take the prediction (x, y, vx,
 * vy of the agents and boxes, and the boxes' theta, omega; walls unchanged).
 * d_n_fallback (device int32, may be NULL) receives the number of envs that
 * fell back. */
int vmas_sur_step(vmas_surrogate *sur, vmas_world *world, const float *d_actions, float limit,
                  int32_t *d_n_fallback, void *stream);
/* Diagnostic: the features of the world's current state as bfloat16 bits,
 * d_node [n_envs * nodes][16], d_edge [6][n_envs * nodes][16] (neighbour
 * slot major), d_mask [6][n_envs * nodes] (1 for a present neighbour); any
 * may be NULL. */
int vmas_sur_debug_features(vmas_surrogate *sur, vmas_world *world, const float *d_actions,
                            uint16_t *d_node, uint16_t *d_edge, float *d_mask, void *stream);
/* Wait for `stream` and return VMAS_EDEVICE (clearing the word) if one of
 * the surrogate's kernels raised its device error word (VMAS_DEVERR_TIMEOUT:
 * a tensor-core GEMM's bounded wait for its copies or MMAs ran out; the CTA
 * left its rows unwritten and freed its tensor memory). */
int vmas_sur_check(vmas_surrogate *sur, void *stream, int32_t *bits);
/* Diagnostic: the surrogate's GEMM, C [M][N] = A B with A(m, k) =
 * trans_a ? a[k lda + m] : a[m lda + k] and B(k, n) = trans_b ? b[n ldb + k]
 * : b[k ldb + n], bfloat16 operands (bits), FP32 accumulation; plus bias [N]
 * (FP32, may be NULL) into d_out_f32 [M][N] (may be NULL) and GELU (gelu != 0)
 * of it rounded into d_out_bf16 [M][N] (may be NULL).  splits > 1 sums K in
 * that many chunks (then no bias, GELU or bfloat16 output).  Untransposed A
 * with transposed B, K a multiple of 8 up to 128, N up to 128 and no split
 * run on the tcgen05 GEMM (tensor memory accumulators, TMA-staged operands);
 * transposed A with untransposed B, M and N up to 128, K >= 4096, a split,
 * no bias on the split-K tcgen05 weight-gradient GEMM (at most `splits`
 * partial blocks; lda, ldb multiples of 8); the rest on the warp-level mma
 * GEMM.  It allocates temporary buffers,
 * waits for `stream`, and returns VMAS_EDEVICE if a bounded wait of the
 * tcgen05 GEMM ran out. */
int vmas_debug_gemm_bf16(int32_t trans_a, int32_t trans_b, int32_t M, int32_t N, int32_t K,
                         const uint16_t *d_a, int32_t lda, const uint16_t *d_b, int32_t ldb,
                         const float *d_bias, int32_t gelu, float *d_out_f32,
                         uint16_t *d_out_bf16, int32_t splits, void *stream);

/* Diagnostic: which GEMM the surrogate's kernels use, process-wide: 0 = the
 * tcgen05 GEMM wherever the shape allows (the default), 1 = the warp-level
 * mma GEMM only (for comparisons), -1 = leave it.  tc_launches (may be NULL)
 * receives the number of tcgen05 GEMM launches in this process so far. */
int vmas_debug_gemm_engine(int32_t engine, int64_t *tc_launches);

/* Test hook for failure detection without a GPU fault, process-wide: while
 * `on` is set, every A-tile barrier of the tcgen05 GEMM, and every stage
 * barrier of the split-K weight-gradient GEMM, expects 16 transaction bytes
 * that no copy delivers, so its bounded waits run out (in
 * a few seconds); each CTA then sets VMAS_DEVERR_TIMEOUT, waits (bounded) for
 * its copies, frees its tensor memory and returns, leaving its rows
 * unwritten, and the context stays usable.  Off by default. */
int vmas_debug_gemm_timeout(int32_t on);

/* Message of the last failure on this thread ("" if none). */
const char *vmas_last_error(void);

/* VMAS_ABI_VERSION of the loaded library. */
int vmas_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VMAS_H_ */
