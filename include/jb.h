/*
 * jb.h -- C ABI of the batched rigid-body step for block-tower collapse
 * episodes ("GPU-Accelerated Inverse Structural Anastylosis from Block
 * Collapse Dynamics").
 *
 * One call advances thousands of independent episodes (towers of boxes on a
 * ground plane) through the paper's step: AABB broadphase (Sec. 6.1,
 * Eq. aabb), OBB separating-axis narrowphase over 15 axes (Sec. 6.2),
 * face-clipped contact manifolds (Sec. 6.2.1), a Projected Gauss-Seidel
 * normal + Coulomb-friction solve (Sec. 7, Eq. keff, Eq. lambda_n,
 * Eq. coulomb_pgs), semi-implicit Euler with quaternion integration
 * (Sec. 4, Eq. newton_euler, Eq. quat_int), Baumgarte position correction
 * (Sec. 7.4, Eq. baumgarte) and the stability / collapse tests of Sec. 8
 * (Eq. stability, Eq. collapse).  Pushes follow Ziglar's thresholds
 * F = k mu_s m g (Sec. 5, Eq. 4 and Eq. 8).
 *
 * Conventions
 *  - SI units, z up, the ground is the plane z = 0 (a static body).
 *  - Quaternions q = [w, x, y, z] (Hamilton product), unit length; angular
 *    velocity in the world frame.  Body frame of a block: x = length,
 *    y = width, z = thickness.
 *  - Per-body arrays are structure-of-arrays, component-major: the c-th
 *    component of body b (global index over all episodes) is arr[c * B + b].
 *    Episodes are concatenated; body_off[e] .. body_off[e+1]-1 are episode
 *    e's bodies and "block" arguments are episode-local indices.
 *  - Memory: the library never allocates device memory.  The caller passes
 *    one device workspace (jb_workspace_bytes) that the batch carves up; all
 *    other pointers are host pointers unless a call says otherwise.  The
 *    library never frees caller memory.
 *  - Work is queued on the stream given at creation; calls that return data
 *    to host memory synchronise that stream before returning.
 *  - Errors: every call returns a jb_status.  Argument errors are detected
 *    synchronously and nothing is launched.  Device-side failures (contact
 *    capacity exceeded, sweep cap hit, non-finite state) are recorded per
 *    episode and surfaced by jb_sync / jb_read_episode_stats.  The message of
 *    the last error on the calling thread is returned by jb_last_error().
 */
#ifndef JB_H
#define JB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t jb_status;
#define JB_OK 0
#define JB_EINVAL (-1)   /* bad argument (null pointer, bad size, bad parameter) */
#define JB_ENOMEM (-2)   /* workspace too small */
#define JB_ECUDA (-3)    /* a CUDA runtime call failed */
#define JB_ERANGE (-4)   /* episode or block index out of range */
#define JB_ESTATE (-5)   /* call not valid in the batch's current state */

/* per-episode status bits (jb_episode_stats.status) */
#define JB_EP_CONTACT_OVERFLOW 1  /* more pairs or candidates than the capacity; extras dropped */
#define JB_EP_NOT_CONVERGED 2     /* residual mode: a solve ended above the tolerance (at pgs_iter_cap,
                                     or stopped by the stall test) at least once */
#define JB_EP_NONFINITE 4         /* a position or velocity became NaN/Inf; episode stopped */
#define JB_EP_TOO_MANY_COLOURS 8  /* colouring overflowed; overflow pairs solved serially */

/* episode phases */
#define JB_PH_FREE 0     /* host-driven (jb_step) */
#define JB_PH_PUSH 1
#define JB_PH_SETTLE 2
#define JB_PH_REST 3     /* collapsed; running until at rest (Sec. 8.3) */
#define JB_PH_DONE 4

/* push axes (block-local, Sec. 5): X = width axis (body y), Y = long axis (body x) */
#define JB_AXIS_X 0
#define JB_AXIS_Y 1

/* Solver parameters.  Defaults (jb_default_params) follow the paper's
 * Appendix A table where it gives a value: dt = 1/240 s, e = 0.10,
 * beta = 0.35, slop = 0.4 mm, AABB eps = 2 mm, g = 9.81. */
typedef struct {
  float dt;                 /* step length, s */
  int32_t n_sub;            /* substeps per step (each a full detect-solve-integrate) */
  int32_t pgs_iters;        /* sweeps per solve in fixed mode (residual_tol == 0) */
  float residual_tol;       /* > 0: residual mode, sweep until residual <= tol (m/s) */
  int32_t pgs_iter_cap;     /* sweep cap in residual mode */
  int32_t pgs_min_iters;    /* sweeps before the first residual check */
  int32_t residual_every;   /* residual mode: at least this many sweeps between checks (>= 1) */
  float restitution;        /* e, applied as (1+e) in the normal row (Sec. 7.1) */
  float beta, slop;         /* Eq. baumgarte */
  float contact_margin;     /* speculative contact margin m_c, m */
  float aabb_eps;           /* Eq. aabb epsilon, m */
  float gravity[3];         /* m/s^2 */
  int32_t warm_start;       /* 0 none, 1 previous-frame impulses, 2 previous-frame where a
                               point matches; on a step where at least half of the
                               episode's pairs are new (no point matched), the warm-start
                               network for the points of the new pairs; zero elsewhere;
                               3 the network for every point (2 and 3 need
                               jb_set_warmstart_mlp) */
  float match_radius;       /* warm-start point match radius, m */
  float fall_frac;          /* Eq. collapse f_d */
  float collapse_ek;        /* Eq. collapse eps_k, J */
  float collapse_theta_deg; /* Eq. collapse theta_th, degrees */
  float rest_ek;            /* Sec. 8.3 rest threshold, J */
  int32_t rest_steps;       /* Sec. 8.3 step budget after collapse */
  float smem_pair_factor;   /* shared-memory solver capacity per episode: factor * bodies + 16
                               contact pairs (0 = 4); steps with more pairs use global memory.
                               Read at batch creation. */
  float sor;                /* relaxation factor omega of the PGS rows, in (0, 2); 0 = 1, the
                               paper's plain projected Gauss-Seidel.  Every row takes
                               proj(lambda - omega (v + b) / k) (projected SOR, Cryer 1971): the
                               fixed points, and so the converged impulses, do not depend on
                               omega; the sweeps needed to reach residual_tol do. */
  int32_t sweep_order;      /* 0: every sweep visits the colours in order; 1: odd sweeps visit
                               them in reverse (symmetric Gauss-Seidel) */
  int32_t residual_every_max; /* residual mode: at most this many sweeps between checks.  Above
                               residual_every, the gap to the next check is half the sweeps
                               the last two residuals predict are still needed (geometric
                               decay), clamped to [residual_every, residual_every_max]; a solve
                               only ends at a check, so this bounds the extra sweeps a
                               converged solve runs.  0 = residual_every (fixed cadence). */
  int32_t stall_window;     /* residual mode, 0 = off: every stall_window sweeps the solve fits
                               the residual's geometric decay over that window and stops when
                               the fit says the tolerance cannot be reached within
                               pgs_iter_cap (no decay, or more sweeps needed than are left).
                               Such a solve counts as capped (JB_EP_NOT_CONVERGED) like one
                               that runs to the cap. */
  int32_t friction_cone;    /* 0: each tangent row clipped to [-mu lambda_n, mu lambda_n] (Eq.
                               coulomb_pgs, the default); 1: a point's two tangent rows take one
                               common step 1/k_t, k_t = max(k_t1, k_t2), and are projected
                               together onto the disc |lambda_t| <= mu lambda_n (the Coulomb cone
                               of the PGS figure).  The residual uses the same projection. */
  int32_t restitution_newton; /* 0: the listing's (1+e) factor in every normal row (Sec. 7.1; at
                               the fixed point v_n = -b, no bounce); 1: Newton restitution, the
                               rows without the factor and a touching point approaching faster
                               than restitution_vmin targets v_n = -e v_n(pre-solve) */
  float restitution_vmin;   /* m/s; <= 0 selects 2 |g| h (resting contacts approach at |g| h) */
  int32_t pgs_accel_period; /* 0: plain projected Gauss-Seidel (the paper).  m > 0: after every m
                               sweeps of a solve, one nonsmooth conjugate-gradient step
                               (Silcowitz, Niebe and Erleben 2010, with a block of m sweeps as
                               the map G): r = G(lambda) - lambda over the block, beta =
                               |r_k|^2 / |r_(k-1)|^2 (0 on the first block and when above 1),
                               lambda <- proj(G(lambda) + beta d), d <- r_k + beta d, the
                               impulse change applied to the bodies.  A fixed point of the sweep
                               is one of this iteration, so the converged impulses are plain
                               PGS's and the residual test is unchanged; the sweeps needed to
                               reach residual_tol fall.  Uses jb_workspace_bytes' scratch. */
  int32_t colour_key;       /* order in which the greedy colouring takes the pairs (the sweep order
                               of the Gauss-Seidel phases; same fixed point): 0 = lower body
                               ascending, upper body descending; 1 = height of the pair's first
                               contact point in 1 mm bins ascending, natural index descending */
} jb_solver_params;

/* Initial scene: host arrays, B = body_off[n_episodes] bodies. */
typedef struct {
  int32_t n_episodes;
  const int32_t* body_off;  /* [E+1], body_off[0] = 0, non-decreasing */
  const float* half;        /* [3][B] half extents, > 0 */
  const float* mass;        /* [B] kg; 0 marks a static box */
  const float* mu;          /* [B] Coulomb coefficient; a pair uses the smaller of its two */
  const float* x;           /* [3][B] centre of mass */
  const float* q;           /* [4][B] orientation (normalised on load) */
  const float* v;           /* [3][B] linear velocity, may be NULL (zero) */
  const float* w;           /* [3][B] angular velocity, may be NULL (zero) */
  const float* ground_mu;   /* [E] ground friction coefficient */
} jb_scene;

/* Tower description (Sec. 3.1: 3 blocks per layer, alternating perpendicular
 * layers, flush, bottom on z = 0; even 0-based levels along world X). */
typedef struct {
  int32_t levels;
  int32_t per_level;        /* blocks per level (3 in the paper) */
  float dims[3];            /* block length, width, thickness, m */
  float mass;               /* nominal block mass, kg */
  float mass_jitter;        /* uniform +- fraction (SplitMix64 draw per block) */
  float mu_s;
} jb_tower_desc;

/* Per-episode push/removal schedule, CSR over moves (host arrays).  Move m
 * pushes `block` along its `axis` with force sign * factor * k * mu_s * m * |g|
 * (Sec. 5 threshold times a factor) at its centre of mass for push_steps
 * steps, then deletes the block if remove != 0, then lets the tower settle for
 * settle_steps steps.  The episode stops early on collapse (Eq. collapse) and
 * then runs until at rest (Sec. 8.3). */
typedef struct {
  const int32_t* off;        /* [E+1] */
  const int32_t* block;      /* [M] episode-local body index */
  const int32_t* axis;       /* [M] JB_AXIS_X / JB_AXIS_Y */
  const float* sign;         /* [M] +1 / -1 */
  const float* factor;       /* [M] */
  const float* k;            /* [M] threshold multiplier (3 or 4 in Sec. 5) */
  const int32_t* remove;     /* [M] */
  const int32_t* push_steps; /* [M] */
  const int32_t* settle_steps; /* [M] */
} jb_protocol;

/* One contact point as read back: pair (a, b) with a = -1 for the ground,
 * SAT axis id (0..2 faces of a, 3..5 faces of b, 6..14 edge pairs a_i x b_j,
 * 15 ground), reference/incident feature ids, the point, the normal (from a
 * to b), the depth (positive = penetrating) and the accumulated impulses
 * (normal, t1, t2) of the last solve. */
typedef struct {
  int32_t a, b, axis, ref_face, inc_face, point;
  float p[3];
  float n[3];
  float t1[3];
  float depth;
  float lambda[3];
} jb_contact;

typedef struct {
  int32_t status;           /* JB_EP_* bits */
  int32_t phase;            /* JB_PH_* */
  int32_t collapsed;        /* Eq. collapse fired */
  int32_t resting;          /* kinetic energy below rest_ek */
  int32_t n_fallen;         /* active blocks displaced more than fall_frac * length */
  int32_t moves_done;
  int32_t n_pairs, n_points;  /* of the last substep */
  int32_t last_sweeps;
  int32_t steps;
  int32_t max_colours;      /* most colours used by one solve (Gauss-Seidel phases per sweep) */
  int32_t capped_solves;    /* residual mode: solves that reached pgs_iter_cap above the tolerance */
  float com_imbalance;      /* minus the support-polygon margin of Eq. stability, m */
  float kinetic;            /* J, active dynamic bodies */
  float last_residual;      /* m/s */
  float max_residual;       /* m/s, over all solves */
  double total_sweeps;
  double solves;
  double body_steps;        /* sum over steps of active dynamic bodies */
  /* work counters (sums over substeps): contact points x sweeps, contact
     points, contact pairs, broadphase pair tests */
  double point_sweeps, point_steps, pair_steps, bp_tests;
  double mlp_points;        /* contact points whose start came from the warm-start network */
  /* Eq. stability on the device after every step (same support polygon and
     COM as com_imbalance): the margin after the last step (m, positive
     inside), the smallest margin over the steps run, the first step (1-based
     count) whose margin was negative and the step at which Eq. collapse
     fired (-1 for none; both since creation or the last jb_set_protocol) */
  float stability_margin;
  float min_stability_margin;
  int32_t first_unstable_step;
  int32_t collapse_step;
} jb_episode_stats;

typedef struct jb_batch jb_batch;

void jb_default_params(jb_solver_params* p);

/* Tower builder (host only, no device work).  jb_tower_layout writes the
 * CSR body offsets [E+1]; jb_tower_init fills half, mass, mu, x, q for all
 * bodies ([3][B], [B], [B], [3][B], [4][B]) and ground_mu [E].  Mass draws:
 * u = splitmix64(seed ^ e*0x9E3779B97F4A7C15 ^ (1<<48) ^ block) >> 11 scaled
 * to [0,1), m = mass * (1 + mass_jitter * (2u - 1)). */
jb_status jb_tower_layout(const jb_tower_desc* towers, int32_t n_episodes, int32_t* body_off);
jb_status jb_tower_init(const jb_tower_desc* towers, int32_t n_episodes, uint64_t seed,
                        const int32_t* body_off, float* half, float* mass, float* mu,
                        float* x, float* q, float* ground_mu);

/* Device workspace needed for a batch with these episode sizes (host body_off)
 * and at most max_moves scheduled moves in total.  Returns 0 on bad input. */
size_t jb_workspace_bytes(int32_t n_episodes, const int32_t* body_off,
                          const jb_solver_params* p, int32_t max_moves);

/* Creates a batch over caller-owned device workspace d_workspace (at least
 * jb_workspace_bytes, 256-byte aligned), uploads the scene and initialises
 * derived state on `cuda_stream` (a cudaStream_t, NULL = legacy default).
 * The batch starts in the host-driven phase with an empty contact cache. */
jb_status jb_batch_create(const jb_scene* scene, const jb_solver_params* p, int32_t max_moves,
                          void* d_workspace, size_t workspace_bytes, void* cuda_stream,
                          jb_batch** out);
void jb_batch_destroy(jb_batch* b);   /* frees the host handle only */

/* Replaces the solver parameters (same batch shape). */
jb_status jb_set_params(jb_batch* b, const jb_solver_params* p);

/* Uploads a schedule (total moves <= max_moves) and starts move 0 of every
 * episode (episodes with no moves are marked done). */
jb_status jb_set_protocol(jb_batch* b, const jb_protocol* prot);
/* Runs every unfinished episode through its schedule for at most max_steps
 * steps in one persistent launch.  Asynchronous. */
jb_status jb_run_protocol(jb_batch* b, int32_t max_steps);

/* Host-driven stepping.  Asynchronous; argument errors (null arrays, n < 0,
 * episode or block out of range: JB_EINVAL / JB_ERANGE) are returned before
 * anything is queued.  Host arrays are read during the call only.
 *
 * jb_apply_push (Sec. 5, Eq. 4 and Eq. 8: a push of F_app along one of the
 * block's own axes, at its centre of mass; the caller picks F_app, e.g.
 * k mu_s m g): for n entries, a constant force force_N (signed, N) along
 * the block's axis (JB_AXIS_X = width axis, JB_AXIS_Y = long axis; the
 * direction is fixed at the call) for n_steps steps. */
jb_status jb_apply_push(jb_batch* b, int32_t n, const int32_t* episode, const int32_t* block,
                        const int32_t* axis, const float* force_N, const int32_t* n_steps);
/* jb_remove_block (the removal rounds of Sec. 12.2 and Sec. 13.1: a block
 * taken out of the tower): deactivates n blocks; they leave the broadphase,
 * their contacts and warm-start entries, and the body-step count, and keep
 * their last pose. */
jb_status jb_remove_block(jb_batch* b, int32_t n, const int32_t* episode, const int32_t* block);
/* jb_step (Sec. 4.2 and Sec. 6-7: forces and the velocity predictor, AABB
 * broadphase, SAT narrowphase and manifold, PGS, integration, Baumgarte
 * correction, n_sub substeps per step): advances every episode in the
 * host-driven phase by n_steps steps. */
jb_status jb_step(jb_batch* b, int32_t n_steps);

/* Waits for queued work; *n_bad_episodes (may be NULL) = episodes whose status is non-zero. */
jb_status jb_sync(jb_batch* b, int32_t* n_bad_episodes);

/* Size classes of the batch (episodes split by body count at creation, each
 * launched as one persistent kernel per jb_step / jb_run_protocol call): the
 * count and, if the arrays are non-NULL, each class's episode count, largest
 * body count and grid size (host arrays of at least 4 entries).  No device
 * work.  (Launch bookkeeping for callers; the paper has no counterpart.) */
jb_status jb_size_classes(const jb_batch* b, int32_t* n_classes, int32_t* episodes, int32_t* max_bodies,
                          int32_t* grid);

/* State transfer (Sec. 4.1: the state S = (x, q, v, w) of every body),
 * [3][B] / [4][B] arrays, host pointers unless device_ptrs != 0 (then device
 * pointers, copied on the batch stream).  Any pointer may be NULL.  Host
 * reads synchronise the batch stream; a NULL batch gives JB_EINVAL.
 * jb_write_state keeps the contact cache unless clear_cache != 0 and, when
 * reset_reference != 0, takes the new poses as the collapse reference. */
jb_status jb_read_state(jb_batch* b, float* x, float* q, float* v, float* w, int32_t device_ptrs);
jb_status jb_write_state(jb_batch* b, const float* x, const float* q, const float* v,
                         const float* w, int32_t device_ptrs, int32_t clear_cache,
                         int32_t reset_reference);
/* Active flags [B] (1 = in the simulation). */
jb_status jb_read_active(jb_batch* b, int32_t* active);

/* Contact points of the last substep of one episode (Sec. 6.2.1: the
 * clipped manifold of each pair, at most 4 points, with the impulses of the
 * Sec. 7 solve), natural order (ground pairs by body, then pairs (a, b)
 * ascending, points in manifold order).  out is a host array of cap entries;
 * *n_out = points written.  JB_ERANGE for a bad episode; JB_ENOMEM if the
 * episode has more than cap points (the first cap are written).
 * Synchronises the batch stream. */
jb_status jb_read_contacts(jb_batch* b, int32_t episode, jb_contact* out, int32_t cap,
                           int32_t* n_out);
/* Per-episode statistics [E] (host array; Sec. 8: the support-polygon margin
 * of Eq. stability as com_imbalance = -margin, the Eq. collapse flag and
 * fallen count, the Sec. 8.3 rest test; plus solver counters).  Computes the
 * margin on the device and synchronises the batch stream. */
jb_status jb_read_episode_stats(jb_batch* b, jb_episode_stats* out);

/* Reference-episode search (Sec. 11.2, the similarity step): among the
 * collapsed episodes, the one whose count of removed blocks is closest to
 * n_removed_hat (lowest index on ties); if none collapsed, the one with the
 * most completed moves (rounds; lowest index on ties).  *episode = the
 * chosen index, *n_removed (may be NULL) = its removed-block count.
 * Synchronous: reads the episode statistics and the active flags. */
jb_status jb_reference_episode(jb_batch* b, int32_t n_removed_hat, int32_t* episode, int32_t* n_removed);

/* Raw snapshot of all mutable device state for exact resume: the Sec. 4.1
 * state of every body, the episode schedule position (Sec. 12.2 rounds), the
 * contact caches that warm-start the Sec. 7.3 solve.  host_buf holds at least
 * jb_state_bytes bytes (JB_ENOMEM otherwise); jb_load_state needs a snapshot
 * of a batch of the same shape.  Both synchronise the batch stream. */
size_t jb_state_bytes(const jb_batch* b);
jb_status jb_save_state(jb_batch* b, void* host_buf, size_t bytes);
jb_status jb_load_state(jb_batch* b, const void* host_buf, size_t bytes);

/* ---- Learned warm start (not in the paper: a small network that predicts
 * a contact point's starting impulses from local features; plain PGS still
 * decides convergence, and the gate compares against it).
 *
 * Features (JB_FEATURES floats per contact point, computed after the force
 * predictor and before the solve, with s_v = 1/(|g| h), s_l = 1/(m_bar |g| h),
 * m_bar = 0.015 kg, L_bar = 0.075 m, h the substep):
 *   0-2   relative point velocity of b w.r.t. a along n, t1, t2, times s_v
 *   3     depth / contact_margin
 *   4-8   n, then t1.x, t1.y (t1.z follows from n by the tangent rule)
 *   9     height of the episode's column above the point: the highest AABB
 *         top of its active dynamic blocks minus the point's z, over 0.15 m
 *         (ten nominal block thicknesses); stands in for the load above
 *   10-11 m_bar / m of a, b (0 for static bodies and the ground)
 *   12-17 body-frame inertia diagonals of a, b over m_bar L_bar^2 (0 if static)
 *   18    friction coefficient
 *   19-21 previous-frame impulses (n, t1, t2) times s_l (0 if unmatched)
 *   22    1 if the point matched a previous-frame point
 *   23    1 if a is the ground
 * Outputs: impulses (n, t1, t2) times s_l, projected to lambda_n >= 0 and
 * |lambda_t| <= mu lambda_n before use.
 * Network: 24 -> 128 -> 128 -> 3, ReLU, parameters W1 [24][128], b1, W2
 * [128][128], b2, W3 [128][3], b3 (row-major [in][out], FP32 master copy,
 * BF16 tensor-core operands with FP32 accumulation). */
#define JB_FEATURES 24
#define JB_REC_FLOATS 27   /* recorder row: features, then converged impulses times s_l */

/* The batch uses the network block d_mlp (device, jb_mlp_bytes, caller
 * owned; NULL removes it) for warm_start 2 and 3. */
jb_status jb_set_warmstart_mlp(jb_batch* b, const void* d_mlp);
/* Training-sample recorder: after every `every`-th converged solve, each
 * contact point appends one JB_REC_FLOATS row to d_rows (device, capacity
 * rows); *d_count (device int32, caller zeroes it) counts rows claimed and may
 * exceed capacity (extra rows are dropped).  capacity 0 turns it off. */
jb_status jb_set_recorder(jb_batch* b, float* d_rows, int32_t capacity, int32_t* d_count, int32_t every);

/* Which points the recorder takes: 0 (the default) every point of a recorded
 * solve; 1 only the points of pairs none of whose points had a previous-frame
 * impulse, the ones the learned warm start predicts in mode 2 (so that the
 * training set has the distribution the network meets).  JB_EINVAL for other
 * values. */
jb_status jb_set_recorder_points(jb_batch* b, int32_t unmatched_only);

size_t jb_mlp_bytes(void);              /* device bytes of a network block */
int32_t jb_mlp_param_count(void);       /* floats of one parameter set */
/* Device scratch of jb_mlp_forward / jb_mlp_grad / jb_mlp_train_step for n
 * rows (the gradient, the loss, an error flag and one row of partial sums per
 * CTA, up to 160 CTAs: about 80 KB per 128 rows, at most 12.8 MB; 0 for
 * n <= 0).  The batch forward and the gradient run in one fused kernel on the
 * tcgen05 tensor cores (BF16 operands in shared memory, FP32 accumulators in
 * tensor memory), one CTA per 128 rows up to one per SM; the rows and
 * activations never go to global memory.  The CTAs' partial sums are added
 * in a fixed order, so the gradient is bitwise reproducible. */
size_t jb_mlp_scratch_bytes(int32_t n);
/* Loads parameters (host, jb_mlp_param_count floats, layout above) into the
 * block, zeroes the AdamW moments and packs the BF16 operands. */
jb_status jb_mlp_load(void* d_mlp, const float* params, void* cuda_stream);
jb_status jb_mlp_save(const void* d_mlp, float* params, void* cuda_stream);
/* y [n][3] = network(x [n][24]); device arrays. */
jb_status jb_mlp_forward(const void* d_mlp, const float* d_x, int32_t n, float* d_y, void* d_scratch,
                         size_t scratch_bytes, void* cuda_stream);
/* Gradient of L = (1/n) sum_rows sum_c (y - t)^2 with respect to the
 * parameters (d_grad, FP32, parameter layout) and L itself (d_loss, may be
 * NULL); t [n][3]. */
jb_status jb_mlp_grad(const void* d_mlp, const float* d_x, const float* d_t, int32_t n, float* d_grad,
                      float* d_loss, void* d_scratch, size_t scratch_bytes, void* cuda_stream);
/* AdamW step `step` (1-based) on the master weights (weight decay on the
 * matrices only), then repack. */
jb_status jb_mlp_adamw(void* d_mlp, const float* d_grad, int32_t step, float lr, float beta1, float beta2,
                       float eps, float weight_decay, void* cuda_stream);
/* jb_mlp_grad on rows [0, n) of (x, t) followed by jb_mlp_adamw. */
jb_status jb_mlp_train_step(void* d_mlp, const float* d_x, const float* d_t, int32_t n, int32_t step, float lr,
                            float beta1, float beta2, float eps, float weight_decay, float* d_loss,
                            void* d_scratch, size_t scratch_bytes, void* cuda_stream);
/* Synchronises the stream and reads the error flag of the last
 * jb_mlp_forward / jb_mlp_grad / jb_mlp_train_step that used this scratch:
 * 1 if a wait of the tensor-core kernel for its own matrix products ran out
 * (about one second; the kernel then skipped its outputs, freed its tensor
 * memory and returned), else 0. */
jb_status jb_mlp_scratch_error(const void* d_scratch, size_t scratch_bytes, void* cuda_stream, int32_t* out);

/* Stepping for callers that cannot allocate device memory.
 *
 * Not part of the paper's method (the paper has no counterpart): an
 * allocation-free variant of jb_batch_create + jb_step for code that runs
 * where device allocation is unavailable or forbidden -- inside a memory pool
 * owned by another framework, in a real-time loop that must not call
 * cudaMalloc, or in a process whose allocator is locked.  It advances
 * n_episodes independent episodes by n_steps host-driven steps (gravity and
 * contacts only; no pushes or schedule), starting with an empty warm-start
 * cache, and writes the new state back in place.
 *
 * Arguments: body_off is a HOST array [n_episodes + 1]; every other array is
 * DEVICE memory in the layout of jb_scene ([3][B], [4][B], [B], [E]); d_x,
 * d_q, d_v, d_w are read and overwritten.  Work is queued on cuda_stream and
 * the call returns without synchronising; the caller synchronises before
 * reading the outputs.
 *
 * It runs the plain solver only: warm_start 0 or 1 (2 and 3 need a network
 * block, which this call has no way to take: JB_EINVAL).
 *
 * Scratch: the library's file-scope device array of JB_NOALLOC_SCRATCH_BYTES
 * (32 MiB; every GPU that loads the library holds it until the process
 * exits).  A batch whose layout needs more returns JB_ENOMEM with the sizes
 * in jb_last_error() and launches nothing.  The call makes no device memory
 * allocation and frees nothing.  Its first call on a device (n_steps 0
 * included) looks up the scratch address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  Each call also copies body_off from
 * the caller's host memory with cudaMemcpyAsync.  All calls share the one array, which keeps the last call's
 * contents (each call re-initialises what must start at zero): calls that
 * overlap on the GPU (different streams, or different host threads) race.
 */
#define JB_NOALLOC_SCRATCH_BYTES (32u << 20)
jb_status jb_step_noalloc(int32_t n_episodes, const int32_t* body_off, const float* d_half,
                          const float* d_mass, const float* d_mu, const float* d_ground_mu,
                          float* d_x, float* d_q, float* d_v, float* d_w,
                          const jb_solver_params* p, int32_t n_steps, void* cuda_stream);

/* Measurement utility (the paper has no counterpart): the FP32 multiply-add
 * rate that bounds the step.  jb_fma_probe queues one launch of `blocks`
 * CTAs of 256 threads, each thread running 8 independent multiply-add chains
 * for `iters` rounds, scalar (packed = 0) or packed two-lane FFMA2
 * (packed = 1), and writes one float per thread to d_sink (device, blocks *
 * 256 floats).  jb_fma_probe_flops gives the launch's flop count (an FMA is 2
 * flops), 0 for bad arguments.  The caller times the launch on cuda_stream. */
jb_status jb_fma_probe(int32_t packed, int32_t blocks, int32_t iters, float* d_sink, void* cuda_stream);
double jb_fma_probe_flops(int32_t packed, int32_t blocks, int32_t iters);

const char* jb_status_str(jb_status s);
const char* jb_last_error(void);
const char* jb_version(void);

#ifdef __cplusplus
}
#endif
#endif
