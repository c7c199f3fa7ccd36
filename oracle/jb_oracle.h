/*
 * FP64 CPU oracle for the batched rigid-body step of block-tower collapse
 * episodes ("GPU-Accelerated Inverse Structural Anastylosis from Block
 * Collapse Dynamics", Sec. 4 rigid body, Sec. 6 collision, Sec. 7 PGS,
 * Sec. 8 stability).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, sequential statement of
 * the method that the CUDA path is checked against.  It shares no code,
 * header, table or helper with the CUDA library, and nothing in the product
 * path may link or call it: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg use it.
 *
 * Units SI, z up, quaternions q = [w, x, y, z] (Hamilton), angular velocity in
 * the world frame.  Arrays crossing this header are structure-of-arrays,
 * component-major: x[c * B + b].
 *
 * Every step function is pinned by the tests to closed forms, brute force,
 * invariants or the paper's printed thresholds.  Parity unpinned: whole
 * collapse episodes (or_run_protocol over a push/removal schedule that ends
 * in a collapse) are chaotic; their outcomes are compared only statistically.
 * The X-axis Ziglar factor k = 4 enters only as a schedule input, pinned to
 * the paper's printed force and not to a derivation.
 */
#ifndef JB_ORACLE_H
#define JB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_world or_world;

typedef struct {
  double dt;             /* step length (s) */
  int n_sub;             /* substeps per step, each a full detect-solve-integrate */
  int pgs_iters;         /* sweeps in fixed-iteration mode (residual_tol == 0) */
  double residual_tol;   /* > 0: sweep until the residual <= tol (m/s) */
  int pgs_iter_cap;      /* sweep cap in residual mode */
  int pgs_min_iters;     /* sweeps before the first residual check */
  double restitution;    /* e in the normal-row update */
  double beta, slop;     /* position correction */
  double contact_margin; /* speculative contact margin m_c */
  double aabb_eps;       /* broadphase epsilon */
  double gravity[3];
  int warm_start;        /* 0 none, 1 previous frame */
  double match_radius;   /* warm-start point matching radius (m) */
  double fall_frac, collapse_ek, collapse_theta_deg, rest_ek;
  int rest_steps;
  int friction_cone;     /* 0: box clip per tangent row (Eq. coulomb_pgs); 1: the two tangent
                            rows of a point projected together onto the disc |lambda_t| <=
                            mu lambda_n (the Coulomb cone of the PGS figure) */
  int restitution_newton; /* 0: the listing's (1+e) factor in every normal row (no bounce at
                            the fixed point); 1: Newton restitution, rows without the factor
                            and a touching point approaching faster than restitution_vmin
                            targets v_n = -e v_n(pre-solve) */
  double restitution_vmin; /* m/s; <= 0 selects 2 |g| h */
  int colour_order;      /* 0: Gauss-Seidel in natural pair order (the listing); 1 and 2: in the
                            GPU library's colour order: greedy lowest-free colouring of the pairs
                            taken by (1) lower body a ascending, upper body b descending or (2)
                            the height of their first point in 1 mm bins ascending, natural index
                            descending; colours ascending, natural index ascending within a
                            colour.  Static bodies
                            (the ground) do not constrain the colouring.  Same fixed point.  This
                            restates the GPU's schedule so that a fixed number of unconverged
                            sweeps can be compared iterate for iterate; it is opt-in for that test
                            alone and is never used by a pin or a converged-parity test. */
  int pgs_accel_period;      /* 0: plain projected Gauss-Seidel (the paper).  m > 0: after every m
                            sweeps one nonsmooth conjugate-gradient step (see solve()); the
                            converged impulses are those of plain PGS. */
  double sat_tie;        /* SAT axis-choice hysteresis (m); <= 0 selects the default 1e-5 (a later
                            face axis replaces the best only if smaller by this much) */
} or_params;

/* episode statistics, one row of OR_NSTAT doubles per episode */
enum {
  OR_ST_STATUS = 0, OR_ST_COLLAPSED, OR_ST_RESTING, OR_ST_NFALLEN, OR_ST_COM_IMB,
  OR_ST_EK, OR_ST_LAST_RES, OR_ST_LAST_SWEEPS, OR_ST_TOTAL_SWEEPS, OR_ST_SOLVES,
  OR_ST_STEPS, OR_ST_BODY_STEPS, OR_ST_PHASE, OR_ST_MOVES_DONE, OR_ST_NPAIRS,
  OR_ST_NPOINTS, OR_ST_MAX_RES, OR_NSTAT
};
enum { OR_PH_FREE = 0, OR_PH_PUSH, OR_PH_SETTLE, OR_PH_REST, OR_PH_DONE };
enum { OR_STATUS_NOT_CONVERGED = 2, OR_STATUS_NONFINITE = 4 };

/* contact record: OR_CREC doubles per pair
   [0] a (-1 ground) [1] b [2] axis [3] ref_face [4] inc_face [5] n_points
   [6..8] n [9..11] t1 [12] delta [13] mu [14] depth_max
   then 4 x { p[3], depth, lambda[3] (n, t1, t2), local_in_A[3] } */
#define OR_CREC 55

#define OR_NFEAT 24   /* warm-start features per contact point */
#define OR_REC 27     /* recorder row: features, then converged impulses over m_bar |g| h */

or_world* or_create(int n_episodes, const int* body_off, const double* half,
                    const double* mass, const double* mu, const double* x,
                    const double* q, const double* v, const double* w,
                    const double* ground_mu, const or_params* p);
void or_destroy(or_world* W);
int or_set_protocol(or_world* W, const int* off, const int* block, const int* axis,
                    const double* sign, const double* factor, const double* k,
                    const int* remove, const int* push_steps, const int* settle_steps);
/* runs every unfinished episode through its schedule; returns max steps taken */
int or_run_protocol(or_world* W, int max_steps, int n_threads);
/* host-driven stepping (no schedule) */
void or_step(or_world* W, int n_steps, int n_threads);
int or_apply_push(or_world* W, int episode, int block, int axis, double force, int n_steps);
int or_remove_block(or_world* W, int episode, int block);
void or_get_state(const or_world* W, double* x, double* q, double* v, double* w);
void or_set_state(or_world* W, const double* x, const double* q, const double* v,
                  const double* w);
void or_clear_cache(or_world* W);
/* Training-sample recorder: after every `every`-th converged solve (counted
   per episode), each contact point appends one OR_REC row (caller buffer of
   `capacity` rows; or_recorded returns rows claimed, may exceed capacity). */
void or_set_recorder(or_world* W, double* rows, int capacity, int every);
long or_recorded(const or_world* W);
int or_get_contacts(const or_world* W, int episode, double* out, int cap);
void or_get_stats(or_world* W, double* out);
double or_com_imbalance(const or_world* W, int episode);
/* Reference-episode search (Sec. 11.2): argmin over collapsed episodes of
   |removed blocks - n_hat| (lowest index on ties), else the episode with the
   most completed moves; returns the index, *n_removed its removed count. */
int or_reference_episode(const or_world* W, int n_hat, int* n_removed);
/* Eq. collapse terms of an episode's current state against its reference
   poses: kinetic energy (J), largest displacement over block length, largest
   tilt of a thickness axis (rad), blocks displaced by more than fall_frac. */
void or_collapse_terms(const or_world* W, int episode, double* ek, double* dx_ratio, double* theta,
                       int* n_fallen);
int or_active(const or_world* W, int body);

/* stage-level entry points (pins) */
int or_sat(const double* xA, const double* qA, const double* hA,
           const double* xB, const double* qB, const double* hB, double margin,
           double* delta15, int* valid15, int* axis, double* n, double* dmin);
/* the axis choice alone, on given separations (15 axes, validity flags) */
int or_sat_select(const double* delta15, const int* valid15, double* dmin);
int or_pair_manifold(const double* xA, const double* qA, const double* hA,
                     const double* xB, const double* qB, const double* hB,
                     double margin, double* out /* OR_CREC */);
int or_ground_manifold(const double* x, const double* q, const double* h,
                       double margin, double* out /* OR_CREC */);
void or_rotmat(const double* q, double* R /* row-major 3x3 */);
void or_body_inertia(double mass, const double* half, double* I /* diag */);
double or_support_margin(int n_pts, const double* xy /* 2*n */, const double* com);
int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
