// Internal layout of a batch on the device: the descriptor every kernel
// receives by value, the per-episode state record and the shared-memory plan
// of one episode (one warp).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/jb.h"

namespace jbk {

constexpr int kWarpsPerCta = 1;          // one warp (episode) per CTA
constexpr int kMaxSizeClasses = 4;       // episode size classes per batch
constexpr int kMaxColours = 64;          // colour kSerial is solved by one lane
constexpr int kSerial = kMaxColours - 1;
constexpr int kMaxPts = 4;               // points per pair (Sec. 6.2.1, step d)
constexpr int kNatPtFloats = 12;         // p[3], depth, local[3], lambda[3], pad[2]
constexpr int kNatPairFloats = 8;        // n[3], depth_max, t1[3], mu
constexpr int kSrtPairFloats = 8;        // n[3], t1[3], mu, depth_max
constexpr int kSrtPtFloats = 13;         // p[3], 1/W_rr[3], W_01 W_02 W_12, bias, lambda[3]
// Record strides of the colour-sorted arrays (record-major, odd strides so
// that 32 lanes on consecutive slots hit 32 different banks).
constexpr int kPairStride = kSrtPairFloats + 1;             // floats per pair header
constexpr int kPtStride = kSrtPtFloats * kMaxPts + 1;       // floats per pair's points

// body flags
constexpr int kActive = 1;
constexpr int kStatic = 2;

// launch modes of the episode kernel
constexpr int kModeFree = 0;
constexpr int kModeProtocol = 1;

// Pair capacity of an episode with nb bodies.  An intact tower needs about
// 3.6 pairs per body; piles after a collapse need more.
__host__ __device__ inline int pair_capacity(int nb) { return 8 * nb + 16; }
// Broadphase candidate capacity (shared memory, u32 per candidate).
__host__ __device__ inline int cand_capacity(int nb) { return 16 * nb + 64; }

struct EpState {
  int32_t phase, mi, remaining, pb, rest_left;
  int32_t collapsed, resting, status;
  int32_t cur, npairs, ncolours, npoints;
  int32_t last_sweeps, steps, n_fallen, max_colours, capped;
  float last_res, max_res, kinetic, com_imb;
  double total_sweeps, solves, body_steps;
  double point_sweeps, point_steps, pair_steps, bp_tests, mlp_points;
  float margin, min_margin;            // Eq. stability after the last step, smallest so far
  int32_t first_unstable, collapse_step;   // 1-based step counts, -1 = none
};

struct Params {
  float dt;
  int n_sub, pgs_iters;
  float residual_tol;
  int pgs_iter_cap, pgs_min_iters, residual_every;
  float restitution, beta, slop, contact_margin, aabb_eps;
  float g[3];
  int warm_start;
  float match_radius, fall_frac, collapse_ek, collapse_cos, rest_ek;
  int rest_steps;
  float sor;        // PGS relaxation factor omega (1 = plain PGS)
  int sweep_order;  // 1: odd sweeps run the colours in reverse
  int residual_every_max;  // >= residual_every
  int stall_window;        // 0 = off
  int friction_cone;       // 1: disc projection of the tangent pair
  int restitution_newton;  // 1: bounce target instead of the (1+e) factor
  float restitution_vmin;  // m/s (resolved: > 0)
  int accel_period;        // 0 = plain PGS; m > 0: a conjugate-gradient step every m sweeps
  int colour_key;          // 0: (a asc, b desc); 1: (height bin asc, natural index desc)
};

// One contact buffer (the batch holds two: this step's and the previous one).
// "Natural" arrays are indexed by the pair's position in natural order;
// "sorted" arrays by its slot in colour order.  Per-episode regions start at
// pair_off[e] (pairs) and 4 * pair_off[e] (points).
struct ContactBuf {
  uint32_t* nat_key;    // ((a + 1) << 16) | b, a = -1 for the ground
  uint32_t* nat_feat;   // axis | ref_face << 8 | inc_face << 16 | np << 24
  uint32_t* nat_slot;   // slot | colour << 16
  float* nat_pt;        // [P * 4][kNatPtFloats]; lambda = final impulses of the step
  float* nat_pf;        // [P][kNatPairFloats]
  // colour-sorted solver arrays, used when a step's pairs exceed the
  // shared-memory capacity (stride Pc per field)
  float* srt_f;         // per episode: [Pc][kPairStride]
  uint32_t* srt_ab;     // local a | local b << 16 (ground = nb)
  int32_t* srt_np;
  float* srt_pt;        // per episode: [Pc][kPtStride], point k field f at k * 13 + f
  float* nat_x;         // [P * 4][kFeatures] warm-start features of each point
};

// Per colour-sorted slot, the acceleration state of one solve: the impulses
// at the start of the sweep block [4][3], then the conjugate direction [4][3].
constexpr int kAccFloats = 24;

constexpr int kFeatures = 24;    // warm-start network inputs per contact point
constexpr int kRecFloats = 27;   // recorder row: features, then converged impulses (n, t1, t2)
// normalisation scales of the features (nominal block mass and length)
constexpr float kFeatMass = 0.015f;
constexpr float kFeatLen = 0.075f;
// load-above feature: column height above a contact point in units of ten
// nominal block thicknesses (0.15 m)
constexpr float kFeatColumnInv = 1.f / 0.15f;

struct Dev {
  int E, B, nb_max, pc_max;
  const int32_t* body_off;
  const int64_t* pair_off;
  // bodies
  float *x, *q, *v, *w, *half, *mass, *invm, *invI, *mu, *x0, *z0, *f;
  int32_t *flags, *f_steps;
  const float* ground_mu;
  EpState* ep;
  // schedule
  int32_t *mv_off, *mv_block, *mv_axis, *mv_remove, *mv_push, *mv_settle;
  float *mv_sign, *mv_factor, *mv_k;
  ContactBuf buf[2];
  float* acc;             // [P][kAccFloats] per-solve acceleration state (scratch)
  int32_t* work_counter;
  const int32_t* order;   // episode processing order [E]
  Params P;
  int smem_per_warp;      // bytes
  int ps;                 // pairs whose solver arrays fit in shared memory
  // warm-start network (caller-owned block) and training-sample recorder
  const unsigned char* mlp;
  float* rec;
  int32_t* rec_count;
  int rec_cap, rec_every;
  int rec_unmatched;      // 1: the recorder takes only the points of pairs with no previous-frame impulse
};

// Error reporting shared by the library's translation units.
jb_status fail(jb_status s, const char* fmt, ...);

// Shared-memory plan of one episode (bytes from the warp's base).
struct SmemPlan {
  int nbs;                // body slots (nb_max + 1, the last one is the ground)
  int off_f;              // float arrays
  int off_flags;
  int off_mask;
  int off_cand;
  int off_col;
  int off_sf, off_ab, off_np, off_sp;   // colour-sorted solver arrays (ps pairs)
  int bytes;
};

constexpr int kBodyFloats = 36;  // x3 q4 v3 w3 half3 R9 Iw6 ext3 invm mu
constexpr int kBodyStride = kBodyFloats + 1;   // record-major, odd stride

// Pairs of an episode whose solver arrays are kept in shared memory: an
// intact tower needs about 3.6 per body.
__host__ __device__ inline int smem_pairs(int nb_max, int pc_max) {
  int p = 4 * nb_max + 16;
  return p < pc_max ? p : pc_max;
}

__host__ __device__ inline SmemPlan smem_plan(int nb_max, int pc_max, int ps) {
  SmemPlan s;
  s.nbs = nb_max + 1;
  int o = 0;
  s.off_mask = o; o += 8 * s.nbs;
  s.off_f = o; o += 4 * kBodyStride * s.nbs;
  s.off_flags = o; o += 4 * s.nbs;
  o = (o + 15) & ~15;   // the candidate array is reused for float2 corner lists
  s.off_cand = o; o += 4 * cand_capacity(nb_max);
  s.off_col = o; o += 4 * 3 * (kMaxColours + 1);
  o = (o + 15) & ~15;
  s.off_sf = o; o += 4 * kPairStride * ps;
  s.off_ab = o; o += 4 * ps;
  s.off_np = o; o += 4 * ps;
  s.off_sp = o; o += 4 * kPtStride * ps;
  o = (o + 15) & ~15;
  s.bytes = o;
  return s;
}

}  // namespace jbk
