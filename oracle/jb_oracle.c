/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see jb_oracle.h).
 *
 * A plain sequential statement of one time step of the paper's rigid-body
 * engine, written in the paper's order:
 *   Sec. 4.2  external forces and semi-implicit Euler (Eq. newton_euler),
 *   Sec. 6.1  AABB broadphase (Eq. aabb),
 *   Sec. 6.2  OBB separating-axis test over 15 axes,
 *   Sec. 6.2.1 contact manifold by Sutherland-Hodgman face clipping,
 *   Sec. 7.1  Jacobian / effective mass (Eq. keff), normal impulse (Eq. lambda_n),
 *   Sec. 7.2  box Coulomb friction (Eq. coulomb_pgs),
 *   Sec. 7.3  sequential Projected Gauss-Seidel (Listing "PGS core"),
 *   Sec. 4.1  quaternion integration (Eq. quat_int),
 *   Sec. 7.4  Baumgarte position correction (Eq. baumgarte),
 *   Sec. 8    support polygon margin (Eq. stability), collapse (Eq. collapse),
 *             rest test (Sec. 8.3).
 * Where the paper is silent or garbled, the reading taken is stated at the
 * point of use ("reading:").  Gauss-Seidel runs in natural order: ground pairs
 * by body, then pairs (i, j) ascending, points in manifold order, rows n, t1, t2.
 */
#include "jb_oracle.h"


#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXP 4          /* contact points per pair (Sec. 6.2.1 step d) */
#define TIE_ABS 1e-5    /* reading: SAT axis hysteresis (m), far below the 0.4 mm slop */
#define EDGE_REL 0.05   /* reading: cross axis must beat the face axis by 5% */
#define CROSS_EPS 1e-6  /* reading: skip degenerate cross axes */
#define INC_TIE 1e-9    /* reading: incident-face choice hysteresis */
#define CLIP_EPS 1e-6   /* reading: the reference face is enlarged by 1 um for clipping */
#define MERGE_EPS 1e-6  /* reading: clipped vertices closer than 1 um are one vertex */
#define DEPTH_TIE 1e-6  /* reading: depths within 1 um tie (lowest index wins) */
#define AREA_TIE 1e-9   /* reading: squared distances / areas within 1e-9 m^2 tie */
#define OR_PI 3.14159265358979323846

typedef struct {
  double x[3], q[4], v[3], w[3];
  double half[3];
  double mass, invm, invI[3], mu;
  int active, is_static;
  double R[3][3], Iw[3][3];     /* rotation, world inverse inertia (per substep) */
  double x0[3], z0[3];          /* initial position and thickness axis */
  double f[3];                  /* external force */
  int f_steps;
} or_body;

typedef struct {
  int a, b;                     /* episode-local; a = -1 is the ground */
  int axis, ref_face, inc_face, np;
  double n[3], t1[3], t2[3];
  double delta, depth_max, mu;
  double p[MAXP][3], depth[MAXP], local[MAXP][3];
  double rA[MAXP][3], rB[MAXP][3];
  double k[MAXP][3];            /* inverse effective mass of rows n, t1, t2 */
  double bias[MAXP];
  double lam[MAXP][3];
  int matched[MAXP];
  double feat[MAXP][OR_NFEAT];
  double lam_start[MAXP][3];    /* acceleration: impulses at the start of the sweep block */
  double dir[MAXP][3];          /* acceleration: conjugate direction */
} or_pair;

typedef struct {
  int nb;
  or_body* b;
  or_body ground;               /* static, zero velocity, identity frame */
  double ground_mu;
  or_pair *pairs, *prev;
  int np, cap, nprev, capprev;
  int* order;            /* sweep order of the pairs (colour_order); ocap entries */
  int ocap;
  /* schedule */
  int n_moves, mi, phase, remaining, pb, rest_left;
  const int *mv_block, *mv_axis, *mv_remove, *mv_push, *mv_settle;
  const double *mv_sign, *mv_factor, *mv_k;
  /* statistics */
  int status, collapsed, resting, last_sweeps;
  long steps, total_sweeps, solves;
  double body_steps, last_res, max_res, ek;
} or_episode;

struct or_world {
  int E, B;
  int* body_off;
  or_episode* ep;
  or_params P;
  /* training-sample recorder */
  double* rec;
  int rec_cap, rec_every;
  long rec_count;
  /* schedule storage */
  int *m_block, *m_axis, *m_remove, *m_push, *m_settle;
  double *m_sign, *m_factor, *m_k;
};

/* ------------------------------------------------------------------ vectors */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c) {
  double t0 = a[1] * b[2] - a[2] * b[1], t1 = a[2] * b[0] - a[0] * b[2], t2 = a[0] * b[1] - a[1] * b[0];
  c[0] = t0; c[1] = t1; c[2] = t2;
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void axpy3(double s, const double* x, double* y) { y[0] += s * x[0]; y[1] += s * x[1]; y[2] += s * x[2]; }
static void matvec3(const double M[3][3], const double* x, double* y) {
  double t[3];
  for (int i = 0; i < 3; ++i) t[i] = M[i][0] * x[0] + M[i][1] * x[1] + M[i][2] * x[2];
  y[0] = t[0]; y[1] = t[1]; y[2] = t[2];
}
static void col3(const double R[3][3], int k, double* c) { c[0] = R[0][k]; c[1] = R[1][k]; c[2] = R[2][k]; }
static double sgn(double v) { return v >= 0.0 ? 1.0 : -1.0; }
static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------- Sec. 4.1 rotation, inertia */
/* Eq. rotmat: rotation matrix of the unit quaternion q = [w, x, y, z]. */
static void rotmat(const double* q, double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - z * w);     R[0][2] = 2 * (x * z + y * w);
  R[1][0] = 2 * (x * y + z * w);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - x * w);
  R[2][0] = 2 * (x * z - y * w);     R[2][1] = 2 * (y * z + x * w);     R[2][2] = 1 - 2 * (x * x + y * y);
}
void or_rotmat(const double* q, double* R) { rotmat(q, (double(*)[3])R); }

/* Eq. inertia: I_body = m/12 diag(w^2+h^2, l^2+h^2, l^2+w^2), l, w, h = full
   dimensions along body x, y, z. */
void or_body_inertia(double m, const double* half, double* I) {
  double l = 2 * half[0], w = 2 * half[1], h = 2 * half[2];
  I[0] = m / 12.0 * (w * w + h * h);
  I[1] = m / 12.0 * (l * l + h * h);
  I[2] = m / 12.0 * (l * l + w * w);
}

/* Sec. 4.1.2: I_world^-1 = R I_body^-1 R^T. */
static void update_frame(or_body* B) {
  rotmat(B->q, B->R);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += B->R[i][k] * B->invI[k] * B->R[j][k];
      B->Iw[i][j] = s;
    }
}

/* --------------------------------------------------------- Sec. 6.2 SAT ----- */
typedef struct { double x[3]; double R[3][3]; double h[3]; } box_t;

/* Projected radius of a box on unit axis u: r = sum_i h_i |a_i . u|. */
static double proj_radius(const box_t* b, const double* u) {
  double r = 0, a[3];
  for (int i = 0; i < 3; ++i) { col3(b->R, i, a); r += b->h[i] * fabs(dot3(a, u)); }
  return r;
}

/* All 15 axes: A0..A2, B0..B2, then A_i x B_j (i-major).  delta = rA + rB - |d.u|.
   Reading: cross axes with |A_i x B_j| < 1e-6 are skipped (parallel edges). */
static void sat15(const box_t* A, const box_t* B, double delta[15], int valid[15], double U[15][3]) {
  double d[3] = {B->x[0] - A->x[0], B->x[1] - A->x[1], B->x[2] - A->x[2]};
  for (int k = 0; k < 15; ++k) {
    double u[3];
    if (k < 3) col3(A->R, k, u);
    else if (k < 6) col3(B->R, k - 3, u);
    else {
      double a[3], b[3];
      col3(A->R, (k - 6) / 3, a); col3(B->R, (k - 6) % 3, b);
      cross3(a, b, u);
      double l = norm3(u);
      if (l < CROSS_EPS) { valid[k] = 0; delta[k] = 0; U[k][0] = U[k][1] = U[k][2] = 0; continue; }
      u[0] /= l; u[1] /= l; u[2] /= l;
    }
    valid[k] = 1;
    U[k][0] = u[0]; U[k][1] = u[1]; U[k][2] = u[2];
    delta[k] = proj_radius(A, u) + proj_radius(B, u) - fabs(dot3(d, u));
  }
}

/* Axis choice.  Reading (the paper only says "the axis with minimum delta"):
   face axes in order A0..B2, a later one replaces the current best only if
   smaller by TIE_ABS; likewise among cross axes; a cross axis wins only if
   delta_edge < delta_face - (0.05 |delta_face| + TIE_ABS).  The hysteresis
   keeps nearly parallel choices stable: stacked blocks have A's and B's face
   normals and the crossed-edge axis all near z, and a smaller tolerance lets
   micro-radian tilts flip the pair between them (and between 4-point face
   and 1-point edge manifolds) from step to step.  Contact exists iff the
   minimum delta over all valid axes exceeds -margin (speculative contacts). */
static int sat_select_tie(const double delta[15], const int valid[15], double* dmin_out, double tie) {
  double dmin = delta[0];
  for (int k = 1; k < 15; ++k) if (valid[k] && delta[k] < dmin) dmin = delta[k];
  *dmin_out = dmin;
  int bf = 0;
  for (int k = 1; k < 6; ++k) if (delta[k] < delta[bf] - tie) bf = k;
  int be = -1;
  for (int k = 6; k < 15; ++k)
    if (valid[k] && (be < 0 || delta[k] < delta[be] - tie)) be = k;
  if (be >= 0 && delta[be] < delta[bf] - (EDGE_REL * fabs(delta[bf]) + tie)) return be;
  return bf;
}
static int sat_select(const double delta[15], const int valid[15], double* dmin_out) {
  return sat_select_tie(delta, valid, dmin_out, TIE_ABS);
}

/* ------------------------------------------------- Sec. 6.2.1 manifold ----- */
typedef struct { int n; double p[8][3]; } poly_t;

/* Sutherland-Hodgman: keep the part of the polygon with (p - c).u <= h. */
static void clip_plane(const poly_t* in, poly_t* out, const double* c, const double* u, double h) {
  out->n = 0;
  if (in->n == 0) return;
  for (int i = 0; i < in->n; ++i) {
    const double* S = in->p[(i + in->n - 1) % in->n];
    const double* E = in->p[i];
    double dS = (S[0] - c[0]) * u[0] + (S[1] - c[1]) * u[1] + (S[2] - c[2]) * u[2] - h;
    double dE = (E[0] - c[0]) * u[0] + (E[1] - c[1]) * u[1] + (E[2] - c[2]) * u[2] - h;
    if (dE <= 0) {
      if (dS > 0 && out->n < 8) {
        double t = dS / (dS - dE);
        for (int j = 0; j < 3; ++j) out->p[out->n][j] = S[j] + t * (E[j] - S[j]);
        out->n++;
      }
      if (out->n < 8) { memcpy(out->p[out->n], E, sizeof(double) * 3); out->n++; }
    } else if (dS <= 0 && out->n < 8) {
      double t = dS / (dS - dE);
      for (int j = 0; j < 3; ++j) out->p[out->n][j] = S[j] + t * (E[j] - S[j]);
      out->n++;
    }
  }
}

/* Area of the convex hull of 4 coplanar-ish points measured across n. */
static double tri_area(const double* a, const double* b, const double* c, const double* n) {
  double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]}, w[3];
  cross3(u, v, w);
  return 0.5 * fabs(dot3(w, n));
}
static double quad_area(const double* a, const double* b, const double* c, const double* d, const double* n) {
  const double* P[4] = {a, b, c, d};
  double s[3] = {0, 0, 0}, t[3];
  for (int i = 0; i < 4; ++i) { cross3(P[i], P[(i + 1) % 4], t); axpy3(1.0, t, s); }
  return 0.5 * fabs(dot3(s, n));
}
static double hull4_area(const double* a, const double* b, const double* c, const double* d, const double* n) {
  double m = quad_area(a, b, c, d, n), t;
  if ((t = quad_area(a, b, d, c, n)) > m) m = t;
  if ((t = quad_area(a, c, b, d, n)) > m) m = t;
  if ((t = tri_area(a, b, c, n)) > m) m = t;
  if ((t = tri_area(a, b, d, n)) > m) m = t;
  if ((t = tri_area(a, c, d, n)) > m) m = t;
  if ((t = tri_area(b, c, d, n)) > m) m = t;
  return m;
}

/* Reading of "sample up to 4 points": (1) deepest, (2) farthest from (1),
   (3) largest triangle with (1),(2), (4) largest added hull area; scores within
   a tie tolerance count as equal and the lowest index wins; output in that
   order.  Applied only when more than 4 remain. */
static int reduce4(int n, double P[][3], double* D, const double* nrm, int* sel) {
  if (n <= 4) { for (int i = 0; i < n; ++i) sel[i] = i; return n; }
  int used[8] = {0};
  /* each pick: the first index whose score is within the tie tolerance of the best */
  double dmax = D[0];
  for (int i = 1; i < n; ++i) if (D[i] > dmax) dmax = D[i];
  int i1 = 0;
  while (D[i1] < dmax - DEPTH_TIE) ++i1;
  used[i1] = 1;
  double sc[8], best;
  best = -1;
  for (int i = 0; i < n; ++i) {
    double d[3] = {P[i][0] - P[i1][0], P[i][1] - P[i1][1], P[i][2] - P[i1][2]};
    sc[i] = used[i] ? -1 : dot3(d, d);
    if (sc[i] > best) best = sc[i];
  }
  int i2 = 0;
  while (used[i2] || sc[i2] < best - AREA_TIE) ++i2;
  used[i2] = 1;
  best = -1;
  for (int i = 0; i < n; ++i) {
    sc[i] = used[i] ? -1 : tri_area(P[i1], P[i2], P[i], nrm);
    if (sc[i] > best) best = sc[i];
  }
  int i3 = 0;
  while (used[i3] || sc[i3] < best - AREA_TIE) ++i3;
  used[i3] = 1;
  double base = tri_area(P[i1], P[i2], P[i3], nrm);
  best = -1;
  for (int i = 0; i < n; ++i) {
    sc[i] = used[i] ? -1 : hull4_area(P[i1], P[i2], P[i3], P[i], nrm) - base;
    if (sc[i] > best) best = sc[i];
  }
  int i4 = 0;
  while (used[i4] || sc[i4] < best - AREA_TIE) ++i4;
  sel[0] = i1; sel[1] = i2; sel[2] = i3; sel[3] = i4;
  return 4;
}

/* Reading of the tangent basis: t1 = normalize(e - (e.n) n) with e = world X,
   or world Y when |n.X| > 0.9; t2 = n x t1. */
static void tangent_basis(const double* n, double* t1, double* t2) {
  double e[3] = {1, 0, 0};
  if (fabs(n[0]) > 0.9) { e[0] = 0; e[1] = 1; }
  double en = dot3(e, n);
  double t[3] = {e[0] - en * n[0], e[1] - en * n[1], e[2] - en * n[2]};
  double l = norm3(t);
  t1[0] = t[0] / l; t1[1] = t[1] / l; t1[2] = t[2] / l;
  cross3(n, t1, t2);
}

/* Points are written to pr->p / depth; returns the count kept. */
static int finish_points(or_pair* pr, int n, double P[][3], double* D, const double* nrm) {
  int sel[4];
  int m = reduce4(n, P, D, nrm, sel);
  double dm = -1e300;
  for (int i = 0; i < m; ++i) {
    memcpy(pr->p[i], P[sel[i]], sizeof(double) * 3);
    pr->depth[i] = D[sel[i]];
    if (D[sel[i]] > dm) dm = D[sel[i]];
  }
  pr->np = m;
  pr->depth_max = dm;
  return m;
}

/* Face-face manifold.  Reading of steps a-d: the reference face is the face of
   the SAT-axis owner whose outward normal is along the contact direction, the
   incident face is the other box's face most anti-parallel to it; the incident
   quad is clipped by the reference face's four side planes (the face enlarged
   by CLIP_EPS, so edges lying on a side plane, as in a flush tower, are not
   split by rounding); per-point depth is the distance below the reference
   face; points with depth > -margin are kept, coincident ones once; the
   contact point is the midpoint between the incident point and the face. */
static int face_manifold(const box_t* A, const box_t* B, int axis, const double* n, double margin, or_pair* pr) {
  const box_t *ref, *inc;
  int ra;
  double nref[3];
  if (axis < 3) { ref = A; inc = B; ra = axis; nref[0] = n[0]; nref[1] = n[1]; nref[2] = n[2]; }
  else { ref = B; inc = A; ra = axis - 3; nref[0] = -n[0]; nref[1] = -n[1]; nref[2] = -n[2]; }
  double ax[3];
  col3(ref->R, ra, ax);
  double sr = sgn(dot3(ax, nref));
  double cr[3] = {ref->x[0] + sr * ref->h[ra] * ax[0], ref->x[1] + sr * ref->h[ra] * ax[1],
                  ref->x[2] + sr * ref->h[ra] * ax[2]};
  int r1 = (ra + 1) % 3, r2 = (ra + 2) % 3;
  double u1[3], u2[3];
  col3(ref->R, r1, u1); col3(ref->R, r2, u2);
  /* incident face */
  int ji = 0; double bestd = -1;
  for (int j = 0; j < 3; ++j) {
    double c[3]; col3(inc->R, j, c);
    double dd = fabs(dot3(c, nref));
    if (dd > bestd + INC_TIE) { bestd = dd; ji = j; }
  }
  double bj[3]; col3(inc->R, ji, bj);
  double si = -sgn(dot3(bj, nref));
  double ci[3] = {inc->x[0] + si * inc->h[ji] * bj[0], inc->x[1] + si * inc->h[ji] * bj[1],
                  inc->x[2] + si * inc->h[ji] * bj[2]};
  int j1 = (ji + 1) % 3, j2 = (ji + 2) % 3;
  double v1[3], v2[3];
  col3(inc->R, j1, v1); col3(inc->R, j2, v2);
  const double s1[4] = {1, -1, -1, 1}, s2[4] = {1, 1, -1, -1};
  poly_t a, b;
  a.n = 4;
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k)
      a.p[i][k] = ci[k] + s1[i] * inc->h[j1] * v1[k] + s2[i] * inc->h[j2] * v2[k];
  double mu1[3] = {-u1[0], -u1[1], -u1[2]}, mu2[3] = {-u2[0], -u2[1], -u2[2]};
  clip_plane(&a, &b, cr, u1, ref->h[r1] + CLIP_EPS);
  clip_plane(&b, &a, cr, mu1, ref->h[r1] + CLIP_EPS);
  clip_plane(&a, &b, cr, u2, ref->h[r2] + CLIP_EPS);
  clip_plane(&b, &a, cr, mu2, ref->h[r2] + CLIP_EPS);
  double P[8][3], D[8];
  int m = 0;
  for (int i = 0; i < a.n; ++i) {
    double rel[3] = {cr[0] - a.p[i][0], cr[1] - a.p[i][1], cr[2] - a.p[i][2]};
    double dep = dot3(rel, nref);
    if (!(dep > -margin)) continue;
    int dup = 0;
    for (int j = 0; j < m && !dup; ++j) {
      double q[3] = {a.p[i][0] - (P[j][0] - 0.5 * D[j] * nref[0]), a.p[i][1] - (P[j][1] - 0.5 * D[j] * nref[1]),
                     a.p[i][2] - (P[j][2] - 0.5 * D[j] * nref[2])};
      dup = dot3(q, q) < MERGE_EPS * MERGE_EPS;
    }
    if (dup) continue;
    for (int k = 0; k < 3; ++k) P[m][k] = a.p[i][k] + 0.5 * dep * nref[k];
    D[m] = dep;
    ++m;
  }
  pr->ref_face = 2 * ra + (sr > 0 ? 0 : 1) + (axis < 3 ? 0 : 8);
  pr->inc_face = 2 * ji + (si > 0 ? 0 : 1);
  return finish_points(pr, m, P, D, n);
}

/* Reading for edge-edge contacts (the paper is silent): one point at the
   midpoint of the closest points of the two supporting edges, depth = delta. */
static int edge_manifold(const box_t* A, const box_t* B, int axis, const double* n, double delta, or_pair* pr) {
  int i = (axis - 6) / 3, j = (axis - 6) % 3;
  double pa[3] = {A->x[0], A->x[1], A->x[2]}, pb[3] = {B->x[0], B->x[1], B->x[2]};
  for (int m = 0; m < 3; ++m) {
    double c[3];
    if (m != i) { col3(A->R, m, c); axpy3(sgn(dot3(c, n)) * A->h[m], c, pa); }
    if (m != j) { col3(B->R, m, c); axpy3(-sgn(dot3(c, n)) * B->h[m], c, pb); }
  }
  double ea[3], eb[3];
  col3(A->R, i, ea); col3(B->R, j, eb);
  double r[3] = {pa[0] - pb[0], pa[1] - pb[1], pa[2] - pb[2]};
  double bb = dot3(ea, eb), c = dot3(ea, r), f = dot3(eb, r);
  double den = 1.0 - bb * bb;
  double s = den > 1e-12 ? (bb * f - c) / den : 0.0;
  s = clampd(s, -A->h[i], A->h[i]);
  double t = clampd(f + s * bb, -B->h[j], B->h[j]);
  double P[1][3], D[1] = {delta};
  for (int k = 0; k < 3; ++k) P[0][k] = 0.5 * ((pa[k] + s * ea[k]) + (pb[k] + t * eb[k]));
  pr->ref_face = 16 + i;
  pr->inc_face = 16 + j;
  return finish_points(pr, 1, P, D, n);
}

/* Box-box narrowphase; returns 1 and fills axis, n, delta, points if in contact. */
static int box_pair_tie(const box_t* A, const box_t* B, double margin, or_pair* pr, double* dmin_out, double tie);
static int box_pair(const box_t* A, const box_t* B, double margin, or_pair* pr, double* dmin_out) {
  return box_pair_tie(A, B, margin, pr, dmin_out, TIE_ABS);
}
static int box_pair_tie(const box_t* A, const box_t* B, double margin, or_pair* pr, double* dmin_out, double tie) {
  double delta[15], U[15][3];
  int valid[15];
  sat15(A, B, delta, valid, U);
  double dmin;
  int ax = sat_select_tie(delta, valid, &dmin, tie);
  if (dmin_out) *dmin_out = dmin;
  if (!(dmin > -margin)) return 0;
  double d[3] = {B->x[0] - A->x[0], B->x[1] - A->x[1], B->x[2] - A->x[2]};
  double n[3] = {U[ax][0], U[ax][1], U[ax][2]};
  if (dot3(n, d) < 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
  pr->axis = ax;
  pr->delta = delta[ax];
  memcpy(pr->n, n, sizeof n);
  int m = ax < 6 ? face_manifold(A, B, ax, n, margin, pr) : edge_manifold(A, B, ax, n, delta[ax], pr);
  return m > 0;
}

/* Reading for ground contacts: the ground z = 0 is body A with n = +z; the
   box corners with z < margin are candidates (depth = -z), reduced to 4. */
static int ground_pair(const box_t* B, double margin, or_pair* pr) {
  double P[8][3], D[8];
  int m = 0;
  for (int c = 0; c < 8; ++c) {
    double s0 = (c & 1) ? 1 : -1, s1 = (c & 2) ? 1 : -1, s2 = (c & 4) ? 1 : -1;
    double p[3];
    for (int k = 0; k < 3; ++k)
      p[k] = B->x[k] + s0 * B->h[0] * B->R[k][0] + s1 * B->h[1] * B->R[k][1] + s2 * B->h[2] * B->R[k][2];
    if (p[2] < margin) {
      D[m] = -p[2];
      P[m][0] = p[0]; P[m][1] = p[1]; P[m][2] = p[2] + 0.5 * D[m];
      ++m;
    }
  }
  if (m == 0) return 0;
  double n[3] = {0, 0, 1};
  memcpy(pr->n, n, sizeof n);
  pr->axis = 15;
  pr->ref_face = 0;
  pr->inc_face = 0;
  finish_points(pr, m, P, D, n);
  pr->delta = pr->depth_max;
  return 1;
}

static void box_of(const or_body* b, box_t* out) {
  memcpy(out->x, b->x, sizeof out->x);
  memcpy(out->R, b->R, sizeof out->R);
  memcpy(out->h, b->half, sizeof out->h);
}

/* -------------------------------------------------------------- episode ---- */
static or_body* body_ref(or_episode* E, int i) { return i < 0 ? &E->ground : &E->b[i]; }

static void push_pair(or_episode* E, const or_pair* p) {
  if (E->np == E->cap) {
    E->cap = E->cap ? 2 * E->cap : 64;
    E->pairs = (or_pair*)realloc(E->pairs, sizeof(or_pair) * E->cap);
  }
  E->pairs[E->np++] = *p;
}

/* Sec. 6.1 Eq. aabb broadphase + Sec. 6.2 narrowphase, natural pair order. */
static void detect(or_episode* E, const or_params* P) {
  E->np = 0;
  double ext[E->nb > 0 ? E->nb : 1][3];
  for (int i = 0; i < E->nb; ++i)
    for (int k = 0; k < 3; ++k)
      ext[i][k] = fabs(E->b[i].R[k][0]) * E->b[i].half[0] + fabs(E->b[i].R[k][1]) * E->b[i].half[1] +
                  fabs(E->b[i].R[k][2]) * E->b[i].half[2];
  or_pair pr;
  /* ground pairs first (ground = body -1) */
  for (int j = 0; j < E->nb; ++j) {
    or_body* B = &E->b[j];
    if (!B->active || B->is_static) continue;
    if (B->x[2] - ext[j][2] > P->aabb_eps) continue;
    box_t bx; box_of(B, &bx);
    memset(&pr, 0, sizeof pr);
    if (ground_pair(&bx, P->contact_margin, &pr)) {
      pr.a = -1; pr.b = j;
      pr.mu = fmin(E->ground_mu, B->mu);
      push_pair(E, &pr);
    }
  }
  for (int i = 0; i < E->nb; ++i) {
    or_body* A = &E->b[i];
    if (!A->active) continue;
    for (int j = i + 1; j < E->nb; ++j) {
      or_body* B = &E->b[j];
      if (!B->active || (A->is_static && B->is_static)) continue;
      int ov = 1;
      for (int k = 0; k < 3; ++k)
        if (fabs(A->x[k] - B->x[k]) > ext[i][k] + ext[j][k] + P->aabb_eps) ov = 0;
      if (!ov) continue;
      box_t ba, bb; box_of(A, &ba); box_of(B, &bb);
      memset(&pr, 0, sizeof pr);
      if (box_pair_tie(&ba, &bb, P->contact_margin, &pr, NULL, P->sat_tie > 0 ? P->sat_tie : TIE_ABS)) {
        pr.a = i; pr.b = j;
        pr.mu = fmin(A->mu, B->mu);
        push_pair(E, &pr);
      }
    }
  }
}

static double rel_vel(const or_body* A, const or_body* B, const double* rA, const double* rB, const double* d);

/* Sec. 7.1 Eq. keff (read as the inverse effective mass) for each row, the
   speculative bias, the tangent basis, and A-local point coordinates. */
static void setup(or_episode* E, double h, const or_params* P) {
  const double vmin = P->restitution_vmin > 0 ? P->restitution_vmin : 2.0 * norm3(P->gravity) * h;
  for (int c = 0; c < E->np; ++c) {
    or_pair* pr = &E->pairs[c];
    or_body *A = body_ref(E, pr->a), *B = body_ref(E, pr->b);
    tangent_basis(pr->n, pr->t1, pr->t2);
    const double* dirs[3] = {pr->n, pr->t1, pr->t2};
    for (int i = 0; i < pr->np; ++i) {
      for (int k = 0; k < 3; ++k) { pr->rA[i][k] = pr->p[i][k] - A->x[k]; pr->rB[i][k] = pr->p[i][k] - B->x[k]; }
      /* local = R_A^T (p - x_A) */
      for (int k = 0; k < 3; ++k)
        pr->local[i][k] = A->R[0][k] * pr->rA[i][0] + A->R[1][k] * pr->rA[i][1] + A->R[2][k] * pr->rA[i][2];
      for (int r = 0; r < 3; ++r) {
        double ca[3], cb[3], ia[3], ib[3];
        cross3(pr->rA[i], dirs[r], ca); cross3(pr->rB[i], dirs[r], cb);
        matvec3(A->Iw, ca, ia); matvec3(B->Iw, cb, ib);
        pr->k[i][r] = A->invm + B->invm + dot3(ca, ia) + dot3(cb, ib);
      }
      /* reading: separated points (depth < 0) may close the gap within the step;
         with Newton restitution a touching point approaching faster than vmin
         targets v_n = -e v_n(pre-solve) */
      pr->bias[i] = pr->depth[i] < 0 ? -pr->depth[i] / h : 0.0;
      if (P->restitution_newton && pr->depth[i] >= 0) {
        double un = rel_vel(A, B, pr->rA[i], pr->rB[i], pr->n);
        if (un < -vmin) pr->bias[i] = P->restitution * un;
      }
      pr->lam[i][0] = pr->lam[i][1] = pr->lam[i][2] = 0;
      pr->matched[i] = 0;
    }
  }
}

static int pair_key_cmp(int a1, int b1, int a2, int b2) {
  if (a1 != a2) return a1 < a2 ? -1 : 1;
  if (b1 != b2) return b1 < b2 ? -1 : 1;
  return 0;
}

/* Reading of the warm start: key (a, b, reference face, incident face); a new
   point inherits the impulse of the nearest old point of the same key within
   match_radius in body-A local coordinates. */
static void warm_start_match(or_episode* E, const or_params* P) {
  if (P->warm_start != 1) return;
  for (int c = 0; c < E->np; ++c) {
    or_pair* pr = &E->pairs[c];
    int lo = 0, hi = E->nprev - 1, found = -1;
    while (lo <= hi) {
      int mid = (lo + hi) / 2;
      int s = pair_key_cmp(E->prev[mid].a, E->prev[mid].b, pr->a, pr->b);
      if (s == 0) { found = mid; break; }
      if (s < 0) lo = mid + 1; else hi = mid - 1;
    }
    if (found < 0) continue;
    const or_pair* op = &E->prev[found];
    if (op->ref_face != pr->ref_face || op->inc_face != pr->inc_face) continue;
    for (int i = 0; i < pr->np; ++i) {
      int best = -1; double bd = P->match_radius * P->match_radius;
      for (int j = 0; j < op->np; ++j) {
        double d[3] = {op->local[j][0] - pr->local[i][0], op->local[j][1] - pr->local[i][1],
                       op->local[j][2] - pr->local[i][2]};
        double s = dot3(d, d);
        if (s <= bd) { bd = s; best = j; }
      }
      if (best >= 0) { memcpy(pr->lam[i], op->lam[best], sizeof(double) * 3); pr->matched[i] = 1; }
    }
  }
}

/* Relative velocity of B with respect to A at the point, along dir. */
static double rel_vel(const or_body* A, const or_body* B, const double* rA, const double* rB, const double* d) {
  double wa[3], wb[3];
  cross3(A->w, rA, wa); cross3(B->w, rB, wb);
  double v[3] = {B->v[0] + wb[0] - A->v[0] - wa[0], B->v[1] + wb[1] - A->v[1] - wa[1],
                 B->v[2] + wb[2] - A->v[2] - wa[2]};
  return dot3(v, d);
}

/* Reading of the impulse application: the full 12-DOF impulse acts on both the
   linear and the angular velocity of A (-) and B (+). */
static void apply_impulse(or_body* A, or_body* B, const double* rA, const double* rB, const double* Pv) {
  double t[3], u[3];
  axpy3(-A->invm, Pv, A->v);
  cross3(rA, Pv, t); matvec3(A->Iw, t, u); axpy3(-1.0, u, A->w);
  axpy3(B->invm, Pv, B->v);
  cross3(rB, Pv, t); matvec3(B->Iw, t, u); axpy3(1.0, u, B->w);
}

static void apply_warm_start(or_episode* E) {
  for (int c = 0; c < E->np; ++c) {
    or_pair* pr = &E->pairs[c];
    or_body *A = body_ref(E, pr->a), *B = body_ref(E, pr->b);
    for (int i = 0; i < pr->np; ++i) {
      double Pv[3] = {0, 0, 0};
      axpy3(pr->lam[i][0], pr->n, Pv); axpy3(pr->lam[i][1], pr->t1, Pv); axpy3(pr->lam[i][2], pr->t2, Pv);
      apply_impulse(A, B, pr->rA[i], pr->rB[i], Pv);
    }
  }
}

/* One Gauss-Seidel sweep: Eq. lambda_n (restitution factor applied every
   iteration, as in the listing; bias added for speculative points) and
   Eq. coulomb_pgs (box clip with the just-updated normal impulse). */
/* Disc projection of the tangent impulse (Coulomb cone of the PGS figure):
   (a1, a2) scaled onto |a| <= lim when outside.  Reading: both tangent rows
   take the same step 1/k_t with k_t = max(k_t1, k_t2), so that a sliding
   contact's fixed point has the friction impulse opposite to the sliding
   velocity (with unequal steps it would lean towards the stiffer row). */
static void disc_project(double a1, double a2, double lim, double* p1, double* p2) {
  double m = sqrt(a1 * a1 + a2 * a2);
  double s = m > lim ? lim / m : 1.0;
  *p1 = a1 * s;
  *p2 = a2 * s;
}

static int cmp_int2(const void* x, const void* y) {
  const int *a = (const int*)x, *b = (const int*)y;
  if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
  return (a[1] > b[1]) - (a[1] < b[1]);
}

/* The sweep order of this solve: natural, or the GPU library's colour order
   (see or_params.colour_order).  Only the order of the pair updates
   changes; the rows of a pair and the fixed point do not. */
static void sweep_order(or_episode* E, int colour) {
  const int n = E->np;
  if (E->ocap < n) { E->ocap = n + 64; E->order = (int*)realloc(E->order, sizeof(int) * E->ocap); }
  for (int i = 0; i < n; ++i) E->order[i] = i;
  if (!colour || n <= 0) return;
  int (*kv)[2] = (int(*)[2])malloc(sizeof(int) * 2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    if (colour == 2)   /* height of the first point in 1 mm bins ascending, then index descending */
      kv[i][0] = (int)floor((E->pairs[i].p[0][2] + 5e-4) * 1000.0) + 1;
    else               /* lower body ascending, upper body descending */
      kv[i][0] = ((E->pairs[i].a + 1) << 16) | (0xffff - E->pairs[i].b);
    kv[i][1] = -i;
  }
  qsort(kv, n, sizeof(int) * 2, cmp_int2);
  unsigned long long* used = (unsigned long long*)calloc(E->nb + 1, sizeof(unsigned long long));
  int* col = (int*)malloc(sizeof(int) * (size_t)n);
  for (int t = 0; t < n; ++t) {
    const int p = -kv[t][1];
    const int a = E->pairs[p].a, b = E->pairs[p].b;
    const int sa = a < 0 || E->b[a].is_static, sb = E->b[b].is_static;
    const unsigned long long m = (sa ? 0ull : used[a]) | (sb ? 0ull : used[b]);
    int c = 0;
    while (c < 63 && ((m >> c) & 1ull)) ++c;   /* colour 63 collects the overflow */
    if (c < 63) {
      if (!sa) used[a] |= 1ull << c;
      if (!sb) used[b] |= 1ull << c;
    }
    col[p] = c;
  }
  for (int i = 0; i < n; ++i) { kv[i][0] = col[i]; kv[i][1] = i; }
  qsort(kv, n, sizeof(int) * 2, cmp_int2);
  for (int i = 0; i < n; ++i) E->order[i] = kv[i][1];
  free(kv); free(used); free(col);
}

static void pgs_sweep(or_episode* E, double e, int cone) {
  for (int cc = 0; cc < E->np; ++cc) {
    or_pair* pr = &E->pairs[E->order[cc]];
    or_body *A = body_ref(E, pr->a), *B = body_ref(E, pr->b);
    const double* dirs[3] = {pr->n, pr->t1, pr->t2};
    for (int i = 0; i < pr->np; ++i) {
      if (cone) {
        /* normal row as in Eq. lambda_n, then both tangent rows from the same
           state, projected together onto the disc of radius mu lambda_n */
        double vn = rel_vel(A, B, pr->rA[i], pr->rB[i], dirs[0]);
        double old0 = pr->lam[i][0];
        double n0 = fmax(0.0, old0 - (1.0 + e) * (vn + pr->bias[i]) / pr->k[i][0]);
        pr->lam[i][0] = n0;
        double P0[3] = {(n0 - old0) * dirs[0][0], (n0 - old0) * dirs[0][1], (n0 - old0) * dirs[0][2]};
        apply_impulse(A, B, pr->rA[i], pr->rB[i], P0);
        double v1 = rel_vel(A, B, pr->rA[i], pr->rB[i], dirs[1]);
        double v2 = rel_vel(A, B, pr->rA[i], pr->rB[i], dirs[2]);
        double o1 = pr->lam[i][1], o2 = pr->lam[i][2], n1, n2;
        double kt = fmax(pr->k[i][1], pr->k[i][2]);
        disc_project(o1 - v1 / kt, o2 - v2 / kt, pr->mu * n0, &n1, &n2);
        pr->lam[i][1] = n1;
        pr->lam[i][2] = n2;
        double Pt[3];
        for (int j = 0; j < 3; ++j) Pt[j] = (n1 - o1) * dirs[1][j] + (n2 - o2) * dirs[2][j];
        apply_impulse(A, B, pr->rA[i], pr->rB[i], Pt);
        continue;
      }
      for (int r = 0; r < 3; ++r) {
        double vrel = rel_vel(A, B, pr->rA[i], pr->rB[i], dirs[r]);
        double old = pr->lam[i][r], nw;
        if (r == 0) {
          nw = fmax(0.0, old - (1.0 + e) * (vrel + pr->bias[i]) / pr->k[i][0]);
        } else {
          double lim = pr->mu * pr->lam[i][0];
          nw = clampd(old - vrel / pr->k[i][r], -lim, lim);
        }
        pr->lam[i][r] = nw;
        double Pv[3] = {(nw - old) * dirs[r][0], (nw - old) * dirs[r][1], (nw - old) * dirs[r][2]};
        apply_impulse(A, B, pr->rA[i], pr->rB[i], Pv);
      }
    }
  }
}

/* Reading of the PGS residual (m/s): max over rows of k |P(lambda - (v+b)/k) - lambda|
   with P the row's projection (normal: [0, inf); tangents: [-mu ln, mu ln],
   or with the cone the tangent pair's disc projection), evaluated at the
   current state without updating it. */
static double pgs_residual(or_episode* E, int cone) {
  double r = 0;
  for (int c = 0; c < E->np; ++c) {
    or_pair* pr = &E->pairs[c];
    or_body *A = body_ref(E, pr->a), *B = body_ref(E, pr->b);
    const double* dirs[3] = {pr->n, pr->t1, pr->t2};
    for (int i = 0; i < pr->np; ++i) {
      double tp[3] = {0, 0, 0}, kt = 0;
      if (cone) {
        double v1 = rel_vel(A, B, pr->rA[i], pr->rB[i], dirs[1]);
        double v2 = rel_vel(A, B, pr->rA[i], pr->rB[i], dirs[2]);
        kt = fmax(pr->k[i][1], pr->k[i][2]);
        disc_project(pr->lam[i][1] - v1 / kt, pr->lam[i][2] - v2 / kt, pr->mu * pr->lam[i][0], &tp[1], &tp[2]);
      }
      for (int k = 0; k < 3; ++k) {
        double vrel = rel_vel(A, B, pr->rA[i], pr->rB[i], dirs[k]);
        double l = pr->lam[i][k], proj;
        if (k == 0) proj = fmax(0.0, l - (vrel + pr->bias[i]) / pr->k[i][0]);
        else if (cone) proj = tp[k];
        else {
          double lim = pr->mu * pr->lam[i][0];
          proj = clampd(l - vrel / pr->k[i][k], -lim, lim);
        }
        double rr = (cone && k > 0 ? kt : pr->k[i][k]) * fabs(proj - l);
        if (!(rr <= r)) r = rr;   /* propagates NaN */
      }
    }
  }
  return r;
}

/* Optional acceleration of the sweeps (not in the paper): the nonsmooth
   nonlinear conjugate gradient method of Silcowitz, Niebe and Erleben ("A
   nonsmooth nonlinear conjugate gradient method for interactive contact force
   problems", The Visual Computer, 2010), with one conjugate-gradient step per
   block of m sweeps instead of per sweep.  Treating a block of sweeps as the
   map lambda -> G(lambda), with r = G(lambda) - lambda the change over the
   block:
     beta = |r_k|^2 / |r_(k-1)|^2 (Fletcher-Reeves; beta = 0 for the first
            block and whenever beta > 1, the restart),
     lambda <- proj(G(lambda) + beta d),   d <- r_k + beta d,
   where proj is each row's own projection (lambda_n >= 0, then the friction
   limits with the new lambda_n; the disc with the cone).  Reading: the step is
   projected so that the state stays feasible.  The impulse change of the step
   is applied to the bodies like any other impulse.  A fixed point of the
   sweep has r = 0, so it is a fixed point of this iteration and the converged
   impulses are plain PGS's; only the sweeps needed to reach a tolerance
   change.  These helpers run over the pairs in sweep order. */
static void accel_begin(or_episode* E) {
  for (int c = 0; c < E->np; ++c) {
    or_pair* pr = &E->pairs[c];
    for (int i = 0; i < pr->np; ++i)
      for (int k = 0; k < 3; ++k) { pr->lam_start[i][k] = pr->lam[i][k]; pr->dir[i][k] = 0; }
  }
}

static double accel_change2(const or_episode* E) {
  double s = 0;
  for (int c = 0; c < E->np; ++c) {
    const or_pair* pr = &E->pairs[c];
    for (int i = 0; i < pr->np; ++i)
      for (int k = 0; k < 3; ++k) { double r = pr->lam[i][k] - pr->lam_start[i][k]; s += r * r; }
  }
  return s;
}

static void accel_step(or_episode* E, double beta, int cone) {
  for (int cc = 0; cc < E->np; ++cc) {
    or_pair* pr = &E->pairs[E->order[cc]];
    or_body *A = body_ref(E, pr->a), *B = body_ref(E, pr->b);
    for (int i = 0; i < pr->np; ++i) {
      double nl[3];
      for (int k = 0; k < 3; ++k) nl[k] = pr->lam[i][k] + beta * pr->dir[i][k];
      nl[0] = fmax(0.0, nl[0]);
      const double lim = pr->mu * nl[0];
      if (cone) disc_project(nl[1], nl[2], lim, &nl[1], &nl[2]);
      else { nl[1] = clampd(nl[1], -lim, lim); nl[2] = clampd(nl[2], -lim, lim); }
      double Pv[3] = {0, 0, 0};
      for (int k = 0; k < 3; ++k) {
        const double dl = nl[k] - pr->lam[i][k];
        axpy3(dl, k == 0 ? pr->n : (k == 1 ? pr->t1 : pr->t2), Pv);
        pr->dir[i][k] = (pr->lam[i][k] - pr->lam_start[i][k]) + beta * pr->dir[i][k];
        pr->lam[i][k] = nl[k];
        pr->lam_start[i][k] = nl[k];
      }
      apply_impulse(A, B, pr->rA[i], pr->rB[i], Pv);
    }
  }
}

/* One sweep followed, at the end of every block of pgs_accel_period sweeps, by
   the acceleration step.  *r2_prev carries |r|^2 of the previous block. */
static void sweep_step(or_episode* E, const or_params* P, int sweeps_done, double* r2_prev) {
  pgs_sweep(E, P->restitution_newton ? 0.0 : P->restitution, P->friction_cone);
  const int m = P->pgs_accel_period;
  if (m > 0 && (sweeps_done + 1) % m == 0) {
    const double r2 = accel_change2(E);
    double beta = *r2_prev > 0 ? r2 / *r2_prev : 0.0;
    if (beta > 1.0) beta = 0.0;   /* restart */
    *r2_prev = r2;
    accel_step(E, beta, P->friction_cone);
  }
}

static void solve(or_episode* E, const or_params* P) {
  sweep_order(E, P->colour_order);
  int sweeps = 0;
  double res = 0, r2_prev = 0;
  if (P->pgs_accel_period > 0) accel_begin(E);
  if (E->np > 0) {
    if (P->residual_tol > 0) {
      for (;;) {
        sweep_step(E, P, sweeps, &r2_prev);
        ++sweeps;
        if (sweeps >= P->pgs_min_iters) {
          res = pgs_residual(E, P->friction_cone);
          if (res <= P->residual_tol) break;
          if (!(res == res)) break;
        }
        if (sweeps >= P->pgs_iter_cap) { E->status |= OR_STATUS_NOT_CONVERGED; break; }
      }
    } else {
      for (int s = 0; s < P->pgs_iters; ++s) sweep_step(E, P, s, &r2_prev);
      sweeps = P->pgs_iters;
      res = pgs_residual(E, P->friction_cone);
    }
  }
  E->last_sweeps = sweeps;
  E->last_res = res;
  if (res > E->max_res) E->max_res = res;
  E->total_sweeps += sweeps;
  E->solves += 1;
}

/* Sec. 4.2 position update and Eq. quat_int with world-frame omega
   (reading: q_dot = 1/2 [0, w] (x) q), renormalised. */
static void integrate(or_episode* E, double h) {
  for (int i = 0; i < E->nb; ++i) {
    or_body* B = &E->b[i];
    if (!B->active || B->is_static) continue;
    axpy3(h, B->v, B->x);
    double w0 = 0, w1 = B->w[0], w2 = B->w[1], w3 = B->w[2];
    double q0 = B->q[0], q1 = B->q[1], q2 = B->q[2], q3 = B->q[3];
    /* Hamilton product [0, w] (x) q */
    double d0 = w0 * q0 - w1 * q1 - w2 * q2 - w3 * q3;
    double d1 = w0 * q1 + w1 * q0 + w2 * q3 - w3 * q2;
    double d2 = w0 * q2 - w1 * q3 + w2 * q0 + w3 * q1;
    double d3 = w0 * q3 + w1 * q2 - w2 * q1 + w3 * q0;
    double nq[4] = {q0 + 0.5 * h * d0, q1 + 0.5 * h * d1, q2 + 0.5 * h * d2, q3 + 0.5 * h * d3};
    double l = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
    for (int k = 0; k < 4; ++k) B->q[k] = nq[k] / l;
  }
}

/* Eq. baumgarte, reading: dx_A = -beta max(0, depth - slop) m_A^-1/(m_A^-1 + m_B^-1) n,
   dx_B = +(same with m_B^-1); depth = the pair's deepest point of this substep's
   narrowphase; Jacobi-accumulated over pairs, then applied; translation only. */
static void baumgarte(or_episode* E, const or_params* P) {
  int nb = E->nb;
  double (*dx)[3] = (double(*)[3])calloc(nb > 0 ? nb : 1, sizeof(double) * 3);
  for (int c = 0; c < E->np; ++c) {
    or_pair* pr = &E->pairs[c];
    or_body *A = body_ref(E, pr->a), *B = body_ref(E, pr->b);
    double pen = pr->depth_max - P->slop;
    double wsum = A->invm + B->invm;
    if (pen <= 0 || wsum <= 0) continue;
    double s = P->beta * pen / wsum;
    if (pr->a >= 0) axpy3(-s * A->invm, pr->n, dx[pr->a]);
    axpy3(s * B->invm, pr->n, dx[pr->b]);
  }
  for (int i = 0; i < nb; ++i)
    if (E->b[i].active && !E->b[i].is_static) axpy3(1.0, dx[i], E->b[i].x);
  free(dx);
}

static void save_cache(or_episode* E) {
  if (E->capprev < E->np) {
    E->capprev = E->np;
    E->prev = (or_pair*)realloc(E->prev, sizeof(or_pair) * (E->capprev > 0 ? E->capprev : 1));
  }
  if (E->np) memcpy(E->prev, E->pairs, sizeof(or_pair) * E->np);
  E->nprev = E->np;
}

/* Warm-start network inputs of every point (learned warm start, not in the
   paper): pre-solve relative point velocity of B w.r.t. A along n, t1, t2
   over |g| h; depth over the margin; n; t1.x, t1.y (t1.z follows from n by
   the tangent rule); the height of the episode's column above the point
   (highest AABB top of its active dynamic blocks minus the point's z) over
   ten nominal block thicknesses, a stand-in for the load the point carries;
   m_bar/m of A and B (0 if static); body inertia diagonals over m_bar
   L_bar^2 (0 if static); mu; matched previous-frame impulses over m_bar |g|
   h; matched flag; ground flag. */
#define FEAT_MASS 0.015
#define FEAT_LEN 0.075
#define FEAT_COLUMN 0.15
static void features(or_episode* E, const or_params* P, double h) {
  double gh = norm3(P->gravity) * h;
  double sI = 1.0 / (FEAT_MASS * FEAT_LEN * FEAT_LEN);
  double ztop = 0.0;
  for (int i = 0; i < E->nb; ++i) {
    const or_body* B = &E->b[i];
    if (!B->active || B->is_static) continue;
    double ez = fabs(B->R[2][0]) * B->half[0] + fabs(B->R[2][1]) * B->half[1] + fabs(B->R[2][2]) * B->half[2];
    if (B->x[2] + ez > ztop) ztop = B->x[2] + ez;
  }
  for (int c = 0; c < E->np; ++c) {
    or_pair* pr = &E->pairs[c];
    or_body *A = body_ref(E, pr->a), *B = body_ref(E, pr->b);
    double IA[3] = {0, 0, 0}, IB[3] = {0, 0, 0};
    if (pr->a >= 0 && !A->is_static) { or_body_inertia(A->mass, A->half, IA); for (int k = 0; k < 3; ++k) IA[k] *= sI; }
    if (!B->is_static) { or_body_inertia(B->mass, B->half, IB); for (int k = 0; k < 3; ++k) IB[k] *= sI; }
    for (int i = 0; i < pr->np; ++i) {
      double wa[3], wb[3], u[3];
      cross3(A->w, pr->rA[i], wa); cross3(B->w, pr->rB[i], wb);
      for (int k = 0; k < 3; ++k) u[k] = (B->v[k] + wb[k]) - (A->v[k] + wa[k]);
      double* f = pr->feat[i];
      f[0] = dot3(u, pr->n) / gh; f[1] = dot3(u, pr->t1) / gh; f[2] = dot3(u, pr->t2) / gh;
      f[3] = P->contact_margin > 0 ? pr->depth[i] / P->contact_margin : 0.0;
      for (int k = 0; k < 3; ++k) f[4 + k] = pr->n[k];
      f[7] = pr->t1[0]; f[8] = pr->t1[1];
      f[9] = (ztop - pr->p[i][2]) / FEAT_COLUMN;
      f[10] = FEAT_MASS * A->invm; f[11] = FEAT_MASS * B->invm;
      for (int k = 0; k < 3; ++k) { f[12 + k] = IA[k]; f[15 + k] = IB[k]; }
      f[18] = pr->mu;
      for (int k = 0; k < 3; ++k) f[19 + k] = pr->lam[i][k] / (FEAT_MASS * gh);
      f[22] = pr->matched[i] ? 1.0 : 0.0;
      f[23] = pr->a < 0 ? 1.0 : 0.0;
    }
  }
}

static void record(or_world* W, or_episode* E, const or_params* P, double h) {
  double gh = norm3(P->gravity) * h;
  for (int c = 0; c < E->np; ++c) {
    or_pair* pr = &E->pairs[c];
    for (int i = 0; i < pr->np; ++i) {
      long slot;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
      slot = W->rec_count++;
      if (slot >= W->rec_cap) return;
      double* row = W->rec + (size_t)slot * OR_REC;
      memcpy(row, pr->feat[i], sizeof(double) * OR_NFEAT);
      for (int k = 0; k < 3; ++k) row[OR_NFEAT + k] = pr->lam[i][k] / (FEAT_MASS * gh);
    }
  }
}

/* One substep of length h: forces, detection, setup, warm start, PGS,
   integration, position correction. */
static void substep(or_world* W, or_episode* E, const or_params* P, double h) {
  for (int i = 0; i < E->nb; ++i) {
    or_body* B = &E->b[i];
    if (!B->active || B->is_static) continue;
    /* Sec. 4.2: v += h (g + F/m); reading: no gyroscopic term in the integrator */
    for (int k = 0; k < 3; ++k) B->v[k] += h * (P->gravity[k] + (B->f_steps > 0 ? B->f[k] * B->invm : 0.0));
  }
  for (int i = 0; i < E->nb; ++i) update_frame(&E->b[i]);
  detect(E, P);
  setup(E, h, P);
  warm_start_match(E, P);
  const int rec = W && W->rec && ((E->solves % W->rec_every) == 0);
  if (rec) features(E, P, h);
  apply_warm_start(E);
  solve(E, P);
  if (rec && (P->residual_tol <= 0 || E->last_res <= P->residual_tol)) record(W, E, P, h);
  integrate(E, h);
  baumgarte(E, P);
  save_cache(E);
}

/* Sec. 8.3: E_k = sum 1/2 m |v|^2 + 1/2 w . I_world w. */
static double kinetic(const or_body* B) {
  double I[3], wl[3];
  or_body_inertia(B->mass, B->half, I);
  double R[3][3];
  rotmat(B->q, R);
  for (int k = 0; k < 3; ++k) wl[k] = R[0][k] * B->w[0] + R[1][k] * B->w[1] + R[2][k] * B->w[2];
  return 0.5 * B->mass * dot3(B->v, B->v) + 0.5 * (I[0] * wl[0] * wl[0] + I[1] * wl[1] * wl[1] + I[2] * wl[2] * wl[2]);
}

/* Eq. collapse terms over active dynamic blocks, excluding `skip`.
   Reading: dx = |x - x0|; theta = angle between the current and initial
   thickness axes; fallen = dx > fall_frac * block length. */
static void collapse_terms(or_episode* E, int skip, double* ek, double* dxr, double* th, int* nfallen, double ff) {
  *ek = 0; *dxr = 0; *th = 0; *nfallen = 0;
  for (int i = 0; i < E->nb; ++i) {
    or_body* B = &E->b[i];
    if (!B->active || B->is_static || i == skip) continue;
    *ek += kinetic(B);
    double d[3] = {B->x[0] - B->x0[0], B->x[1] - B->x0[1], B->x[2] - B->x0[2]};
    double r = norm3(d) / (2 * B->half[0]);
    if (r > *dxr) *dxr = r;
    if (r > ff) (*nfallen)++;
    double R[3][3]; rotmat(B->q, R);
    double z[3]; col3(R, 2, z);
    double c = clampd(dot3(z, B->z0), -1.0, 1.0);
    double a = acos(c);
    if (a > *th) *th = a;
  }
}

static int count_dynamic(const or_episode* E) {
  int n = 0;
  for (int i = 0; i < E->nb; ++i) n += E->b[i].active && !E->b[i].is_static;
  return n;
}

static int state_finite(const or_episode* E) {
  for (int i = 0; i < E->nb; ++i) {
    const or_body* B = &E->b[i];
    for (int k = 0; k < 3; ++k)
      if (!isfinite(B->x[k]) || !isfinite(B->v[k]) || !isfinite(B->w[k])) return 0;
  }
  return 1;
}

static void start_move(or_episode* E, const or_params* P) {
  int m = E->mi;
  int blk = E->mv_block[m];
  or_body* B = &E->b[blk];
  double R[3][3]; rotmat(B->q, R);
  /* push axis: block Y = long axis (body x), block X = width axis (body y) */
  double dir[3]; col3(R, E->mv_axis[m] == 1 ? 0 : 1, dir);
  double g = norm3(P->gravity);
  /* Sec. 5: threshold force F = k mu_s m g, scaled by the schedule's factor */
  double F = E->mv_sign[m] * E->mv_factor[m] * E->mv_k[m] * B->mu * B->mass * g;
  for (int k = 0; k < 3; ++k) B->f[k] = F * dir[k];
  B->f_steps = E->mv_push[m];
  E->pb = blk;
  E->phase = OR_PH_PUSH;
  E->remaining = E->mv_push[m];
}

static void end_push(or_episode* E) {
  if (E->pb >= 0) {
    or_body* B = &E->b[E->pb];
    B->f[0] = B->f[1] = B->f[2] = 0; B->f_steps = 0;
  }
}

/* One step (n_sub substeps) plus the episode schedule. */
static void episode_step(or_world* W, or_episode* E, const or_params* P) {
  E->body_steps += count_dynamic(E);
  double h = P->dt / P->n_sub;
  for (int s = 0; s < P->n_sub; ++s) substep(W, E, P, h);
  for (int i = 0; i < E->nb; ++i)
    if (E->b[i].f_steps > 0) E->b[i].f_steps--;
  E->steps++;
  if (!state_finite(E)) { E->status |= OR_STATUS_NONFINITE; E->phase = E->phase == OR_PH_FREE ? OR_PH_FREE : OR_PH_DONE; return; }
  if (E->phase == OR_PH_FREE || E->phase == OR_PH_DONE) return;
  double ek, dxr, th; int nf;
  int skip = E->phase == OR_PH_PUSH ? E->pb : -1;
  collapse_terms(E, skip, &ek, &dxr, &th, &nf, P->fall_frac);
  int coll = dxr > P->fall_frac && ek > P->collapse_ek && th > P->collapse_theta_deg * OR_PI / 180.0;
  if ((E->phase == OR_PH_PUSH || E->phase == OR_PH_SETTLE) && coll) {
    E->collapsed = 1;
    if (E->phase == OR_PH_PUSH) end_push(E);
    E->pb = -1;
    E->phase = OR_PH_REST;
    E->rest_left = P->rest_steps;
    return;
  }
  if (E->phase == OR_PH_PUSH) {
    if (--E->remaining <= 0) {
      end_push(E);
      if (E->mv_remove[E->mi]) { E->b[E->pb].active = 0; }
      E->pb = -1;
      E->phase = OR_PH_SETTLE;
      E->remaining = E->mv_settle[E->mi];
      if (E->remaining <= 0) goto next_move;
    }
    return;
  }
  if (E->phase == OR_PH_SETTLE) {
    if (--E->remaining <= 0) goto next_move;
    return;
  }
  if (E->phase == OR_PH_REST) {
    double eka, d1, d2; int n1;
    collapse_terms(E, -1, &eka, &d1, &d2, &n1, P->fall_frac);
    E->rest_left--;
    if (eka < P->rest_ek) { E->resting = 1; E->phase = OR_PH_DONE; }
    else if (E->rest_left <= 0) E->phase = OR_PH_DONE;
    return;
  }
  return;
next_move:
  E->mi++;
  if (E->mi < E->n_moves) start_move(E, P);
  else E->phase = OR_PH_DONE;
}

/* ------------------------------------------------------------- public API -- */
or_world* or_create(int n_episodes, const int* body_off, const double* half, const double* mass,
                    const double* mu, const double* x, const double* q, const double* v,
                    const double* w, const double* ground_mu, const or_params* p) {
  or_world* W = (or_world*)calloc(1, sizeof(or_world));
  W->E = n_episodes;
  W->B = body_off[n_episodes];
  W->P = *p;
  W->body_off = (int*)malloc(sizeof(int) * (n_episodes + 1));
  memcpy(W->body_off, body_off, sizeof(int) * (n_episodes + 1));
  W->ep = (or_episode*)calloc(n_episodes > 0 ? n_episodes : 1, sizeof(or_episode));
  int NB = W->B;
  for (int e = 0; e < n_episodes; ++e) {
    or_episode* E = &W->ep[e];
    E->nb = body_off[e + 1] - body_off[e];
    E->b = (or_body*)calloc(E->nb > 0 ? E->nb : 1, sizeof(or_body));
    E->ground_mu = ground_mu[e];
    E->ground.q[0] = 1;
    update_frame(&E->ground);
    E->phase = OR_PH_FREE;
    E->pb = -1;
    for (int i = 0; i < E->nb; ++i) {
      int g = body_off[e] + i;
      or_body* B = &E->b[i];
      for (int k = 0; k < 3; ++k) {
        B->x[k] = x[k * NB + g]; B->half[k] = half[k * NB + g];
        B->v[k] = v ? v[k * NB + g] : 0; B->w[k] = w ? w[k * NB + g] : 0;
      }
      double ql = 0;
      for (int k = 0; k < 4; ++k) { B->q[k] = q[k * NB + g]; ql += B->q[k] * B->q[k]; }
      ql = sqrt(ql);
      for (int k = 0; k < 4; ++k) B->q[k] /= ql;
      B->mass = mass[g];
      B->mu = mu[g];
      B->active = 1;
      B->is_static = !(mass[g] > 0);
      if (!B->is_static) {
        double I[3]; or_body_inertia(B->mass, B->half, I);
        B->invm = 1.0 / B->mass;
        for (int k = 0; k < 3; ++k) B->invI[k] = 1.0 / I[k];
      } else {
        B->v[0] = B->v[1] = B->v[2] = B->w[0] = B->w[1] = B->w[2] = 0;
      }
      update_frame(B);
      memcpy(B->x0, B->x, sizeof B->x0);
      col3(B->R, 2, B->z0);
    }
  }
  return W;
}

void or_destroy(or_world* W) {
  if (!W) return;
  for (int e = 0; e < W->E; ++e) { free(W->ep[e].b); free(W->ep[e].pairs); free(W->ep[e].prev); free(W->ep[e].order); }
  free(W->ep); free(W->body_off);
  free(W->m_block); free(W->m_axis); free(W->m_remove); free(W->m_push); free(W->m_settle);
  free(W->m_sign); free(W->m_factor); free(W->m_k);
  free(W);
}

int or_set_protocol(or_world* W, const int* off, const int* block, const int* axis, const double* sign,
                    const double* factor, const double* k, const int* remove, const int* push_steps,
                    const int* settle_steps) {
  int M = off[W->E];
  size_t n = (size_t)(M > 0 ? M : 1);
#define DUP(dst, src, T) do { dst = (T*)malloc(sizeof(T) * n); if (M) memcpy(dst, src, sizeof(T) * M); } while (0)
  DUP(W->m_block, block, int); DUP(W->m_axis, axis, int); DUP(W->m_remove, remove, int);
  DUP(W->m_push, push_steps, int); DUP(W->m_settle, settle_steps, int);
  DUP(W->m_sign, sign, double); DUP(W->m_factor, factor, double); DUP(W->m_k, k, double);
#undef DUP
  for (int e = 0; e < W->E; ++e) {
    or_episode* E = &W->ep[e];
    int o = off[e];
    E->n_moves = off[e + 1] - o;
    for (int m = 0; m < E->n_moves; ++m)
      if (block[o + m] < 0 || block[o + m] >= E->nb) return -1;
    E->mv_block = W->m_block + o; E->mv_axis = W->m_axis + o; E->mv_remove = W->m_remove + o;
    E->mv_push = W->m_push + o; E->mv_settle = W->m_settle + o;
    E->mv_sign = W->m_sign + o; E->mv_factor = W->m_factor + o; E->mv_k = W->m_k + o;
    E->mi = 0;
    if (E->n_moves > 0) start_move(E, &W->P);
    else E->phase = OR_PH_DONE;
  }
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int or_run_protocol(or_world* W, int max_steps, int n_threads) {
  int maxs = 0;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(max : maxs)
#endif
  for (int e = 0; e < W->E; ++e) {
    or_episode* E = &W->ep[e];
    int s = 0;
    while (s < max_steps && E->phase != OR_PH_DONE && E->phase != OR_PH_FREE) { episode_step(W, E, &W->P); ++s; }
    if (s > maxs) maxs = s;
  }
  (void)n_threads;
  return maxs;
}

void or_step(or_world* W, int n_steps, int n_threads) {
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int e = 0; e < W->E; ++e)
    for (int s = 0; s < n_steps; ++s) episode_step(W, &W->ep[e], &W->P);
  (void)n_threads;
}

int or_apply_push(or_world* W, int e, int blk, int axis, double force, int n_steps) {
  if (e < 0 || e >= W->E || blk < 0 || blk >= W->ep[e].nb) return -1;
  or_body* B = &W->ep[e].b[blk];
  double R[3][3]; rotmat(B->q, R);
  double dir[3]; col3(R, axis == 1 ? 0 : 1, dir);
  for (int k = 0; k < 3; ++k) B->f[k] = force * dir[k];
  B->f_steps = n_steps;
  return 0;
}

int or_remove_block(or_world* W, int e, int blk) {
  if (e < 0 || e >= W->E || blk < 0 || blk >= W->ep[e].nb) return -1;
  W->ep[e].b[blk].active = 0;
  return 0;
}

int or_active(const or_world* W, int g) {
  for (int e = 0; e < W->E; ++e)
    if (g < W->body_off[e + 1]) return W->ep[e].b[g - W->body_off[e]].active;
  return 0;
}

void or_get_state(const or_world* W, double* x, double* q, double* v, double* w) {
  int NB = W->B;
  for (int e = 0; e < W->E; ++e)
    for (int i = 0; i < W->ep[e].nb; ++i) {
      int g = W->body_off[e] + i;
      const or_body* B = &W->ep[e].b[i];
      for (int k = 0; k < 3; ++k) {
        if (x) x[k * NB + g] = B->x[k];
        if (v) v[k * NB + g] = B->v[k];
        if (w) w[k * NB + g] = B->w[k];
      }
      if (q) for (int k = 0; k < 4; ++k) q[k * NB + g] = B->q[k];
    }
}

void or_set_state(or_world* W, const double* x, const double* q, const double* v, const double* w) {
  int NB = W->B;
  for (int e = 0; e < W->E; ++e)
    for (int i = 0; i < W->ep[e].nb; ++i) {
      int g = W->body_off[e] + i;
      or_body* B = &W->ep[e].b[i];
      for (int k = 0; k < 3; ++k) {
        if (x) B->x[k] = x[k * NB + g];
        if (v && !B->is_static) B->v[k] = v[k * NB + g];
        if (w && !B->is_static) B->w[k] = w[k * NB + g];
      }
      if (q) {
        double l = 0;
        for (int k = 0; k < 4; ++k) { B->q[k] = q[k * NB + g]; l += B->q[k] * B->q[k]; }
        l = sqrt(l);
        for (int k = 0; k < 4; ++k) B->q[k] /= l;
      }
      update_frame(B);
    }
}

void or_set_recorder(or_world* W, double* rows, int capacity, int every) {
  W->rec = capacity > 0 ? rows : NULL;
  W->rec_cap = capacity;
  W->rec_every = every > 0 ? every : 1;
  W->rec_count = 0;
}

long or_recorded(const or_world* W) { return W->rec_count; }

void or_clear_cache(or_world* W) {
  for (int e = 0; e < W->E; ++e) W->ep[e].nprev = 0;
}

static void write_crec(const or_pair* pr, double* o) {
  memset(o, 0, sizeof(double) * OR_CREC);
  o[0] = pr->a; o[1] = pr->b; o[2] = pr->axis; o[3] = pr->ref_face; o[4] = pr->inc_face; o[5] = pr->np;
  for (int k = 0; k < 3; ++k) { o[6 + k] = pr->n[k]; o[9 + k] = pr->t1[k]; }
  o[12] = pr->delta; o[13] = pr->mu; o[14] = pr->depth_max;
  for (int i = 0; i < pr->np; ++i) {
    double* r = o + 15 + 10 * i;
    for (int k = 0; k < 3; ++k) { r[k] = pr->p[i][k]; r[4 + k] = pr->lam[i][k]; r[7 + k] = pr->local[i][k]; }
    r[3] = pr->depth[i];
  }
}

int or_get_contacts(const or_world* W, int e, double* out, int cap) {
  if (e < 0 || e >= W->E) return -1;
  const or_episode* E = &W->ep[e];
  /* the cache holds the last substep's pairs with their final impulses */
  for (int c = 0; c < E->nprev && c < cap; ++c) write_crec(&E->prev[c], out + (size_t)c * OR_CREC);
  return E->nprev;
}

/* Eq. stability: support polygon = convex hull (Andrew's monotone chain) of
   the xy corners of ground-touching blocks; d = min over the hull edges of
   the signed distance from the COM to the edge's line, positive inside
   (reading: inside, that is the distance to the boundary; outside, it is not
   the distance to the polygon).  Reading for degenerate hulls (fewer than 3
   vertices): minus the distance to the segment or point. */
static int cmp_xy(const void* a, const void* b) {
  const double *p = (const double*)a, *q = (const double*)b;
  if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
  if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
  return 0;
}
static double cross2(const double* o, const double* a, const double* b) {
  return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0]);
}
double or_support_margin(int n, const double* xy, const double* com) {
  if (n <= 0) return -INFINITY;
  double* P = (double*)malloc(sizeof(double) * 2 * n);
  memcpy(P, xy, sizeof(double) * 2 * n);
  qsort(P, n, sizeof(double) * 2, cmp_xy);
  double* H = (double*)malloc(sizeof(double) * 2 * (2 * n + 1));
  int k = 0;
  for (int i = 0; i < n; ++i) {
    while (k >= 2 && cross2(H + 2 * (k - 2), H + 2 * (k - 1), P + 2 * i) <= 0) --k;
    H[2 * k] = P[2 * i]; H[2 * k + 1] = P[2 * i + 1]; ++k;
  }
  for (int i = n - 2, t = k + 1; i >= 0; --i) {
    while (k >= t && cross2(H + 2 * (k - 2), H + 2 * (k - 1), P + 2 * i) <= 0) --k;
    H[2 * k] = P[2 * i]; H[2 * k + 1] = P[2 * i + 1]; ++k;
  }
  int m = k > 1 ? k - 1 : k;   /* hull vertices, counter-clockwise */
  double d;
  if (m >= 3) {
    d = INFINITY;
    for (int i = 0; i < m; ++i) {
      const double *a = H + 2 * i, *b = H + 2 * ((i + 1) % m);
      double ex = b[0] - a[0], ey = b[1] - a[1];
      double s = (ex * (com[1] - a[1]) - ey * (com[0] - a[0])) / sqrt(ex * ex + ey * ey);
      if (s < d) d = s;
    }
  } else if (m == 2) {
    const double *a = H, *b = H + 2;
    double ex = b[0] - a[0], ey = b[1] - a[1];
    double l2 = ex * ex + ey * ey;
    double t = l2 > 0 ? clampd(((com[0] - a[0]) * ex + (com[1] - a[1]) * ey) / l2, 0, 1) : 0;
    double dx = com[0] - (a[0] + t * ex), dy = com[1] - (a[1] + t * ey);
    d = -sqrt(dx * dx + dy * dy);
  } else {
    double dx = com[0] - H[0], dy = com[1] - H[1];
    d = -sqrt(dx * dx + dy * dy);
  }
  free(P); free(H);
  return d;
}

void or_collapse_terms(const or_world* W, int e, double* ek, double* dx_ratio, double* theta, int* n_fallen) {
  collapse_terms((or_episode*)&W->ep[e], -1, ek, dx_ratio, theta, n_fallen, W->P.fall_frac);
}

static int removed_blocks(const or_episode* E) {
  int r = 0;
  for (int i = 0; i < E->nb; ++i) r += !E->b[i].active;
  return r;
}

int or_reference_episode(const or_world* W, int n_hat, int* n_removed) {
  int best = -1;
  for (int e = 0; e < W->E; ++e) {
    if (!W->ep[e].collapsed) continue;
    if (best < 0 || abs(removed_blocks(&W->ep[e]) - n_hat) < abs(removed_blocks(&W->ep[best]) - n_hat)) best = e;
  }
  if (best < 0)
    for (int e = 0; e < W->E; ++e)
      if (best < 0 || W->ep[e].mi > W->ep[best].mi) best = e;
  if (n_removed) *n_removed = best >= 0 ? removed_blocks(&W->ep[best]) : 0;
  return best;
}

double or_com_imbalance(const or_world* W, int e) {
  const or_episode* E = &W->ep[e];
  const double eps = W->P.aabb_eps;
  double com[2] = {0, 0}, mt = 0;
  double* xy = (double*)malloc(sizeof(double) * 16 * (E->nb > 0 ? E->nb : 1));
  int n = 0;
  for (int i = 0; i < E->nb; ++i) {
    const or_body* B = &E->b[i];
    if (!B->active || B->is_static) continue;
    com[0] += B->mass * B->x[0]; com[1] += B->mass * B->x[1]; mt += B->mass;
    double R[3][3]; rotmat(B->q, R);
    double ez = fabs(R[2][0]) * B->half[0] + fabs(R[2][1]) * B->half[1] + fabs(R[2][2]) * B->half[2];
    if (B->x[2] - ez > eps) continue;
    for (int c = 0; c < 8; ++c) {
      double s0 = (c & 1) ? 1 : -1, s1 = (c & 2) ? 1 : -1, s2 = (c & 4) ? 1 : -1;
      for (int k = 0; k < 2; ++k)
        xy[2 * n + k] = B->x[k] + s0 * B->half[0] * R[k][0] + s1 * B->half[1] * R[k][1] + s2 * B->half[2] * R[k][2];
      ++n;
    }
  }
  double r;
  if (mt <= 0 || n == 0) r = 0;
  else {
    com[0] /= mt; com[1] /= mt;
    r = -or_support_margin(n, xy, com);
  }
  free(xy);
  return r;
}

void or_get_stats(or_world* W, double* out) {
  for (int e = 0; e < W->E; ++e) {
    or_episode* E = &W->ep[e];
    double* o = out + (size_t)e * OR_NSTAT;
    double ek, dxr, th; int nf;
    collapse_terms(E, -1, &ek, &dxr, &th, &nf, W->P.fall_frac);
    int npts = 0;
    for (int c = 0; c < E->nprev; ++c) npts += E->prev[c].np;
    o[OR_ST_STATUS] = E->status; o[OR_ST_COLLAPSED] = E->collapsed;
    o[OR_ST_RESTING] = E->resting || ek < W->P.rest_ek; o[OR_ST_NFALLEN] = nf;
    o[OR_ST_COM_IMB] = or_com_imbalance(W, e); o[OR_ST_EK] = ek;
    o[OR_ST_LAST_RES] = E->last_res; o[OR_ST_LAST_SWEEPS] = E->last_sweeps;
    o[OR_ST_TOTAL_SWEEPS] = (double)E->total_sweeps; o[OR_ST_SOLVES] = (double)E->solves;
    o[OR_ST_STEPS] = (double)E->steps; o[OR_ST_BODY_STEPS] = E->body_steps;
    o[OR_ST_PHASE] = E->phase; o[OR_ST_MOVES_DONE] = E->mi; o[OR_ST_NPAIRS] = E->nprev;
    o[OR_ST_NPOINTS] = npts; o[OR_ST_MAX_RES] = E->max_res;
  }
}

/* ------------------------------------------------------- stage entry points */
static void mkbox(const double* x, const double* q, const double* h, box_t* b) {
  double qq[4], l = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) qq[k] = q[k] / l;
  memcpy(b->x, x, sizeof b->x); memcpy(b->h, h, sizeof b->h);
  rotmat(qq, b->R);
}

int or_sat_select(const double* delta15, const int* valid15, double* dmin) {
  return sat_select(delta15, valid15, dmin);
}

int or_sat(const double* xA, const double* qA, const double* hA, const double* xB, const double* qB,
           const double* hB, double margin, double* delta15, int* valid15, int* axis, double* n, double* dmin) {
  box_t A, B; mkbox(xA, qA, hA, &A); mkbox(xB, qB, hB, &B);
  double U[15][3];
  sat15(&A, &B, delta15, valid15, U);
  int ax = sat_select(delta15, valid15, dmin);
  double d[3] = {B.x[0] - A.x[0], B.x[1] - A.x[1], B.x[2] - A.x[2]};
  double s = dot3(U[ax], d) < 0 ? -1 : 1;
  for (int k = 0; k < 3; ++k) n[k] = s * U[ax][k];
  *axis = ax;
  return *dmin > -margin;
}

int or_pair_manifold(const double* xA, const double* qA, const double* hA, const double* xB, const double* qB,
                     const double* hB, double margin, double* out) {
  box_t A, B; mkbox(xA, qA, hA, &A); mkbox(xB, qB, hB, &B);
  or_pair pr; memset(&pr, 0, sizeof pr);
  int ok = box_pair(&A, &B, margin, &pr, NULL);
  pr.a = 0; pr.b = 1;
  if (ok) tangent_basis(pr.n, pr.t1, pr.t2);
  write_crec(&pr, out);
  return ok ? pr.np : 0;
}

int or_ground_manifold(const double* x, const double* q, const double* h, double margin, double* out) {
  box_t B; mkbox(x, q, h, &B);
  or_pair pr; memset(&pr, 0, sizeof pr);
  int ok = ground_pair(&B, margin, &pr);
  pr.a = -1; pr.b = 0;
  if (ok) tangent_basis(pr.n, pr.t1, pr.t2);
  write_crec(&pr, out);
  return ok ? pr.np : 0;
}
