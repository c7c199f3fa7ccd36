// Device kernels of the batched rigid-body step (sm_103a).
//
// One warp owns one episode (a tower) for the whole launch: the episode's
// bodies and, when they fit, its colour-sorted contact pairs and points live
// in shared memory; the natural-order contact records (and the solver arrays
// of steps with more pairs than fit) live in the global workspace.  A
// persistent grid claims episodes from a work counter.  Per substep the warp
// runs (paper sections in brackets):
//   forces and frames [Sec. 4.2, Eq. rotmat]
//   broadphase, all pairs, ballot compaction in natural order [Sec. 6.1, Eq. aabb]
//   SAT over 15 axes + face-clipped manifold, one pair per lane [Sec. 6.2, 6.2.1]
//   warm-start matching against the previous step's contacts
//   greedy edge colouring of the contact graph, redone every step
//   contact setup [Sec. 7.1, Eq. keff]; optionally the learned warm start
//   coloured projected Gauss-Seidel: pairs of one colour share no dynamic body
//   and run in parallel, one per lane, colours in sequence [Sec. 7.1-7.3,
//   Eq. lambda_n, Eq. coulomb_pgs]; residual mode sweeps until the residual
//   <= tol, checked at an adaptive cadence
//   integration [Sec. 4.2, Eq. quat_int] and position correction [Eq. baumgarte]
//   collapse / rest bookkeeping and the push schedule [Sec. 5, Sec. 8]
// Everything is FP32 (the network's operands BF16).  Waits are warp barriers
// only; every loop is bounded.
#include <cfloat>
#include <climits>
#include <cstdint>

#include "jb_internal.cuh"
#include "jb_mlp.cuh"

namespace jbk {

#define FULL 0xffffffffu

// ------------------------------------------------------------ float3 helpers
__device__ __forceinline__ float3 f3(float a, float b, float c) { return make_float3(a, b, c); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float sgnf(float v) { return v >= 0.f ? 1.f : -1.f; }

// ------------------------------------------------------ shared-memory view
enum { FX = 0, FQ = 3, FV = 7, FW = 10, FH = 13, FR = 16, FI = 25, FE = 31, FM = 34, FMU = 35 };

struct Sm {
  int nbs;
  float* F;
  int* flags;
  unsigned long long* mask;
  uint32_t* cand;
  int* cnt;   // [kMaxColours + 1]
  int* off;   // [kMaxColours + 1]
  int* run;   // [kMaxColours + 1]
  float* sf;  // colour-sorted solver arrays for up to ps pairs
  uint32_t* ab;
  int32_t* np;
  float* sp;
  int ps;
  __device__ __forceinline__ float& at(int f, int i) const { return F[i * kBodyStride + f]; }
  __device__ __forceinline__ float3 ld3(int f, int i) const { return f3(at(f, i), at(f + 1, i), at(f + 2, i)); }
  __device__ __forceinline__ void st3(int f, int i, float3 v) const { at(f, i) = v.x; at(f + 1, i) = v.y; at(f + 2, i) = v.z; }
  // column k of the rotation matrix (body axis k in world coordinates)
  __device__ __forceinline__ float3 axis(int i, int k) const { return f3(at(FR + k, i), at(FR + 3 + k, i), at(FR + 6 + k, i)); }
  __device__ __forceinline__ float3 iw_mul(int i, float3 u) const {
    float xx = at(FI, i), yy = at(FI + 1, i), zz = at(FI + 2, i), xy = at(FI + 3, i), xz = at(FI + 4, i), yz = at(FI + 5, i);
    return f3(xx * u.x + xy * u.y + xz * u.z, xy * u.x + yy * u.y + yz * u.z, xz * u.x + yz * u.y + zz * u.z);
  }
};

__device__ __forceinline__ Sm sm_view(unsigned char* base, int nb_max, int pc_max, int ps) {
  SmemPlan p = smem_plan(nb_max, pc_max, ps);
  Sm s;
  s.nbs = p.nbs;
  s.mask = reinterpret_cast<unsigned long long*>(base + p.off_mask);
  s.F = reinterpret_cast<float*>(base + p.off_f);
  s.flags = reinterpret_cast<int*>(base + p.off_flags);
  s.cand = reinterpret_cast<uint32_t*>(base + p.off_cand);
  s.cnt = reinterpret_cast<int*>(base + p.off_col);
  s.off = s.cnt + (kMaxColours + 1);
  s.run = s.off + (kMaxColours + 1);
  s.sf = reinterpret_cast<float*>(base + p.off_sf);
  s.ab = reinterpret_cast<uint32_t*>(base + p.off_ab);
  s.np = reinterpret_cast<int32_t*>(base + p.off_np);
  s.sp = reinterpret_cast<float*>(base + p.off_sp);
  s.ps = ps;
  return s;
}

// ------------------------------------------------------------ narrowphase
struct Box {
  float3 c, a0, a1, a2, h;
  __device__ __forceinline__ float3 ax(int k) const { return k == 0 ? a0 : (k == 1 ? a1 : a2); }
  __device__ __forceinline__ float hk(int k) const { return k == 0 ? h.x : (k == 1 ? h.y : h.z); }
  __device__ __forceinline__ float radius(float3 u) const {
    return h.x * fabsf(dot(a0, u)) + h.y * fabsf(dot(a1, u)) + h.z * fabsf(dot(a2, u));
  }
};

__device__ __forceinline__ Box box_of(const Sm& s, int i) {
  Box b;
  b.c = s.ld3(FX, i);
  b.a0 = s.axis(i, 0); b.a1 = s.axis(i, 1); b.a2 = s.axis(i, 2);
  b.h = s.ld3(FH, i);
  return b;
}

struct Contact {
  int axis, ref_face, inc_face, np;
  float3 n;
  float delta, dmax;
  float3 p[kMaxPts];
  float depth[kMaxPts];
};

constexpr int kDenseChecks = 6;     // residual checks every sweep over this many sweeps after a CG step
constexpr float kTieAbs = 1e-5f;    // SAT axis hysteresis (m): keeps near-parallel axis choices stable
constexpr float kEdgeRel = 0.05f;   // a cross axis must beat the best face axis by 5 %
constexpr float kCrossEps = 1e-6f;  // degenerate cross axes are skipped
constexpr float kIncTie = 1e-9f;
constexpr float kClipEps = 1e-6f;   // reference face enlarged by 1 um for clipping
constexpr float kMergeEps = 1e-6f;  // clipped vertices closer than 1 um are one vertex
constexpr float kDepthTie = 1e-6f;  // depths within 1 um tie (lowest index wins)
constexpr float kAreaTie = 1e-9f;   // squared distances / areas within 1e-9 m^2 tie

__device__ __forceinline__ float3 sat_axis(const Box& A, const Box& B, int k, bool& ok) {
  ok = true;
  if (k < 3) return A.ax(k);
  if (k < 6) return B.ax(k - 3);
  float3 u = cross(A.ax((k - 6) / 3), B.ax((k - 6) % 3));
  float l = sqrtf(dot(u, u));
  if (l < kCrossEps) { ok = false; return f3(0.f, 0.f, 0.f); }
  return (1.f / l) * u;
}

__device__ __forceinline__ float tri_area(float3 a, float3 b, float3 c, float3 n) {
  return 0.5f * fabsf(dot(cross(b - a, c - a), n));
}
__device__ __forceinline__ float quad_area(float3 a, float3 b, float3 c, float3 d, float3 n) {
  float3 s = cross(a, b) + cross(b, c) + cross(c, d) + cross(d, a);
  return 0.5f * fabsf(dot(s, n));
}
__device__ float hull4(float3 a, float3 b, float3 c, float3 d, float3 n) {
  float m = quad_area(a, b, c, d, n);
  m = fmaxf(m, quad_area(a, b, d, c, n));
  m = fmaxf(m, quad_area(a, c, b, d, n));
  m = fmaxf(m, tri_area(a, b, c, n));
  m = fmaxf(m, tri_area(a, b, d, n));
  m = fmaxf(m, tri_area(a, c, d, n));
  m = fmaxf(m, tri_area(b, c, d, n));
  return m;
}

// Keeps at most 4 of m points: deepest; farthest from it; largest triangle;
// largest added hull area, in that order.  Scores within a tie tolerance count
// as equal and the lowest index wins.
__device__ void keep4(int m, const float3* P, const float* D, float3 nrm, Contact& C) {
  if (m <= kMaxPts) {
    float dm = -FLT_MAX;
    for (int i = 0; i < m; ++i) { C.p[i] = P[i]; C.depth[i] = D[i]; dm = fmaxf(dm, D[i]); }
    C.np = m; C.dmax = dm;
    return;
  }
  float sc[8];
  unsigned used = 0;
  float best = -FLT_MAX;
  for (int i = 0; i < m; ++i) best = fmaxf(best, D[i]);
  int i1 = 0;
  while (D[i1] < best - kDepthTie) ++i1;
  used |= 1u << i1;
  best = -1.f;
  for (int i = 0; i < m; ++i) {
    float3 d = P[i] - P[i1];
    sc[i] = (used >> i & 1) ? -1.f : dot(d, d);
    best = fmaxf(best, sc[i]);
  }
  int i2 = 0;
  while ((used >> i2 & 1) || sc[i2] < best - kAreaTie) ++i2;
  used |= 1u << i2;
  best = -1.f;
  for (int i = 0; i < m; ++i) {
    sc[i] = (used >> i & 1) ? -1.f : tri_area(P[i1], P[i2], P[i], nrm);
    best = fmaxf(best, sc[i]);
  }
  int i3 = 0;
  while ((used >> i3 & 1) || sc[i3] < best - kAreaTie) ++i3;
  used |= 1u << i3;
  float base = tri_area(P[i1], P[i2], P[i3], nrm);
  best = -1.f;
  for (int i = 0; i < m; ++i) {
    sc[i] = (used >> i & 1) ? -1.f : hull4(P[i1], P[i2], P[i3], P[i], nrm) - base;
    best = fmaxf(best, sc[i]);
  }
  int i4 = 0;
  while ((used >> i4 & 1) || sc[i4] < best - kAreaTie) ++i4;
  int sel[4] = {i1, i2, i3, i4};
  float dm = -FLT_MAX;
  for (int q = 0; q < 4; ++q) { C.p[q] = P[sel[q]]; C.depth[q] = D[sel[q]]; dm = fmaxf(dm, D[sel[q]]); }
  C.np = 4; C.dmax = dm;
}

// Sutherland-Hodgman against the half-space (p - c).u <= h.
__device__ int clip_poly(const float3* in, int n, float3* out, float3 c, float3 u, float h) {
  int m = 0;
  if (n == 0) return 0;
  float3 S = in[n - 1];
  float dS = dot(S - c, u) - h;
  for (int i = 0; i < n; ++i) {
    float3 E = in[i];
    float dE = dot(E - c, u) - h;
    if (dE <= 0.f) {
      if (dS > 0.f && m < 8) { out[m++] = S + (dS / (dS - dE)) * (E - S); }
      if (m < 8) out[m++] = E;
    } else if (dS <= 0.f && m < 8) {
      out[m++] = S + (dS / (dS - dE)) * (E - S);
    }
    S = E; dS = dE;
  }
  return m;
}

// Clipping runs in coordinates relative to the reference box centre, which
// keeps FP32 rounding of the clip intersections small for boxes far from the
// origin; the points are moved back at the end.
__device__ void face_contact(const Box& A, const Box& B, int axis, float3 n, float margin, Contact& C) {
  Box ref = axis < 3 ? A : B;
  Box inc = axis < 3 ? B : A;
  const float3 origin = ref.c;
  inc.c = inc.c - origin;
  ref.c = f3(0.f, 0.f, 0.f);
  int ra = axis < 3 ? axis : axis - 3;
  float3 nref = axis < 3 ? n : -n;
  float3 ax = ref.ax(ra);
  float sr = sgnf(dot(ax, nref));
  float3 cr = ref.c + (sr * ref.hk(ra)) * ax;
  int r1 = (ra + 1) % 3, r2 = (ra + 2) % 3;
  float3 u1 = ref.ax(r1), u2 = ref.ax(r2);
  float h1 = ref.hk(r1), h2 = ref.hk(r2);
  int ji = 0; float bd = -1.f;
  for (int j = 0; j < 3; ++j) {
    float dd = fabsf(dot(inc.ax(j), nref));
    if (dd > bd + kIncTie) { bd = dd; ji = j; }
  }
  float3 bj = inc.ax(ji);
  float si = -sgnf(dot(bj, nref));
  float3 ci = inc.c + (si * inc.hk(ji)) * bj;
  int j1 = (ji + 1) % 3, j2 = (ji + 2) % 3;
  float3 v1 = inc.hk(j1) * inc.ax(j1), v2 = inc.hk(j2) * inc.ax(j2);
  float3 pa[8], pb[8];
  pa[0] = ci + v1 + v2; pa[1] = ci - v1 + v2; pa[2] = ci - v1 - v2; pa[3] = ci + v1 - v2;
  int m = clip_poly(pa, 4, pb, cr, u1, h1 + kClipEps);
  m = clip_poly(pb, m, pa, cr, -u1, h1 + kClipEps);
  m = clip_poly(pa, m, pb, cr, u2, h2 + kClipEps);
  m = clip_poly(pb, m, pa, cr, -u2, h2 + kClipEps);
  float D[8];
  int k = 0;
  for (int i = 0; i < m; ++i) {
    float dep = dot(cr - pa[i], nref);
    if (!(dep > -margin)) continue;
    bool dup = false;
    for (int j = 0; j < k && !dup; ++j) {
      float3 q = pa[i] - (pb[j] - (0.5f * D[j]) * nref);
      dup = dot(q, q) < kMergeEps * kMergeEps;
    }
    if (dup) continue;
    pb[k] = pa[i] + (0.5f * dep) * nref; D[k] = dep; ++k;
  }
  C.ref_face = 2 * ra + (sr > 0.f ? 0 : 1) + (axis < 3 ? 0 : 8);
  C.inc_face = 2 * ji + (si > 0.f ? 0 : 1);
  keep4(k, pb, D, n, C);
  for (int i = 0; i < C.np; ++i) C.p[i] = C.p[i] + origin;
}

__device__ void edge_contact(const Box& A, const Box& B, int axis, float3 n, float delta, Contact& C) {
  int i = (axis - 6) / 3, j = (axis - 6) % 3;
  float3 pa = f3(0.f, 0.f, 0.f), pb = B.c - A.c;   // relative to A's centre
  for (int m = 0; m < 3; ++m) {
    if (m != i) { float3 c = A.ax(m); pa = pa + (sgnf(dot(c, n)) * A.hk(m)) * c; }
    if (m != j) { float3 c = B.ax(m); pb = pb + (-sgnf(dot(c, n)) * B.hk(m)) * c; }
  }
  float3 ea = A.ax(i), eb = B.ax(j);
  float3 r = pa - pb;
  float bb = dot(ea, eb), c = dot(ea, r), f = dot(eb, r);
  float den = 1.f - bb * bb;
  float s = den > 1e-12f ? (bb * f - c) / den : 0.f;
  s = fminf(fmaxf(s, -A.hk(i)), A.hk(i));
  float t = fminf(fmaxf(f + s * bb, -B.hk(j)), B.hk(j));
  C.p[0] = 0.5f * ((pa + s * ea) + (pb + t * eb)) + A.c;
  C.depth[0] = delta;
  C.dmax = delta;
  C.np = 1;
  C.ref_face = 16 + i;
  C.inc_face = 16 + j;
}

// SAT over the 15 axes; on contact (min delta > -margin) builds the manifold.
__device__ bool box_box(const Box& A, const Box& B, float margin, Contact& C) {
  float3 d = B.c - A.c;
  float delta[15];
  bool valid[15];
  float dmin = FLT_MAX;
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    bool ok;
    float3 u = sat_axis(A, B, k, ok);
    valid[k] = ok;
    delta[k] = ok ? A.radius(u) + B.radius(u) - fabsf(dot(d, u)) : 0.f;
    if (ok) dmin = fminf(dmin, delta[k]);
  }
  if (!(dmin > -margin)) return false;
  int bf = 0;
#pragma unroll
  for (int k = 1; k < 6; ++k) if (delta[k] < delta[bf] - kTieAbs) bf = k;
  int be = -1;
  float dbe = 0.f;
#pragma unroll
  for (int k = 6; k < 15; ++k)
    if (valid[k] && (be < 0 || delta[k] < dbe - kTieAbs)) { be = k; dbe = delta[k]; }
  float dbf = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) if (k == bf) dbf = delta[k];
  int axis = (be >= 0 && dbe < dbf - (kEdgeRel * fabsf(dbf) + kTieAbs)) ? be : bf;
  bool ok;
  float3 n = sat_axis(A, B, axis, ok);
  if (dot(n, d) < 0.f) n = -n;
  C.axis = axis;
  C.n = n;
  C.delta = axis == be ? dbe : dbf;
  if (axis < 6) face_contact(A, B, axis, n, margin, C);
  else edge_contact(A, B, axis, n, C.delta, C);
  return C.np > 0;
}

// Ground plane z = 0 as body a: corners below the margin, n = +z.
__device__ bool ground_contact(const Box& B, float margin, Contact& C) {
  float3 P[8];
  float D[8];
  int m = 0;
  for (int c = 0; c < 8; ++c) {
    float s0 = (c & 1) ? 1.f : -1.f, s1 = (c & 2) ? 1.f : -1.f, s2 = (c & 4) ? 1.f : -1.f;
    float3 p = B.c + (s0 * B.h.x) * B.a0 + (s1 * B.h.y) * B.a1 + (s2 * B.h.z) * B.a2;
    if (p.z < margin) { D[m] = -p.z; P[m] = f3(p.x, p.y, p.z + 0.5f * D[m]); ++m; }
  }
  if (m == 0) return false;
  C.n = f3(0.f, 0.f, 1.f);
  C.axis = 15; C.ref_face = 0; C.inc_face = 0;
  keep4(m, P, D, C.n, C);
  C.delta = C.dmax;
  return true;
}

__device__ __forceinline__ void tangent_basis(float3 n, float3& t1, float3& t2) {
  float3 e = fabsf(n.x) > 0.9f ? f3(0.f, 1.f, 0.f) : f3(1.f, 0.f, 0.f);
  float3 t = e - dot(e, n) * n;
  t1 = rsqrtf(dot(t, t)) * t;
  t2 = cross(n, t1);
}

// ------------------------------------------------------------ warp helpers
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// ------------------------------------------------------------ episode view
struct Ep {
  int e, b0, nb, Pc, lane;
  int64_t poff;
  Sm s;
};

struct BufView {
  uint32_t *key, *feat, *slot;
  float *pt, *pf, *x;
  // colour-sorted solver arrays: shared memory when the step's pairs fit,
  // else this buffer's global copy; field f of slot s at [f * stride + s]
  uint32_t* ab;
  int32_t* np;
  float *sf, *sp;
  int stride;
};

__device__ __forceinline__ BufView buf_view(const Dev& D, int which, const Ep& E) {
  const ContactBuf& b = D.buf[which];
  BufView v;
  v.key = b.nat_key + E.poff;
  v.feat = b.nat_feat + E.poff;
  v.slot = b.nat_slot + E.poff;
  v.pt = b.nat_pt + E.poff * kMaxPts * kNatPtFloats;
  v.pf = b.nat_pf + E.poff * kNatPairFloats;
  v.x = b.nat_x + E.poff * kMaxPts * kFeatures;
  v.ab = b.srt_ab + E.poff;
  v.np = b.srt_np + E.poff;
  v.sf = b.srt_f + E.poff * kPairStride;
  v.sp = b.srt_pt + E.poff * kPtStride;
  v.stride = E.Pc;
  return v;
}

__device__ __forceinline__ void use_smem_solver(BufView& v, const Sm& s) {
  v.ab = s.ab; v.np = s.np; v.sf = s.sf; v.sp = s.sp; v.stride = s.ps;
}

// ---------------------------------------------------------- PGS pair kernels
// Everything a pair pass touches is loaded once into registers: the two
// bodies' velocities, inverse masses and world inverse inertia (symmetric, 6
// floats), the pair's frame and friction coefficient, and its points' lever
// arms, inverse effective masses, biases and impulses.
struct Sym3 { float xx, yy, zz, xy, xz, yz; };
__device__ __forceinline__ float3 mul(const Sym3& I, float3 u) {
  return f3(I.xx * u.x + I.xy * u.y + I.xz * u.z, I.xy * u.x + I.yy * u.y + I.yz * u.z,
            I.xz * u.x + I.yz * u.y + I.zz * u.z);
}
__device__ __forceinline__ Sym3 ld_iw(const Sm& s, int i) {
  Sym3 I;
  I.xx = s.at(FI, i); I.yy = s.at(FI + 1, i); I.zz = s.at(FI + 2, i);
  I.xy = s.at(FI + 3, i); I.xz = s.at(FI + 4, i); I.yz = s.at(FI + 5, i);
  return I;
}

struct PairRegs {
  int a, b, np;
  bool da, db;
  float3 va, wa, vb, wb, xa, xb, n, t1, t2;
  float ima, imb, mu;
  Sym3 Ia, Ib;
};

// The dynamic shared memory of the episode kernel.  Solver passes address it
// through this symbol so that their loads and stores are shared-memory
// accesses whatever the inlining.
extern __shared__ __align__(16) unsigned char jb_smem[];

// Where an episode's solver data lives: byte offsets into jb_smem for the body
// records (kBodyStride floats each) and, when the step's pairs fit, for the colour-sorted
// pair/point records (kPairStride, kPtStride); otherwise global pointers to them.
struct SolverRef {
  uint32_t oF, oflags, oab, onp, osf, osp;
  const uint32_t* gab;
  const int32_t* gnp;
  const float* gsf;
  float* gsp;
  int nbs, S;
  bool shared;
};

__device__ __forceinline__ SolverRef solver_ref(const Sm& s, const BufView& B) {
  SolverRef r;
  auto off = [](const void* p) { return (uint32_t)(reinterpret_cast<const unsigned char*>(p) - jb_smem); };
  r.oF = off(s.F); r.oflags = off(s.flags);
  r.shared = B.ab == s.ab;
  r.oab = off(s.ab); r.onp = off(s.np); r.osf = off(s.sf); r.osp = off(s.sp);
  r.gab = B.ab; r.gnp = B.np; r.gsf = B.sf; r.gsp = B.sp;
  r.nbs = s.nbs; r.S = B.stride;
  return r;
}

// Resolved pointers inside a solver function (shared or global sorted arrays).
template <bool kShared>
struct SolverView {
  float* __restrict__ F;
  const int* __restrict__ flags;
  const uint32_t* __restrict__ ab;
  const int32_t* __restrict__ np;
  const float* __restrict__ sf;
  float* __restrict__ sp;
  int nbs, S;
  __device__ __forceinline__ explicit SolverView(const SolverRef& r) {
    F = reinterpret_cast<float*>(jb_smem + r.oF);
    flags = reinterpret_cast<const int*>(jb_smem + r.oflags);
    if constexpr (kShared) {
      ab = reinterpret_cast<const uint32_t*>(jb_smem + r.oab);
      np = reinterpret_cast<const int32_t*>(jb_smem + r.onp);
      sf = reinterpret_cast<const float*>(jb_smem + r.osf);
      sp = reinterpret_cast<float*>(jb_smem + r.osp);
    } else {
      ab = r.gab; np = r.gnp; sf = r.gsf; sp = r.gsp;
    }
    nbs = r.nbs; S = r.S;
  }
};

#define VF(f, i) V.F[(i) * kBodyStride + (f)]
#define VSP(f, k) V.sp[sl * kPtStride + (k) * kSrtPtFloats + (f)]
#define VSF(f) V.sf[sl * kPairStride + (f)]

template <bool kS>
__device__ __forceinline__ float3 vld3(const SolverView<kS>& V, int f, int i) {
  return f3(VF(f, i), VF(f + 1, i), VF(f + 2, i));
}
template <bool kS>
__device__ __forceinline__ void vst3(const SolverView<kS>& V, int f, int i, float3 x) {
  VF(f, i) = x.x; VF(f + 1, i) = x.y; VF(f + 2, i) = x.z;
}

template <bool kS>
__device__ __forceinline__ void load_pair(const SolverView<kS>& V, int sl, PairRegs& R) {
  uint32_t ab = V.ab[sl];
  R.np = V.np[sl];
  R.a = ab & 0xffff; R.b = ab >> 16;
  R.n = f3(VSF(0), VSF(1), VSF(2));
  R.t1 = f3(VSF(3), VSF(4), VSF(5));
  R.t2 = cross(R.n, R.t1);
  R.mu = VSF(6);
  R.va = vld3(V, FV, R.a); R.wa = vld3(V, FW, R.a);
  R.vb = vld3(V, FV, R.b); R.wb = vld3(V, FW, R.b);
  R.xa = vld3(V, FX, R.a); R.xb = vld3(V, FX, R.b);
  R.ima = VF(FM, R.a); R.imb = VF(FM, R.b);
  R.Ia.xx = VF(FI, R.a); R.Ia.yy = VF(FI + 1, R.a); R.Ia.zz = VF(FI + 2, R.a);
  R.Ia.xy = VF(FI + 3, R.a); R.Ia.xz = VF(FI + 4, R.a); R.Ia.yz = VF(FI + 5, R.a);
  R.Ib.xx = VF(FI, R.b); R.Ib.yy = VF(FI + 1, R.b); R.Ib.zz = VF(FI + 2, R.b);
  R.Ib.xy = VF(FI + 3, R.b); R.Ib.xz = VF(FI + 4, R.b); R.Ib.yz = VF(FI + 5, R.b);
  R.da = !(V.flags[R.a] & kStatic);
  R.db = !(V.flags[R.b] & kStatic);
}

// Velocity of B relative to A at the point (lever arms rA, rB).
__device__ __forceinline__ float3 point_rel_vel(const PairRegs& R, float3 rA, float3 rB) {
  return (R.vb + cross(R.wb, rB)) - (R.va + cross(R.wa, rA));
}

// Applies the impulse P at the point: A gets -P, B gets +P (linear and angular).
__device__ __forceinline__ void apply_point(PairRegs& R, float3 rA, float3 rB, float3 P) {
  R.va = R.va - R.ima * P;
  R.vb = R.vb + R.imb * P;
  R.wa = R.wa - mul(R.Ia, cross(rA, P));
  R.wb = R.wb + mul(R.Ib, cross(rB, P));
}

// The two tangent rows of a point after its normal row.  Box (Eq.
// coulomb_pgs): t1 then t2, each clipped to [-lim, lim], t2 seeing t1's
// change through W_12.  Cone: both rows from the same state with the common
// step ik_t = min(ik1, ik2) (k_t = max(k_t1, k_t2)), projected together onto
// the disc of radius lim.
template <bool kCone>
__device__ __forceinline__ void tangent_rows(float v1, float v2, float l1, float l2, float ik1, float ik2, float w12,
                                             float lim, float om, float& nl1, float& nl2) {
  if constexpr (kCone) {
    const float ikt = om * fminf(ik1, ik2);
    const float a1 = l1 - v1 * ikt, a2 = l2 - v2 * ikt;
    const float m2 = a1 * a1 + a2 * a2;
    const float sc = m2 > lim * lim ? lim * rsqrtf(m2) : 1.f;
    nl1 = a1 * sc;
    nl2 = a2 * sc;
  } else {
    nl1 = fminf(fmaxf(l1 - v1 * (om * ik1), -lim), lim);
    v2 += w12 * (nl1 - l1);
    nl2 = fminf(fmaxf(l2 - v2 * (om * ik2), -lim), lim);
  }
}

// mode 0: apply warm-start impulses; mode 1: one Gauss-Seidel pass over the
// pair's points, rows n, t1, t2 in order (Eq. lambda_n with the listing's
// (1+e) factor, Eq. coulomb_pgs box clip with the just-updated normal
// impulse); mode 2: position correction (Eq. baumgarte, translation only).
//
// Within a point the three rows act at the same lever arms, so the change of
// the point's relative velocity after an impulse change dl along d_s is
// W d_s dl, with W the 3x3 inverse effective mass in the contact frame
// (diagonal: Eq. keff).  The rows therefore run on the three scalar
// velocities and the bodies take the point's summed impulse once: the same
// Gauss-Seidel iterate as updating the bodies after every row.
//
// Mode 1 relaxes every row by om (projected SOR): the caller folds om into
// e1 for the normal row; om = 1 is the paper's plain PGS, bit for bit.
template <int mode, bool kS, bool kCone = false>
__device__ __forceinline__ void pair_pass(const SolverView<kS>& V, int sl, float e1, float om, float beta,
                                          float slop) {
  if constexpr (mode == 2) {
    uint32_t ab = V.ab[sl];
    int a = ab & 0xffff, b = ab >> 16;
    float3 n = f3(VSF(0), VSF(1), VSF(2));
    float pen = VSF(7) - slop;
    float ima = VF(FM, a), imb = VF(FM, b);
    float wsum = ima + imb;
    if (pen > 0.f && wsum > 0.f) {
      float c = beta * pen / wsum;
      if (!(V.flags[a] & kStatic)) vst3(V, FX, a, vld3(V, FX, a) - (c * ima) * n);
      if (!(V.flags[b] & kStatic)) vst3(V, FX, b, vld3(V, FX, b) + (c * imb) * n);
    }
    return;
  }
  PairRegs R;
  load_pair(V, sl, R);
#pragma unroll
  for (int k = 0; k < kMaxPts; ++k) {
    if (k >= R.np) break;
    const float3 p = f3(VSP(0, k), VSP(1, k), VSP(2, k));
    const float3 rA = p - R.xa, rB = p - R.xb;
    float l0 = VSP(10, k), l1 = VSP(11, k), l2 = VSP(12, k);
    if constexpr (mode == 0) {
      apply_point(R, rA, rB, l0 * R.n + l1 * R.t1 + l2 * R.t2);
    } else {
      const float ik0 = VSP(3, k), ik1 = VSP(4, k), ik2 = VSP(5, k);
      const float w01 = VSP(6, k), w02 = VSP(7, k), w12 = VSP(8, k);
      const float bias = VSP(9, k);
      const float3 u = point_rel_vel(R, rA, rB);
      float vn = dot(u, R.n), v1 = dot(u, R.t1), v2 = dot(u, R.t2);
      float nl0 = fmaxf(0.f, l0 - e1 * (vn + bias) * ik0);
      float d0 = nl0 - l0;
      v1 += w01 * d0;
      v2 += w02 * d0;
      float lim = R.mu * nl0;
      float nl1, nl2;
      tangent_rows<kCone>(v1, v2, l1, l2, ik1, ik2, w12, lim, om, nl1, nl2);
      float d1 = nl1 - l1;
      float d2 = nl2 - l2;
      apply_point(R, rA, rB, d0 * R.n + d1 * R.t1 + d2 * R.t2);
      VSP(10, k) = nl0; VSP(11, k) = nl1; VSP(12, k) = nl2;
    }
  }
  if (R.da) { vst3(V, FV, R.a, R.va); vst3(V, FW, R.a, R.wa); }
  if (R.db) { vst3(V, FV, R.b, R.vb); vst3(V, FW, R.b, R.wb); }
}

// Mode 1 of pair_pass in packed FP32 (FFMA2: two lanes of arithmetic per
// instruction).  Body A's and body B's copies of each quantity share a
// float2 (A in .x, B in .y), with A's signs folded in (inverse mass and
// inverse inertia negated), so that the lever arms, the bodies' point
// velocities and the impulse application run once for both bodies.  The
// rows are scalar and identical to pair_pass; the iterate is the same up to
// rounding order.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

template <bool kS, bool kCone>
__device__ __forceinline__ void pair_sweep_packed(const SolverView<kS>& V, int sl, float e1, float om) {
  const uint32_t ab = V.ab[sl];
  const int a = ab & 0xffff, b = ab >> 16;
  const float3 n = f3(VSF(0), VSF(1), VSF(2));
  const float3 t1 = f3(VSF(3), VSF(4), VSF(5));
  const float3 t2 = cross(n, t1);
  const float mu = VSF(6);
  float2 vx = make_float2(VF(FV, a), VF(FV, b)), vy = make_float2(VF(FV + 1, a), VF(FV + 1, b)),
         vz = make_float2(VF(FV + 2, a), VF(FV + 2, b));
  float2 wx = make_float2(VF(FW, a), VF(FW, b)), wy = make_float2(VF(FW + 1, a), VF(FW + 1, b)),
         wz = make_float2(VF(FW + 2, a), VF(FW + 2, b));
  const float2 xx = make_float2(VF(FX, a), VF(FX, b)), xy = make_float2(VF(FX + 1, a), VF(FX + 1, b)),
               xz = make_float2(VF(FX + 2, a), VF(FX + 2, b));
  const float2 im = make_float2(-VF(FM, a), VF(FM, b));
  const float2 Ixx = make_float2(-VF(FI, a), VF(FI, b)), Iyy = make_float2(-VF(FI + 1, a), VF(FI + 1, b)),
               Izz = make_float2(-VF(FI + 2, a), VF(FI + 2, b)), Ixy = make_float2(-VF(FI + 3, a), VF(FI + 3, b)),
               Ixz = make_float2(-VF(FI + 4, a), VF(FI + 4, b)), Iyz = make_float2(-VF(FI + 5, a), VF(FI + 5, b));
  const bool da = !(V.flags[a] & kStatic), db = !(V.flags[b] & kStatic);
  const float2 nt_x = make_float2(n.x, t1.x), nt_y = make_float2(n.y, t1.y), nt_z = make_float2(n.z, t1.z);
  // all kMaxPts point records, unused ones zero (their impulse change is 0):
  // one branch-free block that the compiler can schedule across points
#pragma unroll
  for (int k = 0; k < kMaxPts; ++k) {
    const float px = VSP(0, k), py = VSP(1, k), pz = VSP(2, k);
    // lever arms r = p - x and their negatives, both bodies at once
    const float2 rx = __fadd2_rn(bc2(px), make_float2(-xx.x, -xx.y));
    const float2 ry = __fadd2_rn(bc2(py), make_float2(-xy.x, -xy.y));
    const float2 rz = __fadd2_rn(bc2(pz), make_float2(-xz.x, -xz.y));
    const float2 nrx = __fadd2_rn(xx, bc2(-px)), nry = __fadd2_rn(xy, bc2(-py)), nrz = __fadd2_rn(xz, bc2(-pz));
    // each body's velocity at the point, v + w x r
    float2 sx = __ffma2_rn(wy, rz, vx), sy = __ffma2_rn(wz, rx, vy), sz = __ffma2_rn(wx, ry, vz);
    sx = __ffma2_rn(wz, nry, sx);
    sy = __ffma2_rn(wx, nrz, sy);
    sz = __ffma2_rn(wy, nrx, sz);
    const float ux = sx.y - sx.x, uy = sy.y - sy.x, uz = sz.y - sz.x;
    // (vn, v1) together, v2 alone
    float2 q = __fmul2_rn(bc2(ux), nt_x);
    q = __ffma2_rn(bc2(uy), nt_y, q);
    q = __ffma2_rn(bc2(uz), nt_z, q);
    float vn = q.x, v1 = q.y;
    float v2 = ux * t2.x + uy * t2.y + uz * t2.z;
    const float ik0 = VSP(3, k), ik1 = VSP(4, k), ik2 = VSP(5, k);
    const float w01 = VSP(6, k), w02 = VSP(7, k), w12 = VSP(8, k);
    const float bias = VSP(9, k);
    const float l0 = VSP(10, k), l1 = VSP(11, k), l2 = VSP(12, k);
    float nl0 = fmaxf(0.f, l0 - e1 * (vn + bias) * ik0);
    float d0 = nl0 - l0;
    v1 += w01 * d0;
    v2 += w02 * d0;
    float lim = mu * nl0;
    float nl1, nl2;
    tangent_rows<kCone>(v1, v2, l1, l2, ik1, ik2, w12, lim, om, nl1, nl2);
    float d1 = nl1 - l1;
    float d2 = nl2 - l2;
    const float Px = d0 * n.x + d1 * t1.x + d2 * t2.x;
    const float Py = d0 * n.y + d1 * t1.y + d2 * t2.y;
    const float Pz = d0 * n.z + d1 * t1.z + d2 * t2.z;
    const float2 PX = bc2(Px), PY = bc2(Py), PZ = bc2(Pz);
    // v += (-ima, imb) P;  w += (-Ia, Ib) (r x P)
    vx = __ffma2_rn(im, PX, vx);
    vy = __ffma2_rn(im, PY, vy);
    vz = __ffma2_rn(im, PZ, vz);
    const float2 cx = __ffma2_rn(ry, PZ, __fmul2_rn(nrz, PY));
    const float2 cy = __ffma2_rn(rz, PX, __fmul2_rn(nrx, PZ));
    const float2 cz = __ffma2_rn(rx, PY, __fmul2_rn(nry, PX));
    wx = __ffma2_rn(Ixx, cx, __ffma2_rn(Ixy, cy, __ffma2_rn(Ixz, cz, wx)));
    wy = __ffma2_rn(Ixy, cx, __ffma2_rn(Iyy, cy, __ffma2_rn(Iyz, cz, wy)));
    wz = __ffma2_rn(Ixz, cx, __ffma2_rn(Iyz, cy, __ffma2_rn(Izz, cz, wz)));
    VSP(10, k) = nl0; VSP(11, k) = nl1; VSP(12, k) = nl2;
  }
  if (da) { VF(FV, a) = vx.x; VF(FV + 1, a) = vy.x; VF(FV + 2, a) = vz.x;
            VF(FW, a) = wx.x; VF(FW + 1, a) = wy.x; VF(FW + 2, a) = wz.x; }
  if (db) { VF(FV, b) = vx.y; VF(FV + 1, b) = vy.y; VF(FV + 2, b) = vz.y;
            VF(FW, b) = wx.y; VF(FW + 1, b) = wy.y; VF(FW + 2, b) = wz.y; }
}

// Residual of one pair at the current state (no update): max over rows of
// k |proj(lambda - (v + b) / k) - lambda|, k the inverse effective mass.  It
// only feeds the stopping test and the statistics, so the division by the
// stored 1/k is the fast approximate one (a few ulp).
template <bool kS>
__device__ __forceinline__ float pair_residual(const SolverView<kS>& V, int sl, bool cone) {
  PairRegs R;
  load_pair(V, sl, R);
  float r = 0.f;
#pragma unroll
  for (int k = 0; k < kMaxPts; ++k) {
    if (k >= R.np) break;
    const float3 p = f3(VSP(0, k), VSP(1, k), VSP(2, k));
    const float3 u = point_rel_vel(R, p - R.xa, p - R.xb);
    const float ik0 = VSP(3, k), ik1 = VSP(4, k), ik2 = VSP(5, k), bias = VSP(9, k);
    const float l0 = VSP(10, k), l1 = VSP(11, k), l2 = VSP(12, k);
    float lim = R.mu * l0;
    float p0 = fmaxf(0.f, l0 - (dot(u, R.n) + bias) * ik0);
    float p1, p2, m12;
    if (cone) {
      // the tangent pair's disc projection with the common step (see tangent_rows)
      const float ikt = fminf(ik1, ik2);
      const float a1 = l1 - dot(u, R.t1) * ikt, a2 = l2 - dot(u, R.t2) * ikt;
      const float m2 = a1 * a1 + a2 * a2;
      const float sc = m2 > lim * lim ? lim * rsqrtf(m2) : 1.f;
      p1 = a1 * sc;
      p2 = a2 * sc;
      m12 = __fdividef(fmaxf(fabsf(p1 - l1), fabsf(p2 - l2)), ikt);
    } else {
      p1 = fminf(fmaxf(l1 - dot(u, R.t1) * ik1, -lim), lim);
      p2 = fminf(fmaxf(l2 - dot(u, R.t2) * ik2, -lim), lim);
      m12 = fmaxf(__fdividef(fabsf(p1 - l1), ik1), __fdividef(fabsf(p2 - l2), ik2));
    }
    float m = fmaxf(__fdividef(fabsf(p0 - l0), ik0), m12);
    if (!(m <= r)) r = m;   // keeps NaN
  }
  return r;
}

// Residual of the whole episode (warp max; NaN propagates).
template <bool kS>
__device__ __noinline__ float episode_residual_t(const SolverRef r, int npairs, int lane, bool cone) {
  const SolverView<kS> V(r);
  float res = 0.f;
  for (int sl = lane; sl < npairs; sl += 32) {
    float m = pair_residual(V, sl, cone);
    if (!(m <= res)) res = m;
  }
  bool nan = __any_sync(FULL, !(res == res));
  return nan ? __int_as_float(0x7fc00000) : warp_max(res);
}

// Runs `mode` over every colour, in order or (rev) in reverse order; lanes
// take the slots of a colour.  `off` holds the colour offsets (ncol + 1
// entries).  Pairs of one colour share no body, so their order is free.
template <int mode, bool kS, bool kCone>
__device__ __noinline__ void colour_passes_t(const SolverRef r, const int* __restrict__ off, int ncol, int lane,
                                             float e1, float om, bool rev, float beta, float slop) {
  const SolverView<kS> V(r);
  for (int i = 0; i < ncol; ++i) {
    const int c = rev ? ncol - 1 - i : i;
    int s0 = off[c], s1 = off[c + 1];
    if (c == kSerial) {
      if (lane == 0) {
        if (rev) for (int sl = s1 - 1; sl >= s0; --sl) pair_pass<mode, kS, kCone>(V, sl, e1, om, beta, slop);
        else for (int sl = s0; sl < s1; ++sl) pair_pass<mode, kS, kCone>(V, sl, e1, om, beta, slop);
      }
    } else {
      for (int sl = s0 + lane; sl < s1; sl += 32) {
        if constexpr (mode == 1) pair_sweep_packed<kS, kCone>(V, sl, e1, om);
        else pair_pass<mode, kS, kCone>(V, sl, e1, om, beta, slop);
      }
    }
    __syncwarp();
  }
}

// Only the sweep (mode 1) depends on the friction model; the warm start and
// the position correction run one instantiation.
template <int mode>
__device__ __forceinline__ void colour_passes(const SolverRef& r, const int* off, int ncol, int lane, float e1,
                                              float om, bool rev, float beta, float slop, bool cone = false) {
  if (mode == 1 && cone) {
    if (r.shared) colour_passes_t<mode, true, true>(r, off, ncol, lane, e1, om, rev, beta, slop);
    else colour_passes_t<mode, false, true>(r, off, ncol, lane, e1, om, rev, beta, slop);
  } else {
    if (r.shared) colour_passes_t<mode, true, false>(r, off, ncol, lane, e1, om, rev, beta, slop);
    else colour_passes_t<mode, false, false>(r, off, ncol, lane, e1, om, rev, beta, slop);
  }
}

__device__ __forceinline__ float episode_residual(const SolverRef& r, int npairs, int lane, bool cone) {
  return r.shared ? episode_residual_t<true>(r, npairs, lane, cone) : episode_residual_t<false>(r, npairs, lane, cone);
}

// ------------------------------------------------ nonsmooth CG acceleration
// One conjugate-gradient step per block of m sweeps (Silcowitz, Niebe and
// Erleben's nonsmooth nonlinear conjugate gradient with a block of sweeps as
// the map G): r = G(lambda) - lambda over the block, beta = |r_k|^2 /
// |r_(k-1)|^2 (0 on the first block and on restart, beta > 1), lambda <-
// proj(G(lambda) + beta d), d <- r_k + beta d.  The state lives in the
// global acc array, kAccFloats per colour-sorted slot ([4][3] impulses at
// the block start, then [4][3] direction); unused point records are zero and
// stay zero.  A fixed point of the sweep is one of this iteration.
template <bool kS>
__device__ __noinline__ void accel_begin_t(const SolverRef r, float* __restrict__ acc, int npairs, int lane) {
  const SolverView<kS> V(r);
  for (int sl = lane; sl < npairs; sl += 32) {
    float4* a4 = reinterpret_cast<float4*>(acc + (size_t)sl * kAccFloats);
    float l[12];
#pragma unroll
    for (int k = 0; k < kMaxPts; ++k) { l[3 * k] = VSP(10, k); l[3 * k + 1] = VSP(11, k); l[3 * k + 2] = VSP(12, k); }
    a4[0] = make_float4(l[0], l[1], l[2], l[3]);
    a4[1] = make_float4(l[4], l[5], l[6], l[7]);
    a4[2] = make_float4(l[8], l[9], l[10], l[11]);
    a4[3] = make_float4(0.f, 0.f, 0.f, 0.f);
    a4[4] = a4[3];
    a4[5] = a4[3];
  }
}

// |lambda - lambda_start|^2 over the episode (warp sum).
template <bool kS>
__device__ __noinline__ float accel_change2_t(const SolverRef r, const float* __restrict__ acc, int npairs, int lane) {
  const SolverView<kS> V(r);
  float s2 = 0.f;
  for (int sl = lane; sl < npairs; sl += 32) {
    const float4* a4 = reinterpret_cast<const float4*>(acc + (size_t)sl * kAccFloats);
    const float4 q0 = a4[0], q1 = a4[1], q2 = a4[2];
    const float ls[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
#pragma unroll
    for (int k = 0; k < kMaxPts; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float d = VSP(10 + c, k) - ls[3 * k + c];
        s2 = fmaf(d, d, s2);
      }
  }
  return warp_sum(s2);
}

// The step on one pair: new impulses, direction and block start, and the
// impulse change applied to both bodies.
template <bool kS, bool kCone>
__device__ __forceinline__ void accel_pair(const SolverView<kS>& V, float* __restrict__ acc, int sl, float beta) {
  PairRegs R;
  load_pair(V, sl, R);
  float4* a4 = reinterpret_cast<float4*>(acc + (size_t)sl * kAccFloats);
  float ls[12], dr[12];
  {
    float4 t[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = a4[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ls[4 * i] = t[i].x; ls[4 * i + 1] = t[i].y; ls[4 * i + 2] = t[i].z; ls[4 * i + 3] = t[i].w;
      dr[4 * i] = t[3 + i].x; dr[4 * i + 1] = t[3 + i].y; dr[4 * i + 2] = t[3 + i].z; dr[4 * i + 3] = t[3 + i].w;
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxPts; ++k) {
    const float l0 = VSP(10, k), l1 = VSP(11, k), l2 = VSP(12, k);
    float n0 = fmaxf(0.f, fmaf(beta, dr[3 * k], l0));
    float n1 = fmaf(beta, dr[3 * k + 1], l1), n2 = fmaf(beta, dr[3 * k + 2], l2);
    const float lim = R.mu * n0;
    if constexpr (kCone) {
      const float m2 = n1 * n1 + n2 * n2;
      const float sc = m2 > lim * lim ? lim * rsqrtf(m2) : 1.f;
      n1 *= sc;
      n2 *= sc;
    } else {
      n1 = fminf(fmaxf(n1, -lim), lim);
      n2 = fminf(fmaxf(n2, -lim), lim);
    }
    dr[3 * k] = (l0 - ls[3 * k]) + beta * dr[3 * k];
    dr[3 * k + 1] = (l1 - ls[3 * k + 1]) + beta * dr[3 * k + 1];
    dr[3 * k + 2] = (l2 - ls[3 * k + 2]) + beta * dr[3 * k + 2];
    ls[3 * k] = n0; ls[3 * k + 1] = n1; ls[3 * k + 2] = n2;
    VSP(10, k) = n0; VSP(11, k) = n1; VSP(12, k) = n2;
    const float d0 = n0 - l0, d1 = n1 - l1, d2 = n2 - l2;
    const float3 p = f3(VSP(0, k), VSP(1, k), VSP(2, k));
    apply_point(R, p - R.xa, p - R.xb, d0 * R.n + d1 * R.t1 + d2 * R.t2);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    a4[i] = make_float4(ls[4 * i], ls[4 * i + 1], ls[4 * i + 2], ls[4 * i + 3]);
    a4[3 + i] = make_float4(dr[4 * i], dr[4 * i + 1], dr[4 * i + 2], dr[4 * i + 3]);
  }
  if (R.da) { vst3(V, FV, R.a, R.va); vst3(V, FW, R.a, R.wa); }
  if (R.db) { vst3(V, FV, R.b, R.vb); vst3(V, FW, R.b, R.wb); }
}

// The step over every colour in order (pairs of one colour share no dynamic
// body; the serial colour runs on one lane).
template <bool kS, bool kCone>
__device__ __noinline__ void accel_step_t(const SolverRef r, float* __restrict__ acc, const int* __restrict__ off,
                                          int ncol, int lane, float beta) {
  const SolverView<kS> V(r);
  for (int c = 0; c < ncol; ++c) {
    const int s0 = off[c], s1 = off[c + 1];
    if (c == kSerial) {
      if (lane == 0)
        for (int sl = s0; sl < s1; ++sl) accel_pair<kS, kCone>(V, acc, sl, beta);
    } else {
      for (int sl = s0 + lane; sl < s1; sl += 32) accel_pair<kS, kCone>(V, acc, sl, beta);
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void accel_begin(const SolverRef& r, float* acc, int npairs, int lane) {
  if (r.shared) accel_begin_t<true>(r, acc, npairs, lane);
  else accel_begin_t<false>(r, acc, npairs, lane);
  __syncwarp();
}
__device__ __forceinline__ float accel_change2(const SolverRef& r, const float* acc, int npairs, int lane) {
  return r.shared ? accel_change2_t<true>(r, acc, npairs, lane) : accel_change2_t<false>(r, acc, npairs, lane);
}
__device__ __forceinline__ void accel_step(const SolverRef& r, float* acc, const int* off, int ncol, int lane, float beta,
                                           bool cone) {
  if (cone) {
    if (r.shared) accel_step_t<true, true>(r, acc, off, ncol, lane, beta);
    else accel_step_t<false, true>(r, acc, off, ncol, lane, beta);
  } else {
    if (r.shared) accel_step_t<true, false>(r, acc, off, ncol, lane, beta);
    else accel_step_t<false, false>(r, acc, off, ncol, lane, beta);
  }
}
#undef VSP
#undef VSF

#undef VF

// ----------------------------------------------------- learned warm start
// The warp collects the points to predict (ids p * 4 + k: every point in
// mode 3; in mode 2 the points of new pairs, on steps where at least half of
// the pairs are new) into the
// candidate array (free after the colouring), runs the network on tiles of 16
// rows on the tensor cores and writes the projected impulses (lambda_n >= 0,
// |lambda_t| <= mu lambda_n) as the points' starting impulses.
__device__ __noinline__ int mlp_warm_start(const Dev& D, const Ep& E, const BufView& Bc, int npairs, bool all_points,
                                           float imp_scale, int lane) {
  const bool cone = D.P.friction_cone != 0;
  const Sm& s = E.s;
  const MlpLayout L = mlp_layout();
  const float* P = reinterpret_cast<const float*>(D.mlp);
  const uint2* pk = reinterpret_cast<const uint2*>(D.mlp + L.pack_base);
  const int ccap = cand_capacity(E.nb);
  uint32_t* list = s.cand;
  float* stage = reinterpret_cast<float*>(s.cand + (ccap - 64));   // 16 rows x 4
  const int lcap = ccap - 64;
  const int g = lane >> 2, t = lane & 3;
  int cnt = 0, predicted = 0;
  if (!all_points) {
    // mode 2 predicts only on a step where at least half of the episode's
    // pairs are new (an episode's first step, a large rearrangement): there
    // the network's starts are reliably closer to the converged impulses
    // than zero; a few pairs forming beside many settled ones start at zero
    int nnew = 0;
    for (int p = lane; p < npairs; p += 32) {
      const int np = Bc.feat[p] >> 24;
      const float* pt = Bc.pt + (size_t)p * kMaxPts * kNatPtFloats;
      bool matched = false;
      for (int k = 0; k < np; ++k) matched |= pt[k * kNatPtFloats + 10] != 0.f;
      nnew += matched ? 0 : 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnew += __shfl_xor_sync(FULL, nnew, o);
    if (2 * nnew < npairs) return 0;
  }
  for (int p0 = 0; p0 < npairs; p0 += 32) {
    const int p = p0 + lane;
    int mine = 0;
    uint32_t ids[kMaxPts];
    if (p < npairs) {
      int np = Bc.feat[p] >> 24;
      const float* pt = Bc.pt + (size_t)p * kMaxPts * kNatPtFloats;
      // mode 2: the points of pairs none of whose points inherited an impulse
      // (new pairs); a point that appears in a pair that already carries
      // impulses starts at zero, as in plain PGS
      bool any_matched = false;
      for (int k = 0; k < np; ++k) any_matched |= pt[k * kNatPtFloats + 10] != 0.f;
      for (int k = 0; k < np; ++k)
        if (all_points || !any_matched) ids[mine++] = (uint32_t)(p * kMaxPts + k);
    }
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    for (int i = 0; i < mine; ++i) list[cnt + incl - mine + i] = ids[i];
    cnt += total;
    predicted += total;
    __syncwarp();
    const bool last = p0 + 32 >= npairs;
    if (!(last || cnt + 32 * kMaxPts > lcap)) continue;
    // run the network over list[0, cnt)
    for (int r0 = 0; r0 < cnt; r0 += 16) {
      const int ia = r0 + g, ib = r0 + g + 8;
      const float* xa = ia < cnt ? Bc.x + (size_t)list[ia] * kFeatures : nullptr;
      const float* xb = ib < cnt ? Bc.x + (size_t)list[ib] * kFeatures : nullptr;
      auto x = [&](const float* r, int c) { return (r && c < kFeatures) ? r[c] : 0.f; };
      uint32_t a[2][4];
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        int c = kk * 16 + 2 * t;
        a[kk][0] = pack_bf16x2(x(xa, c), x(xa, c + 1));
        a[kk][1] = pack_bf16x2(x(xb, c), x(xb, c + 1));
        a[kk][2] = pack_bf16x2(x(xa, c + 8), x(xa, c + 9));
        a[kk][3] = pack_bf16x2(x(xb, c + 8), x(xb, c + 9));
      }
      uint32_t h1[8][4], h2[8][4];
      dense_relu_128<2>(a, pk + L.p1, P + L.b1, lane, h1);
      dense_relu_128<8>(h1, pk + L.p2, P + L.b2, lane, h2);
      float y[4];
      dense_out(h2, pk + L.p3, P + L.b3, lane, y);
      if (t < 2) {
        stage[g * 4 + 2 * t] = y[0]; stage[g * 4 + 2 * t + 1] = y[1];
        stage[(g + 8) * 4 + 2 * t] = y[2]; stage[(g + 8) * 4 + 2 * t + 1] = y[3];
      }
      __syncwarp();
      if (lane < 16 && r0 + lane < cnt) {
        uint32_t id = list[r0 + lane];
        int p = id / kMaxPts, k = id % kMaxPts;
        int sl = Bc.slot[p] & 0xffff;
        float mu = Bc.sf[sl * kPairStride + 6];
        float ln = fmaxf(0.f, stage[lane * 4 + 0] * imp_scale);
        float lim = mu * ln;
        float* rec = Bc.sp + sl * kPtStride + k * kSrtPtFloats;
        rec[10] = ln;
        float t1v = stage[lane * 4 + 1] * imp_scale, t2v = stage[lane * 4 + 2] * imp_scale;
        if (cone) {
          const float m2 = t1v * t1v + t2v * t2v;
          const float sc = m2 > lim * lim ? lim * rsqrtf(m2) : 1.f;
          rec[11] = t1v * sc;
          rec[12] = t2v * sc;
        } else {
          rec[11] = fminf(fmaxf(t1v, -lim), lim);
          rec[12] = fminf(fmaxf(t2v, -lim), lim);
        }
      }
      __syncwarp();
    }
    cnt = 0;
    __syncwarp();
  }
  return predicted;
}

// ------------------------------------------------------------------ substep
struct StepOut {
  float res;
  int sweeps, predicted;
  int npairs, npoints, ncol;
  int status;
};

__device__ __forceinline__ void body_frame(const Sm& s, const Dev& D, int gi, int i) {
  float w = s.at(FQ, i), x = s.at(FQ + 1, i), y = s.at(FQ + 2, i), z = s.at(FQ + 3, i);
  float R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
                2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)};
#pragma unroll
  for (int k = 0; k < 9; ++k) s.at(FR + k, i) = R[k];
  float i0 = 0.f, i1 = 0.f, i2 = 0.f;
  if (gi >= 0 && !(s.flags[i] & kStatic)) { i0 = D.invI[gi]; i1 = D.invI[D.B + gi]; i2 = D.invI[2 * D.B + gi]; }
  // I_world^-1 = R diag(invI) R^T (Sec. 4.1.2)
  s.at(FI, i) = R[0] * R[0] * i0 + R[1] * R[1] * i1 + R[2] * R[2] * i2;
  s.at(FI + 1, i) = R[3] * R[3] * i0 + R[4] * R[4] * i1 + R[5] * R[5] * i2;
  s.at(FI + 2, i) = R[6] * R[6] * i0 + R[7] * R[7] * i1 + R[8] * R[8] * i2;
  s.at(FI + 3, i) = R[0] * R[3] * i0 + R[1] * R[4] * i1 + R[2] * R[5] * i2;
  s.at(FI + 4, i) = R[0] * R[6] * i0 + R[1] * R[7] * i1 + R[2] * R[8] * i2;
  s.at(FI + 5, i) = R[3] * R[6] * i0 + R[4] * R[7] * i1 + R[5] * R[8] * i2;
  float hx = s.at(FH, i), hy = s.at(FH + 1, i), hz = s.at(FH + 2, i);
  s.at(FE, i) = fabsf(R[0]) * hx + fabsf(R[1]) * hy + fabsf(R[2]) * hz;
  s.at(FE + 1, i) = fabsf(R[3]) * hx + fabsf(R[4]) * hy + fabsf(R[5]) * hz;
  s.at(FE + 2, i) = fabsf(R[6]) * hx + fabsf(R[7]) * hy + fabsf(R[8]) * hz;
}

__device__ StepOut substep(const Dev& D, const Ep& E, EpState& st, float h) {
  const Sm& s = E.s;
  const Params& Pm = D.P;
  const int lane = E.lane, nb = E.nb, Pc = E.Pc;
  const int G = nb;   // ground slot
  StepOut out;
  out.status = 0;

  // (1) external forces and gravity on the velocity (Sec. 4.2), frames
  for (int i = lane; i < nb; i += 32) {
    int gi = E.b0 + i;
    int fl = s.flags[i];
    if ((fl & kActive) && !(fl & kStatic)) {
      float im = s.at(FM, i);
      bool on = D.f_steps[gi] > 0;
      float fx = on ? D.f[gi] : 0.f, fy = on ? D.f[D.B + gi] : 0.f, fz = on ? D.f[2 * D.B + gi] : 0.f;
      s.at(FV, i) += h * (Pm.g[0] + fx * im);
      s.at(FV + 1, i) += h * (Pm.g[1] + fy * im);
      s.at(FV + 2, i) += h * (Pm.g[2] + fz * im);
    }
    body_frame(s, D, gi, i);
  }
  __syncwarp();

  // (2) broadphase: ground candidates, then pairs (i, j) i < j ascending
  int ncand = 0;
  const int ccap = cand_capacity(nb);
  for (int j0 = 0; j0 < nb; j0 += 32) {
    int j = j0 + lane;
    bool hit = false;
    if (j < nb) {
      int fl = s.flags[j];
      hit = (fl & kActive) && !(fl & kStatic) && (s.at(FX + 2, j) - s.at(FE + 2, j) <= Pm.aabb_eps);
    }
    unsigned bal = __ballot_sync(FULL, hit);
    int idx = ncand + __popc(bal & lanemask_lt(lane));
    if (hit && idx < ccap) s.cand[idx] = (uint32_t)j;   // a = -1 -> key ((a+1) << 16) | b
    ncand += __popc(bal);
  }
  for (int i = 0; i < nb; ++i) {
    int fi = s.flags[i];
    if (!(fi & kActive)) continue;
    float xi = s.at(FX, i), yi = s.at(FX + 1, i), zi = s.at(FX + 2, i);
    float ex = s.at(FE, i), ey = s.at(FE + 1, i), ez = s.at(FE + 2, i);
    for (int j0 = i + 1; j0 < nb; j0 += 32) {
      int j = j0 + lane;
      bool hit = false;
      if (j < nb) {
        int fj = s.flags[j];
        hit = (fj & kActive) && !((fi & kStatic) && (fj & kStatic)) &&
              fabsf(xi - s.at(FX, j)) <= ex + s.at(FE, j) + Pm.aabb_eps &&
              fabsf(yi - s.at(FX + 1, j)) <= ey + s.at(FE + 1, j) + Pm.aabb_eps &&
              fabsf(zi - s.at(FX + 2, j)) <= ez + s.at(FE + 2, j) + Pm.aabb_eps;
      }
      unsigned bal = __ballot_sync(FULL, hit);
      int idx = ncand + __popc(bal & lanemask_lt(lane));
      if (hit && idx < ccap) s.cand[idx] = ((uint32_t)(i + 1) << 16) | (uint32_t)j;
      ncand += __popc(bal);
    }
  }
  if (ncand > ccap) { out.status |= JB_EP_CONTACT_OVERFLOW; ncand = ccap; }
  __syncwarp();

  // (3) narrowphase + manifold, one candidate per lane, natural order kept
  const int cur = st.cur ^ 1;
  BufView Bc = buf_view(D, cur, E);
  BufView Bp = buf_view(D, st.cur, E);
  int npairs = 0, npoints = 0;
  for (int c0 = 0; c0 < ncand; c0 += 32) {
    int c = c0 + lane;
    bool hit = false;
    Contact C;
    uint32_t key = 0;
    if (c < ncand) {
      key = s.cand[c];
      int a = (int)(key >> 16) - 1, b = (int)(key & 0xffff);
      Box Bb = box_of(s, b);
      if (a < 0) hit = ground_contact(Bb, Pm.contact_margin, C);
      else { Box Ab = box_of(s, a); hit = box_box(Ab, Bb, Pm.contact_margin, C); }
    }
    unsigned bal = __ballot_sync(FULL, hit);
    int idx = npairs + __popc(bal & lanemask_lt(lane));
    if (idx >= Pc) hit = false;   // pair capacity: the rest is dropped and flagged
    if (__popc(bal) + npairs > Pc) out.status |= JB_EP_CONTACT_OVERFLOW;
    if (hit) {
      int a = (int)(key >> 16) - 1;
      Bc.key[idx] = key;
      Bc.feat[idx] = (uint32_t)C.axis | ((uint32_t)C.ref_face << 8) | ((uint32_t)C.inc_face << 16) | ((uint32_t)C.np << 24);
      int ia = a < 0 ? G : a;
      float3 xa = s.ld3(FX, ia);
      float3 c0v = s.axis(ia, 0), c1v = s.axis(ia, 1), c2v = s.axis(ia, 2);
      float* pt = Bc.pt + (size_t)idx * kMaxPts * kNatPtFloats;
      for (int k = 0; k < C.np; ++k) {
        float3 r = C.p[k] - xa;
        float* q = pt + k * kNatPtFloats;
        q[0] = C.p[k].x; q[1] = C.p[k].y; q[2] = C.p[k].z; q[3] = C.depth[k];
        q[4] = dot(c0v, r); q[5] = dot(c1v, r); q[6] = dot(c2v, r);   // R_A^T (p - x_A)
        q[7] = 0.f; q[8] = 0.f; q[9] = 0.f;                          // warm-start impulses
        q[10] = 0.f; q[11] = 0.f;
      }
      Bc.slot[idx] = 0xffffu << 16;   // no colour yet
      float* pf = Bc.pf + (size_t)idx * kNatPairFloats;
      pf[0] = C.n.x; pf[1] = C.n.y; pf[2] = C.n.z; pf[3] = C.dmax;
    }
    npairs = min(npairs + __popc(bal), Pc);
    int pts = hit ? C.np : 0;
    npoints += (int)warp_sum((float)pts);
  }
  __syncwarp();

  // (4) warm-start matching against the previous step
  const int nprev = st.npairs;
  const float mr2 = Pm.match_radius * Pm.match_radius;
  for (int p = lane; p < npairs; p += 32) {
    uint32_t key = Bc.key[p];
    int lo = 0, hi = nprev - 1, q = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      uint32_t km = Bp.key[mid];
      if (km == key) { q = mid; break; }
      if (km < key) lo = mid + 1; else hi = mid - 1;
    }
    if (q < 0 || Pm.warm_start == 0) continue;
    uint32_t fn = Bc.feat[p], fo = Bp.feat[q];
    if (((fn ^ fo) & 0x00ffff00u) != 0) continue;
    int npn = fn >> 24, npo = fo >> 24;
    float* ptn = Bc.pt + (size_t)p * kMaxPts * kNatPtFloats;
    const float* pto = Bp.pt + (size_t)q * kMaxPts * kNatPtFloats;
    for (int k = 0; k < npn; ++k) {
      float* a = ptn + k * kNatPtFloats;
      int best = -1;
      float bd = mr2;
      for (int j = 0; j < npo; ++j) {
        const float* o = pto + j * kNatPtFloats;
        float dx = o[4] - a[4], dy = o[5] - a[5], dz = o[6] - a[6];
        float d2 = dx * dx + dy * dy + dz * dz;
        if (d2 <= bd) { bd = d2; best = j; }
      }
      if (best >= 0) {   // the old point's final impulses of the previous step
        const float* o = pto + best * kNatPtFloats;
        a[7] = o[7]; a[8] = o[8]; a[9] = o[9];
        a[10] = 1.f;     // matched
      }
    }
  }
  __syncwarp();

  // (5) colouring, redone every step: greedy (lowest colour free at both
  // dynamic bodies) over the pairs in order of a key: colour_key 0 (lower
  // body a ascending, upper body b descending) or 1 (height of the pair's
  // first point in 1 mm bins ascending, natural index descending).  The
  // colours are swept in index order, so contacts low in the tower tend to be
  // solved first; on 18-level towers either order needs several times fewer
  // sweeps to reach a residual tolerance than colouring in natural order, at
  // the same colour count.  The candidate array (free after the narrowphase)
  // holds the order.
  uint32_t* ord = s.cand;
  {
    const int nchunk = (npairs + 31) / 32;
    for (int p0 = 0; p0 < npairs; p0 += 32) {
      int p = p0 + lane;
      // pair key ((a + 1) << 16) | b -> ((a + 1) << 16) | (0xffff - b); or the height bin
      const bool by_height = Pm.colour_key == 1;
      auto colour_key = [&](int q) {
        if (by_height) {
          const float z = Bc.pt[(size_t)q * kMaxPts * kNatPtFloats + 2];
          int bin = (int)floorf((z + 5e-4f) * 1000.f);
          bin = min(max(bin + 1, 0), 65535);
          return ((uint32_t)bin << 16) | (uint32_t)(0xffff - q);
        }
        const uint32_t k = Bc.key[q];
        return (k & 0xffff0000u) | (0xffffu - (k & 0xffffu));
      };
      uint32_t key = p < npairs ? colour_key(p) : 0xffffffffu;
      // rank among all pairs: keys are distinct
      int rank = 0;
      for (int c = 0; c < nchunk; ++c) {
        int q = c * 32 + lane;
        uint32_t kq = q < npairs ? colour_key(q) : 0xffffffffu;
        for (int j = 0; j < 32; ++j) rank += __shfl_sync(FULL, kq, j) < key;
      }
      if (p < npairs) ord[rank] = (uint32_t)p;
    }
  }
  for (int i = lane; i <= nb; i += 32) s.mask[i] = 0ull;
  __syncwarp();
  bool many = false;
  for (int t = 0; t < npairs; ++t) {
    int p = ord[t];
    uint32_t key = Bc.key[p];
    int a = (int)(key >> 16) - 1, b = (int)(key & 0xffff);
    bool sa = a < 0 || (s.flags[a] & kStatic), sb = (s.flags[b] & kStatic);
    unsigned long long m = (sa ? 0ull : s.mask[a]) | (sb ? 0ull : s.mask[b]);
    int c = __ffsll((long long)~m) - 1;
    if (c < 0 || c >= kSerial) { c = kSerial; many = true; }
    __syncwarp();
    if (lane == 0) {
      if (c < kSerial) {
        if (!sa) s.mask[a] |= 1ull << c;
        if (!sb) s.mask[b] |= 1ull << c;
      }
      Bc.slot[p] = (uint32_t)c << 16;
    }
    __syncwarp();
  }
  if (many) out.status |= JB_EP_TOO_MANY_COLOURS;
  __syncwarp();

  // (6) counting sort by colour (ascending natural index within a colour)
  for (int c = lane; c <= kMaxColours; c += 32) { s.cnt[c] = 0; s.run[c] = 0; }
  __syncwarp();
  for (int p = lane; p < npairs; p += 32) atomicAdd(&s.cnt[Bc.slot[p] >> 16], 1);
  __syncwarp();
  if (lane == 0) {
    int acc = 0;
    for (int c = 0; c < kMaxColours; ++c) { s.off[c] = acc; acc += s.cnt[c]; }
    s.off[kMaxColours] = acc;
  }
  __syncwarp();
  int ncol = 0;
  {
    int last = -1;
    for (int c = lane; c < kMaxColours; c += 32) if (s.cnt[c] > 0) last = c;
    ncol = (int)warp_max((float)last) + 1;
  }
  for (int p0 = 0; p0 < npairs; p0 += 32) {
    int p = p0 + lane;
    int col = p < npairs ? (int)(Bc.slot[p] >> 16) : -1 - lane;
    unsigned grp = __match_any_sync(FULL, col);
    int rank = __popc(grp & lanemask_lt(lane));
    int base = 0;
    if (p < npairs) base = s.off[col] + s.run[col];
    __syncwarp();
    if (p < npairs) {
      Bc.slot[p] = ((uint32_t)col << 16) | (uint32_t)(base + rank);
      if (rank == 0) s.run[col] += __popc(grp);
    }
    __syncwarp();
  }

  // (7) contact setup (Eq. keff) into the colour-sorted solver arrays:
  // shared memory when the pairs fit, else this buffer's global copy
  if (npairs <= s.ps) use_smem_solver(Bc, s);
  const float ih = 1.f / h;
  const bool want_features = (Pm.warm_start >= 2 && D.mlp) || D.rec != nullptr;
  // features of every point for the recorder and for the network on all
  // points (mode 3); mode 2 predicts, and so needs features for, the
  // unmatched points only
  const bool all_features = (D.rec != nullptr && !D.rec_unmatched) || Pm.warm_start == 3;
  const float gmag = sqrtf(Pm.g[0] * Pm.g[0] + Pm.g[1] * Pm.g[1] + Pm.g[2] * Pm.g[2]);
  const float gh = fmaxf(gmag * h, 1e-12f);
  const float inv_gh = 1.f / gh;
  const float imp_scale = kFeatMass * gh;   // impulse unit m_bar g h
  const float inv_imp = 1.f / imp_scale;
  const float inv_mc = Pm.contact_margin > 0.f ? 1.f / Pm.contact_margin : 0.f;
  // top of the episode's column of blocks: the highest AABB top of its active
  // dynamic bodies (load-above feature)
  float ztop = 0.f;
  if (want_features) {
    float zt = 0.f;
    for (int i = lane; i < E.nb; i += 32)
      if ((s.flags[i] & kActive) && !(s.flags[i] & kStatic)) zt = fmaxf(zt, s.at(FX + 2, i) + s.at(FE + 2, i));
    ztop = warp_max(zt);
  }
  for (int p = lane; p < npairs; p += 32) {
    uint32_t key = Bc.key[p];
    int a = (int)(key >> 16) - 1, b = (int)(key & 0xffff);
    int ia = a < 0 ? G : a;
    int sl = Bc.slot[p] & 0xffff;
    uint32_t ft = Bc.feat[p];
    int np = ft >> 24;
    const float* pt = Bc.pt + (size_t)p * kMaxPts * kNatPtFloats;
    float* pf = Bc.pf + (size_t)p * kNatPairFloats;
    float3 n = f3(pf[0], pf[1], pf[2]);
    float dmax = pf[3];
    float3 t1, t2;
    tangent_basis(n, t1, t2);
    float mu = fminf(s.at(FMU, ia), s.at(FMU, b));
    pf[4] = t1.x; pf[5] = t1.y; pf[6] = t1.z; pf[7] = mu;
    float* sf = Bc.sf;
    float* sp = Bc.sp;
    float* hf = sf + sl * kPairStride;
    hf[0] = n.x; hf[1] = n.y; hf[2] = n.z;
    hf[3] = t1.x; hf[4] = t1.y; hf[5] = t1.z;
    hf[6] = mu; hf[7] = dmax;
    Bc.ab[sl] = (uint32_t)ia | ((uint32_t)b << 16);
    Bc.np[sl] = np;
    float3 xa = s.ld3(FX, ia), xb = s.ld3(FX, b);
    float ima = s.at(FM, ia), imb = s.at(FM, b);
    const Sym3 Ia = ld_iw(s, ia), Ib = ld_iw(s, b);
    float3 Ibody_a = f3(0.f, 0.f, 0.f), Ibody_b = f3(0.f, 0.f, 0.f);
    if (want_features) {
      const float sI = 1.f / (kFeatMass * kFeatLen * kFeatLen);
      if (a >= 0 && !(s.flags[a] & kStatic)) {
        int ga = E.b0 + a;
        Ibody_a = f3(sI / D.invI[ga], sI / D.invI[D.B + ga], sI / D.invI[2 * D.B + ga]);
      }
      if (!(s.flags[b] & kStatic)) {
        int gb = E.b0 + b;
        Ibody_b = f3(sI / D.invI[gb], sI / D.invI[D.B + gb], sI / D.invI[2 * D.B + gb]);
      }
    }
    for (int k = 0; k < np; ++k) {
      const float* q = pt + k * kNatPtFloats;
      float3 pp = f3(q[0], q[1], q[2]);
      float3 rA = pp - xa, rB = pp - xb;
      // W_rs = d_r . K d_s, K the point's inverse mass matrix; the diagonal
      // is Eq. keff for the rows n, t1, t2
      float3 ca0 = cross(rA, n), ca1 = cross(rA, t1), ca2 = cross(rA, t2);
      float3 cb0 = cross(rB, n), cb1 = cross(rB, t1), cb2 = cross(rB, t2);
      float3 ia0 = mul(Ia, ca0), ia1 = mul(Ia, ca1), ia2 = mul(Ia, ca2);
      float3 ib0 = mul(Ib, cb0), ib1 = mul(Ib, cb1), ib2 = mul(Ib, cb2);
      float lin = ima + imb;
      float w00 = lin + dot(ca0, ia0) + dot(cb0, ib0);
      float w11 = lin + dot(ca1, ia1) + dot(cb1, ib1);
      float w22 = lin + dot(ca2, ia2) + dot(cb2, ib2);
      float w01 = dot(ca0, ia1) + dot(cb0, ib1);
      float w02 = dot(ca0, ia2) + dot(cb0, ib2);
      float w12 = dot(ca1, ia2) + dot(cb1, ib2);
      float dep = q[3];
      float bias = dep < 0.f ? -dep * ih : 0.f;
      if (Pm.restitution_newton && dep >= 0.f) {
        // Newton restitution: a touching point approaching faster than vmin
        // targets v_n = -e v_n(pre-solve)
        const float3 u0 = (s.ld3(FV, b) + cross(s.ld3(FW, b), rB)) - (s.ld3(FV, ia) + cross(s.ld3(FW, ia), rA));
        const float un = dot(u0, n);
        if (un < -Pm.restitution_vmin) bias = Pm.restitution * un;
      }
#define W(f, v) sp[sl * kPtStride + k * kSrtPtFloats + (f)] = (v)
      W(0, pp.x); W(1, pp.y); W(2, pp.z);
      W(3, 1.f / w00); W(4, 1.f / w11); W(5, 1.f / w22);
      W(6, w01); W(7, w02); W(8, w12); W(9, bias);
      W(10, q[7]); W(11, q[8]); W(12, q[9]);
      if (want_features && (all_features || q[10] == 0.f)) {
        // warm-start features: pre-solve relative velocity in the contact
        // frame, depth, frame (n, t1.x, t1.y; t1.z follows from n), the
        // height of the column above the point, inverse masses, body
        // inertias, mu, previous impulses and two flags, normalised by the
        // nominal block
        const float3 u = (s.ld3(FV, b) + cross(s.ld3(FW, b), rB)) - (s.ld3(FV, ia) + cross(s.ld3(FW, ia), rA));
        float* f = Bc.x + ((size_t)p * kMaxPts + k) * kFeatures;
        f[0] = dot(u, n) * inv_gh; f[1] = dot(u, t1) * inv_gh; f[2] = dot(u, t2) * inv_gh;
        f[3] = dep * inv_mc;
        f[4] = n.x; f[5] = n.y; f[6] = n.z; f[7] = t1.x; f[8] = t1.y; f[9] = (ztop - pp.z) * kFeatColumnInv;
        f[10] = kFeatMass * ima; f[11] = kFeatMass * imb;
        f[12] = Ibody_a.x; f[13] = Ibody_a.y; f[14] = Ibody_a.z;
        f[15] = Ibody_b.x; f[16] = Ibody_b.y; f[17] = Ibody_b.z;
        f[18] = mu;
        f[19] = q[7] * inv_imp; f[20] = q[8] * inv_imp; f[21] = q[9] * inv_imp;
        f[22] = q[10]; f[23] = a < 0 ? 1.f : 0.f;
      }
    }
    // unused point records of the pair: zero inverse mass and impulses, so
    // that the sweep can run all kMaxPts points without a branch (a zero
    // record's impulse change is exactly zero)
    for (int k = np; k < kMaxPts; ++k)
      for (int f = 0; f < kSrtPtFloats; ++f) W(f, 0.f);
#undef W
  }
  __syncwarp();

  // (7b) learned warm start: the network predicts the starting impulses of the
  // unmatched points (mode 2) or of all points (mode 3)
  int predicted = 0;
  if (Pm.warm_start >= 2 && D.mlp) predicted = mlp_warm_start(D, E, Bc, npairs, Pm.warm_start == 3, imp_scale, lane);

  // (8) warm start: apply the inherited impulses
  const SolverRef V = solver_ref(s, Bc);
  const float e1 = Pm.restitution_newton ? 1.f : 1.f + Pm.restitution;
  if (Pm.warm_start >= 1) colour_passes<0>(V, s.off, ncol, lane, e1, 1.f, false, Pm.beta, Pm.slop);

  // (9) projected Gauss-Seidel sweeps
  int sweeps = 0;
  float res = 0.f;
  if (npairs > 0) {
    const bool rmode = Pm.residual_tol > 0.f;
    const int cap = rmode ? Pm.pgs_iter_cap : Pm.pgs_iters;
    const int every = Pm.residual_every > 0 ? Pm.residual_every : 1;
    const int every_max = Pm.residual_every_max > every ? Pm.residual_every_max : every;
    const float om = Pm.sor, e1om = Pm.sor * e1;
    int next = rmode ? Pm.pgs_min_iters : cap;   // sweep count of the next residual check
    float prev_res = -1.f;
    int prev_at = 0;
    float win_res = -1.f;   // residual at the start of the current stall window
    int win_at = 0;
    bool stalled = false;
    const int am = Pm.accel_period;
    float* acc = D.acc + E.poff * kAccFloats;
    float r2_prev = 0.f;
    int dense_from = INT_MAX - kDenseChecks;   // start of the dense-check window after a step
    if (am > 0) accel_begin(V, acc, npairs, lane);
    while (sweeps < cap) {
      colour_passes<1>(V, s.off, ncol, lane, e1om, om, Pm.sweep_order == 1 && (sweeps & 1), Pm.beta, Pm.slop,
                       Pm.friction_cone != 0);
      ++sweeps;
      if (am > 0 && sweeps % am == 0) {
        const float r2 = accel_change2(V, acc, npairs, lane);
        float beta = r2_prev > 0.f ? r2 / r2_prev : 0.f;
        if (!(beta <= 1.f)) beta = 0.f;   // restart (and NaN)
        r2_prev = r2;
        accel_step(V, acc, s.off, ncol, lane, beta, Pm.friction_cone != 0);
        if (beta > 0.f) dense_from = sweeps + 2;
      }
      // a conjugate-gradient step first raises the residual (its
      // extrapolation overshoots), then the next sweeps bring it to its
      // lowest for a few sweeps before the plain decay resumes; the checks
      // run every sweep over that window, which a cadence fitted to the
      // plain sweeps' geometric decay would step over
      const bool dense = rmode && sweeps >= dense_from && sweeps < dense_from + kDenseChecks;
      if (sweeps >= next || sweeps == cap || dense) {
        res = episode_residual(V, npairs, lane, Pm.friction_cone != 0);
        if (!rmode || res <= Pm.residual_tol || !(res == res)) break;
        // stall test: fit res = win_res * exp(rate * sweeps) over the window
        // and stop when the fit cannot reach the tolerance within the cap
        if (Pm.stall_window > 0) {
          if (win_res < 0.f) {
            win_res = res;
            win_at = sweeps;
          } else if (sweeps - win_at >= Pm.stall_window) {
            const float rate = res < win_res ? __logf(res / win_res) / (float)(sweeps - win_at) : 0.f;
            if (!(rate < 0.f) || __logf(Pm.residual_tol / res) < rate * (float)(cap - sweeps)) {
              stalled = true;
              break;
            }
            win_res = res;
            win_at = sweeps;
          }
        }
        // check cadence: half the sweeps that the decay rate between the
        // last two checks predicts are still needed, within [every, every_max]
        int gap = every_max;
        if (every_max > every && prev_res > 0.f && res < prev_res) {
          const float per_sweep = __logf(res / prev_res) / (float)(sweeps - prev_at);
          const float need = __logf(Pm.residual_tol / res) / per_sweep;
          gap = need < 2.f * every_max ? max(every, (int)(0.5f * need)) : every_max;
        } else if (every_max == every || prev_res < 0.f) {
          gap = every;
        }
        prev_res = res;
        prev_at = sweeps;
        next = sweeps + gap;
      }
    }
    if (rmode && (sweeps >= cap || stalled) && !(res <= Pm.residual_tol)) out.status |= JB_EP_NOT_CONVERGED;
  }
  // final impulses back to the natural arrays (warm-start cache, readback)
  for (int p = lane; p < npairs; p += 32) {
    int sl = Bc.slot[p] & 0xffff;
    int np = Bc.feat[p] >> 24;
    float* pt = Bc.pt + (size_t)p * kMaxPts * kNatPtFloats;
    for (int k = 0; k < np; ++k) {
      float* q = pt + k * kNatPtFloats;
      const float* rec = Bc.sp + sl * kPtStride + k * kSrtPtFloats;
      q[7] = rec[10]; q[8] = rec[11]; q[9] = rec[12];
    }
  }
  // training-sample recorder: converged solves only, every rec_every-th solve
  if (D.rec && npairs > 0 && (res <= Pm.residual_tol || Pm.residual_tol <= 0.f) &&
      ((long long)st.solves % D.rec_every) == 0) {
    for (int p = lane; p < npairs; p += 32) {
      int np = Bc.feat[p] >> 24;
      const float* pt = Bc.pt + (size_t)p * kMaxPts * kNatPtFloats;
      bool any_matched = false;
      for (int k = 0; k < np; ++k) any_matched |= pt[k * kNatPtFloats + 10] != 0.f;
      if (D.rec_unmatched && any_matched) continue;
      for (int k = 0; k < np; ++k) {
        int slot = atomicAdd(D.rec_count, 1);
        if (slot >= D.rec_cap) break;
        float* row = D.rec + (size_t)slot * kRecFloats;
        const float* f = Bc.x + ((size_t)p * kMaxPts + k) * kFeatures;
        for (int j = 0; j < kFeatures; ++j) row[j] = f[j];
        const float* q = pt + k * kNatPtFloats;
        row[24] = q[7] * inv_imp; row[25] = q[8] * inv_imp; row[26] = q[9] * inv_imp;
      }
    }
  }

  // (10) semi-implicit position update and quaternion integration (Eq. quat_int)
  for (int i = lane; i < nb; i += 32) {
    int fl = s.flags[i];
    if (!(fl & kActive) || (fl & kStatic)) continue;
    float3 v = s.ld3(FV, i), w = s.ld3(FW, i);
    s.st3(FX, i, s.ld3(FX, i) + h * v);
    float q0 = s.at(FQ, i), q1 = s.at(FQ + 1, i), q2 = s.at(FQ + 2, i), q3 = s.at(FQ + 3, i);
    // [0, w] (x) q, world-frame angular velocity
    float d0 = -w.x * q1 - w.y * q2 - w.z * q3;
    float d1 = w.x * q0 + w.y * q3 - w.z * q2;
    float d2 = -w.x * q3 + w.y * q0 + w.z * q1;
    float d3 = w.x * q2 - w.y * q1 + w.z * q0;
    float hh = 0.5f * h;
    q0 += hh * d0; q1 += hh * d1; q2 += hh * d2; q3 += hh * d3;
    float il = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    s.at(FQ, i) = q0 * il; s.at(FQ + 1, i) = q1 * il; s.at(FQ + 2, i) = q2 * il; s.at(FQ + 3, i) = q3 * il;
  }
  __syncwarp();

  // (11) position correction (Eq. baumgarte), colour by colour
  colour_passes<2>(V, s.off, ncol, lane, e1, 1.f, false, Pm.beta, Pm.slop);

  st.cur = cur;
  st.npairs = npairs;
  st.ncolours = ncol;
  out.res = res;
  out.sweeps = sweeps;
  out.predicted = predicted;
  out.npairs = npairs;
  out.npoints = npoints;
  out.ncol = ncol;
  return out;
}

// ----------------------------------------------------------------- episode
__device__ __forceinline__ float body_kinetic(const Sm& s, const Dev& D, int gi, int i) {
  float m = D.mass[gi];
  float3 v = s.ld3(FV, i), w = s.ld3(FW, i);
  // body-frame angular velocity R^T w and I = 1 / invI
  float wl0 = dot(s.axis(i, 0), w), wl1 = dot(s.axis(i, 1), w), wl2 = dot(s.axis(i, 2), w);
  float I0 = 1.f / D.invI[gi], I1 = 1.f / D.invI[D.B + gi], I2 = 1.f / D.invI[2 * D.B + gi];
  return 0.5f * m * dot(v, v) + 0.5f * (I0 * wl0 * wl0 + I1 * wl1 * wl1 + I2 * wl2 * wl2);
}

struct Terms { float ek, dxr, cmin; int nfallen; };

// Eq. collapse terms over active dynamic blocks except `skip` (frames must be current).
__device__ Terms collapse_terms(const Dev& D, const Ep& E, int skip) {
  const Sm& s = E.s;
  float ek = 0.f, dxr = 0.f, cmin = 1.f;
  int nf = 0;
  for (int i = E.lane; i < E.nb; i += 32) {
    int fl = s.flags[i];
    if (!(fl & kActive) || (fl & kStatic) || i == skip) continue;
    int gi = E.b0 + i;
    ek += body_kinetic(s, D, gi, i);
    float3 d = s.ld3(FX, i) - f3(D.x0[gi], D.x0[D.B + gi], D.x0[2 * D.B + gi]);
    float r = sqrtf(dot(d, d)) / (2.f * s.at(FH, i));
    dxr = fmaxf(dxr, r);
    nf += r > D.P.fall_frac;
    float3 z = s.axis(i, 2);
    float c = dot(z, f3(D.z0[gi], D.z0[D.B + gi], D.z0[2 * D.B + gi]));
    cmin = fminf(cmin, c);
  }
  Terms t;
  t.ek = warp_sum(ek);
  t.dxr = warp_max(dxr);
  t.cmin = warp_min(cmin);
  t.nfallen = (int)warp_sum((float)nf);
  return t;
}

__device__ void refresh_frames(const Dev& D, const Ep& E) {
  for (int i = E.lane; i < E.nb; i += 32) body_frame(E.s, D, E.b0 + i, i);
  __syncwarp();
}

// Starts move st.mi: a constant force F = sign * factor * k * mu_s * m * |g|
// (Sec. 5) along the block's axis, fixed at the start of the push.
__device__ void start_move(const Dev& D, const Ep& E, EpState& st) {
  int m = D.mv_off[E.e] + st.mi;
  int blk = D.mv_block[m];
  if (E.lane == 0) {
    int gi = E.b0 + blk;
    const Sm& s = E.s;
    float3 dir = s.axis(blk, D.mv_axis[m] == JB_AXIS_Y ? 0 : 1);
    float g = sqrtf(D.P.g[0] * D.P.g[0] + D.P.g[1] * D.P.g[1] + D.P.g[2] * D.P.g[2]);
    float F = D.mv_sign[m] * D.mv_factor[m] * D.mv_k[m] * D.mu[gi] * D.mass[gi] * g;
    D.f[gi] = F * dir.x; D.f[D.B + gi] = F * dir.y; D.f[2 * D.B + gi] = F * dir.z;
    D.f_steps[gi] = D.mv_push[m];
  }
  __syncwarp();
  st.pb = blk;
  st.phase = JB_PH_PUSH;
  st.remaining = D.mv_push[m];
}

__device__ void end_push(const Dev& D, const Ep& E, const EpState& st) {
  if (st.pb >= 0 && E.lane == 0) {
    int gi = E.b0 + st.pb;
    D.f[gi] = 0.f; D.f[D.B + gi] = 0.f; D.f[2 * D.B + gi] = 0.f;
    D.f_steps[gi] = 0;
  }
  __syncwarp();
}

__device__ void next_move(const Dev& D, const Ep& E, EpState& st) {
  st.mi++;
  int nm = D.mv_off[E.e + 1] - D.mv_off[E.e];
  if (st.mi < nm) start_move(D, E, st);
  else st.phase = JB_PH_DONE;
}

// Eq. stability on the warp's current state (frames must be current): the
// signed distance from the COM (xy, mass-weighted over active dynamic blocks)
// to the edges of the convex hull of the xy corners of the ground-touching
// blocks (z - e_z <= aabb_eps), positive inside; minus the distance to the
// hull's segment or point when it has fewer than 3 vertices; 0 when nothing
// touches.  The corners go to the candidate array (free between substeps);
// the hull is found by gift wrapping, each wrap step one warp reduction.
__device__ __forceinline__ bool wrap_better(float2 cur, float2 a, float2 b) {
  // b replaces a as the next hull vertex after cur
  const float cr = (a.x - cur.x) * (b.y - cur.y) - (a.y - cur.y) * (b.x - cur.x);
  const float da = (a.x - cur.x) * (a.x - cur.x) + (a.y - cur.y) * (a.y - cur.y);
  const float db = (b.x - cur.x) * (b.x - cur.x) + (b.y - cur.y) * (b.y - cur.y);
  return cr < 0.f || (cr == 0.f && db > da);
}

__device__ float support_margin_warp(const Dev& D, const Ep& E) {
  const Sm& s = E.s;
  const int lane = E.lane;
  float2* P = reinterpret_cast<float2*>(s.cand);
  float mx = 0.f, my = 0.f, mt = 0.f;
  int cnt = 0;
  for (int i0 = 0; i0 < E.nb; i0 += 32) {
    const int i = i0 + lane;
    bool touch = false;
    if (i < E.nb) {
      const int fl = s.flags[i];
      if ((fl & kActive) && !(fl & kStatic)) {
        const float m = D.mass[E.b0 + i];
        mx += m * s.at(FX, i); my += m * s.at(FX + 1, i); mt += m;
        touch = s.at(FX + 2, i) - s.at(FE + 2, i) <= D.P.aabb_eps;
      }
    }
    const unsigned bal = __ballot_sync(FULL, touch);
    if (touch) {
      const int base = 8 * (cnt + __popc(bal & lanemask_lt(lane)));
      const float3 a0 = s.axis(i, 0), a1 = s.axis(i, 1), a2 = s.axis(i, 2);
      const float hx = s.at(FH, i), hy = s.at(FH + 1, i), hz = s.at(FH + 2, i);
      for (int c = 0; c < 8; ++c) {
        const float s0 = (c & 1) ? hx : -hx, s1 = (c & 2) ? hy : -hy, s2 = (c & 4) ? hz : -hz;
        P[base + c] = make_float2(s.at(FX, i) + s0 * a0.x + s1 * a1.x + s2 * a2.x,
                                  s.at(FX + 1, i) + s0 * a0.y + s1 * a1.y + s2 * a2.y);
      }
    }
    cnt += __popc(bal);
  }
  mx = warp_sum(mx); my = warp_sum(my); mt = warp_sum(mt);
  __syncwarp();
  const int n = 8 * cnt;
  if (!(mt > 0.f) || n == 0) return 0.f;
  const float2 com = make_float2(mx / mt, my / mt);
  // start: the lowest (x, then y) corner
  float2 p0 = make_float2(FLT_MAX, FLT_MAX);
  for (int j = lane; j < n; j += 32) {
    const float2 p = P[j];
    if (p.x < p0.x || (p.x == p0.x && p.y < p0.y)) p0 = p;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float2 q = make_float2(__shfl_xor_sync(FULL, p0.x, o), __shfl_xor_sync(FULL, p0.y, o));
    if (q.x < p0.x || (q.x == p0.x && q.y < p0.y)) p0 = q;
  }
  float dmin = FLT_MAX;
  float2 cur = p0, first = p0;
  int nh = 0;
  for (int it = 0; it < n + 2; ++it) {
    float2 nx = cur;
    bool have = false;
    for (int j = lane; j < n; j += 32) {
      const float2 p = P[j];
      if (p.x == cur.x && p.y == cur.y) continue;
      if (!have || wrap_better(cur, nx, p)) { nx = p; have = true; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float2 q = make_float2(__shfl_xor_sync(FULL, nx.x, o), __shfl_xor_sync(FULL, nx.y, o));
      const bool qh = __shfl_xor_sync(FULL, (int)have, o) != 0;
      if (qh && (!have || wrap_better(cur, nx, q))) { nx = q; have = true; }
    }
    // every lane now holds the same candidate up to ties of equal rank; take lane 0's
    nx = make_float2(__shfl_sync(FULL, nx.x, 0), __shfl_sync(FULL, nx.y, 0));
    have = __shfl_sync(FULL, (int)have, 0) != 0;
    if (!have) break;
    if (nh == 0) first = nx;
    const float ex = nx.x - cur.x, ey = nx.y - cur.y;
    const float len = sqrtf(ex * ex + ey * ey);
    if (len > 0.f) dmin = fminf(dmin, (ex * (com.y - cur.y) - ey * (com.x - cur.x)) / len);
    ++nh;
    cur = nx;
    if (cur.x == p0.x && cur.y == p0.y) break;
  }
  if (nh >= 3) return dmin;
  if (nh == 0) return -sqrtf((com.x - p0.x) * (com.x - p0.x) + (com.y - p0.y) * (com.y - p0.y));
  const float ex = first.x - p0.x, ey = first.y - p0.y;
  const float l2 = ex * ex + ey * ey;
  const float t = l2 > 0.f ? fminf(fmaxf(((com.x - p0.x) * ex + (com.y - p0.y) * ey) / l2, 0.f), 1.f) : 0.f;
  const float dx = com.x - (p0.x + t * ex), dy = com.y - (p0.y + t * ey);
  return -sqrtf(dx * dx + dy * dy);
}

__device__ void run_episode(const Dev& D, int e, int mode, int max_steps, unsigned char* base, int lane) {
  Ep E;
  E.e = e;
  E.lane = lane;
  E.b0 = D.body_off[e];
  E.nb = D.body_off[e + 1] - E.b0;
  E.Pc = pair_capacity(E.nb);
  E.poff = D.pair_off[e];
  E.s = sm_view(base, D.nb_max, D.pc_max, D.ps);
  const Sm& s = E.s;
  EpState st = D.ep[e];
  if (mode == kModeFree && st.phase != JB_PH_FREE) return;
  if (mode == kModeProtocol && (st.phase == JB_PH_FREE || st.phase == JB_PH_DONE)) return;

  for (int i = lane; i < E.nb; i += 32) {
    int gi = E.b0 + i;
    for (int k = 0; k < 3; ++k) {
      s.at(FX + k, i) = D.x[k * D.B + gi];
      s.at(FV + k, i) = D.v[k * D.B + gi];
      s.at(FW + k, i) = D.w[k * D.B + gi];
      s.at(FH + k, i) = D.half[k * D.B + gi];
    }
    for (int k = 0; k < 4; ++k) s.at(FQ + k, i) = D.q[k * D.B + gi];
    s.at(FM, i) = D.invm[gi];
    s.at(FMU, i) = D.mu[gi];
    s.flags[i] = D.flags[gi];
  }
  if (lane == 0) {   // ground slot
    int G = E.nb;
    for (int k = 0; k < 3; ++k) { s.at(FX + k, G) = 0.f; s.at(FV + k, G) = 0.f; s.at(FW + k, G) = 0.f; s.at(FH + k, G) = 0.f; }
    s.at(FQ, G) = 1.f; s.at(FQ + 1, G) = 0.f; s.at(FQ + 2, G) = 0.f; s.at(FQ + 3, G) = 0.f;
    s.at(FM, G) = 0.f;
    s.at(FMU, G) = D.ground_mu[e];
    s.flags[G] = kActive | kStatic;
  }
  __syncwarp();
  if (lane == 0) body_frame(s, D, -1, E.nb);
  __syncwarp();

  const float h = D.P.dt / (float)D.P.n_sub;
  for (int step = 0; step < max_steps; ++step) {
    if (mode == kModeProtocol && st.phase == JB_PH_DONE) break;
    int ndyn = 0, nact = 0;
    for (int i = lane; i < E.nb; i += 32) {
      ndyn += (s.flags[i] & kActive) && !(s.flags[i] & kStatic);
      nact += (s.flags[i] & kActive) != 0;
    }
    ndyn = __reduce_add_sync(FULL, ndyn);
    nact = __reduce_add_sync(FULL, nact);
    st.body_steps += ndyn;
    StepOut o;
    for (int sub = 0; sub < D.P.n_sub; ++sub) {
      o = substep(D, E, st, h);
      st.status |= o.status;
      st.last_sweeps = o.sweeps;
      st.last_res = o.res;
      if (!(o.res <= st.max_res)) st.max_res = o.res;
      st.total_sweeps += o.sweeps;
      st.solves += 1.0;
      st.npoints = o.npoints;
      st.max_colours = max(st.max_colours, o.ncol);
      st.capped += (o.status & JB_EP_NOT_CONVERGED) ? 1 : 0;
      st.point_sweeps += (double)o.npoints * o.sweeps;
      st.point_steps += o.npoints;
      st.pair_steps += o.npairs;
      st.bp_tests += 0.5 * nact * (nact - 1) + ndyn;
      st.mlp_points += o.predicted;
    }
    for (int i = lane; i < E.nb; i += 32) {
      int gi = E.b0 + i;
      if (D.f_steps[gi] > 0) D.f_steps[gi] -= 1;
    }
    st.steps++;
    bool bad = false;
    for (int i = lane; i < E.nb; i += 32) {
      float t = s.at(FX, i) + s.at(FX + 1, i) + s.at(FX + 2, i) + s.at(FV, i) + s.at(FV + 1, i) + s.at(FV + 2, i) +
                s.at(FW, i) + s.at(FW + 1, i) + s.at(FW + 2, i);
      if (!isfinite(t)) bad = true;
    }
    __syncwarp();
    if (__any_sync(FULL, bad)) {
      st.status |= JB_EP_NONFINITE;
      if (st.phase != JB_PH_FREE) st.phase = JB_PH_DONE;
      break;
    }
    // Eq. stability every step: the early-warning margin
    refresh_frames(D, E);
    st.margin = support_margin_warp(D, E);
    st.min_margin = fminf(st.min_margin, st.margin);
    if (st.margin < 0.f && st.first_unstable < 0) st.first_unstable = st.steps;
    if (mode != kModeProtocol) continue;

    int skip = st.phase == JB_PH_PUSH ? st.pb : -1;
    Terms t = collapse_terms(D, E, skip);
    bool coll = t.dxr > D.P.fall_frac && t.ek > D.P.collapse_ek && t.cmin < D.P.collapse_cos;
    if ((st.phase == JB_PH_PUSH || st.phase == JB_PH_SETTLE) && coll) {
      st.collapsed = 1;
      st.collapse_step = st.steps;
      if (st.phase == JB_PH_PUSH) end_push(D, E, st);
      st.pb = -1;
      st.phase = JB_PH_REST;
      st.rest_left = D.P.rest_steps;
      continue;
    }
    if (st.phase == JB_PH_PUSH) {
      if (--st.remaining <= 0) {
        end_push(D, E, st);
        int m = D.mv_off[e] + st.mi;
        if (D.mv_remove[m]) {
          if (lane == 0) s.flags[st.pb] &= ~kActive;
          __syncwarp();
        }
        st.pb = -1;
        st.phase = JB_PH_SETTLE;
        st.remaining = D.mv_settle[m];
        if (st.remaining <= 0) next_move(D, E, st);
      }
    } else if (st.phase == JB_PH_SETTLE) {
      if (--st.remaining <= 0) next_move(D, E, st);
    } else if (st.phase == JB_PH_REST) {
      Terms ta = collapse_terms(D, E, -1);
      st.rest_left--;
      if (ta.ek < D.P.rest_ek) { st.resting = 1; st.phase = JB_PH_DONE; }
      else if (st.rest_left <= 0) st.phase = JB_PH_DONE;
    }
  }

  for (int i = lane; i < E.nb; i += 32) {
    int gi = E.b0 + i;
    for (int k = 0; k < 3; ++k) {
      D.x[k * D.B + gi] = s.at(FX + k, i);
      D.v[k * D.B + gi] = s.at(FV + k, i);
      D.w[k * D.B + gi] = s.at(FW + k, i);
    }
    for (int k = 0; k < 4; ++k) D.q[k * D.B + gi] = s.at(FQ + k, i);
    D.flags[gi] = s.flags[i];
  }
  if (lane == 0) D.ep[e] = st;
  __syncwarp();
}

// Persistent grid: each warp claims episodes from the work counter.
__global__ void __launch_bounds__(kWarpsPerCta * 32) episode_kernel(Dev D, int mode, int max_steps) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = jb_smem + (size_t)warp * D.smem_per_warp;
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(D.work_counter, 1);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx >= D.E) break;
    int e = D.order ? D.order[idx] : idx;
    run_episode(D, e, mode, max_steps, base, lane);
  }
}

// ------------------------------------------------------------ init / commands
// Derived per-body state: normalised q, inverse mass, body inverse inertia
// (Eq. inertia), collapse reference pose; episode state reset.
__global__ void init_bodies_kernel(Dev D) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= D.B) return;
  float q0 = D.q[b], q1 = D.q[D.B + b], q2 = D.q[2 * D.B + b], q3 = D.q[3 * D.B + b];
  float il = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  q0 *= il; q1 *= il; q2 *= il; q3 *= il;
  D.q[b] = q0; D.q[D.B + b] = q1; D.q[2 * D.B + b] = q2; D.q[3 * D.B + b] = q3;
  float m = D.mass[b];
  bool st = !(m > 0.f);
  float l = 2.f * D.half[b], wd = 2.f * D.half[D.B + b], th = 2.f * D.half[2 * D.B + b];
  if (st) {
    D.invm[b] = 0.f;
    for (int k = 0; k < 3; ++k) { D.invI[k * D.B + b] = 0.f; D.v[k * D.B + b] = 0.f; D.w[k * D.B + b] = 0.f; }
  } else {
    D.invm[b] = 1.f / m;
    D.invI[b] = 12.f / (m * (wd * wd + th * th));
    D.invI[D.B + b] = 12.f / (m * (l * l + th * th));
    D.invI[2 * D.B + b] = 12.f / (m * (l * l + wd * wd));
  }
  D.flags[b] = kActive | (st ? kStatic : 0);
  for (int k = 0; k < 3; ++k) { D.x0[k * D.B + b] = D.x[k * D.B + b]; D.f[k * D.B + b] = 0.f; }
  D.f_steps[b] = 0;
  // thickness axis = third column of R(q)
  D.z0[b] = 2.f * (q1 * q3 + q2 * q0);
  D.z0[D.B + b] = 2.f * (q2 * q3 - q1 * q0);
  D.z0[2 * D.B + b] = 1.f - 2.f * (q1 * q1 + q2 * q2);
}

__global__ void init_episodes_kernel(Dev D) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D.E) return;
  EpState s;
  memset(&s, 0, sizeof s);
  s.phase = JB_PH_FREE;
  s.pb = -1;
  s.min_margin = FLT_MAX;
  s.first_unstable = -1;
  s.collapse_step = -1;
  D.ep[e] = s;
}

// Resets the collapse reference to the current poses.
__global__ void reset_reference_kernel(Dev D) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= D.B) return;
  float q0 = D.q[b], q1 = D.q[D.B + b], q2 = D.q[2 * D.B + b], q3 = D.q[3 * D.B + b];
  float il = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  q0 *= il; q1 *= il; q2 *= il; q3 *= il;
  D.q[b] = q0; D.q[D.B + b] = q1; D.q[2 * D.B + b] = q2; D.q[3 * D.B + b] = q3;
  for (int k = 0; k < 3; ++k) D.x0[k * D.B + b] = D.x[k * D.B + b];
  D.z0[b] = 2.f * (q1 * q3 + q2 * q0);
  D.z0[D.B + b] = 2.f * (q2 * q3 - q1 * q0);
  D.z0[2 * D.B + b] = 1.f - 2.f * (q1 * q1 + q2 * q2);
}

// Pair-capacity prefix over the episodes (one thread; used where the host
// keeps no offset table).
__global__ void pair_offsets_kernel(Dev D, int64_t* pair_off) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t acc = 0;
  pair_off[0] = 0;
  for (int e = 0; e < D.E; ++e) {
    acc += pair_capacity(D.body_off[e + 1] - D.body_off[e]);
    pair_off[e + 1] = acc;
  }
}

__global__ void clear_cache_kernel(Dev D) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D.E) return;
  D.ep[e].npairs = 0;
  D.ep[e].ncolours = 0;
}

__device__ __forceinline__ float3 body_axis_g(const Dev& D, int gi, int k) {
  float w = D.q[gi], x = D.q[D.B + gi], y = D.q[2 * D.B + gi], z = D.q[3 * D.B + gi];
  if (k == 0) return f3(1 - 2 * (y * y + z * z), 2 * (x * y + z * w), 2 * (x * z - y * w));
  if (k == 1) return f3(2 * (x * y - z * w), 1 - 2 * (x * x + z * z), 2 * (y * z + x * w));
  return f3(2 * (x * z + y * w), 2 * (y * z - x * w), 1 - 2 * (x * x + y * y));
}

// Starts every episode's schedule (move 0) or marks it done.
__global__ void protocol_start_kernel(Dev D) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D.E) return;
  EpState s = D.ep[e];
  s.mi = 0;
  s.pb = -1;
  s.collapsed = 0;
  s.resting = 0;
  s.min_margin = FLT_MAX;
  s.first_unstable = -1;
  s.collapse_step = -1;
  int m0 = D.mv_off[e], nm = D.mv_off[e + 1] - m0;
  if (nm <= 0) { s.phase = JB_PH_DONE; D.ep[e] = s; return; }
  int blk = D.mv_block[m0];
  int gi = D.body_off[e] + blk;
  float3 dir = body_axis_g(D, gi, D.mv_axis[m0] == JB_AXIS_Y ? 0 : 1);
  float g = sqrtf(D.P.g[0] * D.P.g[0] + D.P.g[1] * D.P.g[1] + D.P.g[2] * D.P.g[2]);
  float F = D.mv_sign[m0] * D.mv_factor[m0] * D.mv_k[m0] * D.mu[gi] * D.mass[gi] * g;
  D.f[gi] = F * dir.x; D.f[D.B + gi] = F * dir.y; D.f[2 * D.B + gi] = F * dir.z;
  D.f_steps[gi] = D.mv_push[m0];
  s.pb = blk;
  s.phase = JB_PH_PUSH;
  s.remaining = D.mv_push[m0];
  D.ep[e] = s;
}

__global__ void push_kernel(Dev D, int n, const int* ep, const int* blk, const int* axis, const float* force, const int* steps) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int gi = D.body_off[ep[i]] + blk[i];
  float3 dir = body_axis_g(D, gi, axis[i] == JB_AXIS_Y ? 0 : 1);
  D.f[gi] = force[i] * dir.x; D.f[D.B + gi] = force[i] * dir.y; D.f[2 * D.B + gi] = force[i] * dir.z;
  D.f_steps[gi] = steps[i];
}

__global__ void remove_kernel(Dev D, int n, const int* ep, const int* blk) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int gi = D.body_off[ep[i]] + blk[i];
  D.flags[gi] &= ~kActive;
  D.f_steps[gi] = 0;
}

// Eq. stability margin and Sec. 8 statistics, one thread per episode.  The
// support polygon is the convex hull (gift wrapping) of the xy corners of the
// ground-touching blocks; imbalance = minus the smallest signed distance from
// the COM to the hull edges (distance to the segment/point if degenerate).
__device__ __forceinline__ float2 corner_xy(const Dev& D, int gi, int c) {
  float3 a0 = body_axis_g(D, gi, 0), a1 = body_axis_g(D, gi, 1), a2 = body_axis_g(D, gi, 2);
  float s0 = (c & 1) ? 1.f : -1.f, s1 = (c & 2) ? 1.f : -1.f, s2 = (c & 4) ? 1.f : -1.f;
  float hx = D.half[gi], hy = D.half[D.B + gi], hz = D.half[2 * D.B + gi];
  return make_float2(D.x[gi] + s0 * hx * a0.x + s1 * hy * a1.x + s2 * hz * a2.x,
                     D.x[D.B + gi] + s0 * hx * a0.y + s1 * hy * a1.y + s2 * hz * a2.y);
}

__device__ __forceinline__ bool touching(const Dev& D, int gi) {
  if (!(D.flags[gi] & kActive) || (D.flags[gi] & kStatic)) return false;
  float3 a0 = body_axis_g(D, gi, 0), a1 = body_axis_g(D, gi, 1), a2 = body_axis_g(D, gi, 2);
  float ez = fabsf(a0.z) * D.half[gi] + fabsf(a1.z) * D.half[D.B + gi] + fabsf(a2.z) * D.half[2 * D.B + gi];
  return D.x[2 * D.B + gi] - ez <= D.P.aabb_eps;
}

__global__ void stats_kernel(Dev D, jb_episode_stats* out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D.E) return;
  int b0 = D.body_off[e], nb = D.body_off[e + 1] - b0;
  EpState st = D.ep[e];
  double cx = 0, cy = 0, mt = 0;
  float ek = 0.f;
  int nf = 0;
  for (int i = 0; i < nb; ++i) {
    int gi = b0 + i;
    if (!(D.flags[gi] & kActive) || (D.flags[gi] & kStatic)) continue;
    float m = D.mass[gi];
    cx += m * D.x[gi]; cy += m * D.x[D.B + gi]; mt += m;
    float3 v = f3(D.v[gi], D.v[D.B + gi], D.v[2 * D.B + gi]);
    float3 w = f3(D.w[gi], D.w[D.B + gi], D.w[2 * D.B + gi]);
    float wl0 = dot(body_axis_g(D, gi, 0), w), wl1 = dot(body_axis_g(D, gi, 1), w), wl2 = dot(body_axis_g(D, gi, 2), w);
    ek += 0.5f * m * dot(v, v) + 0.5f * (wl0 * wl0 / D.invI[gi] + wl1 * wl1 / D.invI[D.B + gi] + wl2 * wl2 / D.invI[2 * D.B + gi]);
    float3 d = f3(D.x[gi] - D.x0[gi], D.x[D.B + gi] - D.x0[D.B + gi], D.x[2 * D.B + gi] - D.x0[2 * D.B + gi]);
    if (sqrtf(dot(d, d)) / (2.f * D.half[gi]) > D.P.fall_frac) ++nf;
  }
  float imb = 0.f;
  if (mt > 0) {
    float comx = (float)(cx / mt), comy = (float)(cy / mt);
    // lowest (x, y) corner as the start of the wrap
    float2 p0 = make_float2(FLT_MAX, FLT_MAX);
    int ncorner = 0;
    for (int i = 0; i < nb; ++i) {
      int gi = b0 + i;
      if (!touching(D, gi)) continue;
      for (int c = 0; c < 8; ++c) {
        float2 p = corner_xy(D, gi, c);
        ++ncorner;
        if (p.x < p0.x || (p.x == p0.x && p.y < p0.y)) p0 = p;
      }
    }
    if (ncorner > 0) {
      float dmin = FLT_MAX;
      float2 cur = p0;
      int nh = 0;
      float2 first_next = p0;
      bool degenerate = true;
      // gift wrapping: next = the point with every other point to its left
      for (int it = 0; it < 8 * nb + 2; ++it) {
        float2 nxt = cur;
        bool have = false;
        for (int i = 0; i < nb; ++i) {
          int gi = b0 + i;
          if (!touching(D, gi)) continue;
          for (int c = 0; c < 8; ++c) {
            float2 p = corner_xy(D, gi, c);
            if (p.x == cur.x && p.y == cur.y) continue;
            if (!have) { nxt = p; have = true; continue; }
            float cr = (nxt.x - cur.x) * (p.y - cur.y) - (nxt.y - cur.y) * (p.x - cur.x);
            float dn = (nxt.x - cur.x) * (nxt.x - cur.x) + (nxt.y - cur.y) * (nxt.y - cur.y);
            float dp = (p.x - cur.x) * (p.x - cur.x) + (p.y - cur.y) * (p.y - cur.y);
            if (cr < 0.f || (cr == 0.f && dp > dn)) nxt = p;
          }
        }
        if (!have) break;
        if (nh == 0) first_next = nxt;
        float ex = nxt.x - cur.x, ey = nxt.y - cur.y;
        float len = sqrtf(ex * ex + ey * ey);
        if (len > 0.f) {
          float sd = (ex * (comy - cur.y) - ey * (comx - cur.x)) / len;
          dmin = fminf(dmin, sd);
        }
        ++nh;
        cur = nxt;
        if (cur.x == p0.x && cur.y == p0.y) break;
      }
      degenerate = nh < 3;
      if (!degenerate) imb = -dmin;
      else if (nh == 0) {
        float dx = comx - p0.x, dy = comy - p0.y;
        imb = sqrtf(dx * dx + dy * dy);
      } else {
        float2 a = p0, b = first_next;
        float ex = b.x - a.x, ey = b.y - a.y;
        float l2 = ex * ex + ey * ey;
        float t = l2 > 0.f ? fminf(fmaxf(((comx - a.x) * ex + (comy - a.y) * ey) / l2, 0.f), 1.f) : 0.f;
        float dx = comx - (a.x + t * ex), dy = comy - (a.y + t * ey);
        imb = sqrtf(dx * dx + dy * dy);
      }
    }
  }
  jb_episode_stats o;
  o.status = st.status;
  o.phase = st.phase;
  o.collapsed = st.collapsed;
  o.resting = st.resting || ek < D.P.rest_ek;
  o.n_fallen = nf;
  o.moves_done = st.mi;
  o.n_pairs = st.npairs;
  o.n_points = st.npoints;
  o.last_sweeps = st.last_sweeps;
  o.steps = st.steps;
  o.max_colours = st.max_colours;
  o.capped_solves = st.capped;
  o.com_imbalance = imb;
  o.kinetic = ek;
  o.last_residual = st.last_res;
  o.max_residual = st.max_res;
  o.total_sweeps = st.total_sweeps;
  o.solves = st.solves;
  o.body_steps = st.body_steps;
  o.point_sweeps = st.point_sweeps;
  o.point_steps = st.point_steps;
  o.pair_steps = st.pair_steps;
  o.bp_tests = st.bp_tests;
  o.mlp_points = st.mlp_points;
  o.stability_margin = st.steps > 0 ? st.margin : 0.f;
  o.min_stability_margin = st.steps > 0 ? st.min_margin : 0.f;
  o.first_unstable_step = st.first_unstable;
  o.collapse_step = st.collapse_step;
  out[e] = o;
}

}  // namespace jbk
