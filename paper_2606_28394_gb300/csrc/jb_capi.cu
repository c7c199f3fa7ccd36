// Host implementation of the C ABI declared in include/jb.h.
//
// The batch never allocates device memory: every device array is carved from
// the caller's workspace.  Layout (each array 256-byte aligned):
//   [persistent] scene + derived body state, episode records, schedule,
//                both contact buffers           (saved by jb_save_state)
//   [scratch]    work counter, command staging, statistics staging
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "jb_internal.cuh"

namespace jbk {
__global__ void episode_kernel(Dev D, int mode, int max_steps);
__global__ void init_bodies_kernel(Dev D);
__global__ void init_episodes_kernel(Dev D);
__global__ void reset_reference_kernel(Dev D);
__global__ void clear_cache_kernel(Dev D);
__global__ void protocol_start_kernel(Dev D);
__global__ void push_kernel(Dev D, int n, const int* ep, const int* blk, const int* axis, const float* force, const int* steps);
__global__ void remove_kernel(Dev D, int n, const int* ep, const int* blk);
__global__ void stats_kernel(Dev D, jb_episode_stats* out);
__global__ void pair_offsets_kernel(Dev D, int64_t* pair_off);
}  // namespace jbk

using namespace jbk;

static thread_local char g_err[512] = "";

jb_status jbk::fail(jb_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t err_ = (call);                                                            \
    if (err_ != cudaSuccess)                                                              \
      return fail(JB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(err_));             \
  } while (0)

struct jb_batch {
  Dev D;
  cudaStream_t stream;
  unsigned char* ws;
  size_t ws_bytes, persist_bytes;
  int E, B, max_moves;
  std::vector<int32_t> body_off;
  std::vector<int64_t> pair_off;
  int32_t* cmd;          // staging for host commands (6 * B ints)
  jb_episode_stats* stats;
  bool has_protocol;
  // Episodes grouped by size: each class has its own shared-memory plan,
  // persistent grid and work queue (a slice of the size-sorted order), and
  // the classes run concurrently on side streams joined to the batch stream.
  struct SizeClass {
    int first, count, nb_max, pc_max, ps, smem, grid;
    cudaStream_t stream;
    cudaEvent_t join;
  };
  std::vector<SizeClass> cls;
  cudaEvent_t fork = nullptr;
  ~jb_batch() {
    for (auto& k : cls) {
      if (k.stream) cudaStreamDestroy(k.stream);
      if (k.join) cudaEventDestroy(k.join);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

// ------------------------------------------------------------ arena layout
namespace {
struct Arena {
  unsigned char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * (n > 0 ? n : 1);
    return p;
  }
};

struct Sizes {
  int E, B, nb_max, pc_max, M;
  int64_t P;
};

// Carves the workspace (base may be null to measure).  Fills D, returns bytes.
size_t carve(unsigned char* base, const Sizes& z, Dev& D, size_t* persist, int32_t** cmd,
             jb_episode_stats** stats) {
  Arena a{base};
  int B = z.B, E = z.E, M = z.M;
  int64_t P = z.P;
  D.body_off = a.take<int32_t>(E + 1);
  D.pair_off = a.take<int64_t>(E + 1);
  D.order = a.take<int32_t>(E);
  D.half = a.take<float>(3 * (size_t)B);
  D.mass = a.take<float>(B);
  D.invm = a.take<float>(B);
  D.invI = a.take<float>(3 * (size_t)B);
  D.mu = a.take<float>(B);
  D.ground_mu = a.take<float>(E);
  D.x = a.take<float>(3 * (size_t)B);
  D.q = a.take<float>(4 * (size_t)B);
  D.v = a.take<float>(3 * (size_t)B);
  D.w = a.take<float>(3 * (size_t)B);
  D.x0 = a.take<float>(3 * (size_t)B);
  D.z0 = a.take<float>(3 * (size_t)B);
  D.f = a.take<float>(3 * (size_t)B);
  D.flags = a.take<int32_t>(B);
  D.f_steps = a.take<int32_t>(B);
  D.ep = a.take<EpState>(E);
  D.mv_off = a.take<int32_t>(E + 1);
  D.mv_block = a.take<int32_t>(M);
  D.mv_axis = a.take<int32_t>(M);
  D.mv_remove = a.take<int32_t>(M);
  D.mv_push = a.take<int32_t>(M);
  D.mv_settle = a.take<int32_t>(M);
  D.mv_sign = a.take<float>(M);
  D.mv_factor = a.take<float>(M);
  D.mv_k = a.take<float>(M);
  for (int k = 0; k < 2; ++k) {
    ContactBuf& c = D.buf[k];
    c.nat_key = a.take<uint32_t>(P);
    c.nat_feat = a.take<uint32_t>(P);
    c.nat_slot = a.take<uint32_t>(P);
    c.nat_pt = a.take<float>((size_t)P * kMaxPts * kNatPtFloats);
    c.nat_pf = a.take<float>((size_t)P * kNatPairFloats);
    c.srt_f = a.take<float>((size_t)P * kPairStride);
    c.srt_ab = a.take<uint32_t>(P);
    c.srt_np = a.take<int32_t>(P);
    c.srt_pt = a.take<float>((size_t)P * kPtStride);
    c.nat_x = a.take<float>((size_t)P * kMaxPts * kFeatures);
  }
  if (persist) *persist = (a.off + 255) & ~size_t(255);
  D.acc = a.take<float>((size_t)P * kAccFloats);
  D.work_counter = a.take<int32_t>(kMaxSizeClasses);
  int32_t* c = a.take<int32_t>(6 * (size_t)std::max(B, 1));
  jb_episode_stats* s = a.take<jb_episode_stats>(E);
  if (cmd) *cmd = c;
  if (stats) *stats = s;
  return (a.off + 255) & ~size_t(255);
}

bool sizes_of(int32_t E, const int32_t* body_off, int32_t max_moves, Sizes& z, std::vector<int64_t>* poff) {
  if (E <= 0 || !body_off || body_off[0] != 0 || max_moves < 0) return false;
  z.E = E;
  z.M = max_moves;
  z.nb_max = 0;
  z.P = 0;
  if (poff) poff->assign(E + 1, 0);
  for (int e = 0; e < E; ++e) {
    int nb = body_off[e + 1] - body_off[e];
    if (nb < 0 || nb > 4000) return false;
    z.nb_max = std::max(z.nb_max, nb);
    z.P += pair_capacity(nb);
    if (poff) (*poff)[e + 1] = z.P;
  }
  z.B = body_off[E];
  z.pc_max = pair_capacity(z.nb_max);
  return true;
}

Params to_params(const jb_solver_params* p) {
  Params q;
  q.dt = p->dt;
  q.n_sub = p->n_sub;
  q.pgs_iters = p->pgs_iters;
  q.residual_tol = p->residual_tol;
  q.pgs_iter_cap = p->pgs_iter_cap;
  q.pgs_min_iters = p->pgs_min_iters;
  q.residual_every = p->residual_every;
  q.restitution = p->restitution;
  q.beta = p->beta;
  q.slop = p->slop;
  q.contact_margin = p->contact_margin;
  q.aabb_eps = p->aabb_eps;
  for (int k = 0; k < 3; ++k) q.g[k] = p->gravity[k];
  q.warm_start = p->warm_start;
  q.match_radius = p->match_radius;
  q.fall_frac = p->fall_frac;
  q.collapse_ek = p->collapse_ek;
  q.collapse_cos = cosf(p->collapse_theta_deg * 3.14159265358979f / 180.f);
  q.rest_ek = p->rest_ek;
  q.rest_steps = p->rest_steps;
  q.sor = p->sor > 0.f ? p->sor : 1.f;
  q.sweep_order = p->sweep_order;
  q.residual_every_max = p->residual_every_max > p->residual_every ? p->residual_every_max : p->residual_every;
  q.stall_window = p->stall_window;
  q.friction_cone = p->friction_cone;
  q.restitution_newton = p->restitution_newton;
  q.accel_period = p->pgs_accel_period;
  q.colour_key = p->colour_key;
  {
    const float g = sqrtf(p->gravity[0] * p->gravity[0] + p->gravity[1] * p->gravity[1] + p->gravity[2] * p->gravity[2]);
    q.restitution_vmin = p->restitution_vmin > 0.f ? p->restitution_vmin : 2.f * g * p->dt / (float)p->n_sub;
  }
  return q;
}

const char* check_params(const jb_solver_params* p) {
  if (!(p->dt > 0.f)) return "dt must be > 0";
  if (p->n_sub < 1) return "n_sub must be >= 1";
  if (p->residual_tol < 0.f) return "residual_tol must be >= 0";
  if (p->residual_tol == 0.f && p->pgs_iters < 0) return "pgs_iters must be >= 0";
  if (p->residual_tol > 0.f && p->pgs_iter_cap < 1) return "pgs_iter_cap must be >= 1";
  if (p->pgs_min_iters < 1) return "pgs_min_iters must be >= 1";
  if (p->residual_every < 1) return "residual_every must be >= 1";
  if (!(p->contact_margin >= 0.f) || !(p->aabb_eps >= p->contact_margin))
    return "need 0 <= contact_margin <= aabb_eps";
  if (p->warm_start < 0 || p->warm_start > 3) return "warm_start must be 0, 1, 2 or 3";
  if (!(p->sor >= 0.f && p->sor < 2.f)) return "sor must be in (0, 2) (0 selects 1)";
  if (p->sweep_order < 0 || p->sweep_order > 1) return "sweep_order must be 0 or 1";
  if (p->residual_every_max < 0) return "residual_every_max must be >= 0";
  if (p->stall_window < 0) return "stall_window must be >= 0";
  if (p->friction_cone < 0 || p->friction_cone > 1) return "friction_cone must be 0 or 1";
  if (p->restitution_newton < 0 || p->restitution_newton > 1) return "restitution_newton must be 0 or 1";
  if (p->pgs_accel_period < 0) return "pgs_accel_period must be >= 0";
  if (p->colour_key < 0 || p->colour_key > 1) return "colour_key must be 0 or 1";
  return nullptr;
}

unsigned grid_of(int n, int t) { return (unsigned)((n + t - 1) / t); }

// The episode kernel's dynamic shared-memory limit is a property of the
// kernel, shared by every batch in the process.  It only ever grows, so a
// batch created later with smaller towers cannot invalidate the launches of
// an earlier one.  Per device (the attribute is per context).
cudaError_t raise_episode_smem_limit(int bytes) {
  static std::mutex mu;
  static int limit[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int& cur = limit[dev & 63];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(episode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

extern "C" {

void jb_default_params(jb_solver_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->dt = 1.f / 240.f;
  p->n_sub = 1;
  p->pgs_iters = 20;
  p->residual_tol = 0.f;
  p->pgs_iter_cap = 20000;
  p->pgs_min_iters = 1;
  p->residual_every = 4;
  p->sor = 1.f;
  p->sweep_order = 0;
  p->residual_every_max = 32;
  p->restitution = 0.10f;
  p->beta = 0.35f;
  p->slop = 4e-4f;
  p->contact_margin = 1e-3f;
  p->aabb_eps = 2e-3f;
  p->gravity[2] = -9.81f;
  p->warm_start = 1;
  p->match_radius = 2e-3f;
  p->fall_frac = 0.5f;
  p->collapse_ek = 5e-5f;
  p->collapse_theta_deg = 30.f;
  p->rest_ek = 1e-7f;
  p->rest_steps = 400;
}

const char* jb_version(void) { return "jb 0.1 sm_103a"; }

const char* jb_status_str(jb_status s) {
  switch (s) {
    case JB_OK: return "ok";
    case JB_EINVAL: return "invalid argument";
    case JB_ENOMEM: return "workspace too small";
    case JB_ECUDA: return "CUDA error";
    case JB_ERANGE: return "index out of range";
    case JB_ESTATE: return "invalid state";
    default: return "unknown status";
  }
}

const char* jb_last_error(void) { return g_err; }

jb_status jb_tower_layout(const jb_tower_desc* t, int32_t E, int32_t* body_off) {
  if (!t || !body_off || E <= 0) return fail(JB_EINVAL, "jb_tower_layout: null pointer or E <= 0");
  body_off[0] = 0;
  for (int e = 0; e < E; ++e) {
    if (t[e].levels < 1 || t[e].per_level < 1) return fail(JB_EINVAL, "tower %d: bad shape", e);
    body_off[e + 1] = body_off[e] + t[e].levels * t[e].per_level;
  }
  return JB_OK;
}

jb_status jb_tower_init(const jb_tower_desc* t, int32_t E, uint64_t seed, const int32_t* body_off, float* half,
                        float* mass, float* mu, float* x, float* q, float* ground_mu) {
  if (!t || !body_off || !half || !mass || !mu || !x || !q || !ground_mu || E <= 0)
    return fail(JB_EINVAL, "jb_tower_init: null pointer or E <= 0");
  const int B = body_off[E];
  const float c = sqrtf(0.5f);
  for (int e = 0; e < E; ++e) {
    const jb_tower_desc& T = t[e];
    if (body_off[e + 1] - body_off[e] != T.levels * T.per_level) return fail(JB_EINVAL, "tower %d: body_off mismatch", e);
    float L = T.dims[0], W = T.dims[1], H = T.dims[2];
    ground_mu[e] = T.mu_s;
    for (int lev = 0; lev < T.levels; ++lev)
      for (int s = 0; s < T.per_level; ++s) {
        int i = lev * T.per_level + s, g = body_off[e] + i;
        half[g] = L / 2; half[B + g] = W / 2; half[2 * B + g] = H / 2;
        double off = (s - (T.per_level - 1) / 2.0) * W;
        double z = lev * (double)H + H / 2.0;
        bool along_x = lev % 2 == 0;
        x[g] = along_x ? 0.f : (float)off;
        x[B + g] = along_x ? (float)off : 0.f;
        x[2 * B + g] = (float)z;
        q[g] = along_x ? 1.f : c; q[B + g] = 0.f; q[2 * B + g] = 0.f; q[3 * B + g] = along_x ? 0.f : c;
        uint64_t key = seed ^ ((uint64_t)e * 0x9E3779B97F4A7C15ull) ^ (1ull << 48) ^ (uint64_t)i;
        double u = (double)(splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
        mass[g] = (float)(T.mass * (1.0 + T.mass_jitter * (2.0 * u - 1.0)));
        mu[g] = T.mu_s;
      }
  }
  return JB_OK;
}

size_t jb_workspace_bytes(int32_t E, const int32_t* body_off, const jb_solver_params* p, int32_t max_moves) {
  Sizes z;
  if (!p || !sizes_of(E, body_off, max_moves, z, nullptr)) return 0;
  Dev D;
  return carve(nullptr, z, D, nullptr, nullptr, nullptr);
}

jb_status jb_batch_create(const jb_scene* sc, const jb_solver_params* p, int32_t max_moves, void* d_ws, size_t bytes,
                          void* stream, jb_batch** out) {
  if (!sc || !p || !out || !d_ws) return fail(JB_EINVAL, "jb_batch_create: null argument");
  *out = nullptr;
  if (const char* m = check_params(p)) return fail(JB_EINVAL, "jb_batch_create: %s", m);
  if (!sc->half || !sc->mass || !sc->mu || !sc->x || !sc->q || !sc->ground_mu)
    return fail(JB_EINVAL, "jb_batch_create: scene has a null array");
  if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) return fail(JB_EINVAL, "workspace must be 256-byte aligned");
  Sizes z;
  std::vector<int64_t> poff;
  if (!sizes_of(sc->n_episodes, sc->body_off, max_moves, z, &poff))
    return fail(JB_EINVAL, "jb_batch_create: bad n_episodes/body_off/max_moves");
  for (int e = 0; e < z.E; ++e)
    if (sc->body_off[e + 1] < sc->body_off[e]) return fail(JB_EINVAL, "body_off must be non-decreasing");
  for (int b = 0; b < z.B; ++b)
    for (int k = 0; k < 3; ++k)
      if (!(sc->half[k * z.B + b] > 0.f)) return fail(JB_EINVAL, "body %d: half extents must be > 0", b);
  jb_batch* bt = new jb_batch();
  size_t need = carve(static_cast<unsigned char*>(d_ws), z, bt->D, &bt->persist_bytes, &bt->cmd, &bt->stats);
  if (bytes < need) {
    delete bt;
    return fail(JB_ENOMEM, "workspace too small: %zu < %zu bytes", bytes, need);
  }
  Dev& D = bt->D;
  D.E = z.E; D.B = z.B; D.nb_max = z.nb_max; D.pc_max = z.pc_max;
  D.P = to_params(p);
  D.ps = smem_pairs(z.nb_max, z.pc_max);
  SmemPlan sp = smem_plan(z.nb_max, z.pc_max, D.ps);
  D.smem_per_warp = sp.bytes;
  bt->stream = static_cast<cudaStream_t>(stream);
  bt->ws = static_cast<unsigned char*>(d_ws);
  bt->ws_bytes = bytes;
  bt->E = z.E; bt->B = z.B; bt->max_moves = max_moves;
  bt->body_off.assign(sc->body_off, sc->body_off + z.E + 1);
  bt->pair_off = poff;
  bt->has_protocol = false;
  // larger towers first: the persistent grid then finishes the long ones early
  std::vector<int32_t> order(z.E);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return sc->body_off[a + 1] - sc->body_off[a] > sc->body_off[b + 1] - sc->body_off[b];
  });
  std::vector<float> zeros3(3 * (size_t)z.B, 0.f);
  cudaStream_t s = bt->stream;
  auto fin = [&](jb_status st) { if (st != JB_OK) delete bt; return st; };
#define CUF(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return fin(fail(JB_ECUDA, "%s: %s", #call, cudaGetErrorString(e_))); } while (0)
  int dev = 0, nsm = 0;
  CUF(cudaGetDevice(&dev));
  CUF(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int smem_max = 0;
  CUF(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // size classes: a new class starts where a tower has at most half the
  // bodies of the current class's largest (order is size-descending)
  {
    const float factor = p->smem_pair_factor > 0.f ? p->smem_pair_factor : 4.f;
    int smem_all = 0;
    for (int i = 0; i < z.E;) {
      jb_batch::SizeClass k{};
      k.first = i;
      k.nb_max = sc->body_off[order[i] + 1] - sc->body_off[order[i]];
      int j = i;
      const bool last = (int)bt->cls.size() == kMaxSizeClasses - 1;
      while (j < z.E && (last || 2 * (sc->body_off[order[j] + 1] - sc->body_off[order[j]]) > k.nb_max)) ++j;
      k.count = j - i;
      k.pc_max = pair_capacity(k.nb_max);
      k.ps = std::min(k.pc_max, (int)(factor * k.nb_max) + 16);
      // very tall towers: keep fewer pairs on chip (steps with more pairs
      // solve from the global copy) so that one episode still fits
      while (k.ps > 0 && kWarpsPerCta * smem_plan(k.nb_max, k.pc_max, k.ps).bytes > smem_max)
        k.ps = std::max(0, k.ps - 16);
      k.smem = kWarpsPerCta * smem_plan(k.nb_max, k.pc_max, k.ps).bytes;
      smem_all = std::max(smem_all, k.smem);
      bt->cls.push_back(k);
      i = j;
    }
    if (smem_all > smem_max)
      return fin(fail(JB_EINVAL, "towers too large for shared memory (%d > %d bytes)", smem_all, smem_max));
    CUF(raise_episode_smem_limit(smem_all));
    for (auto& k : bt->cls) {
      int oc = 0;
      CUF(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, episode_kernel, kWarpsPerCta * 32, k.smem));
      if (oc < 1) return fin(fail(JB_EINVAL, "episode kernel cannot be resident with %d bytes of shared memory", k.smem));
      k.grid = std::max(1, std::min((int)grid_of(k.count, kWarpsPerCta), oc * nsm));
      if (bt->cls.size() > 1) {
        CUF(cudaStreamCreateWithFlags(&k.stream, cudaStreamNonBlocking));
        CUF(cudaEventCreateWithFlags(&k.join, cudaEventDisableTiming));
      }
    }
    if (bt->cls.size() > 1) CUF(cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming));
  }
  const size_t fb = sizeof(float);
  CUF(cudaMemcpyAsync((void*)D.body_off, sc->body_off, sizeof(int32_t) * (z.E + 1), cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync((void*)D.pair_off, poff.data(), sizeof(int64_t) * (z.E + 1), cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync((void*)D.order, order.data(), sizeof(int32_t) * z.E, cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync(D.half, sc->half, 3 * fb * z.B, cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync(D.mass, sc->mass, fb * z.B, cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync(D.mu, sc->mu, fb * z.B, cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync((void*)D.ground_mu, sc->ground_mu, fb * z.E, cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync(D.x, sc->x, 3 * fb * z.B, cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync(D.q, sc->q, 4 * fb * z.B, cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync(D.v, sc->v ? sc->v : zeros3.data(), 3 * fb * z.B, cudaMemcpyHostToDevice, s));
  CUF(cudaMemcpyAsync(D.w, sc->w ? sc->w : zeros3.data(), 3 * fb * z.B, cudaMemcpyHostToDevice, s));
  CUF(cudaMemsetAsync(D.mv_off, 0, sizeof(int32_t) * (z.E + 1), s));
  if (z.B > 0) init_bodies_kernel<<<grid_of(z.B, 256), 256, 0, s>>>(D);
  init_episodes_kernel<<<grid_of(z.E, 256), 256, 0, s>>>(D);
  CUF(cudaGetLastError());
  // zeros3 must outlive the async copies
  CUF(cudaStreamSynchronize(s));
#undef CUF
  *out = bt;
  return JB_OK;
}

void jb_batch_destroy(jb_batch* b) { delete b; }

jb_status jb_set_warmstart_mlp(jb_batch* b, const void* d_mlp) {
  if (!b) return fail(JB_EINVAL, "jb_set_warmstart_mlp: null batch");
  b->D.mlp = static_cast<const unsigned char*>(d_mlp);
  return JB_OK;
}

jb_status jb_set_recorder(jb_batch* b, float* d_rows, int32_t capacity, int32_t* d_count, int32_t every) {
  if (!b) return fail(JB_EINVAL, "jb_set_recorder: null batch");
  if (capacity < 0 || every < 0) return fail(JB_EINVAL, "jb_set_recorder: negative capacity or period");
  if (capacity > 0 && (!d_rows || !d_count || every < 1)) return fail(JB_EINVAL, "jb_set_recorder: null buffer");
  b->D.rec = capacity > 0 ? d_rows : nullptr;
  b->D.rec_count = capacity > 0 ? d_count : nullptr;
  b->D.rec_cap = capacity;
  b->D.rec_every = every > 0 ? every : 1;
  return JB_OK;
}

jb_status jb_set_recorder_points(jb_batch* b, int32_t unmatched_only) {
  if (!b) return fail(JB_EINVAL, "jb_set_recorder_points: null batch");
  if (unmatched_only < 0 || unmatched_only > 1) return fail(JB_EINVAL, "jb_set_recorder_points: 0 or 1");
  b->D.rec_unmatched = unmatched_only;
  return JB_OK;
}

jb_status jb_set_params(jb_batch* b, const jb_solver_params* p) {
  if (!b || !p) return fail(JB_EINVAL, "jb_set_params: null argument");
  if (const char* m = check_params(p)) return fail(JB_EINVAL, "jb_set_params: %s", m);
  b->D.P = to_params(p);
  return JB_OK;
}

jb_status jb_set_protocol(jb_batch* b, const jb_protocol* pr) {
  if (!b || !pr || !pr->off) return fail(JB_EINVAL, "jb_set_protocol: null argument");
  const int E = b->E;
  if (pr->off[0] != 0) return fail(JB_EINVAL, "protocol off[0] must be 0");
  for (int e = 0; e < E; ++e)
    if (pr->off[e + 1] < pr->off[e]) return fail(JB_EINVAL, "protocol offsets must be non-decreasing");
  const int M = pr->off[E];
  if (M > b->max_moves) return fail(JB_ENOMEM, "protocol has %d moves, batch was created for %d", M, b->max_moves);
  if (M > 0 && (!pr->block || !pr->axis || !pr->sign || !pr->factor || !pr->k || !pr->remove || !pr->push_steps ||
                !pr->settle_steps))
    return fail(JB_EINVAL, "jb_set_protocol: null move array");
  for (int e = 0; e < E; ++e) {
    int nb = b->body_off[e + 1] - b->body_off[e];
    for (int m = pr->off[e]; m < pr->off[e + 1]; ++m) {
      if (pr->block[m] < 0 || pr->block[m] >= nb) return fail(JB_ERANGE, "episode %d move %d: block %d out of range", e, m, pr->block[m]);
      if (pr->axis[m] != JB_AXIS_X && pr->axis[m] != JB_AXIS_Y) return fail(JB_EINVAL, "move %d: bad axis", m);
      if (pr->push_steps[m] < 0 || pr->settle_steps[m] < 0) return fail(JB_EINVAL, "move %d: negative duration", m);
    }
  }
  Dev& D = b->D;
  cudaStream_t s = b->stream;
  CU(cudaMemcpyAsync(D.mv_off, pr->off, sizeof(int32_t) * (E + 1), cudaMemcpyHostToDevice, s));
  if (M > 0) {
    CU(cudaMemcpyAsync(D.mv_block, pr->block, 4 * M, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(D.mv_axis, pr->axis, 4 * M, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(D.mv_sign, pr->sign, 4 * M, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(D.mv_factor, pr->factor, 4 * M, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(D.mv_k, pr->k, 4 * M, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(D.mv_remove, pr->remove, 4 * M, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(D.mv_push, pr->push_steps, 4 * M, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(D.mv_settle, pr->settle_steps, 4 * M, cudaMemcpyHostToDevice, s));
  }
  protocol_start_kernel<<<grid_of(E, 256), 256, 0, s>>>(D);
  CU(cudaGetLastError());
  // the host arrays may be released by the caller after return
  CU(cudaStreamSynchronize(s));
  b->has_protocol = true;
  return JB_OK;
}

static jb_status launch_episodes(jb_batch* b, int mode, int n) {
  Dev& D = b->D;
  if (D.P.warm_start >= 2 && !D.mlp)
    return fail(JB_ESTATE, "learned warm start selected but no network set (jb_set_warmstart_mlp)");
  cudaStream_t s = b->stream;
  const bool multi = b->cls.size() > 1;
  CU(cudaMemsetAsync(D.work_counter, 0, sizeof(int32_t) * kMaxSizeClasses, s));
  if (multi) CU(cudaEventRecord(b->fork, s));
  for (size_t c = 0; c < b->cls.size(); ++c) {
    const auto& k = b->cls[c];
    Dev Dc = D;
    Dc.E = k.count;
    Dc.order = D.order + k.first;
    Dc.nb_max = k.nb_max;
    Dc.pc_max = k.pc_max;
    Dc.ps = k.ps;
    Dc.smem_per_warp = k.smem / kWarpsPerCta;
    Dc.work_counter = D.work_counter + c;
    cudaStream_t ks = multi ? k.stream : s;
    if (multi) CU(cudaStreamWaitEvent(ks, b->fork, 0));
    episode_kernel<<<k.grid, kWarpsPerCta * 32, k.smem, ks>>>(Dc, mode, n);
    CU(cudaGetLastError());
    if (multi) {
      CU(cudaEventRecord(k.join, ks));
      CU(cudaStreamWaitEvent(s, k.join, 0));
    }
  }
  return JB_OK;
}

jb_status jb_run_protocol(jb_batch* b, int32_t max_steps) {
  if (!b) return fail(JB_EINVAL, "jb_run_protocol: null batch");
  if (max_steps < 0) return fail(JB_EINVAL, "max_steps must be >= 0");
  if (!b->has_protocol) return fail(JB_ESTATE, "jb_run_protocol: no protocol set");
  if (max_steps == 0) return JB_OK;
  return launch_episodes(b, kModeProtocol, max_steps);
}

jb_status jb_step(jb_batch* b, int32_t n) {
  if (!b) return fail(JB_EINVAL, "jb_step: null batch");
  if (n < 0) return fail(JB_EINVAL, "n_steps must be >= 0");
  if (n == 0) return JB_OK;
  return launch_episodes(b, kModeFree, n);
}

static jb_status check_targets(jb_batch* b, int n, const int32_t* ep, const int32_t* blk) {
  if (n < 0 || n > b->B) return fail(JB_EINVAL, "command count %d out of range", n);
  if (n > 0 && (!ep || !blk)) return fail(JB_EINVAL, "null command array");
  for (int i = 0; i < n; ++i) {
    if (ep[i] < 0 || ep[i] >= b->E) return fail(JB_ERANGE, "episode %d out of range", ep[i]);
    int nb = b->body_off[ep[i] + 1] - b->body_off[ep[i]];
    if (blk[i] < 0 || blk[i] >= nb) return fail(JB_ERANGE, "block %d out of range in episode %d", blk[i], ep[i]);
  }
  return JB_OK;
}

jb_status jb_apply_push(jb_batch* b, int32_t n, const int32_t* ep, const int32_t* blk, const int32_t* axis,
                        const float* force, const int32_t* steps) {
  if (!b) return fail(JB_EINVAL, "jb_apply_push: null batch");
  if (jb_status st = check_targets(b, n, ep, blk)) return st;
  if (n == 0) return JB_OK;
  if (!axis || !force || !steps) return fail(JB_EINVAL, "jb_apply_push: null array");
  for (int i = 0; i < n; ++i) {
    if (axis[i] != JB_AXIS_X && axis[i] != JB_AXIS_Y) return fail(JB_EINVAL, "bad axis");
    if (steps[i] < 0) return fail(JB_EINVAL, "negative step count");
  }
  cudaStream_t s = b->stream;
  int32_t* c = b->cmd;
  CU(cudaMemcpyAsync(c, ep, 4 * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(c + n, blk, 4 * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(c + 2 * n, axis, 4 * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(c + 3 * n, force, 4 * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(c + 4 * n, steps, 4 * n, cudaMemcpyHostToDevice, s));
  push_kernel<<<grid_of(n, 128), 128, 0, s>>>(b->D, n, c, c + n, c + 2 * n, reinterpret_cast<const float*>(c + 3 * n), c + 4 * n);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return JB_OK;
}

jb_status jb_remove_block(jb_batch* b, int32_t n, const int32_t* ep, const int32_t* blk) {
  if (!b) return fail(JB_EINVAL, "jb_remove_block: null batch");
  if (jb_status st = check_targets(b, n, ep, blk)) return st;
  if (n == 0) return JB_OK;
  cudaStream_t s = b->stream;
  CU(cudaMemcpyAsync(b->cmd, ep, 4 * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(b->cmd + n, blk, 4 * n, cudaMemcpyHostToDevice, s));
  remove_kernel<<<grid_of(n, 128), 128, 0, s>>>(b->D, n, b->cmd, b->cmd + n);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return JB_OK;
}

jb_status jb_size_classes(const jb_batch* b, int32_t* n_classes, int32_t* episodes, int32_t* max_bodies,
                          int32_t* grid) {
  if (!b || !n_classes) return fail(JB_EINVAL, "jb_size_classes: null argument");
  *n_classes = (int32_t)b->cls.size();
  for (size_t c = 0; c < b->cls.size(); ++c) {
    if (episodes) episodes[c] = b->cls[c].count;
    if (max_bodies) max_bodies[c] = b->cls[c].nb_max;
    if (grid) grid[c] = (int32_t)b->cls[c].grid;
  }
  return JB_OK;
}

jb_status jb_sync(jb_batch* b, int32_t* n_bad) {
  if (!b) return fail(JB_EINVAL, "jb_sync: null batch");
  CU(cudaStreamSynchronize(b->stream));
  if (n_bad) {
    std::vector<EpState> st(b->E);
    CU(cudaMemcpyAsync(st.data(), b->D.ep, sizeof(EpState) * b->E, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    int bad = 0;
    for (auto& s : st) bad += s.status != 0;
    *n_bad = bad;
  }
  return JB_OK;
}

jb_status jb_read_state(jb_batch* b, float* x, float* q, float* v, float* w, int32_t device_ptrs) {
  if (!b) return fail(JB_EINVAL, "jb_read_state: null batch");
  cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t n3 = 3 * sizeof(float) * b->B;
  cudaStream_t s = b->stream;
  if (x) CU(cudaMemcpyAsync(x, b->D.x, n3, k, s));
  if (q) CU(cudaMemcpyAsync(q, b->D.q, 4 * sizeof(float) * b->B, k, s));
  if (v) CU(cudaMemcpyAsync(v, b->D.v, n3, k, s));
  if (w) CU(cudaMemcpyAsync(w, b->D.w, n3, k, s));
  if (!device_ptrs) CU(cudaStreamSynchronize(s));
  return JB_OK;
}

jb_status jb_write_state(jb_batch* b, const float* x, const float* q, const float* v, const float* w,
                         int32_t device_ptrs, int32_t clear_cache, int32_t reset_reference) {
  if (!b) return fail(JB_EINVAL, "jb_write_state: null batch");
  cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t n3 = 3 * sizeof(float) * b->B;
  cudaStream_t s = b->stream;
  if (x) CU(cudaMemcpyAsync(b->D.x, x, n3, k, s));
  if (q) CU(cudaMemcpyAsync(b->D.q, q, 4 * sizeof(float) * b->B, k, s));
  if (v) CU(cudaMemcpyAsync(b->D.v, v, n3, k, s));
  if (w) CU(cudaMemcpyAsync(b->D.w, w, n3, k, s));
  if (b->B > 0 && reset_reference) reset_reference_kernel<<<grid_of(b->B, 256), 256, 0, s>>>(b->D);
  if (clear_cache) clear_cache_kernel<<<grid_of(b->E, 256), 256, 0, s>>>(b->D);
  CU(cudaGetLastError());
  if (!device_ptrs) CU(cudaStreamSynchronize(s));
  return JB_OK;
}

jb_status jb_read_active(jb_batch* b, int32_t* active) {
  if (!b || !active) return fail(JB_EINVAL, "jb_read_active: null argument");
  std::vector<int32_t> fl(b->B);
  CU(cudaMemcpyAsync(fl.data(), b->D.flags, 4 * (size_t)b->B, cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < b->B; ++i) active[i] = (fl[i] & kActive) ? 1 : 0;
  return JB_OK;
}

jb_status jb_read_contacts(jb_batch* b, int32_t e, jb_contact* out, int32_t cap, int32_t* n_out) {
  if (!b || !n_out) return fail(JB_EINVAL, "jb_read_contacts: null argument");
  if (e < 0 || e >= b->E) return fail(JB_ERANGE, "episode %d out of range", e);
  if (cap > 0 && !out) return fail(JB_EINVAL, "jb_read_contacts: null output with cap > 0");
  cudaStream_t s = b->stream;
  EpState st;
  CU(cudaMemcpyAsync(&st, b->D.ep + e, sizeof st, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  const int64_t po = b->pair_off[e];
  const ContactBuf& c = b->D.buf[st.cur];
  const int np = st.npairs;
  std::vector<uint32_t> key(np), feat(np), slot(np);
  std::vector<float> pt((size_t)np * kMaxPts * kNatPtFloats), pf((size_t)np * kNatPairFloats);
  if (np > 0) {
    CU(cudaMemcpyAsync(key.data(), c.nat_key + po, 4 * np, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(feat.data(), c.nat_feat + po, 4 * np, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(slot.data(), c.nat_slot + po, 4 * np, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(pt.data(), c.nat_pt + po * kMaxPts * kNatPtFloats, 4 * pt.size(), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(pf.data(), c.nat_pf + po * kNatPairFloats, 4 * pf.size(), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
  }
  int n = 0;
  for (int p = 0; p < np; ++p) {
    int a = (int)(key[p] >> 16) - 1, bb = (int)(key[p] & 0xffff);
    uint32_t f = feat[p];
    int npt = f >> 24;
    for (int k = 0; k < npt; ++k, ++n) {
      if (n >= cap) continue;
      jb_contact& o = out[n];
      o.a = a; o.b = bb;
      o.axis = f & 0xff; o.ref_face = (f >> 8) & 0xff; o.inc_face = (f >> 16) & 0xff; o.point = k;
      const float* q = pt.data() + ((size_t)p * kMaxPts + k) * kNatPtFloats;
      for (int j = 0; j < 3; ++j) {
        o.p[j] = q[j];
        o.n[j] = pf[kNatPairFloats * p + j];
        o.t1[j] = pf[kNatPairFloats * p + 4 + j];
        o.lambda[j] = q[7 + j];
      }
      o.depth = q[3];
    }
  }
  *n_out = n;
  return JB_OK;
}

jb_status jb_read_episode_stats(jb_batch* b, jb_episode_stats* out) {
  if (!b || !out) return fail(JB_EINVAL, "jb_read_episode_stats: null argument");
  cudaStream_t s = b->stream;
  stats_kernel<<<grid_of(b->E, 128), 128, 0, s>>>(b->D, b->stats);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(out, b->stats, sizeof(jb_episode_stats) * b->E, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return JB_OK;
}

jb_status jb_reference_episode(jb_batch* b, int32_t n_hat, int32_t* episode, int32_t* n_removed) {
  if (!b || !episode) return fail(JB_EINVAL, "jb_reference_episode: null argument");
  std::vector<jb_episode_stats> st(b->E);
  if (jb_status s = jb_read_episode_stats(b, st.data())) return s;
  std::vector<int32_t> act(b->B);
  if (jb_status s = jb_read_active(b, act.data())) return s;
  int best = -1, best_d = 0, best_r = 0;
  for (int e = 0; e < b->E; ++e) {
    if (!st[e].collapsed) continue;
    int r = 0;
    for (int i = b->body_off[e]; i < b->body_off[e + 1]; ++i) r += act[i] == 0;
    const int d = r > n_hat ? r - n_hat : n_hat - r;
    if (best < 0 || d < best_d) { best = e; best_d = d; best_r = r; }
  }
  if (best < 0) {   // nothing collapsed: the episode with the most rounds
    for (int e = 0; e < b->E; ++e)
      if (best < 0 || st[e].moves_done > st[best].moves_done) best = e;
    best_r = 0;
    if (best >= 0)
      for (int i = b->body_off[best]; i < b->body_off[best + 1]; ++i) best_r += act[i] == 0;
  }
  *episode = best;
  if (n_removed) *n_removed = best_r;
  return JB_OK;
}

size_t jb_state_bytes(const jb_batch* b) { return b ? b->persist_bytes : 0; }

jb_status jb_save_state(jb_batch* b, void* host, size_t bytes) {
  if (!b || !host) return fail(JB_EINVAL, "jb_save_state: null argument");
  if (bytes < b->persist_bytes) return fail(JB_ENOMEM, "snapshot buffer too small: %zu < %zu", bytes, b->persist_bytes);
  CU(cudaMemcpyAsync(host, b->ws, b->persist_bytes, cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  return JB_OK;
}

jb_status jb_load_state(jb_batch* b, const void* host, size_t bytes) {
  if (!b || !host) return fail(JB_EINVAL, "jb_load_state: null argument");
  if (bytes != b->persist_bytes) return fail(JB_EINVAL, "snapshot size %zu does not match batch (%zu)", bytes, b->persist_bytes);
  CU(cudaMemcpyAsync(b->ws, host, b->persist_bytes, cudaMemcpyHostToDevice, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  b->has_protocol = true;
  return JB_OK;
}


// ------------------------------------------------- no-allocation stepping
// Scratch for jb_step_noalloc: a fixed device array that lives as long as the
// library is loaded on a device.  Host code must not use the symbol as an
// address; it asks the runtime for the device address once per device.
static __device__ __align__(256) unsigned char jb_static_scratch[JB_NOALLOC_SCRATCH_BYTES];

static std::mutex g_scratch_mutex;
static void* g_scratch_addr[256];

// Device address of jb_static_scratch on the current device (looked up on the
// first call per device).
static jb_status static_scratch_address(void** out) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(JB_ECUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, jb_static_scratch);
    if (err != cudaSuccess || !p)
      return fail(JB_ECUDA, "cudaGetSymbolAddress(jb_static_scratch) failed: %s", cudaGetErrorString(err));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return JB_OK;
}

jb_status jb_step_noalloc(int32_t n_episodes, const int32_t* body_off, const float* d_half, const float* d_mass,
                          const float* d_mu, const float* d_ground_mu, float* d_x, float* d_q, float* d_v,
                          float* d_w, const jb_solver_params* p, int32_t n_steps, void* cuda_stream) {
  if (!body_off || !d_half || !d_mass || !d_mu || !d_ground_mu || !d_x || !d_q || !d_v || !d_w || !p)
    return fail(JB_EINVAL, "jb_step_noalloc: null argument");
  if (n_steps < 0) return fail(JB_EINVAL, "jb_step_noalloc: n_steps must be >= 0");
  if (const char* m = check_params(p)) return fail(JB_EINVAL, "jb_step_noalloc: %s", m);
  if (p->warm_start >= 2)
    return fail(JB_EINVAL, "jb_step_noalloc: warm_start %d needs a network block; this call runs plain PGS "
                           "(warm_start 0 or 1)", p->warm_start);
  Sizes z;
  if (!sizes_of(n_episodes, body_off, 0, z, nullptr))
    return fail(JB_EINVAL, "jb_step_noalloc: bad n_episodes/body_off");
  for (int e = 0; e < z.E; ++e)
    if (body_off[e + 1] < body_off[e]) return fail(JB_EINVAL, "jb_step_noalloc: body_off must be non-decreasing");
  Dev D;
  memset(&D, 0, sizeof D);
  const size_t need = carve(nullptr, z, D, nullptr, nullptr, nullptr);
  if (need > (size_t)JB_NOALLOC_SCRATCH_BYTES)
    return fail(JB_ENOMEM, "jb_step_noalloc: this batch needs %zu bytes of scratch, the static scratch holds %u",
                need, (unsigned)JB_NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  if (jb_status st = static_scratch_address(&base)) return st;   // first call per device: the lookup
  if (n_steps == 0) return JB_OK;
  carve(static_cast<unsigned char*>(base), z, D, nullptr, nullptr, nullptr);
  D.E = z.E; D.B = z.B; D.nb_max = z.nb_max; D.pc_max = z.pc_max;
  D.P = to_params(p);
  D.ps = smem_pairs(z.nb_max, z.pc_max);
  D.smem_per_warp = smem_plan(z.nb_max, z.pc_max, D.ps).bytes;
  D.order = nullptr;   // episodes in index order
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, nsm = 0, occ = 0, smem_max = 0;
  const int smem = kWarpsPerCta * D.smem_per_warp;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > smem_max) return fail(JB_EINVAL, "towers too large for shared memory (%d > %d bytes)", smem, smem_max);
  CU(raise_episode_smem_limit(smem));
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, episode_kernel, kWarpsPerCta * 32, smem));
  if (occ < 1) return fail(JB_EINVAL, "episode kernel cannot be resident with %d bytes of shared memory", smem);
  const unsigned grid = (unsigned)std::max(1, std::min((int)grid_of(z.E, kWarpsPerCta), occ * nsm));
  const size_t fb = sizeof(float);
  // inputs into the scratch copy of the batch layout; everything that must
  // start at zero is written by the init kernels (the array keeps the last
  // call's contents)
  CU(cudaMemcpyAsync((void*)D.body_off, body_off, sizeof(int32_t) * (z.E + 1), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(D.half, d_half, 3 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(D.mass, d_mass, fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(D.mu, d_mu, fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync((void*)D.ground_mu, d_ground_mu, fb * z.E, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(D.x, d_x, 3 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(D.q, d_q, 4 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(D.v, d_v, 3 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(D.w, d_w, 3 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemsetAsync(D.mv_off, 0, sizeof(int32_t) * (z.E + 1), s));
  pair_offsets_kernel<<<1, 1, 0, s>>>(D, const_cast<int64_t*>(D.pair_off));
  if (z.B > 0) init_bodies_kernel<<<grid_of(z.B, 256), 256, 0, s>>>(D);
  init_episodes_kernel<<<grid_of(z.E, 256), 256, 0, s>>>(D);
  CU(cudaMemsetAsync(D.work_counter, 0, sizeof(int32_t), s));
  episode_kernel<<<grid, kWarpsPerCta * 32, smem, s>>>(D, kModeFree, n_steps);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(d_x, D.x, 3 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(d_q, D.q, 4 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(d_v, D.v, 3 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(d_w, D.w, 3 * fb * z.B, cudaMemcpyDeviceToDevice, s));
  return JB_OK;
}

}  // extern "C"
