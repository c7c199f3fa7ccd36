"""Seeded synthetic inputs for block-tower collapse episodes.

This module is the only code shared by the FP64 oracle tests and the CUDA
path.  It builds *inputs* (initial tower poses, per-block masses and friction
coefficients, and the push/removal schedule of every episode) and holds none
of the method's arithmetic: no collision detection, no contact solve, no
integration, no force thresholds.

Tower layout (paper Sec. 3.1: 3 blocks per layer, alternating perpendicular
layers): flush, zero gaps, bottom face on z = 0.  Levels are numbered from the
ground; 0-based level k has its long axis along world X when k is even and
along world Y when k is odd.  Slot s in {0, 1, 2} sits at offset (s - 1) * W
across the long axis, so slot 1 is the middle block.  Block id = 3 * level +
slot.  Body frame: x = length, y = width, z = thickness.

Random draws use SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) as a counter-based generator:
u = splitmix64(seed ^ episode * GOLDEN ^ (stream << 48) ^ index) >> 11, scaled
to [0, 1).  Masses carry a seeded +-jitter; the push schedule (which block,
which axis, which sign, which force factor) is drawn here and handed to both
implementations as plain arrays.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# draw streams
S_MASS, S_NREM, S_BLOCK, S_AXIS, S_SIGN, S_FORCE, S_LEVEL, S_SLOT, S_MU, S_HEIGHT = range(1, 11)

# push axis codes (block-local): 0 = block X (width axis), 1 = block Y (long axis)
AXIS_X, AXIS_Y = 0, 1


def splitmix64(x):
    """SplitMix64 output function applied to state x (uint64 array or scalar)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def u01(seed, episode, stream, index):
    """Counter-based uniform draw in [0, 1) (53-bit)."""
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) ^ (np.asarray(episode, dtype=np.uint64) * GOLDEN)
               ^ (np.uint64(stream) << np.uint64(48)) ^ np.asarray(index, dtype=np.uint64))
    z = splitmix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Tower:
    levels: int = 18
    per_level: int = 3
    dims: tuple = (0.075, 0.025, 0.015)   # L, W, H in metres
    mass: float = 0.015                   # kg
    mass_jitter: float = 0.02             # +- fraction, uniform
    mu: float = 0.40


@dataclass
class Scene:
    """Structure-of-arrays initial state, episodes concatenated (CSR offsets)."""
    body_off: np.ndarray      # int32 [E+1]
    half: np.ndarray          # float32 [3, B] half extents
    mass: np.ndarray          # float32 [B]  (0 = static)
    mu: np.ndarray            # float32 [B]
    x: np.ndarray             # float32 [3, B]
    q: np.ndarray             # float32 [4, B]  (w, x, y, z)
    v: np.ndarray             # float32 [3, B]
    w: np.ndarray             # float32 [3, B]
    ground_mu: np.ndarray     # float32 [E]

    @property
    def n_episodes(self):
        return len(self.body_off) - 1

    @property
    def n_bodies(self):
        return int(self.body_off[-1])


@dataclass
class Protocol:
    """Per-episode push/removal schedule (CSR over moves)."""
    off: np.ndarray           # int32 [E+1]
    block: np.ndarray         # int32 [M] episode-local body index
    axis: np.ndarray          # int32 [M] AXIS_X / AXIS_Y
    sign: np.ndarray          # float32 [M] +-1
    factor: np.ndarray        # float32 [M] multiple of the threshold force
    k: np.ndarray             # float32 [M] threshold multiplier (F = factor*k*mu*m*g)
    remove: np.ndarray        # int32 [M] 1 = delete the block after the push
    push_steps: np.ndarray    # int32 [M]
    settle_steps: np.ndarray  # int32 [M]


def tower_bodies(t: Tower, seed: int, episode: int):
    """Initial poses and masses of one tower (float32)."""
    # tower parameters are single precision, as in the C tower descriptor
    L, W, H = (float(np.float32(d)) for d in t.dims)
    m0, jit = float(np.float32(t.mass)), float(np.float32(t.mass_jitter))
    n = t.levels * t.per_level
    half = np.empty((3, n), np.float32)
    x = np.zeros((3, n), np.float32)
    q = np.zeros((4, n), np.float32)
    c = np.float32(np.sqrt(0.5))
    for lev in range(t.levels):
        for s in range(t.per_level):
            i = lev * t.per_level + s
            half[:, i] = (L / 2, W / 2, H / 2)
            off = (s - (t.per_level - 1) / 2.0) * W
            z = lev * H + H / 2
            if lev % 2 == 0:
                x[:, i] = (0.0, off, z)
                q[:, i] = (1.0, 0.0, 0.0, 0.0)
            else:
                x[:, i] = (off, 0.0, z)
                q[:, i] = (c, 0.0, 0.0, c)     # +90 degrees about z
    u = u01(seed, episode, S_MASS, np.arange(n))
    mass = (m0 * (1.0 + jit * (2.0 * u - 1.0))).astype(np.float32)
    return half, x, q, mass


def build_scene(towers, seed: int) -> Scene:
    parts = [tower_bodies(t, seed, e) for e, t in enumerate(towers)]
    counts = [p[0].shape[1] for p in parts]
    off = np.zeros(len(towers) + 1, np.int32)
    off[1:] = np.cumsum(counts)
    half = np.concatenate([p[0] for p in parts], axis=1)
    x = np.concatenate([p[1] for p in parts], axis=1)
    q = np.concatenate([p[2] for p in parts], axis=1)
    mass = np.concatenate([p[3] for p in parts])
    mu = np.concatenate([np.full(c, t.mu, np.float32) for c, t in zip(counts, towers)])
    B = int(off[-1])
    return Scene(off, np.ascontiguousarray(half), mass, mu, np.ascontiguousarray(x),
                 np.ascontiguousarray(q), np.zeros((3, B), np.float32),
                 np.zeros((3, B), np.float32), np.array([t.mu for t in towers], np.float32))


def custom_scene(boxes, ground_mu=0.4) -> Scene:
    """One episode from explicit boxes: list of dicts with keys half, x, q, mass, mu
    (and optionally v, w).  mass 0 marks a static box."""
    n = len(boxes)
    f = lambda key, dim, default: np.array(
        [np.asarray(b.get(key, default), np.float64).reshape(dim) for b in boxes],
        np.float32).T.reshape(dim, n) if n else np.zeros((dim, 0), np.float32)
    half = f("half", 3, None)
    x = f("x", 3, None)
    q = f("q", 4, (1, 0, 0, 0))
    v = f("v", 3, (0, 0, 0))
    w = f("w", 3, (0, 0, 0))
    mass = np.array([b["mass"] for b in boxes], np.float32)
    mu = np.array([b.get("mu", ground_mu) for b in boxes], np.float32)
    return Scene(np.array([0, n], np.int32), np.ascontiguousarray(half), mass, mu,
                 np.ascontiguousarray(x), np.ascontiguousarray(q), np.ascontiguousarray(v),
                 np.ascontiguousarray(w), np.array([ground_mu], np.float32))


def concat_scenes(scenes) -> Scene:
    offs = [0]
    for s in scenes:
        offs.append(offs[-1] + s.n_bodies)
    cat = lambda a: np.ascontiguousarray(np.concatenate([getattr(s, a) for s in scenes], axis=-1))
    return Scene(np.array(offs, np.int32), cat("half"), cat("mass"), cat("mu"), cat("x"),
                 cat("q"), cat("v"), cat("w"), cat("ground_mu"))


def _protocol(moves, n_episodes) -> Protocol:
    off = np.zeros(n_episodes + 1, np.int32)
    for e in range(n_episodes):
        off[e + 1] = off[e] + len(moves[e])
    flat = [m for ms in moves for m in ms]
    col = lambda i, dt: np.array([m[i] for m in flat], dt)
    return Protocol(off, col(0, np.int32), col(1, np.int32), col(2, np.float32),
                    col(3, np.float32), col(4, np.float32), col(5, np.int32),
                    col(6, np.int32), col(7, np.int32))


def threshold_k(slot, axis, rule="axis"):
    """The Sec. 5 threshold multiplier k of a push (F = k mu_s m g).
    rule "axis": 3 along block Y, 4 along block X, whatever the slot (the
    friction workload's schedule).  rule "ziglar": Tab. ziglar's move
    classes: side_yaxis and center_xaxis 3, side_xaxis 4 (the torque move);
    a centre block pulled along Y meets the same friction as along X (its own
    weight and the layer above on the layer below), so 3 as well."""
    if rule == "ziglar":
        return 4.0 if (axis == AXIS_X and slot != 1) else 3.0
    return 3.0 if axis == AXIS_Y else 4.0


def removal_protocol(towers, seed, push_steps=120, settle_steps=240, max_removals=8, k_rule="axis"):
    """Removal rounds: 1..max_removals removals of non-top blocks, each pushed
    along block X or Y at factor ~ U[0.8, 1.5] of the threshold (threshold_k
    with k_rule), then deleted, then a settle period."""
    moves = []
    for e, t in enumerate(towers):
        n_rem = 1 + int(u01(seed, e, S_NREM, 0) * max_removals)
        live = list(range((t.levels - 1) * t.per_level))   # non-top blocks
        ms = []
        for r in range(n_rem):
            if not live:
                break
            idx = int(u01(seed, e, S_BLOCK, r) * len(live))
            blk = live.pop(idx)
            axis = AXIS_X if u01(seed, e, S_AXIS, r) < 0.5 else AXIS_Y
            sign = 1.0 if u01(seed, e, S_SIGN, r) < 0.5 else -1.0
            factor = 0.8 + 0.7 * float(u01(seed, e, S_FORCE, r))
            k = threshold_k(blk % t.per_level, axis, k_rule)
            ms.append((blk, axis, sign, factor, k, 1, push_steps, settle_steps))
        moves.append(ms)
    return _protocol(moves, len(towers))


# ---------------------------------------------------------------------------
# Workloads.  Solver parameters are plain dicts (keys as in jb_solver_params).

BASE_PARAMS = dict(dt=1.0 / 240.0, n_sub=1, pgs_iters=20, residual_tol=0.0,
                   pgs_iter_cap=1000, pgs_min_iters=1, restitution=0.10, beta=0.35,
                   slop=4e-4, contact_margin=1e-3, aabb_eps=2e-3,
                   gravity=(0.0, 0.0, -9.81), warm_start=1, match_radius=2e-3,
                   fall_frac=0.5, collapse_ek=5e-5, collapse_theta_deg=30.0,
                   rest_ek=1e-7, rest_steps=400, friction_cone=0,
                   restitution_newton=0, restitution_vmin=0.0, colour_order=0,
                   pgs_accel_period=0, sat_tie=0.0)


def params(**kw):
    p = dict(BASE_PARAMS)
    p.update(kw)
    return p


def single_push_workload(seed=0):
    """One 18-level tower (54 blocks), mu 0.40; push the middle block of level 9
    along block Y at 1.05 x threshold (k = 3) for 0.5 s, no deletion, 2 s total."""
    towers = [Tower(mu=0.40)]
    scene = build_scene(towers, seed)
    blk = 8 * 3 + 1
    prot = _protocol([[(blk, AXIS_Y, 1.0, 1.05, 3.0, 0, 120, 360)]], 1)
    return scene, prot, params(pgs_iters=20)


def ziglar_x_rig(mu, dims=(0.075, 0.025, 0.015), mass=0.015, n=1):
    """The top two levels of a tower on a static base (Sec. 5.3's X-axis
    withdrawal): level 0 static (mass 0) along world Y, level 1 (the pushed
    level, bodies 3-5, body 3 the side block at y = -W) along world X, level
    2 (bodies 6-8) along world Y; exact masses (no jitter), mu on every block
    and the ground.  n copies as n episodes."""
    L, W, H = dims
    qy = (float(np.cos(np.pi / 4)), 0.0, 0.0, float(np.sin(np.pi / 4)))
    boxes = []
    for s in range(3):
        boxes.append(dict(half=(L / 2, W / 2, H / 2), x=((s - 1) * W, 0.0, H / 2), q=qy, mass=0.0, mu=mu))
    for s in range(3):
        boxes.append(dict(half=(L / 2, W / 2, H / 2), x=(0.0, (s - 1) * W, 1.5 * H), mass=mass, mu=mu))
    for s in range(3):
        boxes.append(dict(half=(L / 2, W / 2, H / 2), x=((s - 1) * W, 0.0, 2.5 * H), q=qy, mass=mass, mu=mu))
    one = custom_scene(boxes, ground_mu=mu)
    return one if n == 1 else concat_scenes([one] * n)


def friction_workload(seed=1, per_mu=150, mus=(0.25, 0.40, 0.60), k_rule="axis"):
    """450 episodes (150 per mu), 18 levels, removal rounds, 30 sweeps (mode F)
    or residual mode; k_rule as in threshold_k."""
    towers = [Tower(mu=m) for m in mus for _ in range(per_mu)]
    return build_scene(towers, seed), removal_protocol(towers, seed, k_rule=k_rule), params(pgs_iters=30)


def ragged_workload(seed=2, n=4096):
    """n episodes, levels ~ U{6..30}, mu ~ U[0.2, 0.7], removal rounds."""
    towers = []
    for e in range(n):
        lv = 6 + int(u01(seed, e, S_HEIGHT, 0) * 25)
        mu = 0.2 + 0.5 * float(u01(seed, e, S_MU, 0))
        towers.append(Tower(levels=lv, mu=np.float32(mu).item()))
    return build_scene(towers, seed), removal_protocol(towers, seed), params(pgs_iters=30)


def stress_workload(seed=5, n=16384):
    """n x 48-level towers, mu cycling {0.25, 0.40, 0.60}; one X push at 2 x
    threshold (k = 4) on a level ~ U{10..30}, random slot and sign; 720 steps."""
    mus = (0.25, 0.40, 0.60)
    towers = [Tower(levels=48, mu=mus[e % 3]) for e in range(n)]
    moves = []
    for e in range(n):
        lev = 9 + int(u01(seed, e, S_LEVEL, 0) * 21)        # 0-based 9..29
        slot = int(u01(seed, e, S_SLOT, 0) * 3)
        sign = 1.0 if u01(seed, e, S_SIGN, 0) < 0.5 else -1.0
        moves.append([(3 * lev + slot, AXIS_X, sign, 2.0, 4.0, 0, 120, 600)])
    return build_scene(towers, seed), _protocol(moves, n), params()


def subthreshold_workload(seed=11, n=100, levels=6, push_steps=60, settle_steps=120):
    """n towers, mu ~ U[0.25, 0.6]; one push of the middle block of a level in
    1..levels-2 along block Y or X at factor ~ U[0.5, 0.9] of its Tab. ziglar
    threshold (a centre block: k = 3 on either axis), not removed.  Below the
    thresholds nothing should slide out or topple."""
    towers, moves = [], []
    for e in range(n):
        mu = 0.25 + 0.35 * float(u01(seed, e, S_MU, 0))
        towers.append(Tower(levels=levels, mu=np.float32(mu).item()))
        lev = 1 + int(u01(seed, e, S_LEVEL, 0) * (levels - 2))
        axis = AXIS_X if u01(seed, e, S_AXIS, 0) < 0.5 else AXIS_Y
        sign = 1.0 if u01(seed, e, S_SIGN, 0) < 0.5 else -1.0
        factor = 0.5 + 0.4 * float(u01(seed, e, S_FORCE, 0))
        k = threshold_k(1, axis, "ziglar")
        moves.append([(3 * lev + 1, axis, sign, factor, k, 0, push_steps, settle_steps)])
    return build_scene(towers, seed), _protocol(moves, n), params(residual_tol=1e-5, pgs_iter_cap=20000)


def subset(scene: Scene, prot: Protocol, episodes):
    """Sub-batch of the given episodes (same per-episode inputs)."""
    episodes = list(episodes)
    bo = scene.body_off
    idx = np.concatenate([np.arange(bo[e], bo[e + 1]) for e in episodes]) if episodes else np.zeros(0, int)
    off = np.zeros(len(episodes) + 1, np.int32)
    off[1:] = np.cumsum([bo[e + 1] - bo[e] for e in episodes])
    s = Scene(off, np.ascontiguousarray(scene.half[:, idx]), scene.mass[idx], scene.mu[idx],
              np.ascontiguousarray(scene.x[:, idx]), np.ascontiguousarray(scene.q[:, idx]),
              np.ascontiguousarray(scene.v[:, idx]), np.ascontiguousarray(scene.w[:, idx]),
              scene.ground_mu[episodes])
    po = prot.off
    midx = np.concatenate([np.arange(po[e], po[e + 1]) for e in episodes]) if episodes else np.zeros(0, int)
    moff = np.zeros(len(episodes) + 1, np.int32)
    moff[1:] = np.cumsum([po[e + 1] - po[e] for e in episodes])
    p = Protocol(moff, *[getattr(prot, f)[midx] for f in
                         ("block", "axis", "sign", "factor", "k", "remove", "push_steps", "settle_steps")])
    return s, p


def pile_scene(n_boxes=24, seed=0, spread=0.09, height=0.06, dims=(0.075, 0.025, 0.015),
               mass=0.015, mu=0.4):
    """One episode of randomly oriented blocks scattered over a small region
    (many touching or slightly interpenetrating pairs, all contact kinds)."""
    idx = np.arange(n_boxes)
    ux, uy, uz = (u01(seed, 0, S_LEVEL + k, idx) for k in range(3))
    qv = np.stack([u01(seed, 0, S_SLOT + k, idx) * 2.0 - 1.0 for k in range(4)])
    qv /= np.linalg.norm(qv, axis=0, keepdims=True)
    boxes = []
    for i in range(n_boxes):
        boxes.append(dict(half=tuple(d / 2 for d in dims),
                          x=((ux[i] - 0.5) * spread, (uy[i] - 0.5) * spread, 0.012 + uz[i] * height),
                          q=tuple(qv[:, i]), mass=mass, mu=mu))
    return custom_scene(boxes, ground_mu=mu)


def perturbed(scene: Scene, seed: int, dx=3e-4, dang=0.01) -> Scene:
    """Copy of a scene with every pose jittered (translation +-dx, small rotation
    of about dang radians)."""
    B = scene.n_bodies
    idx = np.arange(B)
    d = np.stack([u01(seed, 1, S_LEVEL + k, idx) * 2 - 1 for k in range(3)]) * dx
    r = np.stack([u01(seed, 1, S_SLOT + k, idx) * 2 - 1 for k in range(3)]) * (dang / 2)
    q = scene.q.astype(np.float64)
    dq = np.vstack([np.ones(B), r])
    w1, x1, y1, z1 = dq
    w2, x2, y2, z2 = q
    nq = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                   w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    nq /= np.linalg.norm(nq, axis=0, keepdims=True)
    return Scene(scene.body_off.copy(), scene.half.copy(), scene.mass.copy(), scene.mu.copy(),
                 (scene.x + d).astype(np.float32), nq.astype(np.float32), scene.v.copy(),
                 scene.w.copy(), scene.ground_mu.copy())
