"""FP64 CPU oracle (test infrastructure only).

ctypes wrapper over ``jb_oracle.c``.  Only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import this package; the product path
(the CUDA library and its binding) never does.

The shared library is compiled from source on first use (gcc, -O2, OpenMP
over episodes) and kept beside the source, git-ignored.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "jb_oracle.c")
LIB = os.path.join(HERE, "libjb_oracle.so")

NSTAT = 17
CREC = 55
STAT_NAMES = ["status", "collapsed", "resting", "n_fallen", "com_imbalance", "kinetic",
              "last_residual", "last_sweeps", "total_sweeps", "solves", "steps", "body_steps",
              "phase", "moves_done", "n_pairs", "n_points", "max_residual"]
PH_FREE, PH_PUSH, PH_SETTLE, PH_REST, PH_DONE = range(5)

_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle shared library (idempotent)."""
    with _lock:
        stale = (not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "jb_oracle.h"))))
        if force or stale:
            tmp = LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
                                   "-o", tmp, SRC, "-lm"])
            os.replace(tmp, LIB)
    return LIB


class _Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_sub", C.c_int), ("pgs_iters", C.c_int),
                ("residual_tol", C.c_double), ("pgs_iter_cap", C.c_int),
                ("pgs_min_iters", C.c_int), ("restitution", C.c_double), ("beta", C.c_double),
                ("slop", C.c_double), ("contact_margin", C.c_double), ("aabb_eps", C.c_double),
                ("gravity", C.c_double * 3), ("warm_start", C.c_int),
                ("match_radius", C.c_double), ("fall_frac", C.c_double),
                ("collapse_ek", C.c_double), ("collapse_theta_deg", C.c_double),
                ("rest_ek", C.c_double), ("rest_steps", C.c_int), ("friction_cone", C.c_int),
                ("restitution_newton", C.c_int), ("restitution_vmin", C.c_double), ("colour_order", C.c_int),
                ("pgs_accel_period", C.c_int), ("sat_tie", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        vp = C.c_void_p
        L.or_create.restype = vp
        L.or_create.argtypes = [C.c_int, ip, dp, dp, dp, dp, dp, dp, dp, dp, C.POINTER(_Params)]
        L.or_destroy.argtypes = [vp]
        L.or_set_protocol.argtypes = [vp, ip, ip, ip, dp, dp, dp, ip, ip, ip]
        L.or_run_protocol.argtypes = [vp, C.c_int, C.c_int]
        L.or_step.argtypes = [vp, C.c_int, C.c_int]
        L.or_apply_push.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int]
        L.or_remove_block.argtypes = [vp, C.c_int, C.c_int]
        L.or_get_state.argtypes = [vp, dp, dp, dp, dp]
        L.or_set_state.argtypes = [vp, dp, dp, dp, dp]
        L.or_clear_cache.argtypes = [vp]
        L.or_get_contacts.argtypes = [vp, C.c_int, dp, C.c_int]
        L.or_get_stats.argtypes = [vp, dp]
        L.or_collapse_terms.argtypes = [vp, C.c_int, dp, dp, dp, ip]
        L.or_reference_episode.argtypes = [vp, C.c_int, ip]
        L.or_com_imbalance.argtypes = [vp, C.c_int]
        L.or_com_imbalance.restype = C.c_double
        L.or_active.argtypes = [vp, C.c_int]
        L.or_sat.argtypes = [dp, dp, dp, dp, dp, dp, C.c_double, dp, ip, ip, dp, dp]
        L.or_sat_select.argtypes = [dp, ip, dp]
        L.or_pair_manifold.argtypes = [dp, dp, dp, dp, dp, dp, C.c_double, dp]
        L.or_ground_manifold.argtypes = [dp, dp, dp, C.c_double, dp]
        L.or_rotmat.argtypes = [dp, dp]
        L.or_body_inertia.argtypes = [C.c_double, dp, dp]
        L.or_set_recorder.argtypes = [vp, dp, C.c_int, C.c_int]
        L.or_recorded.argtypes = [vp]
        L.or_recorded.restype = C.c_long
        L.or_support_margin.argtypes = [C.c_int, dp, dp]
        L.or_support_margin.restype = C.c_double
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def make_params(p: dict) -> _Params:
    out = _Params()
    for name, _ in _Params._fields_:
        val = p[name]
        if name == "gravity":
            out.gravity = (C.c_double * 3)(*val)
        else:
            setattr(out, name, val)
    return out


class World:
    """An oracle batch of episodes built from a synth.Scene."""

    def __init__(self, scene, params: dict):
        L = lib()
        self.E = scene.n_episodes
        self.B = scene.n_bodies
        self.params = dict(params)
        self._keep = [_i(scene.body_off), _d(scene.half), _d(scene.mass), _d(scene.mu),
                      _d(scene.x), _d(scene.q), _d(scene.v), _d(scene.w), _d(scene.ground_mu)]
        self._p = make_params(params)
        self.h = L.or_create(self.E, *[k[1] for k in self._keep], C.byref(self._p))
        self.body_off = np.asarray(scene.body_off)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    def set_protocol(self, prot):
        args = [_i(prot.off), _i(prot.block), _i(prot.axis), _d(prot.sign), _d(prot.factor),
                _d(prot.k), _i(prot.remove), _i(prot.push_steps), _i(prot.settle_steps)]
        self._prot_keep = args
        rc = lib().or_set_protocol(self.h, *[a[1] for a in args])
        if rc != 0:
            raise ValueError("bad protocol")

    def run_protocol(self, max_steps=10 ** 9, threads=0):
        return lib().or_run_protocol(self.h, max_steps, threads)

    def step(self, n=1, threads=0):
        lib().or_step(self.h, n, threads)

    def apply_push(self, e, block, axis, force, n_steps):
        return lib().or_apply_push(self.h, e, block, axis, force, n_steps)

    def remove_block(self, e, block):
        return lib().or_remove_block(self.h, e, block)

    def state(self):
        x = np.zeros((3, self.B)); q = np.zeros((4, self.B))
        v = np.zeros((3, self.B)); w = np.zeros((3, self.B))
        lib().or_get_state(self.h, *[_d(a)[1] for a in (x, q, v, w)])
        return x, q, v, w

    def set_state(self, x, q, v, w):
        arrs = [_d(a) for a in (x, q, v, w)]
        lib().or_set_state(self.h, *[a[1] for a in arrs])

    def set_recorder(self, capacity, every=1):
        """Record (features, converged impulses) rows; returns the buffer."""
        self._rec = np.zeros((max(capacity, 1), 27))
        lib().or_set_recorder(self.h, self._rec.ctypes.data_as(C.POINTER(C.c_double)), int(capacity), int(every))
        return self._rec

    def recorded(self):
        n = lib().or_recorded(self.h)
        return self._rec[:min(n, len(self._rec))]

    def clear_cache(self):
        lib().or_clear_cache(self.h)

    def contacts(self, e):
        L = lib()
        n = L.or_get_contacts(self.h, e, None, 0)
        out = np.zeros((max(n, 1), CREC))
        L.or_get_contacts(self.h, e, out.ctypes.data_as(C.POINTER(C.c_double)), n)
        return out[:n]

    def stats(self):
        out = np.zeros((self.E, NSTAT))
        lib().or_get_stats(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        return {name: out[:, i].copy() for i, name in enumerate(STAT_NAMES)}

    def collapse_terms(self, e):
        """(kinetic J, max displacement / block length, max tilt rad, fallen count)."""
        ek, dx, th = (np.zeros(1) for _ in range(3))
        nf = np.zeros(1, np.int32)
        lib().or_collapse_terms(self.h, e, ek.ctypes.data_as(C.POINTER(C.c_double)),
                                dx.ctypes.data_as(C.POINTER(C.c_double)), th.ctypes.data_as(C.POINTER(C.c_double)),
                                nf.ctypes.data_as(C.POINTER(C.c_int)))
        return float(ek[0]), float(dx[0]), float(th[0]), int(nf[0])

    def reference_episode(self, n_hat):
        r = np.zeros(1, np.int32)
        e = lib().or_reference_episode(self.h, int(n_hat), r.ctypes.data_as(C.POINTER(C.c_int)))
        return int(e), int(r[0])

    def com_imbalance(self, e):
        return lib().or_com_imbalance(self.h, e)

    def active(self):
        return np.array([lib().or_active(self.h, g) for g in range(self.B)], bool)


def sat(xA, qA, hA, xB, qB, hB, margin=1e-3):
    """Stage entry point: SAT over 15 axes for one OBB pair."""
    L = lib()
    arrs = [_d(a) for a in (xA, qA, hA, xB, qB, hB)]
    delta = np.zeros(15); valid = np.zeros(15, np.int32); axis = np.zeros(1, np.int32)
    n = np.zeros(3); dmin = np.zeros(1)
    hit = L.or_sat(*[a[1] for a in arrs], margin, delta.ctypes.data_as(C.POINTER(C.c_double)),
                   valid.ctypes.data_as(C.POINTER(C.c_int)), axis.ctypes.data_as(C.POINTER(C.c_int)),
                   n.ctypes.data_as(C.POINTER(C.c_double)), dmin.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(hit=bool(hit), delta=delta, valid=valid.astype(bool), axis=int(axis[0]), n=n, dmin=float(dmin[0]))


def sat_select(delta, valid):
    """Stage entry point: the SAT axis choice (tolerant ties, edge rule) on
    given separations of the 15 axes; returns (axis, dmin)."""
    d = np.ascontiguousarray(delta, np.float64)
    v = np.ascontiguousarray(valid, np.int32)
    dmin = np.zeros(1)
    ax = lib().or_sat_select(d.ctypes.data_as(C.POINTER(C.c_double)), v.ctypes.data_as(C.POINTER(C.c_int)),
                             dmin.ctypes.data_as(C.POINTER(C.c_double)))
    return int(ax), float(dmin[0])


def sat_decisions_clear(scene, margin=1e-3, eps=3e-7, trials=300, seed=0):
    """True when no discrete contact decision of the scene's box pairs is
    within eps of flipping: no pair separation within 10 eps of -margin, and
    no pair whose chosen SAT axis changes when its 15 separations move by
    up to +-eps (random sign patterns).  Inputs that pass have the same
    contact features in any precision whose separation error is below eps."""
    rng = np.random.default_rng(seed)
    P = rng.integers(-1, 2, (trials, 15)) * eps
    X, Q, H = (np.asarray(getattr(scene, k), np.float64) for k in ("x", "q", "half"))
    bo = scene.body_off
    for e in range(len(bo) - 1):
        for a in range(bo[e], bo[e + 1]):
            for b in range(a + 1, bo[e + 1]):
                r = sat(X[:, a], Q[:, a], H[:, a], X[:, b], Q[:, b], H[:, b], margin)
                if abs(r["dmin"] + margin) < 10 * eps:
                    return False
                if r["hit"] and any(sat_select(r["delta"] + p, r["valid"])[0] != r["axis"] for p in P):
                    return False
    return True


def _crec_dict(rec):
    npnt = int(rec[5])
    pts = rec[15:15 + 40].reshape(4, 10)[:npnt]
    return dict(a=int(rec[0]), b=int(rec[1]), axis=int(rec[2]), ref_face=int(rec[3]),
                inc_face=int(rec[4]), np=npnt, n=rec[6:9].copy(), t1=rec[9:12].copy(),
                delta=rec[12], mu=rec[13], depth_max=rec[14], p=pts[:, 0:3].copy(),
                depth=pts[:, 3].copy(), lam=pts[:, 4:7].copy(), local=pts[:, 7:10].copy())


def pair_manifold(xA, qA, hA, xB, qB, hB, margin=1e-3):
    L = lib()
    arrs = [_d(a) for a in (xA, qA, hA, xB, qB, hB)]
    out = np.zeros(CREC)
    L.or_pair_manifold(*[a[1] for a in arrs], margin, out.ctypes.data_as(C.POINTER(C.c_double)))
    return _crec_dict(out)


def ground_manifold(x, q, h, margin=1e-3):
    L = lib()
    arrs = [_d(a) for a in (x, q, h)]
    out = np.zeros(CREC)
    L.or_ground_manifold(*[a[1] for a in arrs], margin, out.ctypes.data_as(C.POINTER(C.c_double)))
    return _crec_dict(out)


def contact_dicts(recs):
    return [_crec_dict(r) for r in recs]


def rotmat(q):
    R = np.zeros(9)
    lib().or_rotmat(_d(q)[1], R.ctypes.data_as(C.POINTER(C.c_double)))
    return R.reshape(3, 3)


def body_inertia(mass, half):
    I = np.zeros(3)
    lib().or_body_inertia(mass, _d(half)[1], I.ctypes.data_as(C.POINTER(C.c_double)))
    return I


def support_margin(xy, com):
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    return lib().or_support_margin(len(xy), _d(xy)[1], _d(com)[1])


def num_threads():
    return lib().or_num_threads()
