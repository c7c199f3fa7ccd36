"""Batched rigid-body step for block-tower collapse episodes on GB300 (sm_103a).

Thin ctypes binding over the C ABI in ``include/jb.h`` (``libjb.so``, built
in-tree by ``paper_2606_28394_gb300.build``).  The functions keep the C names
(``jb_batch_create``, ``jb_run_protocol``, ...) and only marshal arguments:
every step of the simulation runs in the library's CUDA kernels.  PyTorch is
used for device memory (the batch workspace) and for the current CUDA stream.

There is no CPU fallback: if ``libjb.so`` is missing, importing this package
raises ImportError.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjb.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python paper_2606_28394_gb300/build.py or __graft_entry__.build())")

_lib = C.CDLL(LIB_PATH)

JB_OK, JB_EINVAL, JB_ENOMEM, JB_ECUDA, JB_ERANGE, JB_ESTATE = 0, -1, -2, -3, -4, -5
JB_EP_CONTACT_OVERFLOW, JB_EP_NOT_CONVERGED, JB_EP_NONFINITE, JB_EP_TOO_MANY_COLOURS = 1, 2, 4, 8
JB_PH_FREE, JB_PH_PUSH, JB_PH_SETTLE, JB_PH_REST, JB_PH_DONE = range(5)
JB_AXIS_X, JB_AXIS_Y = 0, 1


class jb_solver_params(C.Structure):
    _fields_ = [("dt", C.c_float), ("n_sub", C.c_int32), ("pgs_iters", C.c_int32),
                ("residual_tol", C.c_float), ("pgs_iter_cap", C.c_int32),
                ("pgs_min_iters", C.c_int32), ("residual_every", C.c_int32),
                ("restitution", C.c_float), ("beta", C.c_float), ("slop", C.c_float),
                ("contact_margin", C.c_float), ("aabb_eps", C.c_float),
                ("gravity", C.c_float * 3), ("warm_start", C.c_int32),
                ("match_radius", C.c_float), ("fall_frac", C.c_float),
                ("collapse_ek", C.c_float), ("collapse_theta_deg", C.c_float),
                ("rest_ek", C.c_float), ("rest_steps", C.c_int32),
                ("smem_pair_factor", C.c_float), ("sor", C.c_float), ("sweep_order", C.c_int32),
                ("residual_every_max", C.c_int32), ("stall_window", C.c_int32),
                ("friction_cone", C.c_int32), ("restitution_newton", C.c_int32),
                ("restitution_vmin", C.c_float), ("pgs_accel_period", C.c_int32),
                ("colour_key", C.c_int32)]


_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)


class jb_scene(C.Structure):
    _fields_ = [("n_episodes", C.c_int32), ("body_off", _ip), ("half", _fp), ("mass", _fp),
                ("mu", _fp), ("x", _fp), ("q", _fp), ("v", _fp), ("w", _fp),
                ("ground_mu", _fp)]


class jb_tower_desc(C.Structure):
    _fields_ = [("levels", C.c_int32), ("per_level", C.c_int32), ("dims", C.c_float * 3),
                ("mass", C.c_float), ("mass_jitter", C.c_float), ("mu_s", C.c_float)]


class jb_protocol(C.Structure):
    _fields_ = [("off", _ip), ("block", _ip), ("axis", _ip), ("sign", _fp), ("factor", _fp),
                ("k", _fp), ("remove", _ip), ("push_steps", _ip), ("settle_steps", _ip)]


class jb_contact(C.Structure):
    _fields_ = [("a", C.c_int32), ("b", C.c_int32), ("axis", C.c_int32),
                ("ref_face", C.c_int32), ("inc_face", C.c_int32), ("point", C.c_int32),
                ("p", C.c_float * 3), ("n", C.c_float * 3), ("t1", C.c_float * 3),
                ("depth", C.c_float), ("lambda_", C.c_float * 3)]


class jb_episode_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("phase", C.c_int32), ("collapsed", C.c_int32),
                ("resting", C.c_int32), ("n_fallen", C.c_int32), ("moves_done", C.c_int32),
                ("n_pairs", C.c_int32), ("n_points", C.c_int32), ("last_sweeps", C.c_int32),
                ("steps", C.c_int32), ("max_colours", C.c_int32), ("capped_solves", C.c_int32),
                ("com_imbalance", C.c_float), ("kinetic", C.c_float),
                ("last_residual", C.c_float), ("max_residual", C.c_float),
                ("total_sweeps", C.c_double), ("solves", C.c_double),
                ("body_steps", C.c_double), ("point_sweeps", C.c_double),
                ("point_steps", C.c_double), ("pair_steps", C.c_double),
                ("bp_tests", C.c_double), ("mlp_points", C.c_double),
                ("stability_margin", C.c_float), ("min_stability_margin", C.c_float),
                ("first_unstable_step", C.c_int32), ("collapse_step", C.c_int32)]


_vp = C.c_void_p
_sig = {
    "jb_default_params": (None, [C.POINTER(jb_solver_params)]),
    "jb_tower_layout": (C.c_int32, [C.POINTER(jb_tower_desc), C.c_int32, _ip]),
    "jb_tower_init": (C.c_int32, [C.POINTER(jb_tower_desc), C.c_int32, C.c_uint64, _ip, _fp, _fp,
                                  _fp, _fp, _fp, _fp]),
    "jb_workspace_bytes": (C.c_size_t, [C.c_int32, _ip, C.POINTER(jb_solver_params), C.c_int32]),
    "jb_batch_create": (C.c_int32, [C.POINTER(jb_scene), C.POINTER(jb_solver_params), C.c_int32,
                                    _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "jb_batch_destroy": (None, [_vp]),
    "jb_set_params": (C.c_int32, [_vp, C.POINTER(jb_solver_params)]),
    "jb_set_protocol": (C.c_int32, [_vp, C.POINTER(jb_protocol)]),
    "jb_run_protocol": (C.c_int32, [_vp, C.c_int32]),
    "jb_apply_push": (C.c_int32, [_vp, C.c_int32, _ip, _ip, _ip, _fp, _ip]),
    "jb_remove_block": (C.c_int32, [_vp, C.c_int32, _ip, _ip]),
    "jb_step": (C.c_int32, [_vp, C.c_int32]),
    "jb_sync": (C.c_int32, [_vp, _ip]),
    "jb_size_classes": (C.c_int32, [_vp, _ip, _ip, _ip, _ip]),
    "jb_reference_episode": (C.c_int32, [_vp, C.c_int32, _ip, _ip]),
    "jb_read_state": (C.c_int32, [_vp, _vp, _vp, _vp, _vp, C.c_int32]),
    "jb_write_state": (C.c_int32, [_vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32]),
    "jb_read_active": (C.c_int32, [_vp, _ip]),
    "jb_read_contacts": (C.c_int32, [_vp, C.c_int32, C.POINTER(jb_contact), C.c_int32, _ip]),
    "jb_read_episode_stats": (C.c_int32, [_vp, C.POINTER(jb_episode_stats)]),
    "jb_state_bytes": (C.c_size_t, [_vp]),
    "jb_save_state": (C.c_int32, [_vp, _vp, C.c_size_t]),
    "jb_load_state": (C.c_int32, [_vp, _vp, C.c_size_t]),
    "jb_set_warmstart_mlp": (C.c_int32, [_vp, _vp]),
    "jb_set_recorder": (C.c_int32, [_vp, _vp, C.c_int32, _vp, C.c_int32]),
    "jb_set_recorder_points": (C.c_int32, [_vp, C.c_int32]),
    "jb_mlp_bytes": (C.c_size_t, []),
    "jb_mlp_param_count": (C.c_int32, []),
    "jb_mlp_scratch_bytes": (C.c_size_t, [C.c_int32]),
    "jb_mlp_load": (C.c_int32, [_vp, _fp, _vp]),
    "jb_mlp_save": (C.c_int32, [_vp, _fp, _vp]),
    "jb_mlp_forward": (C.c_int32, [_vp, _vp, C.c_int32, _vp, _vp, C.c_size_t, _vp]),
    "jb_mlp_grad": (C.c_int32, [_vp, _vp, _vp, C.c_int32, _vp, _vp, _vp, C.c_size_t, _vp]),
    "jb_mlp_scratch_error": (C.c_int32, [_vp, C.c_size_t, _vp, C.POINTER(C.c_int32)]),
    "jb_mlp_adamw": (C.c_int32, [_vp, _vp, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float,
                                 C.c_float, _vp]),
    "jb_mlp_train_step": (C.c_int32, [_vp, _vp, _vp, C.c_int32, C.c_int32, C.c_float, C.c_float,
                                      C.c_float, C.c_float, C.c_float, _vp, _vp, C.c_size_t, _vp]),
    "jb_step_noalloc": (C.c_int32, [C.c_int32, _ip, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                    C.POINTER(jb_solver_params), C.c_int32, _vp]),
    "jb_fma_probe": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32, _vp, _vp]),
    "jb_fma_probe_flops": (C.c_double, [C.c_int32, C.c_int32, C.c_int32]),
    "jb_status_str": (C.c_char_p, [C.c_int32]),
    "jb_last_error": (C.c_char_p, []),
    "jb_version": (C.c_char_p, []),
}
EXPORTS = tuple(_sig)
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class JBError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.jb_last_error().decode()
        super().__init__(f"{where}: {_lib.jb_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def check(status, where="jb"):
    if status != JB_OK:
        raise JBError(status, where)
    return status


# ------------------------------------------------------------------ helpers
def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pf(a):
    return a.ctypes.data_as(_fp)


def _pi(a):
    return a.ctypes.data_as(_ip)


def default_params(**kw) -> jb_solver_params:
    p = jb_solver_params()
    jb_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "gravity":
            p.gravity = (C.c_float * 3)(*v)
        elif hasattr(p, k):
            setattr(p, k, v)
    return p


def params_from_dict(d: dict) -> jb_solver_params:
    keys = {f for f, _ in jb_solver_params._fields_}
    return default_params(**{k: v for k, v in d.items() if k in keys})


class Batch:
    """A batch of episodes on the current CUDA device.

    The workspace is a torch uint8 tensor sized by jb_workspace_bytes; work is
    queued on ``stream`` (default: torch's current stream)."""

    def __init__(self, scene, params, max_moves=0, stream=None, device=None, workspace=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        if isinstance(params, dict):
            params = params_from_dict(params)
        self.params = params
        self.E = int(scene.n_episodes)
        self.B = int(scene.n_bodies)
        self._scene_arrays = [_i32(scene.body_off), _f32(scene.half), _f32(scene.mass),
                              _f32(scene.mu), _f32(scene.x), _f32(scene.q), _f32(scene.v),
                              _f32(scene.w), _f32(scene.ground_mu)]
        bo, half, mass, mu, x, q, v, w, gmu = self._scene_arrays
        self.body_off = bo
        nbytes = jb_workspace_bytes(self.E, _pi(bo), C.byref(params), int(max_moves))
        if nbytes == 0:
            raise JBError(JB_EINVAL, "jb_workspace_bytes")
        with torch.cuda.device(self.device):
            if workspace is not None and workspace.numel() >= nbytes + 256 and workspace.is_cuda:
                self.workspace = workspace
            else:
                self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream or torch.cuda.current_stream(self.device)
        ptr = self.workspace.data_ptr()
        self._ws_ptr = (ptr + 255) & ~255
        sc = jb_scene(self.E, _pi(bo), _pf(half), _pf(mass), _pf(mu), _pf(x), _pf(q), _pf(v),
                      _pf(w), _pf(gmu))
        h = C.c_void_p()
        check(jb_batch_create(C.byref(sc), C.byref(params), int(max_moves), C.c_void_p(self._ws_ptr),
                              nbytes, C.c_void_p(self.stream.cuda_stream), C.byref(h)),
              "jb_batch_create")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            jb_batch_destroy(h)
            self.h = None

    # -- schedule and stepping
    def set_params(self, params):
        """Replace the solver parameters (jb_set_params); smem_pair_factor is fixed at creation."""
        if isinstance(params, dict):
            params = params_from_dict(params)
        self.params = params
        check(jb_set_params(self.h, C.byref(params)), "jb_set_params")

    def set_protocol(self, prot):
        """Upload the push/removal schedule (CSR over episodes) and start every episode's first move."""
        arrs = [_i32(prot.off), _i32(prot.block), _i32(prot.axis), _f32(prot.sign),
                _f32(prot.factor), _f32(prot.k), _i32(prot.remove), _i32(prot.push_steps),
                _i32(prot.settle_steps)]
        pr = jb_protocol(_pi(arrs[0]), _pi(arrs[1]), _pi(arrs[2]), _pf(arrs[3]), _pf(arrs[4]),
                         _pf(arrs[5]), _pi(arrs[6]), _pi(arrs[7]), _pi(arrs[8]))
        check(jb_set_protocol(self.h, C.byref(pr)), "jb_set_protocol")

    def run_protocol(self, max_steps=1 << 30):
        """Run every unfinished episode through its schedule, at most max_steps steps, in one
        persistent launch per size class (asynchronous on the batch stream)."""
        check(jb_run_protocol(self.h, int(max_steps)), "jb_run_protocol")

    def step(self, n=1):
        """Advance every episode n steps with no schedule (host-driven; asynchronous)."""
        check(jb_step(self.h, int(n)), "jb_step")

    def apply_push(self, episode, block, axis, force, n_steps):
        """Constant force (N, signed) along a block's X (width) or Y (length) axis at its
        centre of mass for n_steps steps; arrays or scalars, episode-local block ids."""
        ep, bl, ax, st = (_i32(np.atleast_1d(a)) for a in (episode, block, axis, n_steps))
        f = _f32(np.atleast_1d(force))
        check(jb_apply_push(self.h, len(ep), _pi(ep), _pi(bl), _pi(ax), _pf(f), _pi(st)),
              "jb_apply_push")

    def remove_block(self, episode, block):
        """Take blocks out of the simulation (inactive from the next step)."""
        ep, bl = _i32(np.atleast_1d(episode)), _i32(np.atleast_1d(block))
        check(jb_remove_block(self.h, len(ep), _pi(ep), _pi(bl)), "jb_remove_block")

    def reference_episode(self, n_removed_hat):
        """(episode, removed blocks): the collapsed episode whose removed-block
        count is closest to n_removed_hat, else the one with the most rounds."""
        e, r = C.c_int32(0), C.c_int32(0)
        check(jb_reference_episode(self.h, int(n_removed_hat), C.byref(e), C.byref(r)), "jb_reference_episode")
        return e.value, r.value

    def size_classes(self):
        """[(episodes, largest body count, grid)] per size class (one
        episode-kernel launch each per step or protocol call)."""
        n = C.c_int32(0)
        e, nb, g = (np.zeros(4, np.int32) for _ in range(3))
        check(jb_size_classes(self.h, C.byref(n), _pi(e), _pi(nb), _pi(g)), "jb_size_classes")
        return [(int(e[i]), int(nb[i]), int(g[i])) for i in range(n.value)]

    def sync(self):
        """Wait for queued work; returns the number of episodes with a non-zero status."""
        n = C.c_int32(0)
        check(jb_sync(self.h, C.byref(n)), "jb_sync")
        return n.value

    # -- readback
    def state(self):
        """(x [3,B], q [4,B], v [3,B], w [3,B]) as float32 host arrays."""
        x = np.zeros((3, self.B), np.float32); q = np.zeros((4, self.B), np.float32)
        v = np.zeros((3, self.B), np.float32); w = np.zeros((3, self.B), np.float32)
        check(jb_read_state(self.h, x.ctypes.data, q.ctypes.data, v.ctypes.data, w.ctypes.data, 0),
              "jb_read_state")
        return x, q, v, w

    def write_state(self, x=None, q=None, v=None, w=None, clear_cache=False, reset_reference=False):
        """Overwrite any of x, q, v, w (host arrays); optionally forget the warm-start cache
        or take the new poses as the collapse reference."""
        arrs = [None if a is None else _f32(a) for a in (x, q, v, w)]
        ptrs = [None if a is None else a.ctypes.data for a in arrs]
        check(jb_write_state(self.h, *ptrs, 0, int(clear_cache), int(reset_reference)),
              "jb_write_state")

    def active(self):
        """Per-body flags: True while the body is in the simulation."""
        a = np.zeros(self.B, np.int32)
        check(jb_read_active(self.h, _pi(a)), "jb_read_active")
        return a.astype(bool)

    def contacts(self, episode):
        """The last substep's contact points of one episode (list of jb_contact)."""
        n = C.c_int32(0)
        check(jb_read_contacts(self.h, int(episode), None, 0, C.byref(n)), "jb_read_contacts")
        buf = (jb_contact * max(n.value, 1))()
        check(jb_read_contacts(self.h, int(episode), buf, n.value, C.byref(n)), "jb_read_contacts")
        return [buf[i] for i in range(n.value)]

    def stats(self):
        """Per-episode statistics as a dict of arrays (jb_episode_stats fields)."""
        buf = (jb_episode_stats * self.E)()
        check(jb_read_episode_stats(self.h, buf), "jb_read_episode_stats")
        out = {}
        for name, _ in jb_episode_stats._fields_:
            out[name] = np.array([getattr(buf[i], name) for i in range(self.E)])
        return out

    def save_state(self):
        """Snapshot of the batch's device state as a host byte array (jb_save_state)."""
        n = jb_state_bytes(self.h)
        buf = np.empty(n, np.uint8)
        check(jb_save_state(self.h, buf.ctypes.data, n), "jb_save_state")
        return buf

    def load_state(self, buf):
        """Restore a snapshot taken by save_state on a batch of the same shape."""
        buf = np.ascontiguousarray(buf, np.uint8)
        check(jb_load_state(self.h, buf.ctypes.data, buf.nbytes), "jb_load_state")


def contacts_as_arrays(contacts):
    """List of jb_contact -> dict of numpy arrays."""
    n = len(contacts)
    out = dict(a=np.zeros(n, int), b=np.zeros(n, int), axis=np.zeros(n, int),
               ref_face=np.zeros(n, int), inc_face=np.zeros(n, int), point=np.zeros(n, int),
               p=np.zeros((n, 3)), n=np.zeros((n, 3)), t1=np.zeros((n, 3)),
               depth=np.zeros(n), lam=np.zeros((n, 3)))
    for i, c in enumerate(contacts):
        for k in ("a", "b", "axis", "ref_face", "inc_face", "point", "depth"):
            out[k][i] = getattr(c, k)
        out["p"][i] = list(c.p); out["n"][i] = list(c.n); out["t1"][i] = list(c.t1)
        out["lam"][i] = list(c.lambda_)
    return out

