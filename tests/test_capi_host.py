"""C-ABI library checks that need no GPU: it loads, exports every entry point
declared in include/jb.h, and its host-only helpers behave."""
import ctypes as C
import os
import re

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "jb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jb_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("jb_batch_create", "jb_step", "jb_run_protocol", "jb_apply_push", "jb_remove_block",
                 "jb_read_state", "jb_read_contacts", "jb_read_episode_stats", "jb_sync",
                 "jb_save_state", "jb_load_state", "jb_batch_destroy", "jb_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2606_28394_gb300 as jb
    lib = C.CDLL(jb.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(jb.EXPORTS)


def test_default_params_follow_the_paper_table():
    import paper_2606_28394_gb300 as jb
    p = jb.default_params()
    assert abs(p.dt - 1 / 240) < 1e-9 and abs(p.restitution - 0.10) < 1e-7
    assert abs(p.beta - 0.35) < 1e-7 and abs(p.slop - 4e-4) < 1e-10 and abs(p.aabb_eps - 2e-3) < 1e-10
    assert abs(p.gravity[2] + 9.81) < 1e-6


def test_tower_builder_matches_generator_bit_exactly():
    import paper_2606_28394_gb300 as jb
    towers = [synth.Tower(levels=18, mu=0.4), synth.Tower(levels=7, mu=0.25), synth.Tower(levels=30, mu=0.6)]
    seed = 12345
    ref = synth.build_scene(towers, seed)
    E = len(towers)
    desc = (jb.jb_tower_desc * E)()
    for i, t in enumerate(towers):
        desc[i].levels = t.levels; desc[i].per_level = t.per_level
        desc[i].dims = (C.c_float * 3)(*t.dims); desc[i].mass = t.mass
        desc[i].mass_jitter = t.mass_jitter; desc[i].mu_s = t.mu
    off = np.zeros(E + 1, np.int32)
    assert jb.jb_tower_layout(desc, E, off.ctypes.data_as(jb._ip)) == 0
    assert (off == ref.body_off).all()
    B = int(off[-1])
    half = np.zeros((3, B), np.float32); mass = np.zeros(B, np.float32); mu = np.zeros(B, np.float32)
    x = np.zeros((3, B), np.float32); q = np.zeros((4, B), np.float32); gmu = np.zeros(E, np.float32)
    f = lambda a: a.ctypes.data_as(jb._fp)
    assert jb.jb_tower_init(desc, E, seed, off.ctypes.data_as(jb._ip), f(half), f(mass), f(mu), f(x), f(q), f(gmu)) == 0
    assert (half == ref.half).all() and (mass == ref.mass).all() and (mu == ref.mu).all()
    assert (x == ref.x).all() and (q == ref.q).all() and (gmu == ref.ground_mu).all()


def test_host_argument_errors_need_no_device():
    import paper_2606_28394_gb300 as jb
    p = jb.default_params()
    off = np.array([0, 3], np.int32)
    assert jb.jb_workspace_bytes(0, off.ctypes.data_as(jb._ip), C.byref(p), 0) == 0
    assert jb.jb_workspace_bytes(1, off.ctypes.data_as(jb._ip), C.byref(p), 0) > 0
    assert jb.jb_tower_layout(None, 1, off.ctypes.data_as(jb._ip)) == jb.JB_EINVAL
    assert b"null" in jb.jb_last_error()
    h = C.c_void_p()
    assert jb.jb_batch_create(None, C.byref(p), 0, None, 0, None, C.byref(h)) == jb.JB_EINVAL


def _c_layouts(structs):
    """sizeof and field offsets of the header's structs, from gcc."""
    import subprocess
    import tempfile
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "jb.h"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe], text=True)
    return dict(line.rsplit(" ", 1) for line in out.strip().splitlines())


def test_binding_struct_layouts_match_the_header():
    """Every ctypes mirror of a header struct has the C compiler's size and
    field offsets (a reordered or missing field would silently corrupt the
    call)."""
    import paper_2606_28394_gb300 as jb
    mirrors = {n: getattr(jb, n) for n in ("jb_solver_params", "jb_scene", "jb_tower_desc", "jb_protocol",
                                           "jb_contact", "jb_episode_stats")}
    cname = lambda f: f[:-1] if f.endswith("_") else f     # lambda_ mirrors the C field lambda
    got = _c_layouts({n: [cname(f) for f, _ in m._fields_] for n, m in mirrors.items()})
    for n, m in mirrors.items():
        assert int(got[n]) == C.sizeof(m), n
        for f, _ in m._fields_:
            assert int(got[f"{n}.{cname(f)}"]) == getattr(m, f).offset, (n, f)


def test_too_small_workspace_is_refused_before_any_device_work():
    """A workspace smaller than jb_workspace_bytes is refused with
    JB_ENOMEM from the host-side size check (no device memory is touched,
    so a dummy address is safe)."""
    import paper_2606_28394_gb300 as jb
    sc = synth.build_scene([synth.Tower(levels=2)], 0)
    prm = jb.default_params()
    arrs = [np.ascontiguousarray(a, t) for a, t in ((sc.body_off, np.int32), (sc.half, np.float32),
                                                   (sc.mass, np.float32), (sc.mu, np.float32),
                                                   (sc.x, np.float32), (sc.q, np.float32), (sc.v, np.float32),
                                                   (sc.w, np.float32), (sc.ground_mu, np.float32))]
    fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
    scene = jb.jb_scene(1, arrs[0].ctypes.data_as(C.POINTER(C.c_int32)), *[fp(a) for a in arrs[1:]])
    need = jb.jb_workspace_bytes(1, arrs[0].ctypes.data_as(C.POINTER(C.c_int32)), C.byref(prm), 0)
    assert need > 256
    h = C.c_void_p()
    rc = jb.jb_batch_create(C.byref(scene), C.byref(prm), 0, C.c_void_p(0x1000), need - 256, None, C.byref(h))
    assert rc == jb.JB_ENOMEM and not h.value
    assert b"too small" in jb.jb_last_error()


def _scene_struct(jb, sc, keep):
    arrs = [np.ascontiguousarray(a, t) for a, t in ((sc.body_off, np.int32), (sc.half, np.float32),
                                                   (sc.mass, np.float32), (sc.mu, np.float32),
                                                   (sc.x, np.float32), (sc.q, np.float32), (sc.v, np.float32),
                                                   (sc.w, np.float32), (sc.ground_mu, np.float32))]
    keep.extend(arrs)
    fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
    return jb.jb_scene(sc.n_episodes, arrs[0].ctypes.data_as(C.POINTER(C.c_int32)), *[fp(a) for a in arrs[1:]])


def test_corrupt_inputs_are_refused_before_any_device_work():
    """Host-side validation of jb_batch_create (error codes and messages; no
    device memory is touched, so a dummy workspace address is safe):
    non-positive half extents, a decreasing body_off, and out-of-range solver
    parameters are JB_EINVAL."""
    import paper_2606_28394_gb300 as jb
    good = synth.build_scene([synth.Tower(levels=2), synth.Tower(levels=1)], 0)
    cases = []
    sc = synth.build_scene([synth.Tower(levels=2), synth.Tower(levels=1)], 0)
    sc.half[1, 3] = 0.0
    cases.append(("half extents", sc, {}))
    sc = synth.build_scene([synth.Tower(levels=2), synth.Tower(levels=1)], 0)
    sc.body_off = np.array([0, 6, 4, 9], np.int32)
    cases.append(("body_off", sc, {}))
    for bad in (dict(sor=2.5), dict(friction_cone=3), dict(residual_every=0), dict(warm_start=7),
                dict(dt=0.0), dict(restitution_newton=2), dict(stall_window=-1)):
        cases.append((None, good, bad))
    for expect, sc, bad in cases:
        keep = []
        scene = _scene_struct(jb, sc, keep)
        p = jb.default_params(**bad)
        h = C.c_void_p()
        rc = jb.jb_batch_create(C.byref(scene), C.byref(p), 0, C.c_void_p(0x1000), 1 << 30, None, C.byref(h))
        assert rc == jb.JB_EINVAL and not h.value, (expect, bad)
        if expect:
            assert expect.encode() in jb.jb_last_error(), jb.jb_last_error()
