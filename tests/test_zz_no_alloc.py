"""jb_step_noalloc: stepping for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code running inside another framework's
memory pool, a real-time loop that must not allocate, a process whose device
allocator is locked.  jb_step_noalloc serves them from a fixed device array
inside the library instead of a caller workspace.  These checks call it
through the C ABI, twice in a row on one device (the second call reuses the
scratch the first one left behind), and compare its output with the
allocating entry points (jb_batch_create + jb_step) from the same state, at
the tolerances of the other GPU tests: positions within 1e-5 m, velocities
within 1e-4 m/s.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda:0")


def test_noalloc_matches_allocating_path_on_two_calls(cuda_device):
    import torch
    import paper_2606_28394_gb300 as jb

    towers = [synth.Tower(levels=4, mu=0.3), synth.Tower(levels=6, mu=0.5), synth.Tower(levels=5, mu=0.7)]
    scene = synth.perturbed(synth.build_scene(towers, 11), 12, dx=2e-4, dang=0.01)
    prm = synth.params(residual_tol=1e-5, pgs_iter_cap=20000)
    p = jb.params_from_dict(prm)
    half, mass, mu, gmu = (_dev(torch, a) for a in (scene.half, scene.mass, scene.mu, scene.ground_mu))
    x, q, v, w = (_dev(torch, a) for a in (scene.x, scene.q, scene.v, scene.w))
    off = np.ascontiguousarray(scene.body_off, np.int32)
    stream = torch.cuda.current_stream()
    diag = np.sqrt((scene.half.astype(float) ** 2).sum(0))
    n_steps = 12
    state = (scene.x, scene.q, scene.v, scene.w)
    for call in range(2):
        ref = synth.Scene(scene.body_off, scene.half, scene.mass, scene.mu, *state, scene.ground_mu)
        b = jb.Batch(ref, prm)
        b.step(n_steps)
        xr, qr, vr, wr = b.state()
        rc = jb.jb_step_noalloc(scene.n_episodes, off.ctypes.data_as(jb._ip), half.data_ptr(), mass.data_ptr(),
                                mu.data_ptr(), gmu.data_ptr(), x.data_ptr(), q.data_ptr(), v.data_ptr(),
                                w.data_ptr(), C.byref(p), n_steps, stream.cuda_stream)
        assert rc == jb.JB_OK, jb.jb_last_error()
        torch.cuda.synchronize()
        xs, qs, vs, ws = (t.cpu().numpy() for t in (x, q, v, w))
        assert np.abs(xs - xr).max() < 1e-5, (call, np.abs(xs - xr).max())
        assert np.abs(vs - vr).max() < 1e-4, (call, np.abs(vs - vr).max())
        assert (np.abs(ws - wr).max(0) * diag).max() < 1e-4, call
        assert np.abs(qs - qr).max() < 1e-5, call
        state = (xs, qs, vs, ws)


def test_noalloc_rejects_batches_beyond_the_scratch(cuda_device):
    import torch
    import paper_2606_28394_gb300 as jb

    towers = [synth.Tower(levels=18) for _ in range(200)]
    off = np.zeros(len(towers) + 1, np.int32)
    off[1:] = np.cumsum([54] * len(towers))
    p = jb.default_params()
    dummy = torch.zeros(4 * int(off[-1]), device="cuda:0")
    ptr = dummy.data_ptr()
    rc = jb.jb_step_noalloc(len(towers), off.ctypes.data_as(jb._ip), ptr, ptr, ptr, ptr, ptr, ptr, ptr, ptr,
                            C.byref(p), 1, None)
    assert rc == jb.JB_ENOMEM
    assert b"static scratch" in jb.jb_last_error()
