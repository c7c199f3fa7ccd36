"""Autotuner for the batched step.

Picks the per-episode shared-memory solver capacity (smem_pair_factor: pairs
per body kept on chip before a step falls back to global memory, which sets
how many episodes fit per SM) and the residual-check cadence
(residual_every, residual_every_max) by timing short trials of the actual
workload with CUDA events: the first `trial_steps` physics steps of a sample
of its episodes.
Choices are cached in a JSON file keyed by GPU name and a hash of the
workload's shape and solver parameters.
"""
from __future__ import annotations

import hashlib
import json
import os

from types import SimpleNamespace

import numpy as np

from . import Batch

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), ".autotune_cache.json")
FACTORS = (3.6, 4.0, 5.0)
CADENCE = ((4, 4), (4, 32), (2, 32))   # (residual_every, residual_every_max)
TUNED = ("smem_pair_factor", "residual_every", "residual_every_max")


def subset(scene, prot, episodes):
    """Scene and schedule of the given episodes (plain array slicing)."""
    episodes = np.asarray(list(episodes), int)
    bo, po = np.asarray(scene.body_off), np.asarray(prot.off)
    bidx = np.concatenate([np.arange(bo[e], bo[e + 1]) for e in episodes])
    midx = np.concatenate([np.arange(po[e], po[e + 1]) for e in episodes] + [np.zeros(0, int)])
    boff = np.zeros(len(episodes) + 1, np.int32)
    boff[1:] = np.cumsum(bo[episodes + 1] - bo[episodes])
    moff = np.zeros(len(episodes) + 1, np.int32)
    moff[1:] = np.cumsum(po[episodes + 1] - po[episodes])
    col = lambda a: np.ascontiguousarray(np.asarray(a)[..., bidx])
    s = SimpleNamespace(body_off=boff, half=col(scene.half), mass=col(scene.mass), mu=col(scene.mu),
                        x=col(scene.x), q=col(scene.q), v=col(scene.v), w=col(scene.w),
                        ground_mu=np.asarray(scene.ground_mu)[episodes], n_episodes=len(episodes),
                        n_bodies=int(boff[-1]))
    pr = SimpleNamespace(off=moff, **{f: np.asarray(getattr(prot, f))[midx] for f in
                                      ("block", "axis", "sign", "factor", "k", "remove", "push_steps",
                                       "settle_steps")})
    return s, pr


def _key(scene, params, gpu):
    h = hashlib.sha1()
    h.update(np.asarray(scene.body_off, np.int64).tobytes())
    h.update(json.dumps({k: v for k, v in sorted(params.items()) if k not in TUNED},
                        default=str).encode())
    return f"{gpu}:{h.hexdigest()[:16]}"


def _gpu_trial(s, p, prm, trial_steps, device):
    """Milliseconds (CUDA events) of `trial_steps` steps of the sample."""
    import torch
    b = Batch(s, prm, max_moves=int(p.off[-1]), device=device)
    b.set_protocol(p)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.run_protocol(trial_steps)
    e1.record(b.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def tune(scene, prot, params, trial_steps=120, sample=64, device="cuda", use_cache=True, log=None,
         trial=None, gpu_name=None, cache_path=None):
    """Returns a copy of params with the fastest (smem_pair_factor,
    residual_every, residual_every_max) on a trial of the workload, and the
    timing table.  `trial(scene, prot, params) -> ms`, `gpu_name` and
    `cache_path` default to timing the library on the current GPU and the
    package's cache file."""
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name(torch.device(device))
    if trial is None:
        trial = lambda s, p, prm: _gpu_trial(s, p, prm, trial_steps, device)
    cache_path = cache_path or CACHE
    key = _key(scene, params, gpu_name)
    cache = {}
    if use_cache and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        return dict(params, **cache[key]["best"]), cache[key]["table"]
    idx = np.linspace(0, scene.n_episodes - 1, min(sample, scene.n_episodes)).round().astype(int)
    s, p = subset(scene, prot, idx)
    table = []
    for fac in FACTORS:
        for ev, evm in CADENCE:
            prm = dict(params, smem_pair_factor=fac, residual_every=ev, residual_every_max=evm)
            ms = trial(s, p, prm)
            table.append({"smem_pair_factor": fac, "residual_every": ev, "residual_every_max": evm, "ms": ms})
            if log:
                log(f"factor {fac} cadence {ev}..{evm}: {ms:.1f} ms")
    best = min(table, key=lambda r: r["ms"])
    choice = {k: best[k] for k in TUNED}
    if use_cache:
        cache[key] = {"best": choice, "table": table}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return dict(params, **choice), table
