"""Autotuner for the batched step.

Picks, by timing short trials of the actual workload with CUDA events (the
first `trial_steps` physics steps of a sample of its episodes):
  - smem_pair_factor: pairs per body whose solver records stay in shared
    memory before a step falls back to global memory; it sets how many
    episodes fit per SM (the episode-to-SM packing);
  - the residual-check cadence (residual_every, residual_every_max);
  - pgs_accel_period: how often the conjugate-gradient step runs (0 = plain
    PGS), i.e. the iteration schedule;
  - colour_key: the order in which the greedy colouring takes the pairs, i.e.
    the colour schedule of a sweep.
The search is coordinate descent: each knob in turn over its candidates with
the others at their best so far, two rounds (a trial already timed is not
repeated).  One warp per episode and one episode per CTA are fixed by the
kernel (a tower's largest colour holds about 20 pairs, so more lanes per
episode would idle, and a CTA per episode lets size classes share SMs).
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
ACCEL = (0, 32, 64, 128)
KEYS = (0, 1)
TUNED = ("smem_pair_factor", "residual_every", "residual_every_max", "pgs_accel_period", "colour_key")
# the knobs of the coordinate descent, each a list of settings
KNOBS = (
    ("smem_pair_factor", [{"smem_pair_factor": f} for f in FACTORS]),
    ("cadence", [{"residual_every": a, "residual_every_max": b} for a, b in CADENCE]),
    ("pgs_accel_period", [{"pgs_accel_period": m} for m in ACCEL]),
    ("colour_key", [{"colour_key": k} for k in KEYS]),
)
DEFAULTS = {"smem_pair_factor": 4.0, "residual_every": 4, "residual_every_max": 32, "pgs_accel_period": 64,
            "colour_key": 0}


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
    timed = {}

    def run(choice):
        key_ = tuple(choice[k] for k in TUNED)
        if key_ not in timed:
            ms = trial(s, p, dict(params, **choice))
            timed[key_] = ms
            table.append(dict(choice, ms=ms))
            if log:
                log(f"{choice}: {ms:.1f} ms")
        return timed[key_]

    choice = {k: params.get(k, DEFAULTS[k]) for k in TUNED}
    best_ms = run(choice)
    for _ in range(2):
        for _name, settings in KNOBS:
            for st in settings:
                cand = dict(choice, **st)
                ms = run(cand)
                if ms < best_ms:
                    best_ms, choice = ms, cand
    if use_cache:
        cache[key] = {"best": choice, "table": table}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return dict(params, **choice), table
