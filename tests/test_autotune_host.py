"""The autotuner's selection and cache logic on the host, with a fake trial
in place of the GPU timing (CPU only)."""
import json

import pytest

import synth


def autotune():
    try:
        from paper_2606_28394_gb300 import autotune as a
    except ImportError:
        pytest.skip("library not built")
    return a


def test_picks_the_fastest_trial_and_caches_it(tmp_path):
    a = autotune()
    scene, prot, prm = synth.ragged_workload(seed=7, n=12)
    calls = []

    def trial(s, p, q):
        calls.append(q)
        assert s.n_episodes == 8          # the sample, evenly spaced over the batch
        # fastest: factor 5, checks every 2..32, the step every 128 sweeps, height key
        return (10.0 + abs(q["smem_pair_factor"] - 5.0) + (0 if q["residual_every"] == 2 else 1)
                + abs(q["pgs_accel_period"] - 128) / 64 + (0 if q["colour_key"] == 1 else 0.5))

    cache = str(tmp_path / "cache.json")
    tuned, table = a.tune(scene, prot, prm, sample=8, trial=trial, gpu_name="fake", cache_path=cache)
    # coordinate descent: distinct trials only, fewer than the full grid
    grid = len(a.FACTORS) * len(a.CADENCE) * len(a.ACCEL) * len(a.KEYS)
    assert len(calls) == len(table) < grid
    assert len({tuple(c[k] for k in a.TUNED) for c in calls}) == len(calls)
    assert (tuned["smem_pair_factor"], tuned["residual_every"], tuned["residual_every_max"]) == (5.0, 2, 32)
    assert (tuned["pgs_accel_period"], tuned["colour_key"]) == (128, 1)
    assert tuned["residual_tol"] == prm["residual_tol"]           # the rest of params untouched
    stored = json.load(open(cache))
    assert len(stored) == 1 and list(stored.values())[0]["best"]["smem_pair_factor"] == 5.0
    # second call: answered from the cache, no trials
    calls.clear()
    tuned2, _ = a.tune(scene, prot, prm, sample=8, trial=trial, gpu_name="fake", cache_path=cache)
    assert not calls and tuned2 == tuned
    # another GPU or other solver parameters: a new key, new trials
    a.tune(scene, prot, prm, sample=8, trial=trial, gpu_name="other", cache_path=cache)
    a.tune(scene, prot, dict(prm, residual_tol=1e-6), sample=8, trial=trial, gpu_name="fake", cache_path=cache)
    assert len(calls) == 2 * len(table) and len(json.load(open(cache))) == 3
