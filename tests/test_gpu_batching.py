"""Ragged batches: episodes of different sizes run in size classes (own
shared-memory plan, grid and work queue, concurrent streams).  Classes only
schedule: every episode's trajectory is bit-identical to running it alone.
The autotuner returns one of its candidate configurations."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def jb():
    import paper_2606_28394_gb300 as m
    return m


def test_size_classes_do_not_change_results(cuda_device):
    levels = [25, 4, 13, 6, 18, 9]
    towers = [synth.Tower(levels=l, mu=0.3 + 0.05 * i) for i, l in enumerate(levels)]
    scene = synth.perturbed(synth.build_scene(towers, 21), 22, dx=1e-4, dang=0.005)
    prm = synth.params(residual_tol=1e-5, pgs_iter_cap=20000)
    b = jb().Batch(scene, prm)
    # bodies 75, 54, 39 | 27, 18 | 12: a class ends at half its largest tower
    assert [c[:2] for c in b.size_classes()] == [(3, 75), (2, 27), (1, 12)]
    b.step(6)
    x, q, v, w = b.state()
    st = b.stats()
    for e in range(len(towers)):
        one = synth.subset(scene, synth._protocol([[]] * len(towers), len(towers)), [e])[0]
        a = jb().Batch(one, prm)
        a.step(6)
        xe, qe, ve, we = a.state()
        lo, hi = scene.body_off[e], scene.body_off[e + 1]
        for big, small in ((x, xe), (q, qe), (v, ve), (w, we)):
            assert np.array_equal(big[:, lo:hi], small), e
        assert a.stats()["total_sweeps"][0] == st["total_sweeps"][e]


def test_autotuner_returns_a_candidate(cuda_device):
    from paper_2606_28394_gb300 import autotune
    scene, prot, prm = synth.ragged_workload(seed=7, n=16)
    prm = dict(prm, residual_tol=1e-5, pgs_iter_cap=5000)
    tuned, table = autotune.tune(scene, prot, prm, trial_steps=8, sample=8, use_cache=False)
    assert tuned["smem_pair_factor"] in autotune.FACTORS
    assert (tuned["residual_every"], tuned["residual_every_max"]) in autotune.CADENCE
    assert tuned["pgs_accel_period"] in autotune.ACCEL and tuned["colour_key"] in autotune.KEYS
    # coordinate descent: distinct trials, the choice the fastest of them
    assert 1 < len(table) < len(autotune.FACTORS) * len(autotune.CADENCE) * len(autotune.ACCEL) * len(autotune.KEYS)
    assert all(r["ms"] > 0 for r in table)
    best = min(table, key=lambda r: r["ms"])
    assert all(tuned[k] == best[k] for k in autotune.TUNED)


def test_ragged_batch_one_step_parity(cuda_device):
    """Towers of 3, 7, 12 and 5 levels (three size classes) in one batch, one
    step at PGS residual 1e-6 on both sides: the same bounds as the
    single-tower parity cases."""
    towers = [synth.Tower(levels=l, mu=m) for l, m in ((3, 0.3), (7, 0.5), (12, 0.4), (5, 0.6))]
    scene = synth.perturbed(synth.build_scene(towers, 4), 13, dx=2e-4, dang=0.01)
    # FP32 and FP64 may take a near-tied SAT axis choice differently (a
    # different, equally valid manifold); the jitter seed is one whose
    # decisions are all clear by 3e-7 m (most seeds have one or two pairs
    # within that of the 10 um tie or the edge-rule threshold).
    assert oracle.sat_decisions_clear(scene)
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000)
    b = jb().Batch(scene, prm)
    s64 = synth.Scene(scene.body_off, *[getattr(scene, k).astype(np.float64) for k in
                                        ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")])
    w = oracle.World(s64, prm)
    b.step(1)
    w.step(1)
    st, so = b.stats(), w.stats()
    assert (st["status"] == 0).all() and (st["last_residual"] <= 1e-6).all()
    assert (so["last_residual"] <= 1e-6).all()
    xg, qg, vg, wg = b.state()
    xo, qo, vo, wo = w.state()
    assert np.abs(xg - xo).max() < 1e-5
    diag = np.sqrt((scene.half.astype(float) ** 2).sum(0))
    assert np.abs(vg - vo).max() < 1e-4 and (np.abs(wg - wo).max(0) * diag).max() < 1e-4


def test_step_loop_captures_in_a_cuda_graph(cuda_device):
    """jb_step launches only stream-ordered work (a counter reset, the
    per-class episode kernels forked onto side streams and joined back by
    events), so a host step loop can be captured into a CUDA graph together
    with the caller's own device work and replayed.  Replays give exactly
    the states of direct stepping."""
    import torch
    towers = [synth.Tower(levels=l) for l in (20, 5, 11, 7)]     # three size classes
    scene = synth.perturbed(synth.build_scene(towers, 31), 32, dx=1e-4, dang=0.005)
    prm = synth.params(residual_tol=1e-5, pgs_iter_cap=20000)
    ref = jb().Batch(scene, prm)
    ref.step(6)
    s = torch.cuda.Stream()
    b = jb().Batch(scene, prm, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.step(1)
        b.step(1)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for u, v in zip(ref.state(), b.state()):
        assert np.array_equal(u, v)
    assert (b.stats()["steps"] == 6).all()


def test_global_memory_fallback_matches_shared_memory(cuda_device):
    """Steps whose pairs exceed the on-chip capacity solve from the global
    copy of the colour-sorted arrays.  Forcing that path (capacity 0.5 pairs
    per body) gives the same converged states as the shared-memory path."""
    scene = synth.perturbed(synth.build_scene([synth.Tower(levels=12)], 8), 9, dx=1e-4, dang=0.005)
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000)
    a = jb().Batch(scene, prm)
    g = jb().Batch(scene, dict(prm, smem_pair_factor=0.5))
    a.step(3)
    g.step(3)
    for u, v in zip(a.state(), g.state()):
        assert np.abs(u - v).max() < 1e-5
    assert (g.stats()["status"] & ~jb().JB_EP_NOT_CONVERGED == 0).all()


def test_very_tall_tower_fits_by_shrinking_the_on_chip_capacity(cuda_device):
    """A 100-level tower (300 bodies, ~1,080 pairs) does not fit shared
    memory at the default capacity; the batch keeps fewer pairs on chip and
    its steps run from the global copy.  Two steps: no error bits other than
    the cap, and the flush tower stays put."""
    scene = synth.build_scene([synth.Tower(levels=100)], 0)
    b = jb().Batch(scene, synth.params(residual_tol=1e-5, pgs_iter_cap=4000))
    assert b.size_classes()[0][1] == 300
    b.step(2)
    st = b.stats()
    assert (st["status"] & ~jb().JB_EP_NOT_CONVERGED) == 0
    x = b.state()[0]
    assert np.abs(x - scene.x).max() < 1e-3


def test_empty_episode_and_fully_removed_tower(cuda_device):
    """Degenerate inputs: an episode with no bodies between two towers, and a
    tower whose blocks are all removed.  Both step as no-ops (no error bits,
    no body-steps, COM imbalance 0 as in the oracle), and the other episodes
    are bit-identical to a batch without them."""
    prm = synth.params(residual_tol=1e-5, pgs_iter_cap=20000)
    sc = synth.build_scene([synth.Tower(levels=3), synth.Tower(levels=0), synth.Tower(levels=2)], 0)
    assert list(sc.body_off) == [0, 9, 9, 15]
    b = jb().Batch(sc, prm)
    b.remove_block([2] * 6, list(range(6)))
    b.step(3)
    st = b.stats()
    assert (st["status"] == 0).all()
    assert st["body_steps"][1] == 0 and st["body_steps"][2] == 0
    assert st["com_imbalance"][1] == 0
    w = oracle.World(synth.Scene(sc.body_off, *[getattr(sc, k).astype(np.float64) for k in
                                                ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")]), prm)
    w.step(3)
    assert w.stats()["com_imbalance"][1] == 0
    alone = jb().Batch(synth.build_scene([synth.Tower(levels=3)], 0), prm)
    alone.step(3)
    for big, small in zip(b.state(), alone.state()):
        assert np.array_equal(big[:, :9], small)
    assert not b.active()[9:].any()


def test_reference_episode_search(cuda_device):
    """jb_reference_episode on a batch after removal rounds: the collapsed
    episode with the removed-block count closest to n_hat (else the most
    rounds), against the definition over the batch's statistics and active
    flags."""
    towers = [synth.Tower(levels=5, mu=m) for m in (0.25, 0.4, 0.6) * 4]
    sc = synth.build_scene(towers, 21)
    prot = synth.removal_protocol(towers, 21, push_steps=40, settle_steps=80, max_removals=4)
    b = jb().Batch(sc, synth.params(pgs_iters=10), max_moves=int(prot.off[-1]))
    b.set_protocol(prot)
    b.run_protocol()
    st, act = b.stats(), b.active()
    removed = [int((~act[sc.body_off[e]:sc.body_off[e + 1]]).sum()) for e in range(len(towers))]
    for n_hat in range(6):
        cand = [e for e in range(len(towers)) if st["collapsed"][e]]
        want = (min(cand, key=lambda e: (abs(removed[e] - n_hat), e)) if cand
                else min(range(len(towers)), key=lambda e: (-st["moves_done"][e], e)))
        assert b.reference_episode(n_hat) == (want, removed[want])


def test_nonfinite_episode_is_isolated(cuda_device):
    """Fault injection on the host: a NaN velocity written into one body of
    the middle episode.  That episode is flagged non-finite and stops; its
    neighbours run exactly as in a batch without the NaN."""
    towers = [synth.Tower(levels=4), synth.Tower(levels=4), synth.Tower(levels=4)]
    sc = synth.build_scene(towers, 12)
    prm = synth.params(residual_tol=1e-5, pgs_iter_cap=20000)
    clean, bad = jb().Batch(sc, prm), jb().Batch(sc, prm)
    v = sc.v.astype(np.float32).copy()
    v[0, 12 + 5] = np.nan
    bad.write_state(v=v)
    clean.step(3)
    bad.step(3)
    st = bad.stats()
    assert st["status"][1] & jb().JB_EP_NONFINITE
    assert st["status"][0] == 0 and st["status"][2] == 0
    for u, w in zip(clean.state(), bad.state()):
        assert np.array_equal(u[:, :12], w[:, :12]) and np.array_equal(u[:, 24:], w[:, 24:])
