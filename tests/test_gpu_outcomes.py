"""Whole-episode outcomes on the headline workload (Sec. 8.2 Eq. collapse,
Sec. 8.1 Eq. stability, Sec. 13.1's removal rounds): the GPU's FP32 batch in
the benchmark's configuration (coloured PGS with the conjugate-gradient step
every 64 sweeps, residual <= 1e-5 m/s) against the FP64 oracle's plain
sequential PGS on a 150-episode subset (50 per friction level, stored by
tests/golden/make_friction_outcomes.py).  Collapses are chaotic, so the two
are compared as distributions per mu: two-sample Kolmogorov-Smirnov p > 0.01
for the fallen-block count and the COM imbalance; the mean COM imbalance of
the towers left standing on both sides within 5 %; the all-episode means of
the fallen count and the COM imbalance, and the collapse counts, within three
standard errors of their difference (with 50 chaotic episodes the standard
error of a mean fallen count is about a quarter of it, and a few collapsed
piles with their COM far off the support dominate the imbalance mean, so a
5 % bound there would test noise)."""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "friction150_outcomes.txt")


def jb():
    import paper_2606_28394_gb300 as m
    return m


def test_friction_workload_outcome_distributions_match_the_oracle(cuda_device):
    from scipy.stats import ks_2samp
    gold = np.loadtxt(GOLDEN)
    idx = gold[:, 0].astype(int)
    scene, prot, prm = synth.friction_workload(seed=1)
    prm = dict(prm, residual_tol=1e-5, pgs_iter_cap=20000, pgs_accel_period=64)
    b = jb().Batch(scene, prm, max_moves=int(prot.off[-1]))
    b.set_protocol(prot)
    b.run_protocol(1 << 30)
    st = b.stats()
    assert (st["phase"] == jb().JB_PH_DONE).all()
    assert (st["status"] & (jb().JB_EP_NONFINITE | jb().JB_EP_CONTACT_OVERFLOW) == 0).all()
    mu = scene.ground_mu[idx]
    assert np.allclose(mu, gold[:, 1], atol=5e-3)
    report = {}
    for m in (0.25, 0.40, 0.60):
        sel = np.abs(gold[:, 1] - m) < 5e-3
        e = idx[sel]
        fo, fg = gold[sel, 3], st["n_fallen"][e].astype(float)
        io, ig = gold[sel, 4], st["com_imbalance"][e].astype(float)
        co, cg = gold[sel, 2], st["collapsed"][e].astype(float)
        p_f = ks_2samp(fo, fg).pvalue
        p_i = ks_2samp(io, ig).pvalue
        se = lambda a, b: np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b)) + 1e-12
        both = (co == 0) & (cg == 0)
        report[m] = (p_f, p_i, fo.mean(), fg.mean(), io.mean(), ig.mean(), co.sum(), cg.sum(),
                     io[both].mean(), ig[both].mean())
        assert p_f > 0.01 and p_i > 0.01, report[m]
        assert abs(ig[both].mean() - io[both].mean()) <= 0.05 * abs(io[both].mean()), report[m]
        assert abs(fg.mean() - fo.mean()) <= 3 * se(fo, fg), report[m]
        assert abs(ig.mean() - io.mean()) <= 3 * se(io, ig), report[m]
        assert abs(cg.mean() - co.mean()) <= 3 * se(co, cg), report[m]
    print(report)
