"""Warm-start network on the GPU (BF16 tensor-core operands, FP32
accumulation) against the FP64 oracle network, and the learned warm start in
the episode kernel.

Tolerances (BF16 operands carry 8 mantissa bits): forward outputs within 2e-2
relative (Frobenius); gradients with cosine similarity > 0.99 per tensor and
the loss within 2e-2 relative; AdamW on an exact FP32 gradient within 1e-6
relative; recorded features within 2e-3 (they are normalised to O(1))."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def jb():
    import paper_2606_28394_gb300 as m
    return m


def ws():
    from paper_2606_28394_gb300 import warmstart
    return warmstart


def features_like(rng, n):
    X = rng.normal(0, 1, (n, 24))
    X[:, 4:10] = rng.normal(0, 1, (n, 6))
    X[:, 22:24] = rng.integers(0, 2, (n, 2))
    return X


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda:0")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_forward_matches_fp64_oracle(cuda_device):
    rng = np.random.default_rng(0)
    theta = omlp.init(2).astype(np.float32)
    theta[omlp.N_IN * 128:omlp.N_IN * 128 + 128] = rng.normal(0, 0.1, 128)   # b1
    net = ws().Network(theta)
    for n in (1, 15, 16, 17, 1000):
        X = features_like(rng, n).astype(np.float32)
        y = net.forward(to_dev(X)).cpu().numpy()
        yr, _ = omlp.forward(theta.astype(np.float64), X.astype(np.float64))
        assert rel(y, yr) < 2e-2, (n, rel(y, yr))


def test_gradients_match_fp64_oracle(cuda_device):
    rng = np.random.default_rng(1)
    theta = omlp.init(3).astype(np.float32) * 0.8
    net = ws().Network(theta)
    X = features_like(rng, 3001).astype(np.float32)
    T = rng.normal(0, 1, (3001, 3)).astype(np.float32)
    g, loss = net.grad(to_dev(X), to_dev(T))
    g = g.cpu().numpy()
    gr, lr = omlp.grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(float(loss.item()) - lr) / lr < 2e-2
    o = 0
    for name, shape in omlp.SHAPES:
        k = int(np.prod(shape))
        a, b = g[o:o + k], gr[o:o + k]
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        assert cos > 0.99, (name, cos)
        o += k


def test_adamw_step_matches_formula(cuda_device):
    import torch
    rng = np.random.default_rng(2)
    theta = omlp.init(4).astype(np.float32)
    net = ws().Network(theta)
    g = rng.normal(size=omlp.N_PARAM).astype(np.float32)
    gd = to_dev(g)
    lr, wd = 1e-3, 1e-2
    for step in (1, 2):
        jb().check(jb().jb_mlp_adamw(net.block.data_ptr(), gd.data_ptr(), step, C.c_float(lr), C.c_float(0.9),
                                     C.c_float(0.999), C.c_float(1e-8), C.c_float(wd),
                                     torch.cuda.current_stream().cuda_stream))
    got = net.params().astype(np.float64)
    t = theta.astype(np.float64)
    m = v = np.zeros_like(t)
    for step in (1, 2):
        t, m, v = omlp.adamw(t, g.astype(np.float64), m, v, step, lr, wd=wd)
    assert rel(got, t) < 1e-6


def test_training_fits_a_teacher_network(cuda_device):
    rng = np.random.default_rng(3)
    teacher = omlp.init(10) * 0.5
    X = features_like(rng, 40000)
    T, _ = omlp.forward(teacher, X)
    rows = to_dev(np.hstack([X, T]).astype(np.float32))
    net, hist = ws().train(rows, epochs=12, batch=4096, lr=2e-3, seed=1)
    assert hist[-1][2] < 0.3 * hist[0][2], hist


def test_recorded_features_match_oracle(cuda_device):
    import torch
    scene = synth.perturbed(synth.build_scene([synth.Tower(levels=4, mu=0.5)], 1), 5, dx=2e-4, dang=0.01)
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000)
    b = jb().Batch(scene, prm)
    cap = 4096
    rows = torch.zeros((cap, 27), dtype=torch.float32, device="cuda:0")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    jb().check(jb().jb_set_recorder(b.h, rows.data_ptr(), cap, cnt.data_ptr(), 1))
    b.step(1)
    g = rows[: int(cnt.item())].cpu().numpy().astype(np.float64)
    s64 = synth.Scene(scene.body_off, *[getattr(scene, k).astype(np.float64) for k in
                                        ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")])
    w = oracle.World(s64, prm)
    w.set_recorder(cap, 1)
    w.step(1)
    o = w.recorded()
    assert len(g) == len(o) > 0
    key = lambda r: np.lexsort(np.round(r[:, :24], 2).T[::-1])
    gf, of = g[key(g), :24], o[key(o), :24]
    assert np.abs(gf - of).max() < 2e-3, np.abs(gf - of).max()


@pytest.mark.parametrize("mode", [2, 3])
def test_learned_warm_start_converges_to_the_same_state(cuda_device, mode):
    """Whatever the network predicts, the projected starting impulses only
    change where Gauss-Seidel starts: the converged state matches the oracle
    as for plain PGS (both at residual 1e-6)."""
    scene = synth.perturbed(synth.build_scene([synth.Tower(levels=4, mu=0.5)], 1), 5, dx=2e-4, dang=0.01)
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000, warm_start=mode)
    net = ws().Network(omlp.init(7).astype(np.float32) * 0.05)
    b = jb().Batch(scene, prm)
    jb().check(jb().jb_set_warmstart_mlp(b.h, net.block.data_ptr()))
    b.step(3)
    st = b.stats()
    assert st["status"][0] == 0 and st["last_residual"][0] <= 1e-6
    x, q, v, w = b.state()
    # oracle from the GPU's state after two steps, one more step each
    b2 = jb().Batch(scene, prm)
    jb().check(jb().jb_set_warmstart_mlp(b2.h, net.block.data_ptr()))
    b2.step(2)
    xs, qs, vs, wsv = b2.state()
    s64 = synth.Scene(scene.body_off, *[getattr(scene, k).astype(np.float64) for k in
                                        ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")])
    o = oracle.World(s64, dict(prm, warm_start=1))
    o.set_state(xs.astype(float), qs.astype(float), vs.astype(float), wsv.astype(float))
    o.step(1)
    xo, qo, vo, wo = o.state()
    assert np.abs(x - xo).max() < 1e-5
    diag = np.sqrt((scene.half.astype(float) ** 2).sum(0))
    assert np.abs(v - vo).max() < 1e-4 and (np.abs(w - wo).max(0) * diag).max() < 1e-4


@pytest.mark.parametrize("n", [1, 127, 300, 20000])
def test_tensor_core_kernel_matches_a_bf16_faithful_reference(cuda_device, n):
    """The fused tcgen05 kernel against a PyTorch FP32 computation of the
    same network with the kernel's BF16 roundings (inputs, weights, hidden
    activations, the scaled output error and the backward activations) and
    FP32 sums.  Only the summation order differs, but an activation that
    lands near a BF16 rounding boundary can round the other way (2^-8
    relative), so the forward agrees to 1e-3 relative and every gradient
    block to 1e-2 relative of its largest entry with cosine above 0.9999.
    n = 1 and 127 are one partial tile, 300 a ragged third tile, and 20000
    rows are 157 tiles, more than one per SM, so CTAs accumulate the weight
    sums in tensor memory across tiles."""
    import torch
    torch.manual_seed(n)
    net = ws().Network(device="cuda:0", seed=3)
    p = torch.from_numpy(net.params()).to("cuda:0")
    sizes = [(24, 128), (128,), (128, 128), (128,), (128, 3), (3,)]
    parts, o = [], 0
    for sh in sizes:
        k = int(np.prod(sh))
        parts.append(p[o:o + k].view(*sh))
        o += k
    W1, b1, W2, b2, W3, b3 = parts
    bf = lambda t: t.to(torch.bfloat16).float()
    x = torch.randn(n, 24, device="cuda:0")
    t = 0.1 * torch.randn(n, 3, device="cuda:0")
    h1 = bf(torch.relu(bf(x) @ bf(W1) + b1))
    h2 = bf(torch.relu(h1 @ bf(W2) + b2))
    y_ref = h2 @ bf(W3) + b3
    y = net.forward(x)
    assert float((y - y_ref).abs().max()) <= 1e-3 * float(y_ref.abs().max())
    g, loss = net.grad(x, t)
    net.check_kernel()
    e = y_ref - t
    assert abs(float(loss) - float((e * e).sum()) / n) <= 1e-4 * float((e * e).sum()) / n
    dy = bf(2.0 / n * e)
    dh2 = bf((dy @ bf(W3).T) * (h2 > 0))
    dh1 = bf((dh2 @ bf(W2).T) * (h1 > 0))
    ref = [bf(x).T @ dh1, dh1.sum(0), h1.T @ dh2, dh2.sum(0), h2.T @ dy, dy.sum(0)]
    o = 0
    for r in ref:
        k = r.numel()
        got = g[o:o + k].view_as(r)
        o += k
        assert float((got - r).abs().max()) <= 1e-2 * float(r.abs().max()) + 1e-12
        cos = torch.nn.functional.cosine_similarity(got.flatten(), r.flatten(), dim=0)
        assert float(cos) > 0.9999


def test_collection_and_training_are_bitwise_reproducible(cuda_device):
    """Two runs of the same collection and training give the same rows and
    the same parameters, bit for bit: the recorded rows are put in an order
    fixed by their contents, and the tensor-core kernel adds its CTAs'
    partial gradients in CTA order (more rows than one CTA takes, so several
    CTAs contribute)."""
    import torch
    sc, pr, prm = synth.friction_workload(seed=3001)
    prm = dict(prm, residual_tol=1e-5, pgs_iter_cap=20000, pgs_accel_period=64)
    s_tr, p_tr = synth.subset(sc, pr, range(0, 450, 45))
    runs = []
    for _ in range(2):
        rows = ws().collect(s_tr, p_tr, prm, capacity=200000, every=1, max_steps=60, unmatched_only=True)
        net, hist = ws().train(rows, epochs=3, batch=2048, lr=1e-3, seed=0)
        runs.append((rows, net.params(), hist))
    (r0, p0, h0), (r1, p1, h1) = runs
    assert r0.shape[0] > 4 * 128
    assert torch.equal(r0, r1)
    assert np.array_equal(p0, p1)
    assert [h[1:] for h in h0] == [h[1:] for h in h1]


def test_learned_warm_start_without_network_is_refused(cuda_device):
    scene = synth.build_scene([synth.Tower(levels=2)], 0)
    b = jb().Batch(scene, synth.params(warm_start=2))
    with pytest.raises(jb().JBError):
        b.step(1)


def test_trained_network_gains_on_cold_contacts(cuda_device):
    """What the trained network gains over the method without it, where it
    acts: contacts with no previous impulse.  Trained on the plain solver's
    converged impulses of 30 removal-round towers (other seeds), it starts
    cold contacts of fresh towers closer to their solution than zero
    impulses do, so PGS reaches the same residual in fewer sweeps."""
    sc, pr, prm = synth.friction_workload(seed=3001)
    prm = dict(prm, residual_tol=1e-5, pgs_iter_cap=20000)
    s_tr, p_tr = synth.subset(sc, pr, range(0, 450, 15))
    rows = ws().collect(s_tr, p_tr, prm, capacity=600000, every=2, max_steps=240)
    net, _ = ws().train(rows, epochs=10, batch=8192, lr=1e-3, seed=0)
    ev, pev, _ = synth.friction_workload(seed=4001)
    s_ev, _ = synth.subset(ev, pev, range(0, 450, 45))
    plain, learned, gain = ws().cold_start_gain(s_ev, prm, net, steps=12)
    print(f"cold contacts: plain {plain:.0f}, learned {learned:.0f} sweeps per solve (gain {gain:.2f})")
    assert gain > 1.1, (plain, learned)


def test_trained_network_against_plain_pgs_on_identical_states(cuda_device):
    """The learned warm start against the method without it, plain PGS with
    previous-frame warm start, solved as the benchmark solves (residual
    1e-5, the conjugate-gradient step every 64 sweeps), on the first 24
    steps of removal-round towers of fresh seeds.  Both arms start every
    matched point from its previous impulse; they differ at the points of
    new pairs (every pair of the first step, pairs that form later), where
    plain PGS starts from zero and the learned arm from the network, trained
    on the plain solver's converged impulses at such points of other seeds.
    Every step is solved by both arms from the same snapshot along plain
    PGS's trajectory (warmstart.paired): whole trajectories of the two arms
    part after the first solve (a stack's impulses over redundant supports
    are not unique), and comparing them measures where each trajectory went
    as much as what the network saves.  From identical states the network's
    starts save sweeps on the first step, where it predicts every point, no
    later step costs more in all, and no solve fails to reach the
    residual."""
    sc, pr, prm = synth.friction_workload(seed=3001)
    prm = dict(prm, residual_tol=1e-5, pgs_iter_cap=20000, pgs_accel_period=64)
    s_tr, p_tr = synth.subset(sc, pr, range(0, 450, 15))
    rows = ws().collect(s_tr, p_tr, prm, capacity=400000, every=1, max_steps=240, unmatched_only=True)
    assert rows.shape[0] > 1000 and (rows[:, 22] == 0).all()
    net, _ = ws().train(rows, epochs=30, batch=8192, lr=1e-3, seed=0)
    ev, pev, _ = synth.friction_workload(seed=4001)
    s_ev, p_ev = synth.subset(ev, pev, range(0, 450, 10))
    out = ws().paired(s_ev, p_ev, prm, net, steps=24, mode=2)
    first = out["plain"][0] / out["learned"][0]
    print(f"identical states, 24 steps: plain {out['plain'].sum():.0f}, learned {out['learned'].sum():.0f} sweeps "
          f"(gain {out['gain']:.3f}); first step {out['plain'][0]:.0f} vs {out['learned'][0]:.0f} ({first:.3f})")
    assert out["plain_capped"] == 0 and out["learned_capped"] == 0
    assert first > 1.03, out
    assert out["learned"][1:].sum() <= 1.01 * out["plain"][1:].sum(), out
    assert out["gain"] > 1.0, out
