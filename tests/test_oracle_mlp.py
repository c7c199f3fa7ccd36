"""Pins of the FP64 warm-start network and of the oracle's feature recorder
(CPU only): finite differences, closed forms, the AdamW formulas, and hand
values of the features of a block resting on the ground."""
import math

import numpy as np

import oracle
import synth
from oracle import mlp


def data(rng, n=37):
    X = rng.normal(size=(n, mlp.N_IN))
    T = rng.normal(size=(n, mlp.N_OUT))
    return X, T


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    theta = mlp.init(1) * 0.7
    theta += rng.normal(0, 0.05, theta.shape)     # nonzero biases
    X, T = data(rng)
    g, L = mlp.grad(theta, X, T)
    assert abs(L - mlp.loss(theta, X, T)) < 1e-12
    idx = rng.choice(mlp.N_PARAM, 300, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta); e[i] = h
        fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_zero_weights_give_bias_and_its_gradient():
    rng = np.random.default_rng(4)
    p = mlp.unflatten(np.zeros(mlp.N_PARAM))
    p["b3"] = np.array([0.3, -0.2, 1.1])
    theta = mlp.flatten(p)
    X, T = data(rng, 11)
    Y, _ = mlp.forward(theta, X)
    assert np.allclose(Y, p["b3"])
    g = mlp.unflatten(mlp.grad(theta, X, T)[0])
    assert np.allclose(g["b3"], 2 * (p["b3"] - T).mean(0))
    # no gradient reaches the weights through dead (zero) ReLUs except W3's inputs, which are zero
    assert np.abs(g["W3"]).max() == 0 and np.abs(g["W1"]).max() == 0


def test_positive_region_is_the_linear_map():
    rng = np.random.default_rng(5)
    p = {"W1": rng.uniform(0.01, 0.1, (24, 128)), "b1": rng.uniform(0, 0.1, 128),
         "W2": rng.uniform(0.01, 0.1, (128, 128)), "b2": rng.uniform(0, 0.1, 128),
         "W3": rng.normal(size=(128, 3)), "b3": rng.normal(size=3)}
    X = rng.uniform(0, 1, (9, 24))
    Y, _ = mlp.forward(mlp.flatten(p), X)
    lin = ((X @ p["W1"] + p["b1"]) @ p["W2"] + p["b2"]) @ p["W3"] + p["b3"]
    assert np.allclose(Y, lin, rtol=1e-12, atol=1e-12)


def test_adamw_first_step_formula():
    rng = np.random.default_rng(6)
    theta = rng.normal(size=mlp.N_PARAM)
    g = rng.normal(size=mlp.N_PARAM)
    lr, wd = 1e-3, 1e-2
    new, m, v = mlp.adamw(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr, wd=wd, eps=0.0)
    # first step: mhat = g, vhat = g^2 -> update -lr sign(g); decay on weights only
    decay = np.where(mlp.is_bias_mask(), 0.0, wd)
    assert np.allclose(new, theta * (1 - lr * decay) - lr * np.sign(g), rtol=0, atol=1e-15)


def test_recorder_features_of_a_resting_block():
    hx, hy, hz = 0.0375, 0.0125, 0.0075
    m, mu = 0.015, 0.4
    sc = synth.custom_scene([dict(half=(hx, hy, hz), x=(0, 0, hz), mass=m, mu=mu)], ground_mu=mu)
    for k in ("half", "x", "q", "v", "w", "mass", "mu", "ground_mu"):
        setattr(sc, k, getattr(sc, k).astype(float))
    sc.half[:, 0] = (hx, hy, hz); sc.x[:, 0] = (0, 0, hz); sc.mass[:] = m
    W = oracle.World(sc, synth.params(residual_tol=1e-10, pgs_iter_cap=20000))
    W.set_recorder(64, 1)
    W.step(2)
    rows = W.recorded()
    assert len(rows) == 8      # 4 ground points, two steps
    I = oracle.body_inertia(m, [hx, hy, hz]) / (0.015 * 0.075 ** 2)
    gh = 9.81 / 240.0
    for r in rows[:4]:        # first step: nothing to match yet
        assert np.allclose(r[0:3], [-1, 0, 0], atol=1e-12)        # u = -g h along n
        assert abs(r[3]) < 1e-9                                   # touching
        assert np.allclose(r[4:9], [0, 0, 1, 1, 0])
        assert abs(r[9] - 2 * hz / 0.15) < 1e-9                   # column of one block above z = 0
        assert r[10] == 0 and abs(r[11] - 0.015 / m) < 1e-12
        assert np.allclose(r[12:15], 0) and np.allclose(r[15:18], I)
        assert abs(r[18] - mu) < 1e-7 and np.allclose(r[19:23], 0) and r[23] == 1
    assert abs(rows[:4, 24].sum() - m / 0.015) < 1e-9               # total normal impulse m g h
    for r, prev in zip(rows[4:], rows[:4]):   # second step: matched, previous impulses
        assert r[22] == 1
    assert abs(rows[4:, 19].sum() - m / 0.015) < 1e-9


def test_warm_start_match_radius():
    """Warm-start matching (same pair and features, nearest old point within
    2 mm in body-A coordinates): a block on a static block of the same size
    keeps its four points' impulses when slid 1 mm along its length between
    steps.  Slid 3 mm, the two corners on the static block's far edge stay
    put and match; the two that moved with the top block's end do not, and
    start from zero (the recorder's matched flag and previous impulses)."""
    hx, hy, hz = 0.0375, 0.0125, 0.0075
    for shift, n_matched in ((1e-3, 4), (3e-3, 2)):
        sc = synth.custom_scene([dict(half=(hx, hy, hz), x=(0, 0, hz), mass=0.0, mu=0.4),
                                 dict(half=(hx, hy, hz), x=(0, 0, 3 * hz), mass=0.015, mu=0.4)], ground_mu=0.4)
        for k in ("half", "x", "q", "v", "w", "mass", "mu", "ground_mu"):
            setattr(sc, k, getattr(sc, k).astype(float))
        sc.half[:, :] = np.array([hx, hy, hz])[:, None]
        sc.x[:, 0] = (0, 0, hz); sc.x[:, 1] = (0, 0, 3 * hz); sc.mass[:] = (0.0, 0.015)
        W = oracle.World(sc, synth.params(residual_tol=1e-10, pgs_iter_cap=20000))
        W.set_recorder(64, 1)
        W.step(1)
        x, q, v, w = W.state()
        x = x.copy(); x[0, 1] += shift         # slide the top block along its length
        W.set_state(x, q, np.zeros_like(v), np.zeros_like(w))
        W.step(1)
        rows = W.recorded()
        second = rows[4:8]                      # the block-on-block pair's four points, second step
        assert len(second) == 4
        assert int(second[:, 22].sum()) == n_matched
        assert np.all(second[second[:, 22] == 0, 19:22] == 0)
        if n_matched == 4:
            assert abs(second[:, 19].sum() - 0.015 / 0.015) < 1e-6   # previous total normal impulse m g h


def test_recorder_features_of_a_moving_spinning_pair():
    """The A28 features of a block-on-block pair in the air, both moving and
    spinning, masses 2:1: per point, the relative velocity
    (v_B + w_B x r_B) - (v_A + w_A x r_A) after the gravity predictor, in
    the contact frame, over g h; then depth / margin, n, t1.x, t1.y, the
    column height above the point over 0.15 m, the scaled inverse masses
    and inertias of A and B in that order, mu, zero impulses, and the
    unmatched and not-ground flags."""
    hx, hy, hz = 0.0375, 0.0125, 0.0075
    mA, mB, mu, pen = 0.030, 0.015, 0.4, 1e-4
    vA, wA = np.array([0.1, -0.05, 0.02]), np.array([0.5, -0.3, 0.8])
    vB, wB = np.array([-0.07, 0.12, -0.03]), np.array([-0.4, 0.6, 0.2])
    xA, xB = np.array([0.0, 0.0, 1.0]), np.array([0.01, 0.0, 1.0 + 2 * hz - pen])
    sc = synth.custom_scene([dict(half=(hx, hy, hz), x=tuple(xA), v=tuple(vA), w=tuple(wA), mass=mA, mu=mu),
                             dict(half=(hx, hy, hz), x=tuple(xB), v=tuple(vB), w=tuple(wB), mass=mB, mu=mu)],
                            ground_mu=mu)
    for k in ("half", "x", "q", "v", "w", "mass", "mu", "ground_mu"):
        setattr(sc, k, getattr(sc, k).astype(float))
    sc.half[:, :] = np.array([hx, hy, hz])[:, None]
    sc.x[:, 0], sc.x[:, 1] = xA, xB
    sc.v[:, 0], sc.v[:, 1], sc.w[:, 0], sc.w[:, 1] = vA, vB, wA, wB
    sc.mass[:] = (mA, mB); sc.mu[:] = mu
    prm = synth.params(residual_tol=1e-10, pgs_iter_cap=20000)
    W = oracle.World(sc, prm)
    W.set_recorder(64, 1)
    W.step(1)
    rows = W.recorded()
    C = oracle.contact_dicts(W.contacts(0))
    assert len(C) == 1 and (C[0]["a"], C[0]["b"]) == (0, 1) and C[0]["np"] == 4 and len(rows) == 4
    c = C[0]
    gh = 9.81 / 240.0
    g = np.array([0.0, 0.0, -9.81]) / 240.0            # the predictor's h g
    n, t1 = c["n"], c["t1"]
    t2 = np.cross(n, t1)
    scale_I = 1.0 / (0.015 * 0.075 ** 2)
    I_box = lambda m: m / 3.0 * np.array([hy * hy + hz * hz, hx * hx + hz * hz, hx * hx + hy * hy])
    for r, p, d in zip(rows, c["p"], c["depth"]):
        u = (vB + g + np.cross(wB, p - xB)) - (vA + g + np.cross(wA, p - xA))
        assert np.allclose(r[0:3] * gh, [u @ n, u @ t1, u @ t2], atol=1e-13)
        assert abs(r[3] - d / prm["contact_margin"]) < 1e-12
        assert np.allclose(r[4:7], n) and np.allclose(r[7:9], t1[:2])
        # the column above the interface: B's top (1 + 3 hz - pen) minus the
        # point, halfway into the overlap (1 + hz - pen / 2)
        assert abs(p[2] - (1.0 + hz - pen / 2)) < 1e-12
        assert abs(r[9] - (2 * hz - pen / 2) / 0.15) < 1e-10
        assert abs(r[10] - 0.015 / mA) < 1e-12 and abs(r[11] - 0.015 / mB) < 1e-12
        assert np.allclose(r[12:15], I_box(mA) * scale_I, rtol=1e-12)
        assert np.allclose(r[15:18], I_box(mB) * scale_I, rtol=1e-12)
        assert abs(r[18] - mu) < 1e-12 and np.all(r[19:23] == 0) and r[23] == 0


def test_warm_start_match_follows_body_a():
    """Warm-start matching compares points in body A's coordinates: the same
    block-on-block pair, moved rigidly as a whole between steps (turned 20 deg
    about z and shifted 5 cm), keeps all four points' impulses although every
    point moved by more than the 2 mm radius in world coordinates."""
    hx, hy, hz = 0.0375, 0.0125, 0.0075
    sc = synth.custom_scene([dict(half=(hx, hy, hz), x=(0, 0, hz), mass=0.0, mu=0.4),
                             dict(half=(hx, hy, hz), x=(0, 0, 3 * hz), mass=0.015, mu=0.4)], ground_mu=0.4)
    for k in ("half", "x", "q", "v", "w", "mass", "mu", "ground_mu"):
        setattr(sc, k, getattr(sc, k).astype(float))
    sc.half[:, :] = np.array([hx, hy, hz])[:, None]
    sc.x[:, 0] = (0, 0, hz); sc.x[:, 1] = (0, 0, 3 * hz); sc.mass[:] = (0.0, 0.015)
    W = oracle.World(sc, synth.params(residual_tol=1e-10, pgs_iter_cap=20000))
    W.set_recorder(64, 1)
    W.step(1)
    p1 = oracle.contact_dicts(W.contacts(0))[0]["p"]
    x, q, v, w = (a.copy() for a in W.state())
    ang, shift = np.radians(20.0), np.array([0.05, 0.02, 0.0])
    Rz = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]])
    qz = np.array([np.cos(ang / 2), 0, 0, np.sin(ang / 2)])
    for j in range(2):
        x[:, j] = Rz @ x[:, j] + shift
        a, b = qz, q[:, j]                      # q <- qz (x) q
        q[:, j] = [a[0] * b[0] - a[3] * b[3], a[0] * b[1] - a[3] * b[2],
                   a[0] * b[2] + a[3] * b[1], a[0] * b[3] + a[3] * b[0]]
    W.set_state(x, q, np.zeros_like(v), np.zeros_like(w))
    W.step(1)
    c2 = oracle.contact_dicts(W.contacts(0))
    assert len(c2) == 1 and c2[0]["np"] == 4
    moved = np.linalg.norm(c2[0]["p"][:, None, :] - p1[None, :, :], axis=2).min(axis=1)
    assert moved.min() > 0.01                   # far beyond the match radius in world terms
    second = W.recorded()[4:8]
    assert np.all(second[:, 22] == 1)
    assert abs(second[:, 19].sum() - 1.0) < 1e-6   # the previous total normal impulse m g h


def test_column_height_feature_of_a_block_on_its_edge():
    """Feature 9 (the column height above a contact point over 0.15 m) of a
    block resting on one long edge, turned 30 degrees about its length axis
    and 20 degrees about z: the top of the column is the block's centre
    height plus its rotated AABB half-height, sum_j |R_zj| h_j, and every
    ground point lies on z = 0 (touching), so every row carries
    (x_z + e_z) / 0.15; t1.x, t1.y are the ground frame's (1, 0)."""
    hx, hy, hz = 0.0375, 0.0125, 0.0075
    a, c = np.radians(30.0), np.radians(20.0)
    qx = np.array([np.cos(a / 2), np.sin(a / 2), 0.0, 0.0])
    qz = np.array([np.cos(c / 2), 0.0, 0.0, np.sin(c / 2)])
    w0, x0, y0, z0 = qz
    w1, x1, y1, z1 = qx
    q = np.array([w0 * w1 - x0 * x1 - y0 * y1 - z0 * z1, w0 * x1 + x0 * w1 + y0 * z1 - z0 * y1,
                  w0 * y1 - x0 * z1 + y0 * w1 + z0 * x1, w0 * z1 + x0 * y1 - y0 * x1 + z0 * w1])   # qz (x) qx
    R = oracle.rotmat(q)
    ez = abs(R[2, 0]) * hx + abs(R[2, 1]) * hy + abs(R[2, 2]) * hz
    sc = synth.custom_scene([dict(half=(hx, hy, hz), x=(0, 0, ez), q=tuple(q), mass=0.015, mu=0.4)], ground_mu=0.4)
    for k in ("half", "x", "q", "v", "w", "mass", "mu", "ground_mu"):
        setattr(sc, k, getattr(sc, k).astype(float))
    sc.half[:, 0] = (hx, hy, hz); sc.x[:, 0] = (0, 0, ez); sc.q[:, 0] = q; sc.mass[:] = 0.015
    W = oracle.World(sc, synth.params(residual_tol=1e-10, pgs_iter_cap=20000))
    W.set_recorder(64, 1)
    W.step(1)
    rows = W.recorded()
    C = oracle.contact_dicts(W.contacts(0))
    assert len(C) == 1 and C[0]["a"] == -1 and len(rows) == C[0]["np"] >= 2   # an edge: 2 corners
    assert np.allclose(C[0]["p"][:, 2], 0.0, atol=1e-9)
    assert np.allclose(rows[:, 9], 2 * ez / 0.15, atol=1e-9)
    assert np.allclose(rows[:, 7:9], [1.0, 0.0], atol=1e-12)
