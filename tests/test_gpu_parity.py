"""GPU (FP32, coloured PGS) against the FP64 oracle, through the C ABI.

Tolerances:
  - contact sets: identical pairs (a, b, SAT axis, reference/incident features)
    except pairs whose separation is within 1e-6 m of the -margin threshold;
    depths and point offsets along the normal within 2e-6 m (FP32 rounding of
    0.3 m coordinates is ~3e-8 m per operation), offsets in the contact plane
    within 2e-5 m (a clip vertex where an incident edge meets a side plane at
    a shallow angle theta is only determined to ~eps32 |x| / sin(theta)),
    normals within 1e-5;
  - one step from an identical state with both solvers converged to a PGS
    residual <= 1e-5 m/s: positions within 1e-5 m, velocities within 1e-4 m/s
    (angular velocity scaled by the block's half diagonal).  The residual
    bounds the relative velocity at each contact; a body's velocity adds those
    along its chain of contacts to the ground, so on an n-level stack two
    solutions at residual tol may differ by up to ~2 n tol.  The parity cases
    therefore converge both solvers to 1e-6 (which is <= 1e-5), giving
    2 * 18 * 1e-6 < 1e-4 on the 18-level tower.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

MC = 1e-3   # contact margin


def jb():
    import paper_2606_28394_gb300 as m
    return m


def as64(scene):
    s = synth.Scene(scene.body_off, *[getattr(scene, k).astype(np.float64) for k in
                                      ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")])
    return s


def gpu_contacts(batch, e):
    arr = jb().contacts_as_arrays(batch.contacts(e))
    pairs = {}
    for i in range(len(arr["a"])):
        key = (int(arr["a"][i]), int(arr["b"][i]))
        d = pairs.setdefault(key, dict(axis=int(arr["axis"][i]), ref=int(arr["ref_face"][i]),
                                       inc=int(arr["inc_face"][i]), n=arr["n"][i], p=[], depth=[], lam=[]))
        d["p"].append(arr["p"][i]); d["depth"].append(arr["depth"][i]); d["lam"].append(arr["lam"][i])
    return pairs


def oracle_contacts(world, e):
    out = {}
    for r in oracle.contact_dicts(world.contacts(e)):
        out[(r["a"], r["b"])] = dict(axis=r["axis"], ref=r["ref_face"], inc=r["inc_face"], n=r["n"],
                                     p=list(r["p"]), depth=list(r["depth"]), lam=list(r["lam"]))
    return out


def near_threshold(scene, e, key, tol=1e-6):
    """True if the pair's detection sits within tol of the margin threshold (FP64)."""
    a, b = key
    o = scene.body_off[e]
    S = as64(scene)
    xb, qb, hb = S.x[:, o + b], S.q[:, o + b], S.half[:, o + b]
    if a < 0:
        R = oracle.rotmat(qb / np.linalg.norm(qb))
        zs = [xb[2] + R[2] @ (np.array([sx, sy, sz]) * hb) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
        return min(abs(z - MC) for z in zs) < tol
    r = oracle.sat(S.x[:, o + a], S.q[:, o + a], S.half[:, o + a], xb, qb, hb, margin=MC)
    return abs(r["dmin"] + MC) < tol


def compare_contact_sets(scene, g, o, e=0):
    only_g = set(g) - set(o)
    only_o = set(o) - set(g)
    for key in only_g | only_o:
        assert near_threshold(scene, e, key), ("pair only on one side", key, key in g)
    n_pts = 0
    for key in set(g) & set(o):
        G, O = g[key], o[key]
        assert (G["axis"], G["ref"], G["inc"]) == (O["axis"], O["ref"], O["inc"]), key
        assert np.abs(np.asarray(G["n"]) - O["n"]).max() < 1e-5, key
        pg, po = np.asarray(G["p"]), np.asarray(O["p"])
        dg, do = np.asarray(G["depth"]), np.asarray(O["depth"])
        if len(pg) != len(po):
            # only allowed when a point sits at the depth threshold
            assert np.min(np.abs(np.r_[dg, do] + MC)) < 1e-6, key
            continue
        nrm = np.asarray(O["n"])
        for i in range(len(pg)):
            j = np.argmin(np.linalg.norm(po - pg[i], axis=1))
            d = po[j] - pg[i]
            # across the face: FP32 rounding of the geometry; along the face: a
            # clip vertex on an edge meeting a side plane at a shallow angle
            # theta moves by ~eps32 |x| / sin(theta)
            assert abs(d @ nrm) < 2e-6 and abs(do[j] - dg[i]) < 2e-6, (key, pg[i], po[j])
            assert np.linalg.norm(d - (d @ nrm) * nrm) < 2e-5, (key, pg[i], po[j])
        n_pts += len(pg)
    return n_pts


def step_both(scene, prm, n=1):
    b = jb().Batch(scene, prm)
    w = oracle.World(as64(scene), prm)
    b.step(n)
    w.step(n)
    return b, w


SCENES = {
    "tower18": lambda: synth.build_scene([synth.Tower()], 0),
    "tower18_perturbed": lambda: synth.perturbed(synth.build_scene([synth.Tower()], 0), 3, dx=3e-4, dang=0.02),
    "pile": lambda: synth.pile_scene(28, seed=5),
    "pile2": lambda: synth.pile_scene(40, seed=11, spread=0.12),
    # 48 levels (the full-collapse stress towers): 144 bodies, ~530 pairs; a
    # jitter seed whose SAT decisions are all clear of ties
    "tower48_perturbed": lambda: synth.perturbed(synth.build_scene([synth.Tower(levels=48)], 0), 9,
                                                 dx=3e-4, dang=0.02),
}


@pytest.mark.parametrize("name", sorted(SCENES))
def test_contact_sets_match_oracle(cuda_device, name):
    scene = SCENES[name]()
    if name == "tower48_perturbed":
        assert oracle.sat_decisions_clear(scene)
    prm = synth.params(pgs_iters=1)
    b, w = step_both(scene, prm)
    g, o = gpu_contacts(b, 0), oracle_contacts(w, 0)
    assert len(o) > 0
    n = compare_contact_sets(scene, g, o)
    assert n > 0


def test_free_fall_closed_form_fp32(cuda_device):
    sc = synth.custom_scene([dict(half=(0.0375, 0.0125, 0.0075), x=(0, 0, 2.0), mass=0.015)])
    b = jb().Batch(sc, synth.params())
    n = 37
    b.step(n)
    x, _, v, _ = b.state()
    h = 1 / 240
    assert abs(v[2, 0] + 9.81 * n * h) < 2e-6
    assert abs(x[2, 0] - (2.0 - 9.81 * h * h * n * (n + 1) / 2)) < 2e-6


def velocity_error(scene, v1, w1, v2, w2):
    diag = np.sqrt((scene.half.astype(float) ** 2).sum(0))
    return np.max(np.abs(v1 - v2)), np.max(np.abs(w1 - w2).max(0) * diag)


@pytest.mark.parametrize("name,tol", [("tower4_perturbed", 1e-6), ("pile", 1e-6), ("tower18", 1e-6),
                                      ("tower24", 1e-6)])
def test_one_step_converged_parity(cuda_device, name, tol):
    if name == "tower24":
        scene = synth.build_scene([synth.Tower(levels=24)], 0)
    elif name == "tower4_perturbed":
        scene = synth.perturbed(synth.build_scene([synth.Tower(levels=4, mu=0.5)], 1), 5, dx=2e-4, dang=0.01)
    elif name == "pile":
        scene = synth.pile_scene(28, seed=5)
    else:
        scene = synth.build_scene([synth.Tower()], 0)
    prm = synth.params(residual_tol=tol, pgs_iter_cap=200000)
    b, w = step_both(scene, prm)
    st = b.stats()
    assert st["status"][0] == 0 and st["last_residual"][0] <= tol
    so = w.stats()
    assert so["last_residual"][0] <= tol
    xg, qg, vg, wg = b.state()
    xo, qo, vo, wo = w.state()
    assert np.abs(xg - xo).max() < 1e-5
    ev, ew = velocity_error(scene, vg, wg, vo, wo)
    assert ev < 1e-4 and ew < 1e-4, (ev, ew)


def test_resting_tower_18_levels_gpu(cuda_device):
    """The GPU path on the 18-level resting tower for 2 s: max penetration
    < 1e-5 m and max point speed < 1e-4 m/s (as the oracle's pin)."""
    scene = synth.build_scene([synth.Tower()], 0)
    b = jb().Batch(scene, synth.params(residual_tol=1e-6, pgs_iter_cap=50000))
    diag = np.sqrt((scene.half.astype(float) ** 2).sum(0))
    maxpen = maxspeed = 0.0
    for _ in range(48):
        b.step(10)
        _, _, v, w = b.state()
        arr = jb().contacts_as_arrays(b.contacts(0))
        maxpen = max(maxpen, arr["depth"].max())
        maxspeed = max(maxspeed, (np.linalg.norm(v, axis=0) + np.linalg.norm(w, axis=0) * diag).max())
    assert maxpen < 1e-5 and maxspeed < 1e-4, (maxpen, maxspeed)


def test_push_force_threshold_gpu(cuda_device):
    m = 0.0196
    sc = synth.custom_scene([dict(half=(0.0405, 0.013, 0.009), x=(0, 0, 3.0), mass=m, mu=0.4)])
    b = jb().Batch(sc, synth.params(), max_moves=1)
    b.set_protocol(synth._protocol([[(0, synth.AXIS_Y, 1.0, 1.0, 3.0, 0, 1, 0)]], 1))
    b.run_protocol(1)
    _, _, v, _ = b.state()
    F = m * v[0, 0] * 240
    assert abs(F * 1e3 - 230.7) < 0.06


def test_determinism_and_snapshot_resume(cuda_device):
    scene = synth.perturbed(synth.build_scene([synth.Tower(levels=6), synth.Tower(levels=5)], 2), 4)
    prm = synth.params(residual_tol=1e-5, pgs_iter_cap=20000)
    a = jb().Batch(scene, prm)
    a.step(10)
    snap = a.save_state()
    a.step(15)
    xa = a.state()
    b = jb().Batch(scene, prm)
    b.step(25)
    xb = b.state()
    for u, v in zip(xa, xb):
        assert np.array_equal(u, v)
    a.load_state(snap)
    a.step(15)
    for u, v in zip(a.state(), xb):
        assert np.array_equal(u, v)


def test_protocol_runs_and_matches_oracle_outcomes(cuda_device):
    """Removal rounds on short towers that all stand: both sides run the same schedule to the end, every tower stands
    with nothing fallen on both, and the body-step counts are identical (the
    schedule decides them when nothing collapses).  Outcome statistics of
    collapsing episodes are compared on the headline workload in
    test_gpu_outcomes.py."""
    towers = [synth.Tower(levels=5, mu=m) for m in (0.25, 0.4, 0.6, 0.4)]
    scene = synth.build_scene(towers, 9)
    prot = synth.removal_protocol(towers, 9, push_steps=30, settle_steps=60, max_removals=2)
    prm = synth.params(residual_tol=1e-5, pgs_iter_cap=20000)
    b = jb().Batch(scene, prm, max_moves=int(prot.off[-1]))
    b.set_protocol(prot)
    b.run_protocol()
    w = oracle.World(as64(scene), prm)
    w.set_protocol(prot)
    w.run_protocol()
    sg, so = b.stats(), w.stats()
    assert (sg["phase"] == jb().JB_PH_DONE).all()
    assert (so["phase"] == oracle.PH_DONE).all()
    assert (sg["moves_done"] == so["moves_done"]).all()
    assert (so["collapsed"] == 0).all() and (so["n_fallen"] == 0).all()
    assert (sg["collapsed"] == 0).all() and (sg["n_fallen"] == 0).all()
    assert np.array_equal(sg["body_steps"], so["body_steps"])


def test_host_commands_and_removal(cuda_device):
    scene = synth.build_scene([synth.Tower(levels=3)], 0)
    b = jb().Batch(scene, synth.params())
    b.remove_block([0], [7])
    b.apply_push([0], [1], [synth.AXIS_Y], [0.5], [20])
    b.step(20)
    act = b.active()
    assert not act[7] and act.sum() == 8
    for c in b.contacts(0):
        assert 7 not in (c.a, c.b)
    with pytest.raises(jb().JBError):
        b.remove_block([0], [99])
    with pytest.raises(jb().JBError):
        b.apply_push([1], [0], [0], [0.1], [1])


@pytest.mark.parametrize("sor,order", [(1.4, 0), (1.0, 1), (1.3, 1)])
@pytest.mark.parametrize("name", ["tower4_perturbed", "tower18", "pile"])
def test_relaxed_and_symmetric_sweeps_converge_to_the_oracle(cuda_device, name, sor, order):
    """Over-relaxed rows (projected SOR) and reversed odd sweeps change the
    iterates, not the fixed point: converged to 1e-6 the step matches the
    oracle's plain sequential PGS within the same bounds.  On the pile the
    velocity bound is not asserted: its contact system is ill-conditioned,
    so a residual of 1e-6 bounds the velocity error less tightly (an
    over-relaxed iterate stopped at 1e-6 was 2e-4 m/s, angular scaled by the
    half diagonal, from the oracle's, whose own iterate at 1e-6 lies 2e-5
    from its limit); positions and the residual are."""
    if name == "tower4_perturbed":
        scene = synth.perturbed(synth.build_scene([synth.Tower(levels=4, mu=0.5)], 1), 5, dx=2e-4, dang=0.01)
    elif name == "pile":
        scene = synth.pile_scene(28, seed=5)
    else:
        scene = synth.build_scene([synth.Tower()], 0)
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000)
    b = jb().Batch(scene, dict(prm, sor=sor, sweep_order=order))
    w = oracle.World(as64(scene), prm)
    b.step(1)
    w.step(1)
    st = b.stats()
    assert st["status"][0] == 0 and st["last_residual"][0] <= 1e-6
    xg, qg, vg, wg = b.state()
    xo, qo, vo, wo = w.state()
    assert np.abs(xg - xo).max() < 1e-5
    if name != "pile":
        ev, ew = velocity_error(scene, vg, wg, vo, wo)
        assert ev < 1e-4 and ew < 1e-4, (ev, ew)


def test_relaxation_one_is_plain_pgs_bit_for_bit(cuda_device):
    scene = synth.perturbed(synth.build_scene([synth.Tower(levels=6)], 2), 4, dx=2e-4, dang=0.01)
    prm = synth.params(residual_tol=1e-5, pgs_iter_cap=20000)
    a = jb().Batch(scene, prm)
    b = jb().Batch(scene, dict(prm, sor=1.0, sweep_order=0))
    a.step(5)
    b.step(5)
    for u, v in zip(a.state(), b.state()):
        assert np.array_equal(u, v)


def test_bad_relaxation_is_refused(cuda_device):
    scene = synth.build_scene([synth.Tower(levels=2)], 0)
    for bad in (dict(sor=2.0), dict(sor=-0.5), dict(sweep_order=2)):
        with pytest.raises(jb().JBError):
            jb().Batch(scene, synth.params(**bad))


def test_capped_solves_are_counted(cuda_device):
    """A tolerance no solve can reach: every solve ends at the cap and is
    counted, and the episode carries the not-converged flag."""
    scene = synth.perturbed(synth.build_scene([synth.Tower(levels=3)], 1), 2, dx=2e-4, dang=0.01)
    b = jb().Batch(scene, synth.params(residual_tol=1e-12, pgs_iter_cap=40))
    b.step(3)
    st = b.stats()
    assert st["capped_solves"][0] == 3 and st["solves"][0] == 3
    assert st["status"][0] & jb().JB_EP_NOT_CONVERGED
    ok = jb().Batch(scene, synth.params(residual_tol=1e-5, pgs_iter_cap=200000))
    ok.step(3)
    assert ok.stats()["capped_solves"][0] == 0


def test_stall_window_stops_hopeless_solves_early(cuda_device):
    """With a tolerance FP32 cannot reach, the stall test ends each solve
    long before the cap and counts it as capped; off (0), the solve runs to
    the cap."""
    scene = synth.perturbed(synth.build_scene([synth.Tower(levels=3)], 1), 2, dx=2e-4, dang=0.01)
    prm = synth.params(residual_tol=1e-12, pgs_iter_cap=20000)
    b = jb().Batch(scene, dict(prm, stall_window=256))
    b.step(2)
    st = b.stats()
    assert st["capped_solves"][0] == 2 and st["last_sweeps"][0] < 20000 // 4
    off = jb().Batch(scene, prm)
    off.step(1)
    assert off.stats()["last_sweeps"][0] == 20000
    with pytest.raises(jb().JBError):
        jb().Batch(scene, dict(prm, stall_window=-1))


def test_cone_friction_sliding_block_fp32(cuda_device):
    """The cone variant on the GPU: the diagonal slide keeps its direction
    and loses mu g h of speed per step (FP32)."""
    sc = synth.custom_scene([dict(half=(0.0375, 0.0125, 0.0075), x=(0, 0, 0.0075), mass=0.015, mu=0.4)],
                            ground_mu=0.4)
    sc.v[:, 0] = (0.5 * math.cos(math.radians(30)), 0.5 * math.sin(math.radians(30)), 0.0)
    b = jb().Batch(sc, synth.params(residual_tol=1e-7, pgs_iter_cap=200000, friction_cone=1))
    b.step(10)
    x, q, v, w = b.state()
    assert abs(math.hypot(v[0, 0], v[1, 0]) - (0.5 - 10 * 0.4 * 9.81 / 240)) < 2e-6
    assert abs(math.degrees(math.atan2(v[1, 0], v[0, 0])) - 30.0) < 1e-3


@pytest.mark.parametrize("name", ["tower4_perturbed", "tower18", "pile"])
def test_cone_friction_converges_to_the_oracle(cuda_device, name):
    if name == "tower4_perturbed":
        scene = synth.perturbed(synth.build_scene([synth.Tower(levels=4, mu=0.5)], 1), 5, dx=2e-4, dang=0.01)
    elif name == "pile":
        scene = synth.pile_scene(28, seed=5)
    else:
        scene = synth.build_scene([synth.Tower()], 0)
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000, friction_cone=1)
    b, w = step_both(scene, prm)
    st = b.stats()
    assert st["status"][0] == 0 and st["last_residual"][0] <= 1e-6
    assert w.stats()["last_residual"][0] <= 1e-6
    xg, qg, vg, wg = b.state()
    xo, qo, vo, wo = w.state()
    assert np.abs(xg - xo).max() < 1e-5
    if name != "pile":          # the pile's conditioning, as for relaxed sweeps
        ev, ew = velocity_error(scene, vg, wg, vo, wo)
        assert ev < 1e-4 and ew < 1e-4, (ev, ew)


def test_paper_block_with_three_substeps(cuda_device):
    """The paper's own configuration (Appendix A): 8.1 x 2.6 x 1.8 cm blocks
    of 19.6 g and three substeps per step, converged, against the oracle
    with the same settings."""
    tower = synth.Tower(levels=6, dims=(0.081, 0.026, 0.018), mass=0.0196, mu=0.4)
    scene = synth.perturbed(synth.build_scene([tower], 3), 7, dx=2e-4, dang=0.01)
    assert oracle.sat_decisions_clear(scene)
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000, n_sub=3)
    b, w = step_both(scene, prm, n=2)
    assert (b.stats()["status"] == 0).all()
    xg, qg, vg, wg = b.state()
    xo, qo, vo, wo = w.state()
    assert np.abs(xg - xo).max() < 1e-5
    ev, ew = velocity_error(scene, vg, wg, vo, wo)
    assert ev < 1e-4 and ew < 1e-4, (ev, ew)


def test_subthreshold_pushes_agree_with_the_oracle(cuda_device):
    """Whole episodes compared by outcome: 100 12-level towers, one push of
    a middle block at 0.5-0.9 of its Ziglar threshold (Y: 3 mu m g, X:
    4 mu m g), then a settle.  Topple/no-topple and the fallen-block count
    agree on at least 99 %, and the COM imbalance of at least 99 % of the
    standing towers within 1 mm.  Not all: a centre block rests under the
    upper layer's blocks as the middle of three supports, a load split the
    rigid contact problem leaves open, so its friction capacity, and whether
    a push at 0.9 of the nominal threshold moves it, depends on the split
    each solver's sweep order settles on."""
    scene, prot, prm = synth.subthreshold_workload(levels=12)
    b = jb().Batch(scene, prm, max_moves=int(prot.off[-1]))
    b.set_protocol(prot)
    b.run_protocol()
    w = oracle.World(as64(scene), prm)
    w.set_protocol(prot)
    w.run_protocol()
    sg, so = b.stats(), w.stats()
    assert (sg["phase"] == jb().JB_PH_DONE).all() and (so["phase"] == oracle.PH_DONE).all()
    assert (sg["collapsed"] == so["collapsed"]).mean() >= 0.99
    assert (sg["n_fallen"] == so["n_fallen"]).mean() >= 0.99
    standing = (sg["collapsed"] == 0) & (so["collapsed"] == 0)
    assert standing.mean() >= 0.95
    d = np.abs(sg["com_imbalance"][standing] - so["com_imbalance"][standing])
    assert (d < 1e-3).mean() >= 0.99, np.sort(d)[-3:]


def test_single_push_configuration_matches_the_oracle(cuda_device):
    """The single-tower configuration: 18 levels, mu 0.40, the middle block
    of level 9 pushed along Y at 1.05 x 3 mu m g for 0.5 s, 2 s in all, at
    residual 1e-5.  Converged, the loaded block does not slide (friction
    from the blocks above exceeds the push); both agree on that, on the
    outcome and on the final COM imbalance."""
    scene, prot, prm = synth.single_push_workload()
    prm = dict(prm, residual_tol=1e-5, pgs_iter_cap=20000)
    b = jb().Batch(scene, prm, max_moves=int(prot.off[-1]))
    b.set_protocol(prot)
    b.run_protocol()
    w = oracle.World(as64(scene), prm)
    w.set_protocol(prot)
    w.run_protocol()
    sg, so = b.stats(), w.stats()
    assert sg["steps"][0] == so["steps"][0] == 480
    assert sg["collapsed"][0] == so["collapsed"][0] == 0 and sg["n_fallen"][0] == so["n_fallen"][0] == 0
    blk = 8 * 3 + 1
    xg, xo = b.state()[0], w.state()[0]
    assert np.abs(xg[:, blk] - scene.x[:, blk]).max() < 2e-5
    assert np.abs(xo[:, blk] - scene.x[:, blk]).max() < 2e-5
    assert np.abs(xg - xo).max() < 5e-5
    assert abs(sg["com_imbalance"][0] - so["com_imbalance"][0]) < 1e-4


def test_speculative_contact_and_baumgarte_closed_forms_fp32(cuda_device):
    """The oracle's closed-form pins, in FP32 on the GPU: a block 0.5 mm
    above the ground falling at 1 m/s ends the step exactly touching with
    v_z = -gap/h; a block sunk 2 mm is raised by beta (depth - slop)."""
    h, hz, gap, d, beta, slop = 1.0 / 240.0, 0.0075, 5e-4, 2e-3, 0.35, 4e-4
    prm = synth.params(residual_tol=1e-9, pgs_iter_cap=200000)
    sc = synth.custom_scene([dict(half=(0.0375, 0.0125, hz), x=(0, 0, hz + gap), mass=0.015)])
    sc.v[2, 0] = -1.0
    b = jb().Batch(sc, prm)
    b.step(1)
    x, q, v, w = b.state()
    assert abs(x[2, 0] - hz) < 2e-7 and abs(v[2, 0] + gap / h) < 1e-4
    sc2 = synth.custom_scene([dict(half=(0.0375, 0.0125, hz), x=(0, 0, hz - d), mass=0.015)])
    b2 = jb().Batch(sc2, prm)
    b2.step(1)
    x2 = b2.state()[0]
    assert abs(x2[2, 0] - (hz - d + beta * (d - slop))) < 2e-7


def test_episode_statistics_on_hand_set_states(cuda_device):
    """Collapse bookkeeping (Eq. collapse terms, Eq. stability) on states
    written through the C ABI: kinetic energy, fallen count and COM
    imbalance against the oracle on the same states."""
    sc = synth.build_scene([synth.Tower(levels=3, mass_jitter=0.0), synth.Tower(levels=5)], 0)
    b = jb().Batch(sc, synth.params())
    w = oracle.World(as64(sc), synth.params())
    x, q, v, om = (a.astype(np.float64).copy() for a in (sc.x, sc.q, sc.v, sc.w))
    L = 2 * float(sc.half[0, 4])
    x[0, 4] += 0.6 * L
    x[1, 12] -= 0.3 * L
    ang = math.radians(40.0)
    c, s = math.cos(ang / 2), math.sin(ang / 2)
    q0 = q[:, 7].copy()
    q[:, 7] = [c * q0[0] - s * q0[1], c * q0[1] + s * q0[0], c * q0[2] - s * q0[3], c * q0[3] + s * q0[2]]
    v[:, 2] = (0.3, 0, 0)
    om[:, 15] = (0, 0, 2.0)
    b.write_state(x, q, v, om)
    w.set_state(x, q, v, om)
    sg = b.stats()
    for e in range(2):
        ek, dxr, th, nf = w.collapse_terms(e)
        assert sg["n_fallen"][e] == nf
        assert abs(sg["kinetic"][e] - ek) <= 1e-5 * ek + 1e-12
        assert abs(sg["com_imbalance"][e] - w.com_imbalance(e)) < 1e-6


@pytest.mark.parametrize("accel", [0, 64])
def test_full_friction_batch_sampled_against_the_oracle(cuda_device, accel):
    """The 450-episode batch in the benchmark's launch configuration (one
    persistent launch, every episode resident; plain and accelerated
    sweeps): one converged step from the initial state on the GPU, and six
    sampled episodes recomputed by the oracle's plain PGS, within the
    one-step parity bounds."""
    scene, prot, prm = synth.friction_workload(seed=1)
    prm = dict(prm, residual_tol=1e-6, pgs_iter_cap=200000)
    b = jb().Batch(scene, dict(prm, pgs_accel_period=accel))
    b.step(1)
    st = b.stats()
    assert (st["status"] == 0).all() and (st["last_residual"] <= 1e-6).all()
    x, q, v, w = b.state()
    sample = [0, 77, 151, 224, 300, 449]
    sub, _ = synth.subset(scene, prot, sample)
    o = oracle.World(as64(sub), prm)
    o.step(1)
    xo, qo, vo, wo = o.state()
    idx = np.concatenate([np.arange(scene.body_off[e], scene.body_off[e + 1]) for e in sample])
    assert np.abs(x[:, idx] - xo).max() < 1e-5
    ev, ew = velocity_error(sub, v[:, idx], w[:, idx], vo, wo)
    assert ev < 1e-4 and ew < 1e-4, (ev, ew)


def test_newton_restitution_fp32_and_parity(cuda_device):
    """Newton restitution on the GPU: the touching block moving down at
    1 m/s bounces at e (1 + g h); the default keeps the listing's (1+e)
    factor and stops it.  A flush 4-level tower landing at 0.3 m/s bounces
    as one body at e (0.3 + g h), the oracle's state with the same option."""
    h, e, hz = 1.0 / 240.0, 0.1, 0.0075
    for newton, expect in ((1, e * (1.0 + 9.81 * h)), (0, 0.0)):
        sc = synth.custom_scene([dict(half=(0.0375, 0.0125, hz), x=(0, 0, hz), mass=0.015)])
        sc.v[2, 0] = -1.0
        b = jb().Batch(sc, synth.params(residual_tol=1e-8, pgs_iter_cap=200000, restitution_newton=newton))
        b.step(1)
        assert abs(b.state()[2][2, 0] - expect) < 2e-5, (newton, b.state()[2][2, 0])
    scene = synth.build_scene([synth.Tower(levels=4, mu=0.5)], 1)
    scene.v[2, :] = -0.3       # the whole tower lands: only the ground contacts approach
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000, restitution_newton=1)
    b, w = step_both(scene, prm)
    assert b.stats()["status"][0] == 0
    xg, qg, vg, wg = b.state()
    xo, qo, vo, wo = w.state()
    assert np.abs(vg[2] - e * (0.3 + 9.81 * h)).max() < 1e-5
    assert np.abs(xg - xo).max() < 1e-5
    ev, ew = velocity_error(scene, vg, wg, vo, wo)
    assert ev < 1e-4 and ew < 1e-4, (ev, ew)


@pytest.mark.parametrize("accel,key", [(0, 0), (4, 0), (0, 1)])
@pytest.mark.parametrize("name", ["tower18", "tower4_perturbed", "tower30"])
def test_fixed_sweeps_match_the_oracle_in_colour_order(cuda_device, name, accel, key):
    """With the oracle sweeping in the library's colour order, the iterates
    themselves agree, not only the fixed point: one step of 20 fixed sweeps
    (far from converged) gives the same state up to FP32 rounding.  This
    checks the sweep arithmetic (the point-block rows, the packed impulse
    application, the colour schedule) row for row, and with accel = 4 the
    five conjugate-gradient steps in between (direction, beta, restart,
    projection, impulse application); with key = 1 the height-bin colouring.
    A 30-level tower's colours hold 28-46 pairs, so there lanes also sweep
    two pairs of a colour in one pass."""
    if name == "tower18":
        scene = synth.build_scene([synth.Tower()], 0)
    elif name == "tower30":
        scene = synth.build_scene([synth.Tower(levels=30)], 0)
    else:
        scene = synth.perturbed(synth.build_scene([synth.Tower(levels=4, mu=0.5)], 1), 5, dx=2e-4, dang=0.01)
    prm = synth.params(pgs_iters=20, pgs_accel_period=accel)
    b = jb().Batch(scene, dict(prm, colour_key=key))
    w = oracle.World(as64(scene), dict(prm, colour_order=1 + key))
    b.step(1)
    w.step(1)
    xg, qg, vg, wg = b.state()
    xo, qo, vo, wo = w.state()
    assert np.abs(xg - xo).max() < 1e-6
    ev, ew = velocity_error(scene, vg, wg, vo, wo)
    assert ev < 1e-5 and ew < 1e-5, (ev, ew)
    # the natural order's iterate is measurably different: the agreement is the order's
    wn = oracle.World(as64(scene), prm)
    wn.step(1)
    assert np.abs(wn.state()[2] - vo).max() > 1e-5
    if accel:
        # and so is the plain solve's in the same order: the agreement is the acceleration's
        wp = oracle.World(as64(scene), dict(prm, colour_order=1 + key, pgs_accel_period=0))
        wp.step(1)
        assert np.abs(wp.state()[2] - vo).max() > 1e-5


@pytest.mark.parametrize("period", [8, 64])
@pytest.mark.parametrize("name", ["tower4_perturbed", "tower18", "pile"])
def test_accelerated_solve_converges_to_the_oracle(cuda_device, name, period):
    """The conjugate-gradient acceleration changes the iterates and the sweep
    count, not the fixed point: converged to 1e-6 the GPU's accelerated step
    matches the oracle's plain sequential PGS within the one-step bounds
    (the pile: positions and the residual, as for the relaxed sweeps), in
    fewer sweeps than the GPU's own plain solve."""
    if name == "tower4_perturbed":
        scene = synth.perturbed(synth.build_scene([synth.Tower(levels=4, mu=0.5)], 1), 5, dx=2e-4, dang=0.01)
    elif name == "pile":
        scene = synth.pile_scene(28, seed=5)
    else:
        scene = synth.build_scene([synth.Tower()], 0)
    prm = synth.params(residual_tol=1e-6, pgs_iter_cap=200000)
    b = jb().Batch(scene, dict(prm, pgs_accel_period=period))
    p = jb().Batch(scene, prm)
    w = oracle.World(as64(scene), prm)
    b.step(1)
    p.step(1)
    w.step(1)
    st = b.stats()
    assert st["status"][0] == 0 and st["last_residual"][0] <= 1e-6
    if name == "tower18":
        assert st["last_sweeps"][0] < p.stats()["last_sweeps"][0], (st["last_sweeps"][0], p.stats()["last_sweeps"][0])
    xg, qg, vg, wg = b.state()
    xo, qo, vo, wo = w.state()
    assert np.abs(xg - xo).max() < 1e-5
    if name != "pile":
        ev, ew = velocity_error(scene, vg, wg, vo, wo)
        assert ev < 1e-4 and ew < 1e-4, (ev, ew)
