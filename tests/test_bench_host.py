"""Host-side logic of the benchmark (CPU only): the algorithmic flop count,
the friction-table outcomes and the multi-rank reduction's shape."""
import numpy as np

import bench
import synth


def fake_stats(n, **kw):
    st = {k: np.zeros(n) for k in ("point_sweeps", "point_steps", "pair_steps", "bp_tests", "body_steps",
                                   "collapsed", "moves_done", "mlp_points")}
    st.update({k: np.asarray(v, float) for k, v in kw.items()})
    return st


def test_algorithmic_flops_per_unit():
    st = fake_stats(2, point_sweeps=[10, 5], point_steps=[2, 0], pair_steps=[1, 1], bp_tests=[3, 0],
                    body_steps=[4, 4])
    want = 162 * 15 + 180 * 2 + 750 * 2 + 12 * 3 + 60 * 8
    assert bench.algorithmic_flops(st) == want
    # an intact 18-level episode-step at 30 sweeps (768 points, 192 pairs, 1,431 candidate pairs) is ~4.05 Mflop
    ex = fake_stats(1, point_sweeps=[768 * 30], point_steps=[768], pair_steps=[192], bp_tests=[1431],
                    body_steps=[54])
    assert abs(bench.algorithmic_flops(ex) - 4.05e6) < 0.02e6


def test_outcomes_table_counts_moves_and_collapses():
    towers = [synth.Tower(levels=4, mu=m) for m in (0.25, 0.25, 0.6)]
    scene = synth.build_scene(towers, 0)
    # three moves each: (block, axis, sign, factor, k, remove, push, settle)
    moves = [[(1, synth.AXIS_X, 1, 1, 4, 1, 1, 1), (3, synth.AXIS_Y, 1, 1, 3, 1, 1, 1), (4, synth.AXIS_Y, 1, 1, 3, 1, 1, 1)],
             [(0, synth.AXIS_Y, 1, 1, 3, 1, 1, 1), (7, synth.AXIS_X, 1, 1, 4, 1, 1, 1), (2, synth.AXIS_X, 1, 1, 4, 1, 1, 1)],
             [(4, synth.AXIS_X, 1, 1, 4, 1, 1, 1), (5, synth.AXIS_Y, 1, 1, 3, 1, 1, 1), (6, synth.AXIS_Y, 1, 1, 3, 1, 1, 1)]]
    prot = synth._protocol(moves, 3)
    # episode 0 finished all three moves; episode 1 collapsed during its 2nd
    # move; episode 2 collapsed during its 1st
    st = fake_stats(3, moves_done=[3, 1, 0], collapsed=[0, 1, 1])
    out = bench.outcomes(scene, prot, st)
    assert out["0.25"] == {"episodes": 2, "collapsed": 1, "mean_rounds": 2.0, "torque_move_pct": 25.0}
    assert out["0.60"]["collapsed"] == 1 and out["0.60"]["mean_rounds"] == 0.0
    by = out["by_move"]
    # attempted: ep0 blocks 1(centre,X) 3(side,Y) 4(centre,Y); ep1 0(side,Y) 7(centre,X, collapse);
    # ep2 4(centre,X, collapse)
    assert by["centre_x"] == {"moves": 3, "collapses": 2, "rate": 2 / 3}
    assert by["centre_y"]["moves"] == 1 and by["centre_y"]["collapses"] == 0
    assert by["side_y"] == {"moves": 2, "collapses": 0, "rate": 0.0}
