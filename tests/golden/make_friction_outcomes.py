"""Writes friction150_outcomes.txt: the FP64 oracle's episode outcomes on a
150-episode subset of the 450-episode removal-round workload (every third
episode: 50 per friction level mu_s in {0.25, 0.40, 0.60}; workload seed 1),
plain sequential PGS in natural order at residual <= 1e-5 m/s (sweep cap
20,000), whole schedules.  The outcomes are those of Sec. 8 (Eq. collapse;
the fallen-block count; the COM imbalance of Eq. stability, minus the
support margin) and of the removal rounds of Sec. 13.1 (moves done).

Run from the repository root:  python tests/golden/make_friction_outcomes.py
It calls only oracle/ and synth/ (about 30-60 min on 8 cores)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "friction150_outcomes.txt")
EPISODES = list(range(0, 450, 3))


def main():
    scene, prot, prm = synth.friction_workload(seed=1)
    prm = dict(prm, residual_tol=1e-5, pgs_iter_cap=20000)
    s, p = synth.subset(scene, prot, EPISODES)
    s64 = synth.Scene(s.body_off, *[getattr(s, k).astype(np.float64) for k in
                                    ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")])
    w = oracle.World(s64, prm)
    w.set_protocol(p)
    t0 = time.time()
    w.run_protocol(max_steps=1 << 30, threads=0)
    dt = time.time() - t0
    st = w.stats()
    with open(OUT, "w") as f:
        f.write("# FP64 oracle outcomes, friction workload (seed 1), episodes 0, 3, ..., 447 of 450;\n")
        f.write("# plain PGS, natural order, residual <= 1e-5 m/s, cap 20000; written by make_friction_outcomes.py\n")
        f.write(f"# oracle run {dt:.0f} s on {oracle.num_threads()} threads\n")
        f.write("# columns: episode mu_s collapsed n_fallen com_imbalance_m moves_done steps status\n")
        for i, e in enumerate(EPISODES):
            f.write(f"{e} {float(s.ground_mu[i]):.2f} {int(st['collapsed'][i])} {int(st['n_fallen'][i])} "
                    f"{float(st['com_imbalance'][i]):.6e} {int(st['moves_done'][i])} {int(st['steps'][i])} "
                    f"{int(st['status'][i])}\n")
    print(OUT, dt)


if __name__ == "__main__":
    main()
