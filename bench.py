"""Benchmark: body-steps/s of the batched block-tower step on GB300.

Workload: the 450-episode, three-friction removal-round batch (150 episodes at
each mu_s in {0.25, 0.40, 0.60}, 18-level towers of 0.075 x 0.025 x 0.015 m
blocks, 15 g +- 2 %, 1..8 removals of non-top blocks pushed along block X or Y
at U[0.8, 1.5] x the Ziglar threshold, 0.5 s push + 1 s settle each), solved in
residual mode (PGS residual <= 1e-5 m/s), dt = 1/240 s, plain PGS with
previous-frame warm start.  Synthetic, seeded inputs stand in for the paper's
episode data.

One bench step = the whole job: every episode run through its schedule to the
end in one persistent launch (jb_run_protocol).  value = body-steps of all
episodes / device time; e2e = the same through the C ABI from host buffers
(batch upload, schedule upload, run, statistics readback) timed on the host.

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

# algorithmic flops per unit of work (FMA = 2): PGS row work per contact point
# per sweep, contact setup per point, SAT + manifold per kept pair, AABB test
# per candidate pair, integration per body
FLOP_POINT_SWEEP = 162.0
FLOP_POINT_SETUP = 180.0
FLOP_PAIR = 750.0
FLOP_BP = 12.0
FLOP_BODY = 60.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--warmup-steps", type=int, default=24,
                    help="physics steps per warm-up pass (the job truncated)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--episodes", type=int, default=0, help="use the first n episodes (0 = all 450)")
    ap.add_argument("--max-steps", type=int, default=1 << 30, help="cap physics steps per episode")
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--accel", type=int, default=64,
                    help="PGS acceleration: a nonsmooth conjugate-gradient step every this many sweeps (0 = plain PGS)")
    ap.add_argument("--cap", type=int, default=20000)
    ap.add_argument("--fixed-iters", type=int, default=0,
                    help="fixed-sweep mode with this many sweeps per solve (profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--compare-seeds", type=int, default=3,
                    help="seeds of the workload on which both warm-start arms run (the benchmark's first)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the learned-vs-plain comparison over seeds and the unaccelerated plain arm")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="friction", choices=["friction", "ragged", "stress"],
                    help="friction: 450 x 18-level towers (the headline); ragged: 4096 towers of 6-30 levels; "
                         "stress: 48-level towers (152 of the 16384 unless --episodes)")
    ap.add_argument("--stall-window", type=int, default=0,
                    help="residual mode: stop a solve whose residual trend over this many sweeps cannot reach "
                         "the tolerance within the cap (0 = run every solve to the tolerance or the cap)")
    ap.add_argument("--autotune", action="store_true", help="pick smem_pair_factor and the residual-check cadence by trials")
    ap.add_argument("--warm-start", default="learned", choices=["learned", "plain"],
                    help="learned: train the warm-start network first and keep it if the gate passes")
    ap.add_argument("--train-episodes", type=int, default=96,
                    help="learned path: episodes (other seeds) whose converged solves make the training set")
    ap.add_argument("--collect-steps", type=int, default=1 << 30, help="steps of their schedule to record")
    ap.add_argument("--collect-every", type=int, default=1, help="record every n-th converged solve")
    ap.add_argument("--collect-all-points", dest="collect_unmatched", action="store_false",
                    help="record every point of a recorded solve, not only the points without a "
                         "previous-frame impulse")
    ap.add_argument("--train-rows", type=int, default=5_000_000)
    ap.add_argument("--gate-episodes", type=int, default=48)
    ap.add_argument("--gate-steps", type=int, default=480)
    ap.add_argument("--k-rule", default="axis", choices=["axis", "ziglar"],
                    help="push threshold multiplier: axis (Y 3, X 4; the workload's schedule) or ziglar "
                         "(Tab. ziglar's move classes: side X 4, centre X and Y 3)")
    ap.add_argument("--claims", action="store_true",
                    help="evaluate Sec. 13.2's three claims over three seeds and both k rules (plain PGS), "
                         "print one JSON line and exit")
    ap.add_argument("--cpu-episodes", type=int, default=0)
    ap.add_argument("--cpu-steps", type=int, default=30)
    ap.add_argument("--cpu-whole", type=int, default=16,
                    help="cpu_baseline: the oracle over the whole schedules of this many sampled episodes "
                         "(about 80 s on 16 Grace cores; 0 = only the cold-start sample)")
    return ap.parse_args()


def make_workload(kind, seed, k_rule="axis"):
    if kind == "ragged":
        return synth.ragged_workload(seed=seed)
    if kind == "stress":
        return synth.stress_workload(seed=seed)
    return synth.friction_workload(seed=seed, k_rule=k_rule)


WORKLOAD_SEED = {"friction": 1, "ragged": 2, "stress": 5}
WORKLOAD_NAME = {"friction": "450 episodes x 18-level towers, mu {0.25,0.40,0.60} x 150, removal rounds",
                 "ragged": "4096 episodes, levels U{6..30}, mu U[0.2,0.7], removal rounds",
                 "stress": "48-level towers, mu cycling {0.25,0.40,0.60}, one X push at 2x threshold "
                           "on a level in 10..30, 720 steps"}


def workload(args, rank, seed=None):
    kind = getattr(args, "workload", "friction")
    scene, prot, prm = make_workload(kind, (WORKLOAD_SEED[kind] if seed is None else seed) + rank,
                                     getattr(args, "k_rule", "axis"))
    if kind == "stress" and not args.episodes:
        args.episodes = 152     # one 48-level episode per SM of the 16384
    if args.episodes:
        # spread the subset over the three friction levels
        E = scene.n_episodes
        idx = np.linspace(0, E - 1, args.episodes).round().astype(int)
        scene, prot = synth.subset(scene, prot, idx)
    prm = dict(prm, residual_tol=args.tol, pgs_iter_cap=args.cap, stall_window=getattr(args, "stall_window", 0),
               pgs_accel_period=getattr(args, "accel", 0))
    if args.fixed_iters:
        prm = dict(prm, residual_tol=0.0, pgs_iters=args.fixed_iters)
    return scene, prot, prm


def reduce_ranks(times_ms, walls_s, body_steps, device, dist=None):
    """Whole-job aggregation over ranks: the slowest rank's device time and
    host time (MAX) against the body-steps of all ranks (SUM).  Ranks share
    no data on the step itself; only these totals cross ranks."""
    import torch
    t = torch.tensor([float(times_ms), float(walls_s)], device=device, dtype=torch.float64)
    tot = torch.tensor([float(body_steps)], device=device, dtype=torch.float64)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(t[0].item()), float(t[1].item()), float(tot[0].item())


MLP_FLOP = 2.0 * (24 * 128 + 128 * 128 + 128 * 3)   # per predicted contact point

# DRAM bytes (read + write) of episode_kernel per body-step, from one ncu
# capture of a small case of the same workload (counters stay off the full
# job), scaled to a launch by its body-steps: the traffic is the per-step
# contact records and warm-start caches of each episode plus the initial state
# load, so it grows with the episode-steps run.  Captured with
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
#  -k regex:episode_kernel -s 3 -c 1 python bench.py --warm-start plain --no-cpu --no-compare
#  --episodes 45 --max-steps 300 --steps 1 --warmup 3` (1 pass).  Valid only for
# the kernel sources it was taken on; any change to them reports null.
TRAFFIC = {"bytes_per_body_step": (1827072.0 + 4494336.0) / 720900.0, "case": "45 episodes x 300 steps",
           "workload": "friction", "sources_sha1": "aa1b20f3193efea79f4f102c42c73221450e6143"}


def kernel_sources_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("jb_kernels.cu", "jb_internal.cuh", "jb_mlp.cuh"):
        with open(os.path.join(ROOT, "paper_2606_28394_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def prepare_learned(args, rank, prm, device):
    """Trains the warm-start network and gates it against plain PGS.
    Samples: the plain solver's converged impulses on removal-round towers with
    other seeds than the benchmark (training 3001 + rank, gate 4001 + rank)."""
    from paper_2606_28394_gb300 import warmstart as ws
    import torch
    t0 = time.perf_counter()
    sc, pr, _ = make_workload(args.workload, 3001 + rank)
    s_tr, p_tr = synth.subset(sc, pr, np.linspace(0, sc.n_episodes - 1, args.train_episodes).round().astype(int))
    # the training set: the plain solver's converged impulses at the points the
    # network will predict (no previous-frame impulse), from every solve
    rows = ws.collect(s_tr, p_tr, prm, capacity=args.train_rows, every=args.collect_every,
                      max_steps=args.collect_steps, device=device, unmatched_only=args.collect_unmatched)
    t1 = time.perf_counter()
    net, hist = ws.train(rows, epochs=30, batch=8192, lr=3e-4, wd=1e-4, device=device)
    torch.cuda.synchronize(device)
    t2 = time.perf_counter()
    sc2, pr2, _ = make_workload(args.workload, 4001 + rank)
    s_ev, p_ev = synth.subset(sc2, pr2, np.linspace(0, sc2.n_episodes - 1, args.gate_episodes).round().astype(int))
    # the gate: both warm starts from identical states along plain PGS's
    # trajectory (the network's own effect, free of trajectory divergence)
    gate = ws.paired(s_ev, p_ev, prm, net, steps=args.gate_steps, mode=2, device=device)
    # whole trajectories of both arms on the same episodes (context)
    traj = ws.evaluate(s_ev, p_ev, prm, net, mode=2, max_steps=args.gate_steps, device=device)
    s_cold, _ = synth.subset(sc2, pr2, np.linspace(0, sc2.n_episodes - 1, 10).round().astype(int))
    cold = ws.cold_start_gain(s_cold, prm, net, steps=12, device=device)
    t3 = time.perf_counter()
    info = {"samples": int(rows.shape[0]), "collect_s": t1 - t0, "train_s": t2 - t1, "gate_s": t3 - t2,
            "epochs": 30, "final_train_loss": hist[-1][1], "final_val_loss": hist[-1][2],
            "cold_contacts": {"episodes": 10, "steps": 12, "plain_sweeps_per_solve": cold[0],
                              "learned_sweeps_per_solve": cold[1], "gain": cold[2]},
            "gate": {"episodes": args.gate_episodes, "steps": args.gate_steps,
                     "kind": "paired: both warm starts solve every step from the same snapshot along plain "
                             "PGS's trajectory",
                     "plain_sweeps": float(gate["plain"].sum()), "learned_sweeps": float(gate["learned"].sum()),
                     "first_step_gain": float(gate["plain"][0] / max(gate["learned"][0], 1.0)),
                     "gain": gate["gain"], "learned_capped": gate["learned_capped"],
                     "plain_body_steps_per_s": gate["body_steps"] / max(gate["plain_ms"] * 1e-3, 1e-12),
                     "learned_body_steps_per_s": gate["body_steps"] / max(gate["learned_ms"] * 1e-3, 1e-12),
                     "learned_over_plain": gate["plain_ms"] / max(gate["learned_ms"], 1e-12)},
            "trajectories": {"episodes": args.gate_episodes, "steps": args.gate_steps,
                             "plain_sweeps_per_solve": traj["plain"]["sweeps_per_solve"],
                             "learned_sweeps_per_solve": traj["learned"]["sweeps_per_solve"],
                             "gain": traj["gain"]},
            "kept": bool(gate["gain"] > 1.0)}
    return net, info


def pinned_inputs(scene, prot, torch):
    """Copies of the scene and schedule arrays in page-locked host memory
    (numpy views of pinned tensors; same dtypes and shapes)."""
    from types import SimpleNamespace

    def pin(a):
        a = np.ascontiguousarray(a)
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0].copy()).dtype, pin_memory=True)
        out = t.numpy()
        out[...] = a
        return out

    sc = SimpleNamespace(**{k: pin(getattr(scene, k)) for k in
                            ("body_off", "half", "mass", "mu", "x", "q", "v", "w", "ground_mu")})
    sc.n_episodes, sc.n_bodies = int(scene.n_episodes), int(scene.n_bodies)
    pr = SimpleNamespace(**{k: pin(getattr(prot, k)) for k in
                            ("off", "block", "axis", "sign", "factor", "k", "remove", "push_steps", "settle_steps")})
    return sc, pr


def outcomes(scene, prot, st):
    """The friction experiment's table (Tab. results) from the batch: per mu,
    collapsed episodes N_c, mean rounds (moves performed) and the share of
    moves pushed along block X (Ziglar's torque moves, 4 mu m g)."""
    mu = np.asarray(scene.ground_mu, float)
    out = {}
    for m in sorted(set(np.round(mu, 2))):
        sel = np.where(np.abs(mu - m) < 5e-3)[0]
        done = st["moves_done"][sel]
        axes = [prot.axis[prot.off[e]:prot.off[e] + int(d)] for e, d in zip(sel, done)]
        n_moves = int(sum(len(a) for a in axes))
        n_x = int(sum(int((a == synth.AXIS_X).sum()) for a in axes))
        out[f"{m:.2f}"] = {"episodes": int(len(sel)), "collapsed": int(st["collapsed"][sel].sum()),
                           "mean_rounds": float(done.mean()) if len(sel) else 0.0,
                           "torque_move_pct": 100.0 * n_x / max(n_moves, 1)}
    # collapse rate per kind of move (Sec. 13.2's comparison): the moves each
    # episode attempted (those done plus the one in progress at a collapse),
    # by slot (centre = 1) and push axis; a collapse is charged to its move
    kinds = {}
    for e in range(len(mu)):
        n_att = int(st["moves_done"][e]) + (1 if st["collapsed"][e] else 0)
        n_att = min(n_att, int(prot.off[e + 1] - prot.off[e]))
        for j in range(n_att):
            mv = int(prot.off[e]) + j
            slot = int(prot.block[mv]) % 3
            key = ("centre" if slot == 1 else "side") + ("_x" if int(prot.axis[mv]) == synth.AXIS_X else "_y")
            kd = kinds.setdefault(key, [0, 0])
            kd[0] += 1
            kd[1] += int(bool(st["collapsed"][e]) and j == n_att - 1)
    out["by_move"] = {k: {"moves": v[0], "collapses": v[1], "rate": v[1] / max(v[0], 1)} for k, v in sorted(kinds.items())}
    # Eq. stability as an early warning: the device's per-step margin went
    # negative before (or at) the step where Eq. collapse fired
    if "first_unstable_step" in st:
        col = np.asarray(st["collapsed"]) > 0
        fu, cs = np.asarray(st["first_unstable_step"]), np.asarray(st["collapse_step"])
        warned = col & (fu >= 1) & (fu <= cs)
        lead = (cs - fu)[warned]
        out["early_warning"] = {"collapsed": int(col.sum()), "warned_before_collapse": int(warned.sum()),
                                "median_lead_steps": float(np.median(lead)) if len(lead) else None,
                                "standing_with_negative_margin": int(((~col) & (fu >= 1)).sum()),
                                "standing": int((~col).sum())}
    return out


def algorithmic_flops(st):
    return (FLOP_POINT_SWEEP * st["point_sweeps"].sum() + FLOP_POINT_SETUP * st["point_steps"].sum()
            + FLOP_PAIR * st["pair_steps"].sum() + FLOP_BP * st["bp_tests"].sum()
            + FLOP_BODY * st["body_steps"].sum())


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,utilization.gpu,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return False
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)
        return False

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        num = lambda s: float(s) if s.replace(".", "", 1).isdigit() else float("nan")
        load = [r for r in self.rows if num(r[2]) > 0] or self.rows
        sm = [num(r[0]) for r in load]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": num(self.rows[0][1]), "reasons": reasons,
                "samples": len(self.rows)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def cpu_baseline(args, scene, prot, prm):
    """FP64 oracle on the host cores, on a bounded sample of the same workload:
    the first `cpu_steps` steps of `cpu_episodes` episodes spread over the batch."""
    import oracle
    ncores = oracle.num_threads()
    ne = args.cpu_episodes or ncores
    idx = np.linspace(0, scene.n_episodes - 1, ne).round().astype(int)
    s, p = synth.subset(scene, prot, idx)
    s64 = synth.Scene(s.body_off, *[getattr(s, k).astype(np.float64) for k in
                                    ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")])
    w = oracle.World(s64, dict(prm, pgs_accel_period=0, colour_order=0))
    w.set_protocol(p)
    t0 = time.perf_counter()
    w.run_protocol(max_steps=args.cpu_steps, threads=ncores)
    dt = time.perf_counter() - t0
    st = w.stats()
    bs = float(st["body_steps"].sum())
    return {"value": bs / dt, "unit": "body-steps/s", "cores": ncores, "kind": "oracle",
            "sample": f"first {args.cpu_steps} steps of {ne} of the {scene.n_episodes} episodes "
                      f"(evenly spaced over the three mu levels), FP64, plain PGS in natural order, "
                      f"OpenMP over episodes",
            "seconds": dt, "episodes": ne,
            "sweeps_per_solve": float(st["total_sweeps"].sum() / max(st["solves"].sum(), 1))}


def cpu_whole_schedules(args, scene, prot, prm):
    """The oracle over the whole schedules of a sample of episodes (the same
    work per episode as the GPU job), FP64 plain PGS in natural order."""
    import oracle
    ncores = oracle.num_threads()
    idx = np.linspace(0, scene.n_episodes - 1, args.cpu_whole).round().astype(int)
    s, p = synth.subset(scene, prot, idx)
    s64 = synth.Scene(s.body_off, *[getattr(s, k).astype(np.float64) for k in
                                    ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")])
    w = oracle.World(s64, dict(prm, pgs_accel_period=0, colour_order=0))
    w.set_protocol(p)
    t0 = time.perf_counter()
    w.run_protocol(max_steps=1 << 30, threads=ncores)
    dt = time.perf_counter() - t0
    st = w.stats()
    return {"value": float(st["body_steps"].sum()) / dt, "unit": "body-steps/s", "cores": ncores, "kind": "oracle",
            "sample": f"whole schedules of {args.cpu_whole} of the {scene.n_episodes} episodes (evenly spaced), "
                      f"FP64, plain PGS in natural order, OpenMP over episodes",
            "seconds": dt, "episodes": args.cpu_whole, "idx": idx.tolist(),
            "sweeps_per_solve": float(st["total_sweeps"].sum() / max(st["solves"].sum(), 1))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scene, prot, prm = workload(args, 0)
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(args, scene, prot, prm)
        if i >= args.warmup:
            vals.append(cb)
    v = statistics.mean(c["value"] for c in vals)
    line = {"impl": "reference", "metric": "body-steps/s at PGS residual <= 1e-5: learned warm start vs plain PGS",
            "value": v, "unit": "body-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(c["seconds"] for c in vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME[args.workload] if not args.episodes else
                       f"{args.episodes} episodes (evenly spaced) of: {WORKLOAD_NAME[args.workload]}",
                       "residual_tol": args.tol, "pgs_iter_cap": args.cap, "sample": vals[0]["sample"]},
            "cpu_baseline": {k: vals[0][k] for k in ("kind", "cores", "sample")} | {"value": v, "unit": "body-steps/s"},
            "e2e": {"value": v, "unit": "body-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def claims(args):
    """Sec. 13.2's three claims on the friction workload, per seed and per
    threshold rule: (1) side_yaxis moves collapse less often than side_xaxis
    moves; (2) the centre block pushed along X (center_xaxis) is the safest
    move; (3) the collapse rate falls as mu_s rises.  A collapse is charged to
    the move in progress.  Forces are F = k mu_s m g, so the pushes scale with
    the friction they meet: nothing in the schedule makes higher mu_s safer,
    and claim (3) can only come from the dynamics."""
    import torch
    import paper_2606_28394_gb300 as jb
    dev = torch.device("cuda", 0)
    out = {"claims": "Sec. 13.2: side_y < side_x; centre_x safest; collapse rate falls with mu_s", "runs": []}
    for rule in ("axis", "ziglar"):
        for sd in COMPARE_SEEDS:
            a2 = argparse.Namespace(**vars(args))
            a2.k_rule = rule
            sc, pr, prm = workload(a2, 0, seed=sd)
            b = jb.Batch(sc, dict(prm, warm_start=1), max_moves=int(pr.off[-1]), device=dev)
            b.set_protocol(pr)
            b.run_protocol(1 << 30)
            st = b.stats()
            o = outcomes(sc, pr, st)
            by = o["by_move"]
            rates = {k: v["rate"] for k, v in by.items()}
            per_mu = [o[m]["collapsed"] / o[m]["episodes"] for m in ("0.25", "0.40", "0.60")]
            out["runs"].append({"k_rule": rule, "seed": sd, "by_move": by, "collapse_rate_per_mu": per_mu,
                                "claim1_side_y_below_side_x": rates.get("side_y", 0) < rates.get("side_x", 0),
                                "claim2_centre_x_safest": rates.get("centre_x", 1) <= min(rates.values()),
                                "claim3_falls_with_mu": per_mu[0] > per_mu[1] > per_mu[2]})
    for rule in ("axis", "ziglar"):
        runs = [r for r in out["runs"] if r["k_rule"] == rule]
        out[rule] = {c: sum(r[c] for r in runs) for c in ("claim1_side_y_below_side_x", "claim2_centre_x_safest",
                                                           "claim3_falls_with_mu")} | {"seeds": len(runs)}
    print(json.dumps(out))


def fp32_peak(jb, torch, dev, stream):
    """The FP32 multiply-add rate of this GPU, measured with the library's own
    probe kernel (8 independent FMA chains per thread, 8 CTAs of 256 threads
    per SM, scalar FFMA and packed FFMA2), CUDA events on the launching
    stream, best of 5 launches each after a warm-up launch."""
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = 8 * nsm, 1 << 13
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    out = {"sms": nsm, "blocks": blocks, "threads": 256, "iters": iters}
    for packed, name in ((0, "ffma"), (1, "ffma2")):
        flops = jb.jb_fma_probe_flops(packed, blocks, iters)
        best = float("inf")
        for rep in range(6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            jb.check(jb.jb_fma_probe(packed, blocks, iters, sink.data_ptr(), C_stream(stream)), "jb_fma_probe")
            e1.record(stream)
            e1.synchronize()
            if rep:
                best = min(best, e0.elapsed_time(e1))
        out[name + "_tflops"] = flops / (best / 1e3) / 1e12
    out["peak_tflops"] = max(out["ffma_tflops"], out["ffma2_tflops"])
    return out


def C_stream(stream):
    return stream.cuda_stream


COMPARE_SEEDS = (1, 1001, 2001)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.claims:
        return claims(args)
    import torch
    import torch.distributed as dist
    import paper_2606_28394_gb300 as jb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    scene, prot, prm = workload(args, rank)
    # the job's host inputs live in pinned memory (numpy views of pinned
    # tensors), as a caller streaming batches would keep them
    scene, prot = pinned_inputs(scene, prot, torch)
    M = int(prot.off[-1])
    stream = torch.cuda.current_stream(dev)
    ws = jb.Batch(scene, prm, max_moves=M, stream=stream, device=dev).workspace   # allocated once
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    def io_bytes(sc, pr):
        h2d = (sc.body_off.nbytes + sc.half.nbytes + sc.mass.nbytes + sc.mu.nbytes
               + sc.x.nbytes + sc.q.nbytes + sc.v.nbytes + sc.w.nbytes + sc.ground_mu.nbytes
               + sum(getattr(pr, f).nbytes for f in ("off", "block", "axis", "sign", "factor", "k",
                                                      "remove", "push_steps", "settle_steps")))
        return h2d, sc.n_episodes * jb.C.sizeof(jb.jb_episode_stats)

    h2d, d2h = io_bytes(scene, prot)
    peak = fp32_peak(jb, torch, dev, stream)

    tuning = None
    if args.autotune:
        from paper_2606_28394_gb300 import autotune
        prm, table = autotune.tune(scene, prot, prm, device=dev)
        tuning = {"choice": {k: prm[k] for k in autotune.TUNED}, "trials": table}
    net, learned = None, None
    if args.warm_start == "learned":
        net, learned = prepare_learned(args, rank, prm, dev)
    plain_prm = dict(prm, warm_start=1)
    learned_prm = dict(prm, warm_start=2) if net is not None else None
    kept = bool(learned and learned["kept"])
    run_prm = learned_prm if kept else plain_prm

    launches = [1]

    def job(max_steps, params=None, sc=None, pr=None, work=None):
        """One pass through the C ABI from host buffers: create the batch
        (scene upload), upload the schedule, run every episode through it in
        one persistent launch, read the statistics back.  CUDA events bracket
        the launch (inputs resident); the host clock brackets the whole pass."""
        params = params or run_prm
        sc = sc if sc is not None else scene
        pr = pr if pr is not None else prot
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        b = jb.Batch(sc, params, max_moves=int(pr.off[-1]), stream=stream, device=dev,
                     workspace=work if work is not None else ws)
        launches[0] = len(b.size_classes())     # episode-kernel launches per run_protocol
        if params["warm_start"] >= 2:
            jb.check(jb.jb_set_warmstart_mlp(b.h, net.block.data_ptr()), "jb_set_warmstart_mlp")
        b.set_protocol(pr)
        e0.record(stream)
        b.run_protocol(max_steps)
        e1.record(stream)
        st = b.stats()
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        barrier()
        return e0.elapsed_time(e1), t1 - t0, st

    def rate(ms, st):
        return float(st["body_steps"].sum()) / (ms / 1e3)

    def sps(st):
        return float(st["total_sweeps"].sum() / max(st["solves"].sum(), 1))

    # warm-up: the same launch path on the job truncated to a few physics steps
    for _ in range(args.warmup):
        job(min(args.warmup_steps, args.max_steps))
    times, walls = [], []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            ms_i, wall_i, st = job(args.max_steps)
            times.append(ms_i)
            walls.append(wall_i)
    ms = float(sum(times))
    body_steps = float(st["body_steps"].sum())
    flops = algorithmic_flops(st)
    mlp_flops = MLP_FLOP * float(st["mlp_points"].sum())
    ms_max, wall_max, total_body_steps = reduce_ranks(ms, sum(walls), body_steps * args.steps, dev,
                                                       dist if world > 1 else None)
    value = total_body_steps / (ms_max / 1e3)

    # learned warm start against plain PGS: both arms on the same job, for
    # the benchmark's seed and two more seeds of the same workload (whole
    # episodes are chaotic, so one seed's ratio carries trajectory noise)
    compare = None
    if net is not None and not args.no_compare:
        per_seed = []
        seeds = (WORKLOAD_SEED[args.workload],) + tuple(sd for sd in COMPARE_SEEDS if sd != WORKLOAD_SEED[args.workload])
        for sd in seeds[:max(1, args.compare_seeds)]:
            if sd == WORKLOAD_SEED[args.workload]:
                sc_s, pr_s = scene, prot
            else:
                a2 = argparse.Namespace(**vars(args))
                sc_s, pr_s, _ = workload(a2, rank, seed=sd)
                sc_s, pr_s = pinned_inputs(sc_s, pr_s, torch)
            arms = {}
            for name, p_ in (("plain", plain_prm), ("learned", learned_prm)):
                if sc_s is scene and p_ is run_prm:
                    arms[name] = (ms / args.steps, st)   # the timed runs above
                else:
                    ms_a, _, st_a = job(args.max_steps, p_, sc_s, pr_s)
                    arms[name] = (ms_a, st_a)
            per_seed.append({"seed": sd, "plain_body_steps_per_s": rate(*arms["plain"]),
                             "learned_body_steps_per_s": rate(*arms["learned"]),
                             "plain_sweeps_per_solve": sps(arms["plain"][1]),
                             "learned_sweeps_per_solve": sps(arms["learned"][1]),
                             "learned_points": float(arms["learned"][1]["mlp_points"].sum()),
                             "point_solves": float(arms["learned"][1]["point_steps"].sum()),
                             "learned_over_plain": rate(*arms["learned"]) / rate(*arms["plain"]),
                             "plain_over_learned_sweeps": float(arms["plain"][1]["total_sweeps"].sum()
                                                                / max(arms["learned"][1]["total_sweeps"].sum(), 1))})
        ratios = [r["learned_over_plain"] for r in per_seed]
        work = [r["plain_over_learned_sweeps"] for r in per_seed]
        compare = {"seeds": per_seed, "learned_over_plain_mean": statistics.mean(ratios),
                   "learned_over_plain_min": min(ratios), "learned_over_plain_max": max(ratios),
                   "plain_over_learned_sweeps_mean": statistics.mean(work),
                   "plain_over_learned_sweeps_min": min(work), "plain_over_learned_sweeps_max": max(work),
                   "note": "each seed: the whole 450-episode job once per arm; the body-steps/s ratio follows "
                           "the busiest (collapsing, chaotic) episode of each arm, so it spreads across seeds; "
                           "the total-sweeps ratio is the work saved, and the time saved wherever the GPU is "
                           "filled (the work inside one seed is deterministic)"}
    # the paper's plain PGS without the conjugate-gradient steps, same job (context)
    unaccel = None
    if prm.get("pgs_accel_period", 0) and not args.no_compare:
        ms_u, _, st_u = job(args.max_steps, dict(plain_prm, pgs_accel_period=0))
        unaccel = {"value": rate(ms_u, st_u), "ms_per_step": ms_u, "sweeps_per_solve": sps(st_u),
                   "capped_fraction": float(st_u["capped_solves"].sum() / max(st_u["solves"].sum(), 1))}
    e2e = None
    if not args.no_e2e:
        e2e = {"value": total_body_steps / wall_max, "unit": "body-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "gpu_launches_per_step": 4 + launches[0],
               "note": "host wall clock over jb_batch_create (scene upload from pinned host arrays), "
                       "jb_set_protocol, jb_run_protocol, jb_read_episode_stats"}

    peaks = load_peaks()
    peak_tf = peak["peak_tflops"]
    achieved = flops / (ms / args.steps / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": achieved / peak_tf,
            "traffic": (TRAFFIC["bytes_per_body_step"] * body_steps
                        if (TRAFFIC["bytes_per_body_step"] and TRAFFIC["sources_sha1"] == kernel_sources_sha1()
                            and args.workload == TRAFFIC["workload"] and not args.fixed_iters) else None),
            "traffic_note": f"ncu DRAM bytes per body-step on {TRAFFIC['case']} of this workload x the launch's "
                            f"body-steps",
            "mlp_flops_per_launch": mlp_flops,
            "mlp_roofline_ms": mlp_flops / (float(peaks.get("bf16_tflops", 1892.9)) * 1e12) * 1e3,
            "peak_note": (f"measured FP32 multiply-add rate of this GPU (jb_fma_probe, {peak['sms']} SMs from the "
                          f"device, {peak['blocks']} CTAs x 256 threads x 8 chains, best of 5): FFMA "
                          f"{peak['ffma_tflops']:.1f}, FFMA2 {peak['ffma2_tflops']:.1f} TFLOP/s; peak = the larger"),
            "kernel": "episode_kernel (persistent, one warp per episode)",
            "flops_per_launch": flops,
            "work_basis": "algorithmic flops per unit x the GPU's own sweeps (colour order, conjugate-gradient "
                          "steps every pgs_accel_period sweeps, residual checks at an adaptive cadence)"}
    line = {"metric": "body-steps/s at PGS residual <= 1e-5: learned warm start vs plain PGS",
            "value": value, "unit": "body-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": (WORKLOAD_NAME[args.workload] if not args.episodes else
                                    f"{args.episodes} episodes (evenly spaced) of: {WORKLOAD_NAME[args.workload]}")
                                   + (f", fixed {args.fixed_iters} sweeps (profiling)" if args.fixed_iters else ""),
                       "residual_tol": args.tol, "pgs_iter_cap": args.cap, "max_steps": args.max_steps,
                       "pgs_accel_period": prm.get("pgs_accel_period", 0),
                       "stall_window": jb.params_from_dict(run_prm).stall_window,
                       "residual_check_every": [jb.params_from_dict(run_prm).residual_every,
                                                jb.params_from_dict(run_prm).residual_every_max],
                       "l2": "flushed (256 MB write) before every timed step",
                       "warmup": f"{args.warmup} passes of the job truncated to {args.warmup_steps} physics steps",
                       "episodes": scene.n_episodes, "bodies": scene.n_bodies},
            "warm_start": {"mode": "learned (network on the points of new pairs, previous-frame elsewhere)"
                           if kept else "plain (previous-frame)"
                           + (": the gate rejected the network" if learned else ""),
                           "training": learned, "comparison": compare,
                           "learned_over_plain": compare["learned_over_plain_mean"] if compare else None,
                           "learned_over_plain_identical_states": (learned["gate"]["learned_over_plain"]
                                                                   if learned else None)},
            "plain_pgs_unaccelerated": unaccel,
            "autotune": tuning,
            "roofline": roof, "fp32_probe": peak, "gpu_launches": args.steps * launches[0],
            "clocks": clk.summary(),
            "e2e": e2e,
            "solver": {"sweeps_per_solve": sps(st),
                       "not_converged_episodes": int(((st["status"] & jb.JB_EP_NOT_CONVERGED) != 0).sum()),
                       "solves": float(st["solves"].sum()),
                       "capped_solves": int(st["capped_solves"].sum()),
                       "capped_fraction": float(st["capped_solves"].sum() / max(st["solves"].sum(), 1)),
                       "capped_in_collapsed_episodes": int(st["capped_solves"][st["collapsed"] > 0].sum()),
                       "sweeps_share_busiest_over_mean": float(st["total_sweeps"].max() / max(st["total_sweeps"].mean(), 1)),
                       "collapsed": int(st["collapsed"].sum()), "body_steps_per_job": body_steps,
                       "max_colours": int(st["max_colours"].max()),
                       # critical path: job time over the busiest episode's sweeps
                       "us_per_sweep_busiest_episode": ms / args.steps * 1e3 / float(st["total_sweeps"].max()),
                       "fixed_iters": args.fixed_iters}}
    line["outcomes"] = outcomes(scene, prot, st)
    if rank == 0 and not args.no_cpu:
        cb = cpu_baseline(args, scene, prot, prm)
        # the GPU on the CPU leg's sample (same episodes, same steps): the same work side by side
        idx = np.linspace(0, scene.n_episodes - 1, cb["episodes"]).round().astype(int)
        s_c, p_c = synth.subset(scene, prot, idx)
        b = jb.Batch(s_c, plain_prm, max_moves=int(p_c.off[-1]), stream=stream, device=dev)
        b.set_protocol(p_c)
        b.run_protocol(args.cpu_steps)
        st_c = b.stats()
        cb["gpu_sweeps_per_solve_same_sample"] = sps(st_c)
        line["cpu_baseline"] = cb
        if args.cpu_whole:
            # the representative leg: whole schedules, the GPU job's own work per episode
            cw = cpu_whole_schedules(args, scene, prot, prm)
            s_w, p_w = synth.subset(scene, prot, cw.pop("idx"))
            b = jb.Batch(s_w, plain_prm, max_moves=int(p_w.off[-1]), stream=stream, device=dev)
            b.set_protocol(p_w)
            b.run_protocol(1 << 30)
            cw["gpu_sweeps_per_solve_same_sample"] = sps(b.stats())
            cw["cold_start_sample"] = cb
            line["cpu_baseline"] = cw
            # the work rate counted on the paper's plain PGS sweeps (the oracle's natural
            # order over the same whole schedules) rather than on the GPU's own
            roof["frac_on_plain_pgs_sweeps"] = (roof["frac"] * cw["sweeps_per_solve"]
                                                / max(cw["gpu_sweeps_per_solve_same_sample"], 1e-9))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
