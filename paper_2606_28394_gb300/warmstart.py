"""Learned warm start: collect samples, train, evaluate, gate.

The network and its training run in the library's kernels (jb_mlp_*): BF16
tensor-core operands with FP32 accumulation and FP32 master weights.  This
module only allocates device memory (torch), slices the recorded rows into
minibatches and drives the calls.  Plain PGS with previous-frame warm start
is the yardstick: `evaluate` runs the same episodes with and without the
network and the gate keeps the network only if it needs fewer sweeps per
solve.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import (JB_ECUDA, Batch, JBError, check, jb_mlp_bytes, jb_mlp_forward, jb_mlp_grad, jb_mlp_load, jb_mlp_param_count,
               jb_mlp_save, jb_mlp_scratch_bytes, jb_mlp_scratch_error, jb_mlp_train_step, jb_set_recorder,
               jb_set_recorder_points, jb_set_warmstart_mlp,
               _fp)

N_IN, N_HID, N_OUT = 24, 128, 3
REC = 27


def he_init(seed=0):
    """He-normal weights, zero biases, flat in the layout of jb_mlp_load."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, shape in ((N_IN, (N_IN, N_HID)), (None, (N_HID,)), (N_HID, (N_HID, N_HID)), (None, (N_HID,)),
                          (N_HID, (N_HID, N_OUT)), (None, (N_OUT,))):
        parts.append(rng.normal(0, math.sqrt(2.0 / fan_in), shape).ravel() if fan_in else np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


class Network:
    """A network block on the device (jb_mlp_bytes) plus training scratch."""

    def __init__(self, params=None, device="cuda", seed=0):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.block = torch.zeros(jb_mlp_bytes(), dtype=torch.uint8, device=self.device)
        self.nparam = jb_mlp_param_count()
        self.step_count = 0
        self._scratch = None
        self.load(he_init(seed) if params is None else params)

    @property
    def stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def load(self, params):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == self.nparam
        check(jb_mlp_load(self.block.data_ptr(), p.ctypes.data_as(_fp), self.stream), "jb_mlp_load")
        self.step_count = 0

    def params(self):
        out = np.zeros(self.nparam, np.float32)
        check(jb_mlp_save(self.block.data_ptr(), out.ctypes.data_as(_fp), self.stream), "jb_mlp_save")
        return out

    def scratch(self, n):
        need = jb_mlp_scratch_bytes(int(n))
        if self._scratch is None or self._scratch.numel() < need:
            self._scratch = self.torch.empty(need, dtype=self.torch.uint8, device=self.device)
        return self._scratch

    def check_kernel(self):
        """Raises if the last tensor-core launch on this scratch gave up
        waiting for its matrix products (its outputs are then not valid)."""
        if self._scratch is None:
            return
        flag = C.c_int32(0)
        check(jb_mlp_scratch_error(self._scratch.data_ptr(), self._scratch.numel(), self.stream, C.byref(flag)),
              "jb_mlp_scratch_error")
        if flag.value:
            raise JBError(JB_ECUDA, "warm-start network kernel: a tensor-core wait ran out")

    def forward(self, x):
        """x: float32 device tensor [n, 24] -> [n, 3]."""
        x = x.contiguous()
        n = x.shape[0]
        y = self.torch.empty((n, N_OUT), dtype=self.torch.float32, device=self.device)
        sc = self.scratch(n)
        check(jb_mlp_forward(self.block.data_ptr(), x.data_ptr(), n, y.data_ptr(), sc.data_ptr(), sc.numel(),
                             self.stream), "jb_mlp_forward")
        self.check_kernel()
        return y

    def grad(self, x, t):
        x, t = x.contiguous(), t.contiguous()
        n = x.shape[0]
        g = self.torch.empty(self.nparam, dtype=self.torch.float32, device=self.device)
        loss = self.torch.zeros(1, dtype=self.torch.float32, device=self.device)
        sc = self.scratch(n)
        check(jb_mlp_grad(self.block.data_ptr(), x.data_ptr(), t.data_ptr(), n, g.data_ptr(), loss.data_ptr(),
                          sc.data_ptr(), sc.numel(), self.stream), "jb_mlp_grad")
        return g, loss

    def train_step(self, x, t, lr, wd=1e-4, beta1=0.9, beta2=0.999, eps=1e-8):
        n = x.shape[0]
        self.step_count += 1
        loss = self.torch.zeros(1, dtype=self.torch.float32, device=self.device)
        sc = self.scratch(n)
        check(jb_mlp_train_step(self.block.data_ptr(), x.data_ptr(), t.data_ptr(), n, self.step_count,
                                C.c_float(lr), C.c_float(beta1), C.c_float(beta2), C.c_float(eps), C.c_float(wd),
                                loss.data_ptr(), sc.data_ptr(), sc.numel(), self.stream), "jb_mlp_train_step")
        return loss


def collect(scene, prot, params, capacity, every=1, max_steps=1 << 30, device="cuda", unmatched_only=False):
    """Runs the plain solver through the schedule with the recorder on; returns
    the recorded rows [n, 27] (device tensor): features, then the converged
    impulses in units of m_bar |g| h.  unmatched_only records only the points
    of pairs with no previous-frame impulse (the points mode 2 predicts)."""
    import torch
    prm = dict(params, warm_start=1)
    b = Batch(scene, prm, max_moves=int(prot.off[-1]), device=device)
    rows = torch.zeros((capacity, REC), dtype=torch.float32, device=b.device)
    count = torch.zeros(1, dtype=torch.int32, device=b.device)
    check(jb_set_recorder(b.h, rows.data_ptr(), capacity, count.data_ptr(), every), "jb_set_recorder")
    check(jb_set_recorder_points(b.h, 1 if unmatched_only else 0), "jb_set_recorder_points")
    b.set_protocol(prot)
    b.run_protocol(max_steps)
    b.sync()
    n = min(int(count.item()), capacity)
    rows = rows[:n]
    # the recorder's warps claim rows in whatever order they reach them: put
    # the rows in an order fixed by their contents (a projection on a fixed
    # random direction, in FP64), so that everything downstream repeats
    key = rows.double() @ torch.from_numpy(np.random.default_rng(12345).standard_normal(REC)).to(rows.device)
    return rows[torch.argsort(key, stable=True)].contiguous()


def train(rows, epochs=30, batch=8192, lr=3e-4, wd=1e-4, val_frac=0.2, seed=0, device="cuda", log=None):
    """AdamW with cosine decay to lr / 20 over `epochs` (the paper's training
    recipe, Sec. 9.6), 80/20 split of the rows at random (seeded permutation,
    so training and validation rows come from the same episodes and steps);
    minibatches are contiguous slices of the shuffled training rows from a
    per-epoch random offset.  The reported training loss is over a random
    65,536-row sample of the training rows."""
    import torch
    n = rows.shape[0]
    n_val = int(n * val_frac)
    perm = torch.from_numpy(np.random.default_rng(seed + 1).permutation(n)).to(rows.device)
    rows = rows[perm]
    tr, va = rows[: n - n_val], rows[n - n_val:]
    x_tr, t_tr = tr[:, :N_IN].contiguous(), tr[:, N_IN:].contiguous()
    x_va, t_va = va[:, :N_IN].contiguous(), va[:, N_IN:].contiguous()
    net = Network(device=device, seed=seed)
    rng = np.random.default_rng(seed)
    steps_per_epoch = max(1, (x_tr.shape[0] + batch - 1) // batch)
    total = epochs * steps_per_epoch
    hist = []
    it = 0
    for ep in range(epochs):
        off = int(rng.integers(0, batch)) if x_tr.shape[0] > batch else 0
        for s in range(steps_per_epoch):
            lo = (off + s * batch) % max(1, x_tr.shape[0] - batch + 1) if x_tr.shape[0] > batch else 0
            hi = min(x_tr.shape[0], lo + batch)
            cur = lr / 20 + 0.5 * (lr - lr / 20) * (1 + math.cos(math.pi * it / total))
            net.train_step(x_tr[lo:hi], t_tr[lo:hi], cur, wd)
            it += 1
        net.check_kernel()
        tl = float(net.grad(x_tr[: min(len(x_tr), 65536)], t_tr[: min(len(x_tr), 65536)])[1].item())
        vl = float(net.grad(x_va, t_va)[1].item()) if len(x_va) else float("nan")
        hist.append((ep, tl, vl))
        if log:
            log(f"epoch {ep} train {tl:.4g} val {vl:.4g}")
    return net, hist


def evaluate(scene, prot, params, net, mode=2, max_steps=1 << 30, device="cuda"):
    """Sweeps per solve and body-steps of the plain solver and of the learned
    warm start (mode 2: points of new pairs; 3: all points) on the same episodes,
    and whether the gate keeps the network."""
    import torch
    out = {}
    for name, ws in (("plain", 1), ("learned", mode)):
        b = Batch(scene, dict(params, warm_start=ws), max_moves=int(prot.off[-1]), device=device)
        if ws >= 2:
            check(jb_set_warmstart_mlp(b.h, net.block.data_ptr()), "jb_set_warmstart_mlp")
        b.set_protocol(prot)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.run_protocol(max_steps)
        e1.record(b.stream)
        st = b.stats()
        ms = e0.elapsed_time(e1)
        out[name] = dict(sweeps_per_solve=float(st["total_sweeps"].sum() / max(st["solves"].sum(), 1)),
                         body_steps=float(st["body_steps"].sum()), ms=ms,
                         body_steps_per_s=float(st["body_steps"].sum()) / max(ms * 1e-3, 1e-12),
                         not_converged=int(((st["status"] & 2) != 0).sum()))
    out["gain"] = out["plain"]["sweeps_per_solve"] / max(out["learned"]["sweeps_per_solve"], 1e-9)
    out["keep"] = out["gain"] > 1.0
    return out


def cold_start_gain(scene, params, net, steps=20, mode=2, device="cuda"):
    """Sweeps per solve on contacts with no previous impulse: the warm-start
    cache is cleared before every step, so every point is unmatched.  Plain
    PGS starts those points from zero impulses, the learned warm start from
    the network's prediction; both solve to the same residual.  Returns
    (plain, learned, plain / learned)."""
    out = {}
    for name, ws in (("plain", 1), ("learned", mode)):
        b = Batch(scene, dict(params, warm_start=ws), device=device)
        if ws >= 2:
            check(jb_set_warmstart_mlp(b.h, net.block.data_ptr()), "jb_set_warmstart_mlp")
        for _ in range(steps):
            b.write_state(clear_cache=True)
            b.step(1)
        st = b.stats()
        out[name] = float(st["total_sweeps"].sum() / max(st["solves"].sum(), 1))
    return out["plain"], out["learned"], out["plain"] / max(out["learned"], 1e-9)


def paired(scene, prot, params, net, steps, mode=2, device="cuda"):
    """Sweeps of both warm starts from identical states.  Along plain PGS's
    own trajectory every step is solved twice from the same snapshot (the
    bodies, the schedule position and the previous-frame impulse cache):
    once with the network's starts, once with plain PGS's zero starts at the
    points without a previous impulse; the plain solve carries the trajectory
    on.  Whole trajectories of the two arms part after the first solve (the
    impulses over a stack's redundant supports are not unique, and the
    episodes are chaotic), so comparing them measures where each trajectory
    went as much as what the network saves; this pairing measures only the
    latter.  Returns the per-step sweep sums of both arms, their totals'
    ratio (plain / learned), and the device time of each arm's step launches
    (CUDA events on the batch stream) over the same body-steps."""
    b = Batch(scene, dict(params, warm_start=1), max_moves=int(prot.off[-1]), device=device)
    check(jb_set_warmstart_mlp(b.h, net.block.data_ptr()), "jb_set_warmstart_mlp")
    b.set_protocol(prot)
    import torch
    plain, learned = [], []
    ms = {"plain": 0.0, "learned": 0.0}
    capped = 0
    total = lambda: float(b.stats()["total_sweeps"].sum())

    def timed_step(name):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.run_protocol(1)
        e1.record(b.stream)
        e1.synchronize()
        ms[name] += e0.elapsed_time(e1)

    body_steps = 0.0
    for _ in range(steps):
        snap = b.save_state()
        st0 = b.stats()
        s0, c0 = float(st0["total_sweeps"].sum()), int(st0["capped_solves"].sum())
        b0 = float(st0["body_steps"].sum())
        b.set_params(dict(params, warm_start=mode))
        timed_step("learned")
        st = b.stats()
        learned.append(float(st["total_sweeps"].sum()) - s0)
        capped += int(st["capped_solves"].sum()) - c0
        b.load_state(snap)
        s0 = total()
        b.set_params(dict(params, warm_start=1))
        timed_step("plain")
        st = b.stats()
        plain.append(float(st["total_sweeps"].sum()) - s0)
        body_steps += float(st["body_steps"].sum()) - b0
    plain, learned = np.array(plain), np.array(learned)
    return {"plain": plain, "learned": learned, "gain": float(plain.sum() / max(learned.sum(), 1.0)),
            "plain_capped": int(st["capped_solves"].sum()), "learned_capped": capped,
            # the same body-steps in both arms; device time of the step launches
            "body_steps": body_steps, "plain_ms": ms["plain"], "learned_ms": ms["learned"]}
