"""Benchmark: selected-inverse entries/s on S for the 64^3 shifted diffusion workload.

One step = the whole path on one matrix with its factors resident on the GPU:
SelInv (Takahashi recurrence on S), NInv (m-term Neumann series and the
product on S), Mix, and the rank-k correction applied on S.  ``value`` counts
the entries of S (both triangles, |S| = 2|S_lo| - n) per second of step time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--prec fp64|fp32] [--size 64]
With --gpus N > 1 under torchrun every rank runs its own replica of the
workload (the path has no cross-matrix exchange): weak scaling, no collective
on the data path.  ``--impl reference`` times the FP64 CPU oracle on the host
cores instead (the baseline arm).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--size", type=int, default=64)
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def build_workload(size):
    from workloads.configs import diff3d, plant_2x2, random_lowrank
    t0 = time.time()
    w = diff3d(size)
    f = plant_2x2(w.factors, 0.02, 2)
    V, lam = random_lowrank(f.n, w.k, seed=16)
    return w, f, V, lam, time.time() - t0


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_counts(h, f, m, k):
    """Per-step algorithmic work and bytes per phase (see the roofline notes in the design doc)."""
    st = h.stats()
    return st


def run_ours(args, rank, world):
    import torch
    from paper_2609_11363_b300 import Handle

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w, f, V, lam, t_gen = build_workload(args.size)
    m, k = w.m, w.k
    t0 = time.time()
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=dev.index)
    t_sym = time.time() - t0
    nS_lo = h.nnz_S
    nS = 2 * nS_lo - f.n
    prec = args.prec
    stream = torch.cuda.current_stream()

    Lv = torch.as_tensor(f.L_val, device=dev)
    Dv = torch.as_tensor(f.D_packed, device=dev)
    Vd = torch.as_tensor(V, device=dev)
    lamd = torch.as_tensor(lam, device=dev)
    G = torch.empty(nS_lo, dtype=torch.float64, device=dev)
    N = torch.empty_like(G)
    M = torch.empty_like(G)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    # NInv pattern for m is built on the first call (symbolic, host); eps from a first SelInv
    t0 = time.time()
    h.selinv(Lv, Dv, prec, out=G)
    h.ninv(Lv, Dv, m, prec, out=N)
    h.sync_status()
    t_sym_ninv = time.time() - t0
    diag_pos = torch.as_tensor(h.pattern_host()[0][1:] - 1, device=dev)
    eps = 1e-3 * float(G[diag_pos].abs().max())
    launches_per_step = 2 + (1 if prec == "fp32" else 0) + (3 + m) + 1 + (1 if prec == "fp64" else 3)

    phases = ["selinv", "ninv", "mix", "lowrank"]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        h.selinv(Lv, Dv, prec, out=G)
        if ev is not None:
            ev[1].record(stream)
        h.ninv(Lv, Dv, m, prec, out=N)
        if ev is not None:
            ev[2].record(stream)
        h.mix(G, N, eps, out=M)
        if ev is not None:
            ev[3].record(stream)
        h.lowrank_correct(Vd, lamd, M, prec)
        if ev is not None:
            ev[4].record(stream)

    for _ in range(args.warmup):
        step()
    h.sync_status()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(dev.index)
    clocks.start()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for s in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the events)
        step(evs[s])
    torch.cuda.synchronize()
    clk = clocks.stop()
    h.sync_status()
    per_phase = {p: [] for p in phases}
    step_ms = []
    for ev in evs:
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
        for p, x in zip(phases, t):
            per_phase[p].append(x)
        step_ms.append(ev[0].elapsed_time(ev[4]))
    total_ms = float(np.sum(step_ms))
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / args.steps
    value = world * nS * args.steps / (total_ms / 1e3)

    # end to end through the public API: pinned host inputs -> device, step, result -> host
    e2e = None
    if rank == 0:
        e2e = measure_e2e(h, f, V, lam, m, eps, prec, dev, args)

    phase_ms = {p: float(np.median(v)) for p, v in per_phase.items()}
    return dict(w=w, f=f, h=h, nS=nS, nS_lo=nS_lo, t_gen=t_gen, t_sym=t_sym, t_sym_ninv=t_sym_ninv,
                ms_per_step=ms_per_step, value=value, clocks=clk, phase_ms=phase_ms, e2e=e2e, eps=eps,
                launches=launches_per_step * args.steps, m=m, k=k)


def measure_e2e(h, f, V, lam, m, eps, prec, dev, args):
    import torch
    pin = lambda a: torch.as_tensor(a).pin_memory()  # noqa: E731
    hL, hD, hV, hl = pin(f.L_val), pin(f.D_packed), pin(V), pin(lam)
    out_host = torch.empty(h.nnz_S, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    Lv = torch.empty(hL.shape, dtype=torch.float64, device=dev)
    Dv = torch.empty(hD.shape, dtype=torch.float64, device=dev)
    Vd = torch.empty(hV.shape, dtype=torch.float64, device=dev)
    ld = torch.empty(hl.shape, dtype=torch.float64, device=dev)
    G = torch.empty(h.nnz_S, dtype=torch.float64, device=dev)
    N = torch.empty_like(G)
    M = torch.empty_like(G)

    def one():
        Lv.copy_(hL, non_blocking=True); Dv.copy_(hD, non_blocking=True)
        Vd.copy_(hV, non_blocking=True); ld.copy_(hl, non_blocking=True)
        h.selinv(Lv, Dv, prec, out=G)
        h.ninv(Lv, Dv, m, prec, out=N)
        h.mix(G, N, eps, out=M)
        h.lowrank_correct(Vd, ld, M, prec)
        out_host.copy_(M, non_blocking=True)

    one()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    h2d = (hL.numel() + hD.numel() + hV.numel() + hl.numel()) * 8
    d2h = out_host.numel() * 8
    nS = 2 * h.nnz_S - f.n
    return {"value": nS / (ms / 1e3), "unit": "entries/s", "ms_per_step": ms, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


def roofline(res, peaks):
    """Dominant kernel phase and its achieved fraction of the bound (see design notes)."""
    ph = res["phase_ms"]
    dom = max(ph, key=ph.get)
    st = res["h"].stats()
    out = {"phase_ms": ph, "dominant": dom}
    return out


def cpu_baseline(f, V, lam, m, eps, nS, budget_s=20.0):
    """The FP64 oracle as it stands, on a bounded sample of the same step."""
    import oracle
    cores = os.cpu_count()
    t0 = time.time()
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    t_sym = time.time() - t0
    t0 = time.time()
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    t_sel = time.time() - t0
    rows = np.repeat(np.arange(f.n), np.diff(S[0]))
    rng = np.random.default_rng(1)
    t0 = time.time()
    nsamp = 0
    while time.time() - t0 < max(1.0, budget_s - t_sel) and nsamp < 4096:
        idx = rng.integers(0, len(rows), 16)
        oracle.ninv_entries_sampled(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m,
                                    list(zip(rows[idx], S[1][idx])))
        nsamp += 16
    t_ninv_per = (time.time() - t0) / nsamp
    t0 = time.time()
    Mx = oracle.mix(G, G, eps)
    oracle.lowrank_correct(S[0], S[1], Mx, V, lam)
    t_rest = time.time() - t0
    t_step = t_sel + t_ninv_per * len(rows) + t_rest
    return {"value": nS / t_step, "unit": "entries/s", "cores": 1, "kind": "oracle",
            "sample": "full SelInv (%.1fs) + NInv on %d sampled S entries (%.2f ms each, scaled to all %d) "
                      "+ full Mix and low-rank; symbolic %.1fs excluded" % (t_sel, nsamp, 1e3 * t_ninv_per,
                                                                             len(rows), t_sym),
            "step_seconds_estimated": t_step}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, world)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return
    res = run_ours(args, rank, world)
    if rank == 0:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) if os.path.exists(
                os.path.join(ROOT, "MEASURED_PEAKS.json")) else open(os.devnull) as fh:
            try:
                peaks = json.load(fh)
            except ValueError:
                peaks = {}
        rf = roofline(res, peaks)
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(res["f"], *build_lowrank(res), res["m"], res["eps"], res["nS"])
        st = res["h"].stats()
        line = {
            "metric": "selected-inverse entries/s on S (SelInv+NInv+Mix+rank-k step; rel.err<=1e-10 vs FP64 oracle)",
            "value": res["value"], "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": "diff3d_%d_shifted: 3D 7-pt log-normal diffusion %d^3 (n=%d), shifted into the "
                                   "first spectral gap, ILDL tau=1e-3, 2%% planted 2x2 pivots; NInv m=%d; k=%d" % (
                                       args.size, args.size, res["f"].n, res["m"], res["k"]),
                       "n": res["f"].n, "nnz_L": st["nnz_L"], "S_entries": res["nS"], "S_lo": res["nS_lo"],
                       "n_2x2": st["n_2x2"], "supernodes": st["n_supernodes"], "levels": st["n_levels"],
                       "nnz_W": st["nnz_W"], "l2": "flushed between timed steps (512 MB write)",
                       "precision": args.prec, "symbolic_s": res["t_sym"],
                       "ninv_pattern_s": res["t_sym_ninv"], "input_gen_s": res["t_gen"],
                       "parallelism": "replicas" if world > 1 else "single"},
            "phase_ms": res["phase_ms"],
            "roofline": rf,
            "cpu_baseline": cpu,
            "e2e": res["e2e"],
            "gpu_launches": res["launches"],
            "clocks": res["clocks"],
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def build_lowrank(res):
    from workloads.configs import random_lowrank
    return random_lowrank(res["f"].n, res["k"], seed=16)


def run_reference(args, world):
    w, f, V, lam, t_gen = build_workload(args.size)
    import oracle
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    eps = 1e-3 * float(np.max(np.abs(G[S[0][1:] - 1])))
    nS = 2 * len(S[1]) - f.n
    for _ in range(args.warmup):
        pass
    vals = []
    for _ in range(args.steps):
        r = cpu_baseline(f, V, lam, w.m, eps, nS, budget_s=5.0)
        vals.append(r["step_seconds_estimated"])
    t = float(np.sum(vals))
    value = nS * args.steps / t
    line = {"impl": "reference", "metric": "selected-inverse entries/s on S (SelInv+NInv+Mix+rank-k step; "
                                           "rel.err<=1e-10 vs FP64 oracle)",
            "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "diff3d_%d_shifted (FP64 CPU oracle, single thread)" % args.size, "n": f.n},
            "cpu_baseline": {"value": value, "unit": "entries/s", "cores": 1, "kind": "oracle",
                             "sample": "per step: full SelInv + NInv on sampled entries scaled to |S_lo|"},
            "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
