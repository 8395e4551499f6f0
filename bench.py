"""Benchmark: selected-inverse entries/s on S for the 64^3 shifted diffusion workload.

One step = the whole path on one matrix whose factors are resident on the GPU:
SelInv (Takahashi recurrence on S), NInv (m-term Neumann series and the product
on S), Mix, and the rank-k correction applied on S.  ``value`` counts the
entries of S (both triangles, |S| = 2 |S_lo| - n) per second of step time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--prec fp64|fp32] [--size 64]
With --gpus N > 1 (under torchrun) every rank runs its own replica of the
workload: the path has no exchange step between matrices (weak scaling, no
collective on the data path).  ``--impl reference`` times the FP64 CPU oracle on
the host cores instead (the baseline arm: the paper ships no code).
After the FP64 timed region the same step also runs in the mixed-precision
forms (FP32X2, FP32) on the same inputs: ``forms`` holds their step times and
their error against the FP64 step's result (``--no-forms`` leaves this out).
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

METRIC = "selected-inverse entries/s on S at stated rel. error vs FP64 oracle; % roofline"
# the error each precision form is held to against the FP64 oracle (parity tests)
STATED_ERROR = {"fp64": "entrywise |x-r| <= 1e-10 (|r| + sqrt|r_ii r_jj|)",
                "fp32x2": "entrywise |x-r| <= 1e-10 (|r| + sqrt|r_ii r_jj|)",
                "fp32": "normwise ||x-r||_F <= 1e-5 ||r||_F"}
# B300: 148 SMs; FP64 2 FMA/clk/SM (4 flop), FP32 128 FMA/clk/SM (256 flop)
N_SMS = 148
FP64_FLOP_PER_CLK_SM = 4
FP32_FLOP_PER_CLK_SM = 256


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "fp32x2"],
                   help="fp32x2: FP64 with the NInv product on S in pairs of floats (FP64-class)")
    p.add_argument("--size", type=int, default=64)
    p.add_argument("--ninv-delta", type=float, default=0.0,
                   help="inverse tolerance of NInv: off-diagonal |w| < delta dropped after each Horner step")
    p.add_argument("--workload", default="diff3d",
                   choices=["diff3d", "batch9pt", "learned", "elastic", "covariance", "band", "ninv_own"],
                   help="diff3d: the 64^3 step (default); batch9pt: 256 matrices in one graph-captured launch; "
                        "learned: the trained NInv->SelInv correction on 128^3; elastic: the 27-point 3-dof "
                        "operator (N^3 nodes, --elastic-size N); covariance: the (1-d/3)^4 covariance-type "
                        "matrix on an N x N grid (--cov-size N); band: the dense-row microbenchmark shape "
                        "(--band-n, --band-b, --band-tau), SelInv FP64 vs the tensor-core forms; ninv_own: NInv "
                        "on its own delta-sparsified pattern on the 64^3 factors (--own-deltas)")
    p.add_argument("--own-deltas", default="1e-1,1e-2", help="ninv_own: inverse tolerances to time")
    p.add_argument("--band-n", type=int, default=12288)
    p.add_argument("--band-b", type=int, default=1024)
    p.add_argument("--band-tau", type=float, default=1e-6)
    p.add_argument("--elastic-size", type=int, default=24)
    p.add_argument("--factor-cache", default=None,
                   help="elastic: directory of the on-disk factor cache (the ILDL at 80^3 nodes takes minutes)")
    p.add_argument("--cov-size", type=int, default=200)
    p.add_argument("--spai-iters", type=int, default=20,
                   help="covariance: PCG steps of the SPAI refinement of Mix (Mix-SPAI); 0 = leave it out")
    p.add_argument("--einv-k", type=int, default=3,
                   help="covariance: eigenpairs of the spectral check (Lanczos on A^{-1} - Mix); 0 = skip it")
    p.add_argument("--einv-steps", type=int, default=30, help="covariance: Lanczos steps of the spectral check")
    p.add_argument("--spai-power", type=int, default=2,
                   help="covariance: SPAI pattern P = S + pairs within this graph distance in A")
    p.add_argument("--exact-diag-max-n", type=int, default=10000,
                   help="covariance: also report err_1 of the diagonals against a dense inverse up to this n")
    p.add_argument("--batch", type=int, default=256, help="matrices of the batch9pt workload")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true",
                   help="leave out the FP32X2 and FP32 steps timed after the FP64 line's timed region")
    return p.parse_args()


def build_workload(size):
    from workloads.configs import diff3d, plant_2x2, random_lowrank
    t0 = time.time()
    w = diff3d(size)
    f = plant_2x2(w.factors, 0.02, 2)
    V, lam = random_lowrank(f.n, w.k, seed=16)
    return w, f, V, lam, time.time() - t0


def workload_name(size, f, m, k):
    return ("diff3d_%d_shifted: 3D 7-point log-normal diffusion %d^3 (n=%d), shifted into the first spectral gap, "
            "ILDL tau=1e-3, 2%% planted 2x2 pivots; SelInv + NInv m=%d + Mix + rank-%d correction" % (
                size, size, f.n, m, k))


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


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            try:
                return json.load(fh), "measured"
            except ValueError:
                pass
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def kernel_rooflines(trace, st, m, k, nS_lo, prec, peaks, steps):
    """Per kernel: launches per step, mean launch time, algorithmic work per launch and
    the achieved fraction of its bound (see the design notes for the unit counts)."""
    mhz = float(peaks.get("sm_max_mhz", 2032.0))
    fp64_alu = prec != "fp32"  # fp32x2 keeps SelInv, the Horner steps and the low-rank correction in FP64
    alu_peak = N_SMS * (FP64_FLOP_PER_CLK_SM if fp64_alu else FP32_FLOP_PER_CLK_SM) * mhz * 1e6 / 1e12
    alu_src = "derived: %d SMs x %d %s flop/clk x %.0f MHz" % (
        N_SMS, FP64_FLOP_PER_CLK_SM if fp64_alu else FP32_FLOP_PER_CLK_SM, "FP64" if fp64_alu else "FP32", mhz)
    hbm = float(peaks["hbm_gbs"])
    horner = st["horner_products"] / max(m, 1)  # mean products of one Horner step
    work = {
        "selinv_persistent": ("alu", st["selinv_flops"], "flop"),
        "ninv_horner": ("alu", 2.0 * horner, "flop"),
        "ninv_product": ("alu", 2.0 * st["product_stream"], "flop"),
        "lowrank": ("alu", 2.0 * k * nS_lo, "flop"),
        "mix": ("hbm", 24.0 * nS_lo, "byte"),  # reads G and N, writes M: 3 x 8 B per entry
    }
    if fp64_alu:
        work["ninv_map_horner"] = ("alu", 2.0 * horner, "flop")
        work["ninv_map_product"] = ("alu", 2.0 * st["product_hits"], "flop")
        # pairs of floats: a 2-byte map entry and an 8-byte pair per streamed row, N written
        work["ninv_pair_product"] = ("hbm", 10.0 * st["product_stream"] + 8.0 * nS_lo, "byte")
    else:
        # FP32 map form streams a 2-byte map entry and a 4-byte value per product and
        # writes its targets (Horner); per product-map entry the same, plus N (8 B)
        work["ninv_map_horner"] = ("hbm", 6.0 * horner + 4.0 * st["nnz_W"], "byte")
        work["ninv_map_product"] = ("hbm", 6.0 * st["product_stream"] + 8.0 * nS_lo, "byte")
    out = {}
    for name, (launches, total_ms) in trace.items():
        per_launch_ms = total_ms / launches
        row = {"launches_per_step": launches / steps, "ms_per_launch": per_launch_ms,
               "ms_per_step": total_ms / steps}
        if name in work:
            bound, units, kind = work[name]
            if bound == "alu":
                ach = units / (per_launch_ms * 1e-3) / 1e12
                row.update(bound="alu", achieved=ach, peak=alu_peak, unit="TFLOP/s", frac=ach / alu_peak,
                           peak_source=alu_src, work_per_launch=units)
            else:
                ach = units / (per_launch_ms * 1e-3) / 1e9
                row.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                           peak_source="MEASURED_PEAKS.json hbm_gbs", work_per_launch=units)
        out[name] = row
    return out


# DRAM bytes (read + write) per unit of work from one ncu capture of the same kernel
# build on the 32^3 case of this workload (profiles/ninv_map_kernels_diff3d_32_fp64.md):
# FP64 Horner (hm_step_fx): 2.600 GB over the 757.9 M products of its 4 steps; FP64
# product: 1.996 GB over 811.8 M streamed map entries.  Scaled to a launch here by
# the units it processes.
DRAM_PER_UNIT = {"ninv_map_horner": 2.59975e9 / 757.933257e6, "ninv_map_product": 1.99553e9 / 811.837539e6}


def dram_traffic(kernel, prec, st, m):
    if prec != "fp64" or kernel not in DRAM_PER_UNIT:
        return None, None
    units = st["horner_products"] / max(m, 1) if kernel == "ninv_map_horner" else st["product_stream"]
    return DRAM_PER_UNIT[kernel] * units, ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the FP64 kernel on "
                                           "the 32^3 case, scaled by the units per launch (estimate)")


def aggregate_ranks(total_ms, units_per_step, steps, world, device):
    """Whole-job throughput of `world` replicas: the slowest rank's time (max over ranks)
    and the units every rank processed.  Returns (ms per step, units per second)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    return total_ms / steps, world * units_per_step * steps / (total_ms / 1e3)


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

    # the NInv pattern for m is built by the first call (host, symbolic); eps from a first SelInv
    t0 = time.time()
    h.selinv(Lv, Dv, prec, out=G)
    h.ninv(Lv, Dv, m, prec, out=N, delta=args.ninv_delta)
    h.sync_status()
    t_sym_ninv = time.time() - t0
    diag_pos = torch.as_tensor(h.pattern_host()[0][1:] - 1, device=dev)
    eps = 1e-3 * float(G[diag_pos].abs().max())

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        h.selinv(Lv, Dv, prec, out=G)
        if ev is not None:
            ev[1].record(stream)
        h.ninv(Lv, Dv, m, prec, out=N, delta=args.ninv_delta)
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
    h.trace(True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for s in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the events)
        step(evs[s])
    torch.cuda.synchronize()
    clk = clocks.stop()
    trace = h.trace_read()
    h.trace(False)
    h.sync_status()
    phases = ["selinv", "ninv", "mix", "lowrank"]
    per_phase = {p: [] for p in phases}
    step_ms = []
    for ev in evs:
        for i, p in enumerate(phases):
            per_phase[p].append(ev[i].elapsed_time(ev[i + 1]))
        step_ms.append(ev[0].elapsed_time(ev[4]))
    ms_per_step, value = aggregate_ranks(float(np.sum(step_ms)), nS, args.steps, world, dev)

    e2e = forms = None
    if rank == 0:
        M64 = M.clone()  # the last timed FP64 step's corrected result
        e2e = measure_e2e(h, f, V, lam, m, eps, prec, dev, args)
        if prec == "fp64" and not args.no_forms:
            forms = measure_forms(h, Lv, Dv, Vd, lamd, m, eps, M64, nS, flush, stream, dev, args,
                                  float(np.sum(step_ms)) / args.steps)
    launches = int(sum(c for c, _ in trace.values()))
    return dict(w=w, f=f, h=h, nS=nS, nS_lo=nS_lo, t_gen=t_gen, t_sym=t_sym, t_sym_ninv=t_sym_ninv,
                ms_per_step=ms_per_step, value=value, clocks=clk, eps=eps, e2e=e2e, m=m, k=k, V=V, lam=lam,
                phase_ms={p: float(np.median(v)) for p, v in per_phase.items()}, trace=trace, launches=launches,
                forms=forms)


def measure_forms(h, Lv, Dv, Vd, lamd, m, eps, M64, nS, flush, stream, dev, args, fp64_ms):
    """The same step in the mixed-precision forms, after the FP64 timed region and on
    the same inputs: event-timed steps with L2 flushed between them, and the error
    of each form's corrected result against the FP64 step's, in the measure of the
    form's stated error (entrywise scaled for the pair form, normwise for FP32)."""
    import torch
    rp, col = h.pattern_host()
    rows = torch.as_tensor(np.repeat(np.arange(h.n, dtype=np.int64), np.diff(rp)), device=dev)
    cols = torch.as_tensor(np.asarray(col, dtype=np.int64), device=dev)
    dia = M64[torch.as_tensor(rp[1:] - 1, device=dev)].abs()
    G, N, M = torch.empty_like(M64), torch.empty_like(M64), torch.empty_like(M64)
    out = {}
    for form in ("fp32x2", "fp32"):
        try:
            def step():
                h.selinv(Lv, Dv, form, out=G)
                h.ninv(Lv, Dv, m, form, out=N, delta=args.ninv_delta)
                h.mix(G, N, eps, out=M)
                h.lowrank_correct(Vd, lamd, M, form)

            for _ in range(max(args.warmup, 1)):
                step()
            h.sync_status()
            K = max(1, min(args.steps, 5))
            evs = []
            for _ in range(K):
                flush.zero_()
                e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                e[0].record(stream)
                step()
                e[1].record(stream)
                evs.append(e)
            torch.cuda.synchronize()
            h.sync_status()
            ms = [a.elapsed_time(b) for a, b in evs]
            if form == "fp32x2":
                err = float(((M - M64).abs() / (M64.abs() + torch.sqrt(dia[rows] * dia[cols]))).max())
                measure = "entrywise max |x-r| / (|r| + sqrt|r_ii r_jj|), r = the FP64 step's result"
            else:
                err = float(torch.linalg.norm(M - M64) / torch.linalg.norm(M64))
                measure = "normwise ||x-r||_F / ||r||_F, r = the FP64 step's result"
            out[form] = {"ms_per_step": float(np.mean(ms)), "value": nS * K / (float(np.sum(ms)) / 1e3),
                         "unit": "entries/s", "speedup_vs_fp64": fp64_ms / float(np.mean(ms)), "steps": K,
                         "stated_rel_error": STATED_ERROR[form], "error_vs_fp64": err, "error_measure": measure}
        except Exception as exc:  # the FP64 line stands whatever happens here
            out[form] = {"failed": repr(exc)}
    return out


def measure_e2e(h, f, V, lam, m, eps, prec, dev, args):
    """The same step through the public API with host buffers: pinned host -> device copies
    of L, D, V, lambda and the device -> host copy of the corrected result, all timed."""
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
        h.ninv(Lv, Dv, m, prec, out=N, delta=args.ninv_delta)
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
    nS = 2 * h.nnz_S - f.n
    return {"value": nS / (ms / 1e3), "unit": "entries/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int((hL.numel() + hD.numel() + hV.numel() + hl.numel()) * 8),
            "d2h_bytes_per_step": int(out_host.numel() * 8)}


def trailing_block(f, V, nt):
    """The trailing principal block [c0, n) of the factors (c0 = n - nt, moved down
    so that no 2x2 pivot is cut): the top of the elimination tree.  SelInv, the
    Neumann series and the product on S restricted to this block depend on no
    entry outside it (every column's rows lie below it), so the oracle's full
    step on the block computes exactly the workload's own values there."""
    import scipy.sparse as sp
    n = f.n
    c0 = max(0, n - int(nt))
    while c0 > 0 and not f.pivot_start[c0]:
        c0 -= 1
    L = sp.csr_matrix((f.L_val, f.L_col, f.L_rowptr), shape=(n, n))[c0:, c0:].tocsr()
    L.sort_indices()
    return dict(n=n - c0, c0=c0, rp=L.indptr.astype(np.int64), col=L.indices.astype(np.int32), val=L.data,
                ps=np.ascontiguousarray(f.pivot_start[c0:]), dd=np.ascontiguousarray(f.d_diag[c0:]),
                do=np.ascontiguousarray(f.d_off[c0:]), V=np.ascontiguousarray(V[c0:]))


def oracle_step(b, lam, m, all_threads=False):
    """One whole oracle step on a block: SelInv, NInv (m), Mix with
    eps = 1e-3 max|G_ii| (as the GPU arm), rank-k correction; every phase runs
    in full.  all_threads: SelInv by level sets and NInv in C on every host
    thread (variant (ii)), else the plain oracle as it stands, one thread."""
    import oracle
    n = b["n"]
    t0 = time.perf_counter()
    S = oracle.symbolic_S(n, b["rp"], b["col"], b["ps"])
    t_sym = time.perf_counter() - t0
    t0 = time.perf_counter()
    if all_threads:
        G, _ = oracle.selinv_levels(n, b["rp"], b["col"], b["val"], b["ps"], b["dd"], b["do"], S)
    else:
        G = oracle.selinv(n, b["rp"], b["col"], b["val"], b["ps"], b["dd"], b["do"], S)
    t1 = time.perf_counter()
    if all_threads:
        N = oracle.ninv_threads(n, b["rp"], b["col"], b["val"], b["ps"], b["dd"], b["do"], m, S)
    else:
        N = oracle.ninv(n, b["rp"], b["col"], b["val"], b["ps"], b["dd"], b["do"], m, S)
    t2 = time.perf_counter()
    eps = 1e-3 * float(np.max(np.abs(G[S[0][1:] - 1])))
    M = oracle.lowrank_correct(S[0], S[1], oracle.mix(G, N, eps), b["V"], lam)
    t3 = time.perf_counter()
    nS = 2 * len(S[1]) - n
    return t3 - t0, nS, {"selinv_s": t1 - t0, "ninv_s": t2 - t1, "mix_lowrank_s": t3 - t2, "pattern_s": t_sym,
                         "checksum": float(np.sum(M))}


LADDER = (2048, 4096, 8192, 12288, 16384, 24576, 32768, 49152, 65536, 98304, 131072)


def calibrated_block(f, V, lam, m, target_s):
    """The largest trailing block of the ladder whose plain-oracle step is
    expected within target_s: blocks are timed upward (each timing is a real
    step, the smaller ones serve as warm-up) until one takes more than a third
    of the target (the next would not fit: the step grows 3-5x per doubling)."""
    best = None
    for nt in LADDER + (f.n,):
        nt = min(nt, f.n)
        b = trailing_block(f, V, nt)
        t, nS, parts = oracle_step(b, lam, m)
        if best is None or t <= target_s:
            best = (b, t, nS, parts)
        if t > target_s / 3 or nt >= f.n:
            break
    return best


def cpu_baseline(f, V, lam, m, nS_full):
    """Both CPU baselines, measured (nothing extrapolated): the plain oracle on one
    thread over a trailing block of the workload, and the all-threads variant
    over the whole workload."""
    import oracle
    b, t, nS, parts = calibrated_block(f, V, lam, m, target_s=15.0)
    full = trailing_block(f, V, f.n)
    t_all, nS_all, parts_all = oracle_step(full, lam, m, all_threads=True)
    return {"value": nS / t, "unit": "entries/s", "cores": 1, "kind": "oracle",
            "sample": "plain FP64 oracle (C SelInv, scipy NInv, numpy Mix + rank-k), one host thread, one "
                      "whole step timed on the trailing principal block of the same factors (rows/cols %d..%d, "
                      "n' = %d, |S'| = %d of |S| = %d): the top of the elimination tree, whose values depend on "
                      "nothing outside it; SelInv %.2f s, NInv %.2f s, Mix + rank-k %.2f s" % (
                          b["c0"], f.n - 1, b["n"], nS, nS_full, parts["selinv_s"], parts["ninv_s"],
                          parts["mix_lowrank_s"]),
            "step_seconds": t,
            "all_cores": {"value": nS_all / t_all, "unit": "entries/s", "cores": oracle.host_threads(),
                          "kind": "oracle, variant (ii): SelInv by level sets and NInv in C, OpenMP over all "
                                  "host threads",
                          "sample": "the whole workload (n = %d, |S| = %d), one full step timed" % (f.n, nS_all),
                          "step_seconds": t_all, "selinv_s": parts_all["selinv_s"], "ninv_s": parts_all["ninv_s"],
                          "mix_lowrank_s": parts_all["mix_lowrank_s"]}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if args.impl == "ours" else "gloo")
    if args.workload != "diff3d" and args.impl == "ours":
        run_extra(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return
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
        peaks, peak_kind = load_peaks()
        st = res["h"].stats()
        kr = kernel_rooflines(res["trace"], st, res["m"], res["k"], res["nS_lo"], args.prec, peaks, args.steps)
        dom = max(kr, key=lambda x: kr[x]["ms_per_step"])
        d = kr[dom]
        traffic, traffic_src = dram_traffic(dom, args.prec, st, res["m"])
        roofline = {"kernel": dom, "bound": d.get("bound"), "achieved": d.get("achieved"), "peak": d.get("peak"),
                    "unit": d.get("unit"), "frac": d.get("frac"), "traffic": traffic, "traffic_source": traffic_src,
                    "peak_source": d.get("peak_source"), "ms_per_launch": d["ms_per_launch"],
                    "work_per_launch": d.get("work_per_launch"), "kernels": kr}
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(res["f"], res["V"], res["lam"], res["m"], res["nS"])
        line = {
            "metric": METRIC, "value": res["value"], "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp32x2": "f64+f32x2"}[args.prec],
            "data": "synthetic",
            "config": {"workload": workload_name(args.size, res["f"], res["m"], res["k"]), "n": res["f"].n,
                       "nnz_L": st["nnz_L"], "S_entries": res["nS"], "S_lo": res["nS_lo"], "n_2x2": st["n_2x2"],
                       "supernodes": st["n_supernodes"], "levels": st["n_levels"], "nnz_W": st["nnz_W"],
                       "l2": "flushed between timed steps (512 MB write)", "precision": args.prec,
                       "stated_rel_error": STATED_ERROR[args.prec], "ninv_delta": args.ninv_delta,
                       "symbolic_s": res["t_sym"], "ninv_pattern_s": res["t_sym_ninv"],
                       "input_gen_s": res["t_gen"], "peaks": peak_kind,
                       "parallelism": "replicas" if world > 1 else "single"},
            "phase_ms": res["phase_ms"],
            "forms": res["forms"],
            "roofline": roofline,
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


def _gen_batch_member(seed):
    from workloads.configs import batch9pt_member
    return batch9pt_member(seed).factors


def run_extra(args, rank, world):
    """The other hot-path rows, one JSON line each (not the default benchmark line).

    batch9pt: 256 random-weight 9-point matrices (n uniform in [2048, 65536], seeds
    3000+) in one batched handle; the autotuner picks the SelInv schedule; one step
    = SelInv + NInv (m = 3) in FP32 for all matrices, replayed from a CUDA graph.
    learned: the NInv -> SelInv correction network trained on 3D diffusion 48^3
    (seeds 4000+) and applied to 128^3 (seed 4999); one step = NInv stack (m = 3)
    + features + network, compared with SelInv FP64 on the same matrix.
    """
    import multiprocessing as mp

    import torch
    from paper_2609_11363_b300 import Handle
    from workloads.configs import diff3d

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    peaks, peak_kind = load_peaks()
    if args.workload == "batch9pt":
        from paper_2609_11363_b300.autotune import tune_selinv
        t0 = time.time()
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            fs = pool.map(_gen_batch_member, [3000 + i for i in range(args.batch)])
        t_gen = time.time() - t0
        torch.cuda.set_device(dev)
        Lv = torch.as_tensor(np.concatenate([f.L_val for f in fs]), device=dev)
        Dv = torch.as_tensor(np.concatenate([f.D_packed for f in fs]), device=dev)
        t0 = time.time()
        h, best, table = tune_selinv(fs, Lv, Dv, prec="fp32", caps=(1, 4), bigs=(512, 2048), device=dev.index)
        t_tune = time.time() - t0
        G = torch.empty(h.nnz_S, dtype=torch.float64, device=dev)
        N = torch.empty_like(G)

        def step():
            h.selinv(Lv, Dv, "fp32", out=G)
            h.ninv(Lv, Dv, 3, "fp32", out=N)

        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            step()
            step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        clocks = ClockSampler(dev.index)
        clocks.start()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            graph.replay()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        clk = clocks.stop()
        h.sync_status()
        nS = 2 * h.nnz_S - h.n
        total = float(np.sum(ms))
        st = h.stats()
        # the same work without batching: one handle per matrix, launched one after another
        singles = []
        for b, f in enumerate(fs):
            lay = h.layout()
            hb = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=dev.index, **best)
            Lb = Lv[lay["L"][b]:lay["L"][b + 1]]
            Db = Dv[lay["D"][b]:lay["D"][b + 1]]
            Gb = torch.empty(hb.nnz_S, dtype=torch.float64, device=dev)
            singles.append((hb, Lb, Db, Gb, torch.empty_like(Gb)))

        def loop_step():
            for hb, Lb, Db, Gb, Nb in singles:
                hb.selinv(Lb, Db, "fp32", out=Gb)
                hb.ninv(Lb, Db, 3, "fp32", out=Nb)

        loop_step()
        torch.cuda.synchronize()
        ms_loop = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            loop_step()
            e1.record()
            torch.cuda.synchronize()
            ms_loop.append(e0.elapsed_time(e1))
        for hb, *_ in singles:
            hb.sync_status()
            hb.close()
        del singles
        line = {"metric": METRIC,
                "value": world * nS * args.steps / (total / 1e3), "unit": "entries/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "batch9pt: %d 2D 9-point random-weight Laplacians, n ~ U[2048, 65536], "
                                       "ILDL tau=1e-2, SelInv + NInv m=3 in FP32, one CUDA graph per step" % args.batch,
                           "stated_rel_error": STATED_ERROR["fp32"],
                           "matrices": len(fs), "n_total": h.n, "S_entries": nS, "levels": st["n_levels"],
                           "autotuned": best, "autotune_table_ms": [list(r[:3]) for r in table],
                           "one_handle_per_matrix_ms_per_step": float(np.median(ms_loop)),
                           "autotune_s": t_tune, "input_gen_s": t_gen, "l2": "flushed between timed steps"},
                "clocks": clk, "gpu_launches": None}
        if rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "elastic":
        run_elastic(args, rank, world, dev, peaks)
        return
    if args.workload == "band":
        torch.cuda.set_device(dev)
        run_band(args, rank, world, dev, peaks)
        return
    if args.workload == "covariance":
        run_covariance(args, rank, world, dev)
        return
    if args.workload == "ninv_own":
        torch.cuda.set_device(dev)
        run_ninv_own(args, rank, world, dev)
        return
    # learned correction
    from paper_2609_11363_b300.learned import LearnedCorrection
    torch.cuda.set_device(dev)
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        train_f = pool.map(_gen_diff_spd48, [4000 + i for i in range(64)])
    test_w = diff3d(args.size if args.size != 64 else 128, shifted=False, m=3, seed=4999)
    t_gen = time.time() - t0
    lc = LearnedCorrection(m=3, seed=1, batch=16384, device=dev.index)
    sets = []
    for f in train_f:
        h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=dev.index)
        d = lc.prepare(h, torch.as_tensor(f.L_val, device=dev), torch.as_tensor(f.D_packed, device=dev))
        sets.append({"X": d["X"], "y": d["y"]})  # keep only what training needs
        del d
        h.close()
    fit = lc.fit(sets, epochs=2, lr=2e-3)
    del sets
    torch.cuda.empty_cache()  # the inference matrix's NInv maps take half of the free memory
    f = test_w.factors
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=dev.index)
    Lv = torch.as_tensor(f.L_val, device=dev)
    Dv = torch.as_tensor(f.D_packed, device=dev)
    d = lc.prepare(h, Lv, Dv)
    ev = lc.evaluate(d)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            flush.zero_()  # inputs are smaller than L2: flush it between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))

    def learned_step():
        Nst = h.ninv_stack(Lv, Dv, 3, "fp64")
        X, sc = h.mlp_features(Nst, 3, Lv, Dv)
        lc.mlp.predict(X, sc, Nst[3].contiguous())

    ms_learned = timed(learned_step, args.steps)
    ms_stack = timed(lambda: h.ninv_stack(Lv, Dv, 3, "fp64"), args.steps)
    ms_selinv = timed(lambda: h.selinv(Lv, Dv, "fp64"), args.steps)
    h.sync_status()
    nS = 2 * h.nnz_S - h.n
    line = {"metric": METRIC,
            "value": nS / (ms_learned / 1e3), "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_learned, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+f64", "data": "synthetic",
            "config": {"workload": "learned: 3-layer width-64 BF16 MLP trained on 64 seeds of 3D 7-point "
                                   "log-normal diffusion 48^3, applied to %d^3 (n=%d), tau=1e-3, m=3" % (
                                       round(f.n ** (1 / 3)), f.n),
                       "stated_rel_error": "relative Frobenius error on S against SelInv FP64: reported, not bounded",
                       "train_entries": fit["entries"], "train_steps": fit["steps"], "train_s": fit["seconds"],
                       "ninv_form": "map" if h.stats()["ninv_index_bytes"] > 0 else "hash",
                       "err_vs_selinv_ninv": ev["err_ninv"], "err_vs_selinv_learned": ev["err_learned"],
                       "keep_correction": LearnedCorrection.choose([ev]), "selinv_fp64_ms": ms_selinv,
                       "ninv_stack_ms": ms_stack,
                       "input_gen_s": t_gen},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line))


def run_band(args, rank, world, dev, peaks):
    """The dense-row microbenchmark shape of the paper (n = 12,288, half-bandwidth
    1024, DoDD 1.8, tau = 1e-6 by default): SelInv in FP64 and in the tensor-core
    forms (TF32 / BF16 split operands), entries of S per second, the normwise
    difference from the FP64 result (itself parity-tested against the oracle) and
    the critical-path split of the tensor-core call."""
    import torch
    from paper_2609_11363_b300 import Handle
    from paper_2609_11363_b300.timeline import critical_path, dependencies
    from workloads.configs import band
    t0 = time.time()
    f = band(args.band_n, args.band_b, tau=args.band_tau).factors
    t_gen = time.time() - t0
    t0 = time.time()
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=dev.index, supernode_cap=16)
    t_sym = time.time() - t0
    st = h.stats()
    Lv = torch.as_tensor(f.L_val, device=dev)
    Dv = torch.as_tensor(f.D_packed, device=dev)
    nS = 2 * h.nnz_S - f.n
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res, outs = {}, {}
    clocks = ClockSampler(dev.index)
    clocks.start()
    for prec in ("fp64", "tf32", "bf16"):
        G = torch.empty(h.nnz_S, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            h.selinv(Lv, Dv, prec, out=G)
        h.sync_status()
        h.trace(True)
        ms = []
        steps = args.steps if prec != "fp64" else max(1, min(args.steps, 3))
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            h.selinv(Lv, Dv, prec, out=G)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        tr = h.trace_read()
        h.trace(False)
        h.sync_status()
        outs[prec] = G.cpu().numpy()
        res[prec] = {"ms": float(np.median(ms)), "entries_per_s": nS / (float(np.median(ms)) / 1e3),
                     "kernels": {k: {"launches_per_step": c / steps, "ms_per_step": t / steps} for k, (c, t) in tr.items()}}
    clk = clocks.stop()
    ref = outs["fp64"]
    for prec in ("tf32", "bf16"):
        res[prec]["normwise_vs_fp64"] = float(np.linalg.norm(outs[prec] - ref) / np.linalg.norm(ref))
        res[prec]["speedup_vs_fp64"] = res["fp64"]["ms"] / res[prec]["ms"]
    # critical path of the TF32 call (a separate, recorded call)
    h.timeline(True)
    G = torch.empty(h.nnz_S, dtype=torch.float64, device=dev)
    h.selinv(Lv, Dv, "tf32", out=G)
    h.sync_status()
    stamps = h.timeline_read()
    h.timeline(False)
    sn_start, sn_level = h.supernodes()
    cp = critical_path(stamps, dependencies(f.n, f.L_rowptr, f.L_col, sn_start), sn_level)
    # work of the contraction: per supernode 3 split products of 2 |R|^2 w flops
    tc_flops = 3 * 2.0 * st["tc_pairs"] * 16
    tc_ms = res["tf32"]["kernels"].get("selinv_tc_tf32", {}).get("ms_per_step", res["tf32"]["ms"])
    line = {"metric": METRIC, "workload": "band", "value": res["tf32"]["entries_per_s"], "unit": "entries/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["tf32"]["ms"],
            "higher_is_better": True, "dtype": "tf32 split operands, f32 accumulators, f64 pivots and G_JJ",
            "data": "synthetic",
            "config": {"workload": "band_%d_b%d_tau%g: dense band, half-bandwidth %d, DoDD 1.8, seed 6, natural "
                                   "order; SelInv" % (f.n, args.band_b, args.band_tau, args.band_b),
                       "n": f.n, "nnz_L": st["nnz_L"], "S_entries": nS, "supernodes": st["n_supernodes"],
                       "levels": st["n_levels"], "tc_levels": st["tc_levels"], "tc_pairs": st["tc_pairs"],
                       "tc_mirror_bytes": st["tc_mirror_bytes"], "input_gen_s": t_gen, "symbolic_s": t_sym,
                       "l2": "flushed between timed calls (512 MB write)",
                       "stated_rel_error": {"tf32": "normwise 1e-6", "bf16": "normwise 1e-5"}},
            "forms": res, "critical_path_tf32": cp,
            "tensor_roofline": {"bound": "latency of the level chain", "flops_per_call": tc_flops,
                                "achieved_tflops": tc_flops / (tc_ms * 1e-3) / 1e12,
                                "peak_tflops_tf32": 0.5 * float(peaks.get("bf16_tflops", 1800.0)),
                                "peak_source": "MEASURED_PEAKS.json bf16 x 1/2 (nominal TF32:BF16 ratio)"},
            "clocks": clk}
    line["tensor_roofline"]["frac"] = line["tensor_roofline"]["achieved_tflops"] / line["tensor_roofline"]["peak_tflops_tf32"]
    print(json.dumps(line))


def run_ninv_own(args, rank, world, dev):
    """NInv on its own pattern (Section 2.2): delta sparsifies the series W and the
    product W^T D^{-1} W, so fill and time fall as delta grows.  The 64^3 benchmark
    factors, m = 4; per delta: the call's wall time (it sizes its outputs on the host
    between steps, so it synchronises), the kernel times, the fill of W and of the
    product, against NInv on S."""
    import torch
    from paper_2609_11363_b300 import Handle
    w, f, _, _, t_gen = build_workload(args.size)
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=dev.index)
    Lv = torch.as_tensor(f.L_val, device=dev)
    Dv = torch.as_tensor(f.D_packed, device=dev)
    N = torch.empty(h.nnz_S, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            out.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(out))

    rows = []
    for delta in [float(x) for x in args.own_deltas.split(",")]:
        ms = timed(lambda: h.ninv_own(Lv, Dv, w.m, delta), args.steps)
        h.trace(True)
        cp, r, v, steps = h.ninv_own(Lv, Dv, w.m, delta)
        torch.cuda.synchronize()
        kern = h.trace_read()
        h.trace(False)
        h.sync_status()
        rows.append({"delta": delta, "ms": ms, "nnz_W_by_step": [int(x) for x in steps],
                     "nnz_N_lo": int(r.numel()), "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kern.items()}})
    del cp, r, v
    ms_on_S = timed(lambda: h.ninv(Lv, Dv, w.m, "fp64", out=N), args.steps)  # after: its maps take HBM
    line = {"metric": METRIC, "value": None, "unit": "entries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ninv_own: " + workload_name(args.size, f, w.m, w.k).split(";")[0]
                                   + "; NInv m=%d on its own delta-sparsified pattern" % w.m,
                       "S_lo": int(h.nnz_S), "ninv_on_S_ms": ms_on_S, "by_delta": rows,
                       "timing": "host wall time per call after a device synchronisation, L2 flushed before each",
                       "input_gen_s": t_gen},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line))


def run_elastic(args, rank, world, dev, peaks):
    """27-point 3-dof elastic-like operator on N^3 nodes (n = 3 N^3; the configuration
    is 80^3 nodes, n = 1,536,000), ILDL tau = 1e-4.  One step, inputs resident:
    SelInv in the BF16 tensor-core form (the leading levels on tcgen05 with split
    operands, the rest FP64; pivots and G_JJ FP64) + NInv on its own pattern (m = 2,
    delta = 1e-1, the paper's loose tolerance for Mix) + Mix on that pattern + the
    rank-64 correction on the Mix pattern.  FP64 and FP32 SelInv are timed beside it,
    with the BF16 form's normwise difference from FP64.  At this size the SelInv
    plan is the scan form (no pair lists)."""
    import torch
    from paper_2609_11363_b300 import Handle
    from workloads.configs import elastic3d, random_lowrank
    torch.cuda.set_device(dev)
    t0 = time.time()
    w = elastic3d(args.elastic_size, cache_dir=args.factor_cache)
    f = w.factors
    V, lam = random_lowrank(f.n, w.k, seed=5)
    t_gen = time.time() - t0
    t0 = time.time()
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=dev.index)
    t_sym = time.time() - t0
    Lv = torch.as_tensor(f.L_val, device=dev)
    Dv = torch.as_tensor(f.D_packed, device=dev)
    Vd = torch.as_tensor(V, device=dev)
    ld = torch.as_tensor(lam, device=dev)
    G = torch.empty(h.nnz_S, dtype=torch.float64, device=dev)
    G64 = torch.empty_like(G)
    h.selinv(Lv, Dv, "fp64", out=G64)
    h.sync_status()
    eps = 1e-3 * float(G64.abs().max())  # the diagonal dominates |G| on this SPD operator
    delta, prec = 0.1, "bf16"

    def step():
        h.selinv(Lv, Dv, prec, out=G)
        h.ninv_own(Lv, Dv, w.m, delta, copy=False)
        h.mix_own(G, eps, copy=False)
        h.lowrank_correct_mix_own(Vd, ld, "fp64")

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            flush.zero_()  # L2 flushed between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))

    for _ in range(args.warmup):
        step()
    clk = ClockSampler(dev.index)
    clk.start()
    ms = timed(step, args.steps)
    clocks = clk.stop()
    phases = {"selinv_" + p: timed(lambda p=p: h.selinv(Lv, Dv, p, out=G), args.steps)
              for p in ("fp64", "fp32", "bf16", "tf32")}
    h.selinv(Lv, Dv, prec, out=G)
    diff_bf16 = float(torch.linalg.norm(G - G64) / torch.linalg.norm(G64))
    phases["ninv_own"] = timed(lambda: h.ninv_own(Lv, Dv, w.m, delta, copy=False), args.steps)
    _, _, _, wsteps = h.ninv_own(Lv, Dv, w.m, delta, copy=False)
    phases["mix_own"] = timed(lambda: h.mix_own(G, eps, copy=False), args.steps)
    phases["lowrank_mix"] = timed(lambda: h.lowrank_correct_mix_own(Vd, ld, "fp64"), args.steps)
    # one step traced, and the scan form's exact lookups and pairs of one FP64 SelInv
    h.trace(True)
    step()
    torch.cuda.synchronize()
    kern = h.trace_read()
    h.trace(False)
    h.timeline(True)
    h.selinv(Lv, Dv, "fp64", out=G)
    look, pairs = h.selinv_scan_counts()
    h.timeline(False)
    h.sync_status()
    st = h.stats()
    nS = 2 * h.nnz_S - h.n
    line = {"metric": METRIC, "value": world * nS / (ms / 1e3), "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 split operands + f64", "data": "synthetic",
            "config": {"workload": "elastic: 27-point 3-dof lattice-spring operator %d^3 nodes (n=%d), ILDL tau=1e-4; "
                                   "SelInv BF16/FP32-acc + FP64 pivots, NInv m=%d on its own pattern (delta=%g), "
                                   "Mix on that pattern, rank-%d correction on the Mix pattern"
                                   % (args.elastic_size, f.n, w.m, delta, w.k),
                       "stated_rel_error": {"selinv_bf16": "normwise 1e-5 vs FP64 oracle",
                                            "ninv_mix_lowrank": STATED_ERROR["fp64"]},
                       "selinv_bf16_normwise_vs_fp64": diff_bf16,
                       "nnz_L": st["nnz_L"], "S_entries": nS, "supernodes": st["n_supernodes"],
                       "max_width": st["max_width"], "levels": st["n_levels"], "max_c": st["max_c"],
                       "selinv_form": "scan" if st["selinv_scan"] else "pair lists",
                       "scan_lookups": look, "scan_pairs_lower": pairs, "tc_levels": st["tc_levels"],
                       "tc_supernodes": st["tc_supernodes"], "nnz_W_by_step": [int(x) for x in wsteps],
                       "nnz_N_lo": getattr(h, "own_nnz", None), "nnz_mix_lo": h.mix_own_nnz(), "eps": eps,
                       "phases_ms": phases,
                       "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kern.items()},
                       "input_gen_s": t_gen, "symbolic_s": t_sym, "l2": "flushed between timed steps (512 MB write)"},
            "clocks": clocks, "gpu_launches": int(sum(v[0] for v in kern.values()))}
    if rank == 0:
        print(json.dumps(line))


def run_covariance(args, rank, world, dev):
    """The paper's covariance-type example, (1 - d/3)^4 on an N x N grid, ILDL tau = 1e-3.
    One step = SelInv + NInv (m = 3, inverse tolerance --ninv-delta) + Mix in FP64,
    inputs resident; the phases are timed apart as well."""
    import torch
    from paper_2609_11363_b300 import Handle
    from workloads.configs import covariance
    torch.cuda.set_device(dev)
    t0 = time.time()
    w = covariance(args.cov_size)
    f = w.factors
    t_gen = time.time() - t0
    from paper_2609_11363_b300.autotune import tune_selinv
    Lv = torch.as_tensor(f.L_val, device=dev)
    Dv = torch.as_tensor(f.D_packed, device=dev)
    t0 = time.time()
    h, best, table = tune_selinv(f, Lv, Dv, prec="fp64", caps=(4, 16, 64), bigs=(1024, 4096), device=dev.index)
    t_tune = time.time() - t0
    G = torch.empty(h.nnz_S, dtype=torch.float64, device=dev)
    N = torch.empty_like(G)
    M = torch.empty_like(G)
    h.selinv(Lv, Dv, "fp64", out=G)
    h.ninv(Lv, Dv, w.m, "fp64", out=N, delta=args.ninv_delta)
    eps = 1e-3 * float(G.abs().max())  # SPD: the largest |G| is on the diagonal

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            flush.zero_()  # inputs are smaller than L2: flush it between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))

    t0 = time.time()
    Ac = h.spai_analyse(w.A, power=args.spai_power)
    t_spai_an = time.time() - t0
    Av = torch.as_tensor(Ac.data, device=dev)
    Y = torch.empty(h.nnz_P, dtype=torch.float64, device=dev)
    it = args.spai_iters

    def step():
        h.selinv(Lv, Dv, "fp64", out=G)
        h.ninv(Lv, Dv, w.m, "fp64", out=N, delta=args.ninv_delta)
        h.mix(G, N, eps, out=M)
        if it > 0:
            h.spai(Av, M, it, out=Y)

    for _ in range(args.warmup):
        step()
    ms = timed(step, args.steps)
    ms_sel = timed(lambda: h.selinv(Lv, Dv, "fp64", out=G), args.steps)
    ms_ninv = timed(lambda: h.ninv(Lv, Dv, w.m, "fp64", out=N, delta=args.ninv_delta), args.steps)
    ms_spai = timed(lambda: h.spai(Av, M, it, out=Y), args.steps) if it > 0 else 0.0
    h.sync_status()
    spectral = None
    if args.einv_k > 0:
        # the spectral check of the paper's covariance runs: k requested eigenpairs of
        # E_inv = A^{-1} - Mix, Lanczos with ILDL-preconditioned CG (timed once, synchronous)
        t0 = time.time()
        Ae = h.einv_analyse(w.A)
        t_an = time.time() - t0
        q0 = torch.as_tensor(np.random.default_rng(0).standard_normal(f.n), device=dev)
        Aev = torch.as_tensor(Ae.data, device=dev)
        torch.cuda.synchronize()
        t0 = time.time()
        lam, _, info = h.einv_lanczos(Aev, Lv, Dv, M, q0, args.einv_k, args.einv_steps, cg_tol=1e-10, cg_maxit=500)
        t_lz = time.time() - t0
        stE = h.stats()
        spectral = {"k": args.einv_k, "lanczos_steps": info["steps"], "cg_iterations": info["cg_iterations"],
                    "cg_unconverged": info["cg_unconverged"], "seconds": t_lz, "analyse_s": t_an,
                    "ritz_values": [float(x) for x in lam], "solve_levels": [stE["einv_levels_fwd"],
                                                                             stE["einv_levels_bwd"]]}
    st = h.stats()
    nS = 2 * h.nnz_S - h.n
    gn = float(torch.linalg.vector_norm(G))
    err = {"ninv_vs_selinv": float(torch.linalg.vector_norm(N - G)) / gn,
           "mix_vs_selinv": float(torch.linalg.vector_norm(M - G)) / gn}
    if f.n <= args.exact_diag_max_n:
        # err_1 of the diagonal against diag(A^{-1}) from a dense Cholesky (measurement only)
        rp, _ = h.pattern_host()
        dpos = torch.as_tensor(rp[1:] - 1, device=dev)  # the diagonal ends each row of S_lo
        Ad = torch.as_tensor(w.A.toarray(), device=dev)
        Ai = torch.cholesky_inverse(torch.linalg.cholesky(Ad))
        exact = torch.diagonal(Ai)
        del Ad, Ai
        en = float(exact.abs().sum())
        for nm, X in (("selinv", G), ("ninv", N), ("mix", M)):
            err["err1_diag_%s_vs_exact" % nm] = float((X[dpos] - exact).abs().sum()) / en
        if it > 0:
            prp, _ = h.spai_pattern()
            ppos = torch.as_tensor(prp[1:] - 1, device=dev)
            err["err1_diag_mix_spai_vs_exact"] = float((Y[ppos] - exact).abs().sum()) / en
    line = {"metric": METRIC, "value": world * nS / (ms / 1e3), "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "rel_error_on_S_lo": err, "spectral_check": spectral,
            "config": {"workload": "covariance: (1 - d/3)^4 on a %d x %d grid (n=%d), ILDL tau=1e-3, SelInv + NInv m=%d "
                                   "+ Mix%s, FP64" % (args.cov_size, args.cov_size, f.n, w.m,
                                                      " + SPAI (%d PCG steps on S + distance-%d neighbourhoods of A)"
                                                      % (it, args.spai_power) if it > 0 else ""),
                       "spai_iters": it, "spai_power": args.spai_power, "spai_nnz_P_lo": st["spai_nnz_P"],
                       "spai_fp64_ms": ms_spai, "spai_entries": st["spai_entries"], "spai_analyse_s": t_spai_an,
                       "spai_cols_warp": st["spai_cols_warp"], "spai_cols_cta": st["spai_cols_cta"],
                       "stated_rel_error": STATED_ERROR["fp64"], "ninv_delta": args.ninv_delta,
                       "nnz_A": int(w.A.nnz), "nnz_L": st["nnz_L"], "S_entries": nS, "levels": st["n_levels"],
                       "nnz_W": st["nnz_W"], "ninv_form": "map" if st["ninv_index_bytes"] > 0 else "hash",
                       "selinv_fp64_ms": ms_sel, "ninv_fp64_ms": ms_ninv, "input_gen_s": t_gen,
                       "l2": "flushed (512 MB write) before each timed step",
                       "selinv_schedule": best, "tune_table": table, "tune_s": t_tune},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line))


def _gen_diff_spd48(seed):
    from workloads.configs import diff3d
    return diff3d(48, shifted=False, m=3, seed=seed).factors


def run_reference(args, world):
    """The baseline arm: the plain FP64 oracle as it stands, on one host thread.
    Each step is one whole oracle step (SelInv, NInv, Mix, rank-k) on the same
    trailing block of the workload's factors, sized during the warm-up so that
    the whole run stays within a few minutes."""
    w, f, V, lam, t_gen = build_workload(args.size)
    # the timed steps together take about 150 s at most, and one step 15 s at most:
    # the oracle's memory grows faster than its time with the block (about 34 GB
    # at n' = 24,576 of the 64^3 workload), so a few long steps must not buy a
    # larger block
    budget_s = 150.0
    b, t_cal, nS_b, _ = calibrated_block(f, V, lam, w.m, target_s=min(budget_s / max(args.steps, 1), 15.0))
    for _ in range(max(args.warmup - 1, 0)):
        oracle_step(b, lam, w.m)
    times, parts = [], None
    for _ in range(args.steps):
        t, nS_b, parts = oracle_step(b, lam, w.m)
        times.append(t)
    t = float(np.sum(times))
    value = nS_b * args.steps / t
    sample = ("plain FP64 oracle (C SelInv, scipy NInv, numpy Mix + rank-k), one host thread; every step is a "
              "whole oracle step on the trailing principal block of the same factors (rows/cols %d..%d, n' = %d, "
              "|S'| = %d): the top of the elimination tree, whose values depend on nothing outside it" % (
                  b["c0"], f.n - 1, b["n"], nS_b))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.size, f, w.m, w.k), "n": f.n, "sample_n": b["n"],
                       "sample_S_entries": nS_b, "impl": "FP64 CPU oracle, one host thread"},
            "cpu_baseline": {"value": value, "unit": "entries/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "last_step_parts_s": {k: v for k, v in parts.items() if k.endswith("_s")}},
            "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
