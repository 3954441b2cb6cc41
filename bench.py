"""Benchmark of the EMD misfit hot path: PDHG cell-updates/s and solves/s at a fixed residual.

Workload: one transmissive-geometry gather pair of 3000 time samples x 400 receivers
(dt = 1 ms, dx = 12.5 m; eight direct / refracted / diffracted events, cycle-skipped
prediction plus 30 dB noise), solved by Algorithm 1 until the stopping residual reaches
the target.  One step = one complete solve (prepare, every PDHG pass, finalize).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (launched by torch.distributed.run) every rank solves its own gather of the
same shape: the solves are independent, so there is no data-path collective (weak
scaling).  The reference arm (--impl reference) times the FP64 CPU oracle on a bounded
sample of the same workload.  Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NT, NR, DT, DX = 3000, 400, 1e-3, 12.5
TOL = 1e-2
MG_FACTOR = 10
PROFILE_TILE = 7  # 13 x 120 tiles, two CTAs per SM (tile ids count from 1)
CELL_BYTES = 36  # algorithmic bytes per cell-update of the fused pass (first-try accept)
METRIC = "PDHG cell-updates/s and EMD solves/s at fixed residual; HBM GB/s vs peak"
WORKLOAD = (f"transmissive gather pair {NT}x{NR} (nt x nr), dt=1ms, dx=12.5m, 8 events, "
            f"Algorithm 1 to residual {TOL:g}")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", choices=["transmissive", "marine", "transmissive-mg"], default=None,
                    help="run --warmup solves of a named gather (for ncu) and exit")
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--workload", choices=["transmissive", "uneven48", "uneven48-residual"], default="transmissive",
                    help="uneven48: 48 uneven gathers, batched solve vs one solve per gather")
    return ap.parse_args()


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_shots(sizes, world):
    """Independent solves over `world` ranks: largest first, each to the rank with the
    fewest cells so far (greedy balance by cell count).  Returns one list of shot indices
    per rank; every shot lands on exactly one rank."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for s in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda j: (load[j], j))
        out[r].append(s)
        load[r] += sizes[s]
    return [sorted(x) for x in out]


def max_over_ranks(value, device="cpu"):
    """The largest `value` over all ranks (the whole job's step time); `value` itself
    when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _kernel_hash():
    """Hash of the device code of the fused pass (the benchmark gather never takes the
    resident solve), comments and whitespace removed: a traffic capture stays valid
    across edits of comments only."""
    h = hashlib.sha256()
    for rel in ("paper_1808_07284_gb300/csrc/emd_kernels.cuh", "paper_1808_07284_gb300/csrc/emd_pass_tma.cuh"):
        with open(os.path.join(ROOT, rel)) as fh:
            code = re.sub(r"//[^\n]*", "", fh.read())
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def _traffic():
    """DRAM bytes per pass launch from the committed ncu summary, if it matches these sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_pass_traffic.json")) as fh:
            t = json.load(fh)
        if t.get("sources") == _kernel_hash() and t.get("cells") == NT * NR:
            return float(t["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_baseline(obs, pred, iters=60):
    """The FP64 oracle as it stands, on a bounded sample: `iters` PDHG iterations of the
    same gather (cell-updates/s; numpy elementwise kernels run on one core)."""
    from oracle import emd_oracle as O
    t = time.perf_counter()
    r = O.pdhg(obs, pred, DT, DX, max_iter=iters)
    el = time.perf_counter() - t
    return {"value": NR * NT * r["iters"] / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{r['iters']} PDHG iterations of the {NT}x{NR} gather (FP64 numpy), {el:.1f} s"}


def run_reference(a):
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import synth
    from oracle import emd_oracle as O
    obs, pred = synth.gather_pair_transmissive(nt=NT, nr=NR, dt=DT, dx=DX)
    iters = 25
    for _ in range(a.warmup):
        O.pdhg(obs, pred, DT, DX, max_iter=3)
    times = []
    for _ in range(a.steps):
        t = time.perf_counter()
        r = O.pdhg(obs, pred, DT, DX, max_iter=iters)
        times.append(time.perf_counter() - t)
    el = sum(times)
    v = NR * NT * iters * a.steps / el
    sample = f"{iters} PDHG iterations of the {NT}x{NR} gather per step (FP64 numpy oracle)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "cell-updates/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * el / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (bounded sample: fixed iteration count)", "nt": NT, "nr": NR,
                   "iters_per_step": iters},
        "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_gpu(a):
    import numpy as np
    import torch

    import paper_1808_07284_gb300 as P
    import synth

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    obs, pred = synth.gather_pair_transmissive(nt=NT, nr=NR, dt=DT, dx=DX)
    o = torch.from_numpy(obs).to(dev)
    p = torch.from_numpy(pred).to(dev)
    ws = P.new_workspace(P.emd_workspace_size(NT, NR), dev)
    phi = torch.empty((NR, NT), dtype=torch.float32, device=dev)
    m = torch.empty((2, NR, NT), dtype=torch.float32, device=dev)
    params = P.emd_default_params(max_iter=200000, tol=TOL)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def solve(prm):
        return P.emd_dyn_solve(o, p, DT, DX, prm, phi, m, ws, stream)

    for _ in range(max(a.warmup, 3)):
        res = solve(params)
    torch.cuda.synchronize()

    # ---- timed region: K solves, L2 flushed between them, each timed by CUDA events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    iters, launches = [], 0
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(a.steps):
            flush.zero_()
            ev[s][0].record(stream)
            res = solve(params)
            ev[s][1].record(stream)
            iters.append(res.iters)
            launches += res.launches  # counted by the library: prepare, passes, finalize
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - t0
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    t_step = max_over_ranks(sum(ms) / len(ms) / 1e3, dev)
    cells = NR * NT
    it_mean = float(np.mean(iters))
    value = world * cells * it_mean / t_step

    # ---- per-pass duration, live: two fixed-iteration solves, the difference is pure passes
    def timed_fixed(n):
        prm = P.emd_default_params(max_iter=n)
        solve(prm)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solve(prm)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    n1, n2 = 256, 2304
    t_pass = (timed_fixed(n2) - timed_fixed(n1)) / (n2 - n1)
    peak, peak_kind = _peaks()
    achieved = CELL_BYTES * cells / t_pass / 1e9
    traffic = _traffic()

    # ---- the same gather by the two-grid solve (Sec. 2.2, Sec. 3.3): time coarsened by 10 (the
    #      paper's 3000 -> 301), coarse solve to the same residual, fine solve from its
    #      interpolated solution to the same residual
    mg = P.emd_default_mg_params(factor=MG_FACTOR, coarse_max_iter=200000, coarse_tol=TOL)
    ws_mg = P.new_workspace(P.emd_mg_workspace_size(NT, NR, MG_FACTOR), dev)
    for _ in range(3):
        P.emd_dyn_solve_mg(o, p, DT, DX, params, mg, phi, m, ws_mg, stream)
    mg_ms, mg_runs = [], []
    for s in range(a.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fr, cr = P.emd_dyn_solve_mg(o, p, DT, DX, params, mg, phi, m, ws_mg, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        mg_ms.append(e0.elapsed_time(e1))
        mg_runs.append((fr, cr))
    t_mg = max_over_ranks(sum(mg_ms) / len(mg_ms) / 1e3, dev)
    fr, cr = mg_runs[-1]
    multigrid = {
        "solves_per_s": world / t_mg, "ms_per_solve": 1e3 * t_mg, "factor": MG_FACTOR,
        "coarse_grid": [NR, -(-NT // MG_FACTOR)], "coarse_iters": cr.iters, "fine_iters": fr.iters,
        "residual": fr.residual, "dist": fr.dist, "dist_single_solve": res.dist,
        "speedup_vs_single_solve": t_step / t_mg, "launches_per_solve": fr.launches,
        "note": "coarse and fine solves both run to the residual of the single solve; L2 flushed before each",
    }

    # ---- end to end through the public API: pinned host gathers in, phi and the result out
    h_obs = torch.from_numpy(obs).pin_memory()
    h_pred = torch.from_numpy(pred).pin_memory()
    h_phi = torch.empty((NR, NT), dtype=torch.float32).pin_memory()
    e2e_t = []
    for s in range(max(2, a.steps)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        do = h_obs.to(dev, non_blocking=True)
        dp = h_pred.to(dev, non_blocking=True)
        r = P.emd_dyn_solve(do, dp, DT, DX, params, phi, m, ws, stream)
        h_phi.copy_(phi, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append((time.perf_counter() - t, r.iters))
    e2e_v = world * cells * sum(i for _, i in e2e_t) / sum(t for t, _ in e2e_t)

    if rank == 0:
        cpu = None if a.no_cpu_baseline else _cpu_baseline(obs, pred)
        out = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nt": NT, "nr": NR, "dt": DT, "dx": DX, "tol": TOL,
                       "iters_per_solve": it_mean, "l2": "flushed (256 MB write) before every timed solve",
                       "reductions": "f64 above the warp", "parallelism": f"{world} independent solves"},
            "solves_per_s": world / t_step,
            "multigrid": multigrid,
            "hbm_gbs_algorithmic": achieved,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_solve_tma (one fused PDHG iteration per pass of a persistent launch)",
                         "note": f"{CELL_BYTES} B/cell x {cells} cells per launch over the live per-pass "
                                 f"duration {t_pass * 1e6:.2f} us; peak {peak_kind}; the 43 MB working set "
                                 "is L2-resident between passes"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_v, "unit": "cell-updates/s", "h2d_bytes_per_step": 2 * cells * 4,
                    "d2h_bytes_per_step": cells * 4 + 192},
            "gpu_launches": launches,
            "wall_s_timed": wall,
        }
        cs = clk.summary()
        if cs is not None:
            out["clocks"] = cs
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile(a):
    """Fixed-iteration solves of one gather, nothing timed: the command ncu captures.
    transmissive: the benchmark gather (3000 x 400, 43 MB of state, L2-resident);
    marine: one 8000 x 648 streamer gather (dt = 2 ms, dx = 25 m; 187 MB of state > L2);
    transmissive-mg: the benchmark gather by the two-grid solve, both stages to the benchmark
    residual (--iters is ignored)."""
    import torch

    import paper_1808_07284_gb300 as P
    import synth
    dev = torch.device("cuda:0")
    if a.profile in ("transmissive", "transmissive-mg"):
        obs, pred = synth.gather_pair_transmissive(nt=NT, nr=NR, dt=DT, dx=DX)
        dt, dx = DT, DX
    else:
        obs, pred = synth.gather_pair_marine(shot=0)
        dt, dx = 2e-3, 25.0
    o = torch.from_numpy(obs).to(dev)
    p = torch.from_numpy(pred).to(dev)
    for _ in range(max(1, a.warmup)):
        if a.profile == "transmissive-mg":
            d, phi, m, info = P.emd(o, p, dt, dx, max_iter=200000, tol=TOL, multigrid=dict(
                factor=MG_FACTOR, coarse_max_iter=200000, coarse_tol=TOL))
        else:
            # the tile shape the benchmark's autotuner settles on, fixed: under a profiler
            # the autotuner's trial timings are distorted and it may pick another shape
            d, phi, m, info = P.emd(o, p, dt, dx, max_iter=a.iters, tile=PROFILE_TILE)
    torch.cuda.synchronize()
    print(json.dumps({"profile": a.profile, "shape": list(obs.shape), "iters": info["iters"],
                      "dist": d, "status": info["status"]}))


def run_uneven48(a):
    """48 gathers with nr ~ U{200..640}, nt ~ U{1500..5000} (dt = 1 ms, dx = 12.5 m), 200
    PDHG iterations each (the paper runs 100-200 per EMD): one batched solve against the
    same 48 solves run one after another.  The two produce the same iterates, so they end
    at the same residual."""
    import torch

    import paper_1808_07284_gb300 as P
    import synth
    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    allp = synth.batch_uneven_hyperbolic(n_shots=48)
    mine = shard_shots([o.size for o, _ in allp], world)[rank]
    pairs = [allp[s] for s in mine]
    total_cells = sum(o.size for o, _ in allp)
    O_ = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    P_ = [torch.from_numpy(p).to(dev) for _, p in pairs]
    cells = sum(o.numel() for o in O_)
    iters = 200
    nts, nrs = [o.shape[1] for o in O_], [o.shape[0] for o in O_]
    wsb = P.new_workspace(P.emd_batched_workspace_size(nts, nrs), dev)
    wss = P.new_workspace(max(P.emd_workspace_size(nt, nr) for nt, nr in zip(nts, nrs)), dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def batched():
        return P.emd_batched(O_, P_, DT, DX, workspace=wsb, max_iter=iters)

    def sequential():
        return [P.emd(o, p, DT, DX, workspace=wss, max_iter=iters) for o, p in zip(O_, P_)]

    def timed(fn):
        for _ in range(max(1, a.warmup)):
            fn()
        ts = []
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return sum(ts) / len(ts), out

    tb, (db, _, _, ib) = timed(batched)
    ts_, outs = timed(sequential)
    tb, ts_ = max_over_ranks(tb, dev), max_over_ranks(ts_, dev)
    worst = max(abs(db[b] - outs[b][0]) / abs(outs[b][0]) for b in range(len(pairs)))
    if rank != 0:
        return
    print(json.dumps({
        "metric": "EMD solves/s, 48 uneven gathers (batched vs one solve per gather)",
        "value": 48 / tb, "unit": "solves/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * tb, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "48 uneven hyperbolic gathers, nr~U{200..640}, nt~U{1500..5000}, "
                               "dt=1ms, dx=12.5m, 200 iterations", "cells": total_cells,
                   "parallelism": f"shots sharded over {world} ranks, no collective"},
        "sequential_solves_per_s": 48 / ts_, "batched_speedup": ts_ / tb, "scaling": "strong",
        "cell_updates_per_s_batched": total_cells * iters / tb,
        "hbm_gbs_algorithmic_batched": CELL_BYTES * total_cells * iters / tb / 1e9,
        "max_rel_dist_diff_batched_vs_sequential": worst,
    }), flush=True)


def run_uneven48_residual(a):
    """The 48 uneven gathers of run_uneven48, every solve run to the residual TOL instead of
    a fixed count: one batched solve and one solve per gather, each with and without the
    two-grid warm start (time coarsened by MG_FACTOR, coarse stage to the same residual)."""
    import torch

    import paper_1808_07284_gb300 as P
    import synth
    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    allp = synth.batch_uneven_hyperbolic(n_shots=48)
    mine = shard_shots([o.size for o, _ in allp], world)[rank]
    pairs = [allp[s] for s in mine]
    total_cells = sum(o.size for o, _ in allp)
    O_ = [torch.from_numpy(o).to(dev) for o, _ in pairs]
    P_ = [torch.from_numpy(p).to(dev) for _, p in pairs]
    nts, nrs = [o.shape[1] for o in O_], [o.shape[0] for o in O_]
    mg = dict(factor=MG_FACTOR, coarse_max_iter=200000, coarse_tol=TOL)
    wsb = P.new_workspace(P.emd_batched_mg_workspace_size(nts, nrs, MG_FACTOR), dev)
    wss = P.new_workspace(max(P.emd_mg_workspace_size(nt, nr, MG_FACTOR) for nt, nr in zip(nts, nrs)), dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    kw = dict(max_iter=200000, tol=TOL)

    arms = {
        "batched_two_grid": lambda: P.emd_batched(O_, P_, DT, DX, workspace=wsb, multigrid=mg, **kw),
        "batched": lambda: P.emd_batched(O_, P_, DT, DX, workspace=wsb, **kw),
        "per_gather_two_grid": lambda: _per_gather(P, O_, P_, wss, dict(multigrid=mg, **kw)),
        "per_gather": lambda: _per_gather(P, O_, P_, wss, kw),
    }
    res = {}
    for name, fn in arms.items():
        for _ in range(max(1, a.warmup)):
            fn()
        ts = []
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            d, _, _, infos = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = max_over_ranks(sum(ts) / len(ts), dev)
        res[name] = {"solves_per_s": 48 / t, "ms_per_step": 1e3 * t,
                     "max_residual": max(i["residual"] for i in infos),
                     "fine_iters_mean": sum(i["iters"] for i in infos) / len(infos),
                     "fine_iters_max": max(i["iters"] for i in infos), "dists": d}
    if rank != 0:
        return
    ref = res["per_gather"]["dists"]
    for v in res.values():
        v["max_rel_dist_diff_vs_per_gather"] = max(abs(x - y) / abs(y) for x, y in zip(v.pop("dists"), ref))
    top = res["batched_two_grid"]
    print(json.dumps({
        "metric": "EMD solves/s at fixed residual, 48 uneven gathers",
        "value": top["solves_per_s"], "unit": "solves/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": top["ms_per_step"], "higher_is_better": True, "dtype": "f32",
        "data": "synthetic", "scaling": "strong",
        "config": {"workload": "48 uneven hyperbolic gathers, nr~U{200..640}, nt~U{1500..5000}, dt=1ms, "
                               f"dx=12.5m, every solve to residual {TOL:g}", "cells": total_cells,
                   "two_grid_factor": MG_FACTOR, "parallelism": f"shots sharded over {world} ranks, no collective",
                   "l2": "flushed (256 MB write) before every timed step"},
        "arms": res,
        "batched_vs_per_gather": res["per_gather"]["ms_per_step"] / res["batched"]["ms_per_step"],
        "batched_two_grid_vs_per_gather": res["per_gather"]["ms_per_step"] / top["ms_per_step"],
        "batched_two_grid_vs_per_gather_two_grid":
            res["per_gather_two_grid"]["ms_per_step"] / top["ms_per_step"],
    }), flush=True)


def _per_gather(P, O_, P_, ws, kw):
    out = [P.emd(o, p, DT, DX, workspace=ws, **kw) for o, p in zip(O_, P_)]
    return [x[0] for x in out], None, None, [x[3] for x in out]


def main():
    a = _args()
    if a.workload == "uneven48" and not a.profile and a.impl != "reference":
        run_uneven48(a)
        return
    if a.workload == "uneven48-residual" and not a.profile and a.impl != "reference":
        run_uneven48_residual(a)
        return
    if a.profile:
        run_profile(a)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
