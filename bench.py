#!/usr/bin/env python
"""Benchmark of the column-generation VMAT optimiser on one B300.

A step is one whole plan: 180 column-generation iterations (prices ->
pricing -> aperture column -> master problem) on the prostate-scale phantom
(128x128x64 voxels at 3 mm, 180 beams, 40x40 MLC, 4.51e8 non-zeros of D, FP32
D).  value = column-generation iterations per second over all ranks, inputs
resident in HBM.  Also reported: the roofline of the dominant kernel, the
sparse products' HBM bandwidth, FP16/BF16-D plans with their dose error
against FP64 NumPy products of the same D, an end-to-end figure through the C-ABI from host
buffers, and the oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched by torch.distributed.run, one independent plan per rank
(replicas; weak scaling).
"""
from __future__ import annotations

import argparse
import csv
import dataclasses
import ctypes
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CG iters/s & SpMV HBM GB/s (% of peak); FP16-D vs FP32-D at ≤0.5% dose err"
# DRAM bytes / algorithmic bytes of k_master from one ncu capture of the
# current kernel on the plan's own apertures (bench.py --case master-plan
# --case-cols 90 --case-ctas 73: 65.284864 MB read + 0.806656 MB written
# against 3,922,386,944 algorithmic bytes of that launch); set to None
# whenever the kernel changes until it has been captured again
MASTER_TRAFFIC_RATIO = (65.284864e6 + 0.806656e6) / 3922386944
# L2 sector peak of that capture: 140,826,227 sectors in 1.361408 ms at
# 9.510887% of peak sustained elapsed, 32 B per sector
L2_PEAK_GBS = 140826227 / 1.361408e-3 / 0.09510887 * 32 / 1e9
UNIT = "CG iters/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = []
        reasons = set()
        smax = 0.0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- helpers
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _aggregate(ms_local, ws, steps, units_per_step, device):
    """Whole-job throughput of `ws` replicas (one per GPU, independent plans,
    no data-path collective): the slowest rank's time (all-reduce MAX over
    the timed region) and every rank's units over it."""
    ms = float(ms_local)
    if ws > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ws * steps * units_per_step / (ms / 1e3)


def _workload(name):
    from paper_1005_4396_b300 import inputs
    return {"prostate": inputs.prostate_config, "tiny": inputs.tiny_config,
            "headneck": inputs.headneck_config}[name]()


def _describe(cfg, prob):
    return (f"{cfg.name}: {cfg.nx}x{cfg.ny}x{cfg.nz} voxels at {cfg.h} mm, {cfg.n_angles} beams, "
            f"{cfg.n_rows}x{cfg.n_cols} MLC, {prob.n_beamlets} beamlets, nnz(D)={prob.nnz}, "
            f"{cfg.iterations} CG iterations per plan, master KKT {cfg.kkt_eps:g}")


def _algorithmic_bytes(prob, info, rec):
    """Bytes each kernel must move per launch by its definition (not counting
    re-reads).  master: every PG iteration reads the aperture-dose columns
    twice (gradient pass, direction pass) plus once at entry (the dose at
    exit comes from the carried state), counting only the subtiles of a
    column that hold a nonzero (an
    all-zero subtile carries no information and is not read), and writes z
    and F'.  price: the D rows of the free beams (8 B/nnz FP32 value+index),
    their row pointers, the prices written, F' gathered once.  Also returns
    the master bytes of dense columns (every voxel of every column)."""
    cfg = prob.cfg
    RC = cfg.n_rows * cfg.n_cols
    Va = info["n_active"]
    sv = info["subtile_voxels"]
    vb = 8 if info["d_dtype"] == 1 else 6
    nnz_beam = np.add.reduceat(np.diff(prob.row_ptr), np.arange(0, prob.n_beamlets, RC))
    free_nnz = nnz_beam.sum()
    master, dense, price = [], [], []
    sub = np.cumsum(rec["col_subtiles"].astype(np.float64))
    for t, k in enumerate(rec["k"]):
        P = int(rec["iters"][t])
        master.append((2 * P + 1) * sub[t] * sv * 4 + 8 * Va)
        dense.append((2 * P + 1) * (t + 1) * Va * 4 + 8 * Va)
        free_beams = cfg.n_angles - t
        price.append(free_nnz * vb + free_beams * RC * (8 + 4) + 4 * Va)
        free_nnz -= nnz_beam[k]
    return (np.array(master, dtype=np.float64), np.array(price, dtype=np.float64),
            np.array(dense, dtype=np.float64))


# ---------------------------------------------------------------- FP64 checks
# Dose and gradient errors reported beside the timings are taken against
# plain FP64 NumPy products of the same D (the library is not involved).
def _fluence64(cfg, lleaf, rleaf, y):
    """Beamlet fluence of apertures (open columns [l, r) of each row) with
    intensities y: x_(k,row,c) = y_k where open (Eq. 3)."""
    N, R, C = cfg.n_angles, cfg.n_rows, cfg.n_cols
    c = np.arange(C).reshape(1, 1, C)
    l = np.asarray(lleaf, np.int64).reshape(N, R, 1)
    r = np.asarray(rleaf, np.int64).reshape(N, R, 1)
    return (((c >= l) & (c < r)) * np.asarray(y, np.float64).reshape(N, 1, 1)).reshape(-1)


def _dose64(prob, x):
    """z_j = sum_i D_ij x_i in FP64."""
    w = np.repeat(np.asarray(x, np.float64), np.diff(prob.row_ptr)) * prob.val
    return np.bincount(prob.vox_idx, weights=w, minlength=prob.n_vox)


def _price64(prob, f):
    """g_i = sum_j D_ij f_j in FP64 (empty rows give 0)."""
    prod = prob.val * np.asarray(f, np.float64)[prob.vox_idx]
    g = np.zeros(prob.n_beamlets)
    nz = np.flatnonzero(np.diff(prob.row_ptr) > 0)
    g[nz] = np.add.reduceat(prod, prob.row_ptr[nz])
    return g


def _cost64(prob, z):
    """sum_j F(z_j) (Eq. 1) and F'(z) in FP64."""
    Tv, av, bv = prob.voxel_params()
    e = z - Tv
    return float(np.sum(np.where(e > 0, bv, av) * e * e)), np.where(e > 0, 2 * bv * e, 2 * av * e)


def _gaps(theta, cyclic):
    """(left, right) neighbour and gap of each beam on the arc (None at path ends)."""
    n = len(theta)
    out = []
    for k in range(n):
        lft = k - 1 if k > 0 else (n - 1 if cyclic and n > 1 else None)
        rgt = k + 1 if k < n - 1 else (0 if cyclic and n > 1 else None)
        gl = None if lft is None else (theta[k] - theta[lft] if lft < k else theta[0] + 360.0 - theta[n - 1])
        gr = None if rgt is None else (theta[rgt] - theta[k] if rgt > k else theta[0] + 360.0 - theta[n - 1])
        out.append((lft, gl, rgt, gr))
    return out


def _rate64(theta, y, cyclic):
    """Largest |y_k' - y_k| / gap over neighbouring beams (degrees)."""
    return max([abs(y[r] - y[k]) / g for k, (_, _, r, g) in enumerate(_gaps(theta, cyclic)) if r is not None],
               default=0.0)


def _dG64(theta, y, cyclic):
    """Gradient of the smoothing term of Eq. 2."""
    g = np.zeros(len(y))
    for k, (lft, gl, rgt, gr) in enumerate(_gaps(theta, cyclic)):
        if lft is not None:
            g[k] += 2.0 * (y[k] - y[lft]) / gl
        if rgt is not None:
            g[k] -= 2.0 * (y[rgt] - y[k]) / gr
    return g


def _dose_err(prob, plan_f, plan_ref_dose, lleaf, rleaf, y):
    """max/mean |z - z_FP64| over voxels, in % of the largest prescription."""
    z64 = _dose64(prob, _fluence64(prob.cfg, lleaf, rleaf, y))
    d = np.abs(plan_ref_dose.astype(np.float64) - z64)
    rx = float(prob.T.max())
    return float(d.max() / rx * 100), float(d.mean() / rx * 100)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    from paper_1005_4396_b300 import inputs, vmat
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peak, peak_kind = _peaks()
    cfg = _workload(args.workload)
    prob = inputs.make_problem(cfg)
    plan = vmat.Plan(prob, val_f32=True)
    plan.set_master_method(args.master)
    info = plan.info
    plan.set_profiling(True)

    kkt = max(cfg.kkt_eps, 1e-6)  # FP32 gradients: relative KKT 1e-6 is the reachable floor

    def step():
        plan.reset()
        return plan.colgen_run(kkt_tol=kkt)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = plan.launches()
    inf0 = vmat.vmat_get_info(plan.ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    recs = [step() for _ in range(args.steps)]
    ev1.record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    launches = plan.launches() - l0
    inf1 = vmat.vmat_get_info(plan.ctx)
    ms, value = _aggregate(ev0.elapsed_time(ev1), ws, args.steps, cfg.iterations, "cuda")
    # in-kernel phase clocks of the master (CTA 0) over the timed plans
    pg_iters = inf1["master_pg_iters"] - inf0["master_pg_iters"]
    master_phases = {
        "us_per_iteration": {n: round(1e3 * (inf1["master_ms"][q] - inf0["master_ms"][q]) / max(pg_iters, 1), 3)
                             for q, n in enumerate(["gradient_pass_and_sum", "step", "direction_pass",
                                                    "line_search"])},
        "grid_barriers_per_iteration": round((inf1["master_syncs"] - inf0["master_syncs"]) / max(pg_iters, 1), 3),
        "rejected_trial_steps_per_plan": round((inf1["master_rejected"] - inf0["master_rejected"]) / args.steps, 1),
        "grid_barrier_wait_us_per_iteration": round(
            1e3 * (inf1["master_wait_ms"] - inf0["master_wait_ms"]) / max(pg_iters, 1), 3),
        "note": "globaltimer clocks of CTA 0 inside k_master, per projected-gradient iteration",
    }
    live_calls = inf1["price_calls"][0] - inf0["price_calls"][0]
    price_calls = inf1["price_calls"][1] - inf0["price_calls"][1]
    live_entries = inf1["price_live_entries"] - inf0["price_live_entries"]

    # per-phase device time and the roofline of the dominant kernel
    phase = np.sum([r["phase_ms"] for r in recs], axis=0)  # [n_iter, 4]
    ph_tot = phase.sum(axis=0) / args.steps
    names = ["price_spmv", "pricing", "aperture", "master"]
    mb, pb, db = zip(*[_algorithmic_bytes(prob, info, r) for r in recs])
    mb = np.sum(mb, axis=0) / args.steps
    pb = np.sum(pb, axis=0) / args.steps
    db = np.sum(db, axis=0) / args.steps
    if price_calls and live_calls == price_calls:
        # every pricing read only the live voxels' rows: 8 B per entry read, F' read
        # twice (scan, rows), and per free beamlet its accumulator read and cleared
        # and its price written
        free_beamlets = sum((cfg.n_angles - t) * cfg.n_rows * cfg.n_cols for t in range(cfg.iterations))
        pb = np.array([(8.0 * live_entries + price_calls * 8.0 * info["n_active"]
                        + args.steps * free_beamlets * 20.0) / args.steps])
    master_gbs = mb.sum() / (ph_tot[3] / 1e3) / 1e9
    price_gbs = pb.sum() / (ph_tot[0] / 1e3) / 1e9
    dom = int(np.argmax(ph_tot))
    dom_gbs = {0: price_gbs, 3: master_gbs}.get(dom)
    n_master = len(recs[0]["k"])
    roofline = {
        "kernel": {0: "k_price", 1: "k_pricing", 2: "k_aperture", 3: "k_master"}[dom],
        "bound": "hbm", "achieved": round(dom_gbs, 1) if dom_gbs else None,
        "peak": peak, "unit": "GB/s", "frac": round(dom_gbs / peak, 4) if dom_gbs else None,
        "peak_kind": f"{peak_kind} copy bandwidth",
        # DRAM bytes per launch = measured traffic/algorithmic ratio of one ncu capture of
        # this kernel on a plan's own apertures (half-depth phantom, 90 columns, 30
        # iterations) times this launch's algorithmic bytes
        "traffic": (round(MASTER_TRAFFIC_RATIO * float(mb.sum()) / n_master, 0)
                    if dom == 3 and MASTER_TRAFFIC_RATIO else None),
        "traffic_note": "per launch (average over the plan), scaled from one ncu capture of the "
                        "same kernel on a half-depth prostate plan's own 90 apertures (65 MB of "
                        "nonzero column subtiles, L2-resident): DRAM/algorithmic = 0.0179",
        "l2": ({"achieved": round(dom_gbs, 1), "peak": round(L2_PEAK_GBS, 1), "unit": "GB/s",
                "frac": round(dom_gbs / L2_PEAK_GBS, 4),
                "peak_kind": "L2 sector peak of the ncu capture (34.8 TB/s)"} if dom == 3 else None),
        "launches_per_step": n_master,
        "bytes_per_step": float(mb.sum()),
        "note": ("master algorithmic bytes per launch = (2*P+1) reads of the nonzero subtiles "
                 "of the plan's aperture-dose columns (4 B per voxel) + z and F' written; "
                 "P = projected-gradient iterations of the launch; the nonzero part of the "
                 "columns fits in L2 (126 MB) and is read from DRAM about once per launch, so "
                 "frac (HBM) is not this kernel's bound: it is latency- and barrier-bound "
                 "(l2.frac, and the ncu stall counters)"),
    }
    # stand-alone SpMV bandwidth of the two sparse products at full D (FP32)
    x = torch.rand(prob.n_beamlets, device="cuda")
    f = torch.randn(prob.n_vox, device="cuda")
    z = torch.empty(prob.n_vox, device="cuda")
    g = torch.empty(prob.n_beamlets, device="cuda")
    spmv = {}
    for name, fn, byts in [
            ("dose", lambda: vmat.vmat_dose(plan.ctx, x, z, None, False),
             prob.nnz * 8 + (info["n_active"] + 1) * 8 + info["n_active"] * 8 + prob.n_beamlets * 4),
            ("price", lambda: vmat.vmat_price(plan.ctx, f, g, None),
             prob.nnz * 8 + (prob.n_beamlets + 1) * 8 + prob.n_beamlets * 4 + info["n_active"] * 8)]:
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 20
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        t_ms = a.elapsed_time(b) / n
        gbs = byts / (t_ms / 1e3) / 1e9
        spmv[name] = {"ms": round(t_ms, 4), "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
                      "frac_nominal_8TBs": round(gbs / 8000.0, 4)}
    spmv["note"] = ("host-timed around the C-ABI call (includes its stream synchronisation); "
                    "bytes: 8 B/nnz (FP32 value + int32 index) + row pointers + vectors")
    spmv["price_in_plan_GB/s"] = round(price_gbs, 1)
    spmv["price_in_plan"] = {
        "ms_per_plan": round(float(ph_tot[0]), 3), "live_voxel_form_calls": int(live_calls),
        "calls": int(price_calls),
        "live_entries_per_call": round(live_entries / max(live_calls, 1), 1),
        "fraction_of_D_read_per_call": round(live_entries / max(live_calls, 1) / prob.nnz, 5),
        "note": ("prices of the free beams at each column-generation iteration; the live-voxel "
                 "form reads only the voxel-major rows of voxels with F' != 0 (one-sided Eq. 1); "
                 "GB/s over its algorithmic bytes (8 B per entry read + F' twice + 20 B per free "
                 "beamlet)")}

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded phantom and ray/Gaussian D; no clinical data)",
           "config": {"workload": _describe(cfg, prob), "parallelism": f"replicas x{ws}",
                      "l2": (f"D {prob.nnz * 8 / 1e9:.2f} GB per copy (FP32 value + int32 index), "
                             f"aperture-dose matrix up to {info['n_active'] * cfg.n_angles * 4 / 1e6:.0f} MB; "
                             + ("inputs larger than L2 (126 MB); no flush" if prob.nnz * 8 > 126e6 else
                                "the tiny workload fits in L2; no flush (L2-resident by design)")),
                      "active_voxels": info["n_active"],
                      "master_launch": [info["master_grid"], info["master_block"]]},
           "gpu_launches": int(launches),
           "roofline": roofline, "spmv": spmv,
           "phases_ms_per_plan": {n: round(float(v), 3) for n, v in zip(names, ph_tot)},
           "master_method": {"pg": "projected gradient (Sec. 2.2)",
                             "newton": "projected Newton (option beyond the paper)"}[args.master],
           "master_iters_per_plan": int(np.mean([r["iters"].sum() for r in recs])),
           "master_phases": master_phases,
           "final_cost": float(recs[-1]["cost"][-1]),
           "clocks": clocks}

    if rank == 0 and ws == 1 and not args.quick:
        out["variants"] = run_variants(prob, plan, recs[-1], kkt)  # reads this plan's state first
        out["plan_quality"] = run_quality(prob, plan)  # before the feasibility step changes y
        out["dose_rate_feasibility"] = run_feasibility(prob, plan, recs[-1], kkt)
        out["price_smoothing"] = run_price_smoothing(prob, plan, recs[-1], kkt)
        if args.master == "pg":
            out["projected_newton"] = run_newton(prob, plan, recs[-1], kkt, args)
        out["e2e"] = run_e2e(prob, args)
    plan.close()
    if rank == 0 and ws == 1 and not args.quick:
        extra = {}
        if args.workload == "prostate" and not args.headline_only:
            hn = inputs.make_problem(inputs.headneck_config())
            out["headneck"] = run_workload_leg(hn, args)
            extra["headneck"] = hn
            out["batched"] = run_batched_leg(args)
        out["cpu_baseline"] = run_cpu_baseline(prob, args, extra)
        out["headline"] = ("value, roofline, e2e and cpu_baseline.value: the prostate workload "
                           "(config.workload); headneck and batched are further workloads in the "
                           "same run")
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_quality(prob, plan):
    """Dose-volume histograms of the timed plan (GPU, 1500 bins up to 1.5 x
    the largest prescription) and per-structure figures (mean, D95, D5,
    fraction at or above the largest prescription)."""
    import torch
    from paper_1005_4396_b300 import quality
    rx = float(prob.T.max())
    z = plan.plan_dose()
    plan.dvh(z, 1.5 * rx, 1500)  # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    counts = plan.dvh(z, 1.5 * rx, 1500)
    b.record()
    torch.cuda.synchronize()
    m = quality.dvh_metrics(counts, 1.5 * rx, prob.struct_names, rx)
    return {"dvh_ms": round(a.elapsed_time(b), 3), "prescription": rx,
            "structures": {k: {q: round(v, 4) if isinstance(v, float) else v for q, v in d.items()}
                           for k, d in m.items() if k != "air"}}


def run_feasibility(prob, plan, rec, kkt):
    """Sec. 3 final step on the timed plan: a dose-rate limit of half the
    plan's largest variation between neighbours (the paper gives no value),
    gamma doubled per round until the plan meets it."""
    cfg = prob.cfg
    y = rec["y"]
    top = _rate64(prob.theta_deg, y, cfg.cyclic)
    limit = 0.5 * top
    t0 = time.perf_counter()
    r = plan.dose_rate_feasibility(limit, gamma_factor=2.0, max_rounds=30, kkt_tol=kkt,
                                   allow_infeasible=True)
    dt = time.perf_counter() - t0
    return {"limit_per_degree": limit, "largest_before": top, "rounds": r["rounds"],
            "gamma": r["gamma"], "violation_after": r["violation"], "feasible": r["violation"] <= 0,
            "cost_before": float(rec["cost"][-1]), "cost_after": r["cost"], "ms": round(dt * 1e3, 2),
            "note": "limit proposed here (half the plan's largest |dy|/gap); cost_after uses the final gamma"}


def _plan_parts(prob, r):
    """Eq. 1 voxel cost (FP64 NumPy dose of the plan's fluence), Eq. 2
    smoothing term and largest |dy|/gap of a finished plan, on its own arc."""
    cfg = prob.cfg
    y = r["y"]
    z = _dose64(prob, _fluence64(cfg, r["lleaf"], r["rleaf"], y))
    G = float(np.sum([(y[k2] - y[k]) ** 2 / g for k, (_, _, k2, g) in
                      enumerate(_gaps(prob.theta_deg, cfg.cyclic)) if k2 is not None]))
    return {"voxel_cost": _cost64(prob, z)[0], "G": G, "max_rate_per_degree": _rate64(prob.theta_deg, y, cfg.cyclic)}


def _timed_plan(plan, kkt):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.reset()
    torch.cuda.synchronize()
    a.record()
    r = plan.colgen_run(kkt_tol=kkt)
    b.record()
    torch.cuda.synchronize()
    return r, a.elapsed_time(b) / 1e3


def run_price_smoothing(prob, plan, rec, kkt):
    """The timed plan again with smoothing-aware pricing: each beam priced by
    the exact reduced cost of its new column (beamlet sum + gamma dG/dy_k,
    an option; the paper prices by the beamlet sum)."""
    plan.set_price_smoothing(True)
    try:
        r, s = _timed_plan(plan, kkt)
    finally:
        plan.set_price_smoothing(False)
    n = len(r["k"])
    return {"cg_iters_per_s": round(n / s, 3), "s_per_plan": round(s, 4),
            "master_iters": int(r["iters"].sum()), "final_cost": float(r["cost"][-1]),
            "final_cost_literal_pricing": float(rec["cost"][-1]),
            "iterations_with_other_beam": int(np.sum(r["k"] != rec["k"])),
            "note": "option beyond the paper's literal price; same workload and KKT rule"}


def run_study(args):
    """Pricing study on one workload: the paper's literal aperture price
    against the exact reduced cost (smoothing derivative included), on a ring
    of beams (the smoothing and leaf-travel neighbours wrap around, as the
    arc of a full rotation) and on a path (Eq. 2 as printed, k = 1..N-1).
    Each plan is evaluated in FP64 on its own arc."""
    import torch
    from paper_1005_4396_b300 import inputs, vmat
    torch.cuda.set_device(0)
    cfg = _workload(args.workload)
    base = inputs.make_problem(cfg)
    kkt = max(cfg.kkt_eps, 1e-6)
    rows = []
    for cyclic in (True, False):
        prob = inputs.Problem(**{**base.__dict__, "cfg": dataclasses.replace(cfg, cyclic=cyclic)})
        with vmat.Plan(prob, val_f32=True) as plan:
            for _ in range(args.warmup if cyclic else 1):
                plan.reset()
                plan.colgen_run(kkt_tol=kkt)
            for exact in (False, True):
                plan.set_price_smoothing(exact)
                r, s = _timed_plan(plan, kkt)
                parts = _plan_parts(prob, r)
                rows.append({"arc": "ring" if cyclic else "path",
                             "pricing": "exact reduced cost" if exact else "beamlet sum (paper)",
                             "s_per_plan": round(s, 4), "cg_iters_per_s": round(len(r["k"]) / s, 3),
                             "master_iters": int(r["iters"].sum()),
                             "final_cost": float(r["cost"][-1]),
                             "voxel_cost": round(parts["voxel_cost"], 6),
                             "gamma_G": round(cfg.gamma * parts["G"], 6),
                             "max_rate_per_degree": round(parts["max_rate_per_degree"], 6),
                             "beam_order_head": r["k"][:8].tolist()})
    out = {"metric": "pricing study: CG iters/s and final cost, literal vs exact reduced-cost pricing, ring vs path",
           "value": rows[0]["cg_iters_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
           "dtype": "f32", "data": "synthetic", "config": {"workload": _describe(cfg, base)},
           "gamma": cfg.gamma, "plans": rows}
    print(json.dumps(out), flush=True)


def run_newton(prob, plan, rec_pg, kkt, args):
    """The same plan with the projected-Newton master (an option beyond the
    paper): CG iterations/s, master iterations and where the time goes; its
    plan's dose against the FP64 dose (NumPy) of the same apertures and
    intensities."""
    import torch
    plan.set_master_method("newton")
    try:
        for _ in range(args.warmup):
            plan.reset()
            plan.colgen_run(kkt_tol=kkt)
        recs = []
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.steps):
            plan.reset()
            recs.append(plan.colgen_run(kkt_tol=kkt))
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        r = recs[-1]
        ph = np.sum([q["phase_ms"] for q in recs], axis=0).sum(axis=0) / args.steps
        z = plan.plan_dose().cpu().numpy()
        emax, _ = _dose_err(prob, plan, z, r["lleaf"], r["rleaf"], r["y"])
    finally:
        plan.set_master_method("pg")
    n = len(r["k"])
    return {"value": round(n / (ms / 1e3), 3), "unit": UNIT, "ms_per_plan": round(ms, 3),
            "master_iters_per_plan": int(np.mean([q["iters"].sum() for q in recs])),
            "max_master_iters": int(r["iters"].max()),
            "phases_ms_per_plan": {k: round(float(v), 3) for k, v in
                                   zip(["price_spmv", "pricing", "aperture", "master"], ph)},
            "final_cost": float(r["cost"][-1]), "final_cost_pg": float(rec_pg["cost"][-1]),
            "beams_in_same_order_as_pg": int(np.sum(r["k"] == rec_pg["k"])),
            "max_dose_err_pct_rx": round(emax, 6),
            "note": "same workload and KKT rule; not the paper's method (Sec. 2.2 names the gradient "
                    "projection method), so not the headline value"}


def run_variants(prob, plan32, rec32, kkt=1e-6):
    """FP16-D and BF16-D plans: throughput and dose error against an FP64 product of D."""
    import torch
    from paper_1005_4396_b300 import vmat
    res = {}
    z32 = plan32.plan_dose().cpu().numpy()
    e32 = _dose_err(prob, plan32, z32, rec32["lleaf"], rec32["rleaf"], rec32["y"])
    res["f32"] = {"max_dose_err_pct_rx": round(e32[0], 5), "mean_dose_err_pct_rx": round(e32[1], 6)}
    for dt in ("f16", "bf16"):
        with vmat.Plan(prob, dtype=dt, val_f32=True) as p:
            p.reset()
            p.colgen_run(kkt_tol=kkt)
            p.reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            r = p.colgen_run(kkt_tol=kkt)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            z = p.plan_dose().cpu().numpy()
            emax, emean = _dose_err(prob, p, z, r["lleaf"], r["rleaf"], r["y"])
            same = int(np.sum(r["k"] == rec32["k"]))
            res[dt] = {"cg_iters_per_s": round(len(r["k"]) / t, 3),
                       "max_dose_err_pct_rx": round(emax, 4), "mean_dose_err_pct_rx": round(emean, 5),
                       "within_0.5pct": bool(emax <= 0.5),
                       "final_cost": float(r["cost"][-1]),
                       "beams_in_same_order_as_f32": same,
                       "device_bytes": p.info["device_bytes"]}
    res["note"] = ("dose error: the plan's own dose on the GPU against the FP64 dose (NumPy) of "
                   "the same apertures and intensities, % of the largest prescription")
    return res


def run_workload_leg(prob, args):
    """Another single-plan workload in the default run: one plan per storage
    type of D (FP32, FP16, BF16 with per-beamlet scale), each timed over
    --steps plans after one warm-up, with the plan's own GPU dose against the
    FP64 NumPy dose of its apertures and intensities."""
    import torch
    from paper_1005_4396_b300 import vmat
    cfg = prob.cfg
    kkt = max(cfg.kkt_eps, 1e-6)
    res = {"workload": _describe(cfg, prob)}
    for dt in ("f32", "f16", "bf16"):
        with vmat.Plan(prob, dtype=dt, val_f32=True) as p:
            p.reset()
            p.colgen_run(kkt_tol=kkt)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            for _ in range(args.steps):
                p.reset()
                r = p.colgen_run(kkt_tol=kkt)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3 / args.steps
            z = p.plan_dose().cpu().numpy()
            emax, emean = _dose_err(prob, p, z, r["lleaf"], r["rleaf"], r["y"])
            res[dt] = {"cg_iters_per_s": round(len(r["k"]) / t, 3), "s_per_plan": round(t, 4),
                       "master_iters": int(r["iters"].sum()),
                       "max_dose_err_pct_rx": round(emax, 5), "mean_dose_err_pct_rx": round(emean, 6),
                       "within_0.5pct": bool(emax <= 0.5), "final_cost": float(r["cost"][-1]),
                       "device_bytes": p.info["device_bytes"]}
    res["note"] = ("CUDA events around --steps whole plans (D resident); dose error: the plan's "
                   "own GPU dose against the FP64 dose of the same apertures and intensities, "
                   "% of the largest prescription")
    return res


def run_e2e(prob, args):
    """Same metric through the C-ABI from pinned host buffers: create (H2D of
    D and the problem), one plan, read back the result, destroy."""
    import torch
    from paper_1005_4396_b300 import vmat
    cfg = prob.cfg

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t, t.numpy()

    keep = []
    arrs = {}
    for name, a in [("theta", prob.theta_deg.astype(np.float64)), ("sid", prob.struct_id),
                    ("T", prob.T), ("alpha", prob.alpha), ("beta", prob.beta),
                    ("row_ptr", prob.row_ptr), ("vox", prob.vox_idx),
                    ("val", prob.val.astype(np.float32))]:
        t, v = pinned(a)
        keep.append(t)
        arrs[name] = v
    h2d = sum(v.nbytes for v in arrs.values())
    P = vmat.vmat_problem(prob.n_vox, cfg.n_angles, cfg.n_rows, cfg.n_cols,
                          arrs["theta"].ctypes.data, arrs["sid"].ctypes.data, arrs["T"].size,
                          arrs["T"].ctypes.data, arrs["alpha"].ctypes.data, arrs["beta"].ctypes.data,
                          cfg.gamma, int(cfg.cyclic), cfg.max_leaf_step, prob.nnz,
                          arrs["row_ptr"].ctypes.data, arrs["vox"].ctypes.data, vmat.VMAT_F32,
                          arrs["val"].ctypes.data)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = cfg.iterations
    times = []
    d2h = 0
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = vmat.vmat_create_raw(P, vmat.VMAT_F32, stream)
        r = vmat.vmat_colgen_run(ctx, cfg.n_angles, cfg.n_rows, n, 100000, max(cfg.kkt_eps, 1e-6))
        vmat.vmat_destroy(ctx)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        d2h = sum(r[k].nbytes for k in ("k", "lleaf", "rleaf", "y", "p", "p2", "cost", "rho", "iters"))
    t = min(times[1:]) if len(times) > 1 else times[0]
    return {"value": round(n / t, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "s_per_plan": round(t, 3),
            "note": "vmat_create from pinned host arrays (D copied, transposed on the device) "
                    "+ vmat_colgen_run (180 iterations) + results to host + vmat_destroy"}


def _oracle_sample(prob, n_iter):
    import oracle
    t0 = time.perf_counter()
    rec = oracle.colgen(prob, n_iter=n_iter)
    return time.perf_counter() - t0, rec


def _omp_threads(n):
    """Thread count of the oracle's OpenMP regions started from this thread."""
    import ctypes.util
    name = ctypes.util.find_library("gomp") or "libgomp.so.1"
    ctypes.CDLL(name).omp_set_num_threads(int(n))


def _oracle_operator_rates(prob, seed=5, n_master_cols=None, master_iters=3):
    """Per-operator rates of the FP64 oracle on one workload: dose z = D^T x,
    price g = D F'(z), and one projected-gradient master iteration with half
    the beams holding a seeded deliverable aperture."""
    import oracle
    from paper_1005_4396_b300 import inputs
    cfg = prob.cfg
    x = inputs.rng.uniform(seed, prob.n_beamlets)
    t0 = time.perf_counter()
    z = oracle.dose(prob, x)
    t_dose = time.perf_counter() - t0
    f = oracle.voxel_dcost(z, prob.struct_id, prob.T, prob.alpha, prob.beta)
    t0 = time.perf_counter()
    oracle.price(prob, f)
    t_price = time.perf_counter() - t0
    R = cfg.n_rows
    ll, rr = inputs.random_apertures(seed, cfg)
    ncol = n_master_cols or cfg.n_angles // 2
    beams = np.arange(0, cfg.n_angles, max(1, cfg.n_angles // ncol))[:ncol]
    M = np.array([oracle.aperture_dose(prob, k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
                  for k in beams])
    y0 = np.zeros(cfg.n_angles)
    t0 = time.perf_counter()
    res = oracle.master(M, beams, prob.theta_deg, prob.struct_id, prob.T, prob.alpha, prob.beta,
                        cfg.gamma, cfg.cyclic, y0, eps=0.0, max_iter=master_iters)
    t_master = (time.perf_counter() - t0) / max(res["iters"], 1)
    return {"dose_per_s": round(1 / t_dose, 4), "price_per_s": round(1 / t_price, 4),
            "master_iter_per_s": round(1 / t_master, 4), "master_columns": int(ncol)}


def run_cpu_baseline(prob, args, extra=None):
    """The FP64 oracle on the host cores: the headline sample (first
    --cpu-iters iterations of the timed plan, all threads), then per-operator
    rates at all threads and at one thread on this workload (and on any
    `extra` workloads), and the whole tiny plan at both thread counts."""
    import oracle
    from paper_1005_4396_b300 import inputs
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    _omp_threads(cores)
    n = args.cpu_iters
    dt, _ = _oracle_sample(prob, n)
    out = {"value": round(n / dt, 4), "unit": UNIT, "cores": int(cores), "kind": "oracle",
           "sample": f"first {n} column-generation iterations of the same plan (FP64 oracle, "
                     f"OpenMP over {cores} threads, {dt:.1f} s); early iterations have the "
                     f"fewest columns, so this overstates the oracle's whole-plan rate"}
    if args.quick:
        return out
    tiny = inputs.make_problem(inputs.tiny_config())
    rates = {}
    for threads in (cores, 1):
        _omp_threads(threads)
        key = f"threads_{threads}"
        rates[key] = {}
        t0 = time.perf_counter()
        oracle.colgen(tiny)
        rates[key]["tiny_whole_plan"] = {"s": round(time.perf_counter() - t0, 3),
                                         "cg_iters_per_s": round(tiny.cfg.iterations / (time.perf_counter() - t0), 3)}
        for name, p in [(prob.cfg.name, prob)] + list((extra or {}).items()):
            rates[key][name] = _oracle_operator_rates(p)
    _omp_threads(cores)
    out["operator_rates"] = rates
    out["operator_note"] = ("dose: z = D^T x (serial scatter, the same at every thread count); price: "
                            "g = D F'(z) over all beamlets; master: one projected-gradient iteration "
                            "(two FP64 passes over the columns + exact line search) with half the beams "
                            "holding an aperture; tiny_whole_plan: 36 iterations at KKT 1e-8")
    return out


# ---------------------------------------------------------------- batched plans
def run_batched(args):
    """The batched workload alone (see run_batched_leg), as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    out = run_batched_leg(args)
    print(json.dumps(out), flush=True)


def run_batched_leg(args):
    """Sixteen independent plans of uneven size (seeds 10-25: 90-180 beams,
    40x40 or 60x40 MLC, prostate- or head-and-neck-like, 0.4-2.2 M voxels):
    FP16-D plans in one tuned batch (per-plan SM budgets, plans side by side, one CUDA graph
    launch) against the plain FP32 single-plan loop on the same GPU."""
    import torch
    from paper_1005_4396_b300 import inputs, vmat
    cfgs = inputs.batch_configs(scale=args.batch_scale)
    kkt = 1e-6
    plans16, probs, fp32 = [], [], []
    t_setup = time.perf_counter()
    for c in cfgs:
        prob = inputs.make_problem(c)
        # plain FP32 single-plan loop: whole plan on the whole GPU
        with vmat.Plan(prob, val_f32=True) as p32:
            p32.set_master_method(args.master)
            p32.colgen_run(kkt_tol=kkt)  # warm-up
            p32.reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            r32 = p32.colgen_run(kkt_tol=kkt)
            b.record()
            torch.cuda.synchronize()
            fp32.append(a.elapsed_time(b) / 1e3)
        p16 = vmat.Plan(prob, dtype="f16", val_f32=True)
        p16.set_master_method(args.master)
        plans16.append(p16)
        probs.append(prob if len(probs) < 3 else None)  # keep a few for the dose check
        del prob
    t_setup = time.perf_counter() - t_setup
    batch = vmat.Batch(plans16)
    share, trial = batch.tune(trial_iters=20, kkt_tol=kkt)
    batch.run(kkt_tol=kkt)  # warm-up replay
    outs, plan_ms, total_ms = batch.run(kkt_tol=kkt)
    errs = []
    for prob, plan, out in zip(probs, plans16, outs):
        if prob is None:
            continue
        z = plan.plan_dose().cpu().numpy()
        z64 = _dose64(prob, _fluence64(prob.cfg, out["lleaf"], out["rleaf"], out["y"]))
        errs.append(float(np.abs(z - z64).max() / prob.T.max() * 100))
    n = len(plans16)
    iters = sum(c.n_angles for c in cfgs)
    out = {"metric": "plans/s (FP16-D batched, one graph launch) vs FP32 single-plan loop",
           "master_method": args.master,
           "value": round(n / (total_ms / 1e3), 4), "unit": "plans/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": "f16-D, f32 accumulate", "data": "synthetic",
           "config": {"workload": f"{n} plans, seeds 10-25, grid voxels "
                                  f"{min(c.n_vox for c in cfgs)}-{max(c.n_vox for c in cfgs)}, "
                                  f"beams 90-180, MLC 40x40/60x40, scale {args.batch_scale}",
                      "sm_share": share, "tuner_trial_ms": trial},
           "batched_s": round(total_ms / 1e3, 3),
           "per_plan_wall_s": [round(v / 1e3, 3) for v in plan_ms],
           "fp32_single_plan_loop": {"plans_per_s": round(n / sum(fp32), 4),
                                     "per_plan_s": [round(v, 3) for v in fp32]},
           "cg_iters_per_s_batched": round(iters / (total_ms / 1e3), 2),
           "max_dose_err_pct_rx_sampled": errs,
           "setup_s": round(t_setup, 1)}
    batch.close()
    for p in plans16:
        p.close()
    return out


def run_autograd(args):
    """Differentiable dose + cost on the prostate phantom: 32 fluence vectors
    per call (U(0,1), 288,000 beamlets) forward + hand-written backward, and
    32 aperture-intensity vectors through random deliverable-shaped apertures;
    throughput in vectors/s with CUDA events, and sampled errors against the
    FP64 gradient and central differences of the FP64 cost (h = 1e-3, 8
    directions normalised to |d|_inf = 1)."""
    import torch
    from paper_1005_4396_b300 import autograd, inputs, vmat
    torch.cuda.set_device(0)
    prob = inputs.make_problem(inputs.prostate_config())
    cfg = prob.cfg

    def ocost(x):
        return _cost64(prob, _dose64(prob, x))[0]

    def ograd(x):
        return _price64(prob, _cost64(prob, _dose64(prob, x))[1])

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    out = {"metric": "differentiable dose+cost: fluence vectors/s (forward + backward, 32 per call)",
           "unit": "vectors/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
           "data": "synthetic", "config": {"workload": _describe(cfg, prob), "batch": 32}}
    with vmat.Plan(prob, val_f32=True) as plan:
        Xh = inputs.fluence_batch(91, prob.n_beamlets, 32).T.copy()
        X = torch.tensor(Xh, device="cuda", requires_grad=True)
        l, r = inputs.random_apertures(92, cfg)
        ld, rd = torch.tensor(l, device="cuda"), torch.tensor(r, device="cuda")
        Yh = inputs.rng.uniform(93, cfg.n_angles * 32).astype(np.float32).reshape(cfg.n_angles, 32)
        Y = torch.tensor(Yh, device="cuda", requires_grad=True)

        def step_x():
            X.grad = None
            autograd.dose_cost(plan, X).sum().backward()

        def step_y():
            Y.grad = None
            autograd.aperture_dose_cost(plan, Y, ld, rd).sum().backward()

        for name, fn in (("fluence", step_x), ("intensity", step_y)):
            for _ in range(max(args.warmup, 3)):
                fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            for _ in range(args.steps):
                fn()
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / args.steps
            out[name] = {"ms_per_call": round(ms, 3), "vectors_per_s": round(32 / (ms / 1e3), 1)}
        out["value"] = out["fluence"]["vectors_per_s"]
        # roofline of the fluence call (dose forward + price backward on row tiles):
        # algorithmic bytes = both tiled forms of D once (4 B index + 8 x 4 B values per
        # union entry) + X read + Z and F' written + F' gathered onto active voxels + G
        # written, 128 B per row each
        info = vmat.vmat_get_info(plan.ctx)
        te = info["tile_entries"]
        Va, B, V = info["n_active"], prob.n_beamlets, prob.n_vox
        byts = (te[0] + te[1]) * (4 + 8 * 4) + 128 * (B + 2 * V + 2 * Va + B)
        gbs = byts / (out["fluence"]["ms_per_call"] / 1e3) / 1e9
        peak, peak_kind = _peaks()
        out["roofline"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(gbs / peak, 4), "peak_kind": f"{peak_kind} copy bandwidth",
                           "bytes_per_call": int(byts), "tile_entries": te,
                           "csr_nnz": prob.nnz,
                           "note": "one fluence call: dose forward and price backward on row tiles of D "
                                   "(8 rows per tile); the gathers of X and F' rows are L2 traffic"}
        # errors on sampled vectors
        step_x()
        gx = X.grad.cpu().numpy()
        x = Xh[:, 5].astype(np.float64)
        out["fluence"]["rel_err_vs_fp64_grad"] = rel(gx[:, 5], ograd(x))
        dirs = inputs.rng.normal(94, 8 * prob.n_beamlets).reshape(8, prob.n_beamlets)
        dirs /= np.abs(dirs).max(axis=1, keepdims=True)
        h = 1e-3
        fd = np.array([(ocost(x + h * d) - ocost(x - h * d)) / (2 * h) for d in dirs])
        out["fluence"]["rel_err_vs_central_differences"] = rel(dirs @ gx[:, 5].astype(np.float64), fd)
        step_y()
        gy = Y.grad.cpu().numpy()
        y = Yh[:, 2].astype(np.float64)
        N, R, C = cfg.n_angles, cfg.n_rows, cfg.n_cols
        xf = _fluence64(cfg, l, r, y)
        openm = _fluence64(cfg, l, r, np.ones(N)).reshape(N, R * C)
        g_or = (openm * ograd(xf).reshape(N, R * C)).sum(axis=1) + \
            cfg.gamma * _dG64(prob.theta_deg, y, cfg.cyclic)
        out["intensity"]["rel_err_vs_fp64_grad"] = rel(gy[:, 2], g_or)
    out["note"] = ("one call = forward dose+cost of 32 vectors and the backward of their sum; "
                   "errors: relative 2-norm on one sampled vector")
    print(json.dumps(out), flush=True)


def run_coarse(args):
    """Coarse voxels for unspecified tissue (Sec. 3): the plan optimised on
    the problem whose tissue voxels are merged in 2x2x2 blocks (volume-
    weighted), against the plan optimised at full resolution; both evaluated
    at full resolution (FP64 NumPy dose of each plan's fluence)."""
    import torch
    from paper_1005_4396_b300 import inputs, vmat
    torch.cuda.set_device(0)
    cfg = _workload(args.workload)
    fine = inputs.make_problem(cfg)
    t0 = time.perf_counter()
    cp = inputs.coarse_tissue(fine)
    t_merge = time.perf_counter() - t0
    kkt = max(cfg.kkt_eps, 1e-6)
    res = {}
    for name, prob in (("full", fine), ("coarse_tissue", cp.prob)):
        with vmat.Plan(prob, val_f32=True) as plan:
            for _ in range(args.warmup):
                plan.reset()
                plan.colgen_run(kkt_tol=kkt)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            plan.reset()
            a.record()
            r = plan.colgen_run(kkt_tol=kkt)
            b.record()
            torch.cuda.synchronize()
            s = a.elapsed_time(b) / 1e3
            info = plan.info
        z = _dose64(fine, _fluence64(cfg, r["lleaf"], r["rleaf"], r["y"]))
        c = _cost64(fine, z)[0]
        Gy = float(np.sum([(r["y"][k2] - r["y"][k]) ** 2 / g for k, (_, _, k2, g) in
                           enumerate(_gaps(fine.theta_deg, cfg.cyclic)) if k2 is not None]))
        res[name] = {"s_per_plan": round(s, 4), "cg_iters_per_s": round(len(r["k"]) / s, 2),
                     "active_voxels": info["n_active"], "nnz": prob.nnz,
                     "master_iters": int(r["iters"].sum()),
                     "full_resolution_cost": c + cfg.gamma * Gy}
    out = {"metric": "CG iters/s with coarse tissue voxels, full-resolution cost of the plan",
           "value": res["coarse_tissue"]["cg_iters_per_s"], "unit": UNIT, "n_gpus": 1,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": _describe(cfg, fine)}, "merge_s": round(t_merge, 2), **res,
           "cost_ratio_coarse_over_full": res["coarse_tissue"]["full_resolution_cost"] /
           res["full"]["full_resolution_cost"]}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- profiling cases
def run_case(args):
    """Small cases sized for an ncu capture (a few GB on the device, inputs
    larger than L2): the prostate phantom cut to 32 slices (V_active 221k,
    nnz 2.2e8).  master: --case-cols seeded apertures (150), one master launch of 30
    projected-gradient iterations.  spmv: dose and price SpMV, twice each."""
    import torch
    from paper_1005_4396_b300 import inputs, vmat
    torch.cuda.set_device(0)
    cfg = inputs.prostate_config(nz=32)
    prob = inputs.make_problem(cfg)
    plan = vmat.Plan(prob, val_f32=True)
    if args.case_ctas:
        vmat.vmat_set_master_budget(plan.ctx, args.case_ctas)
    out = {"case": args.case, "nnz": prob.nnz, "active_voxels": plan.info["n_active"]}
    if args.case == "master":
        R = cfg.n_rows
        ll, rr = inputs.random_apertures(7, cfg)
        beams = np.random.default_rng(7).permutation(cfg.n_angles)[:args.case_cols]
        for k in beams:
            plan.add_column(int(k), ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
        y = np.zeros(cfg.n_angles)
        res = plan.master_step(max_iters=30, kkt_tol=1e-9, y=y)
        out.update(columns=int(args.case_cols), master=res)
    elif args.case == "master-plan":
        # the plan's own apertures: --case-cols column-generation iterations
        # (one master launch each), then one more master launch of exactly 30
        # projected-gradient iterations from the plan's y (tolerance 0 never
        # stops early); its working set is that of the plan's hard masters
        rec = plan.colgen_run(n_iters=args.case_cols, kkt_tol=1e-6)
        res = plan.master_step(max_iters=30, kkt_tol=0.0)
        info = vmat.vmat_get_info(plan.ctx)
        sub = int(rec["col_subtiles"].sum())
        alg = (2 * 30 + 1) * sub * info["subtile_voxels"] * 4 + 8 * info["n_active"]
        out.update(columns=int(args.case_cols), master=res, nonzero_subtiles=sub,
                   nonzero_column_MB=round(sub * info["subtile_voxels"] * 4 / 1e6, 2),
                   algorithmic_bytes_last_launch=alg, master_launch=[info["master_grid"], info["master_block"]])
    elif args.case == "price-live":
        # prices at a plan's F' (live-voxel form): --case-cols column-generation
        # iterations (one live-voxel pricing each), then three stand-alone price
        # calls at F' of the plan dose, F' formed here in NumPy (Eq. 1, FP32)
        plan.colgen_run(n_iters=args.case_cols, kkt_tol=1e-6)
        z = plan.plan_dose().cpu().numpy().astype(np.float64)
        e = z - prob.T[prob.struct_id]
        fp = np.where(e > 0, 2 * prob.beta[prob.struct_id] * e,
                      np.where(e < 0, 2 * prob.alpha[prob.struct_id] * e, 0.0)).astype(np.float32)
        f = torch.as_tensor(fp, device="cuda")
        i0 = vmat.vmat_get_info(plan.ctx)
        for _ in range(3):
            plan.price(f)
        torch.cuda.synchronize()
        i1 = vmat.vmat_get_info(plan.ctx)
        calls = i1["price_calls"][0] - i0["price_calls"][0]
        out.update(columns=int(args.case_cols), live_voxels=int(np.count_nonzero(fp)),
                   live_form_calls=int(calls),
                   live_entries_per_call=int((i1["price_live_entries"] - i0["price_live_entries"]) / max(calls, 1)))
    elif args.case == "spmm32":
        # the differentiable forward's batched products: 32 fluence vectors
        X = torch.rand(prob.n_beamlets, 32, device="cuda")
        for _ in range(2):
            Z, Fp, _ = plan.dose_batch32(X)
            plan.price_batch32(Fp)
        torch.cuda.synchronize()
        out.update(n_beamlets=prob.n_beamlets)
    else:
        x = torch.rand(prob.n_beamlets, device="cuda")
        f = torch.randn(prob.n_vox, device="cuda")
        for _ in range(2):
            plan.dose(x)
            plan.price(f)
        torch.cuda.synchronize()
    plan.close()
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    from paper_1005_4396_b300 import inputs
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cfg = _workload(args.workload)
    prob = inputs.make_problem(cfg)
    n = args.cpu_iters
    for _ in range(args.warmup):
        _oracle_sample(prob, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_sample(prob, n)
    dt = time.perf_counter() - t0
    value = args.steps * n / dt
    sample = (f"each step: the first {n} column-generation iterations of the plan "
              f"(FP64 oracle, {cores} threads)")
    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt / args.steps * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": _describe(cfg, prob)}, "impl": "reference",
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": int(cores),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="prostate", choices=["prostate", "tiny", "headneck"])
    ap.add_argument("--cpu-iters", type=int, default=16)
    ap.add_argument("--quick", action="store_true", help="skip variants, e2e and CPU baseline")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the head-and-neck and batched workloads of the default run")
    ap.add_argument("--case", default=None, choices=["master", "master-plan", "spmv", "spmm32", "price-live"],
                    help="small case for an ncu capture instead of the benchmark")
    ap.add_argument("--case-cols", type=int, default=150,
                    help="columns of the --case master launch (150: ~133 MB, above L2)")
    ap.add_argument("--case-ctas", type=int, default=0,
                    help="CTA budget of the --case master kernel (73 on the half-depth phantom "
                         "gives the full prostate's 8 voxels per thread and 384-thread CTAs)")
    ap.add_argument("--batched", action="store_true",
                    help="the sixteen-plan batch (FP16-D, graph) against the FP32 single-plan loop")
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--master", default="pg", choices=["pg", "newton"],
                    help="master method of the timed plan (pg: the paper's gradient projection)")
    ap.add_argument("--coarse", action="store_true",
                    help="coarse tissue voxels (2x2x2) against full resolution, evaluated at full resolution")
    ap.add_argument("--autograd", action="store_true",
                    help="the differentiable dose+cost (32 vectors per call) on the prostate phantom")
    ap.add_argument("--study", default=None, choices=["pricing"],
                    help="pricing: literal vs exact reduced-cost pricing on a ring and on a path of beams")
    args = ap.parse_args()
    if args.study:
        run_study(args)
        return
    if args.autograd:
        run_autograd(args)
        return
    if args.coarse:
        run_coarse(args)
        return
    if args.case:
        run_case(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
