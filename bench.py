#!/usr/bin/env python
"""Benchmark of the batched chemistry solve: cell-steps/s at rtol 1e-4.

Default workload: uneven stiffness, 131072 cells per GPU (half dark, 10%
cloud cells carrying eight aqueous sections on the 232-species multiphase
mechanism, the rest on the 72-species gas mechanism), one 180 s step.  One
bench step = one call of the whole hot path (rate constants, BDF + Newton +
sparse LU for every cell over the outer step): both mechanisms in one
camp_solve_batch call (a persistent grid per mechanism, autotuned launch
shape), captured once in a CUDA graph and replayed, with the inputs resident
in HBM; a fresh copy of the initial state is taken inside every step and L2
is flushed (256 MB write) between timed steps.  The same line carries the
plain FP64 form (one static launch per mechanism per step), the end-to-end
rate through the host-buffer call, the FP64 oracle on the host cores over a
stratified sample, the error against it with every violating cell
arbitrated, and the roofline of the cost models.  Prints one JSON line
(rank 0).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--workload uneven]
    python bench.py --workload gas72|multiphase232|particles|water|small|serving
    python bench.py --impl reference   # the FP64 CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {"small": 1, "gas72": 2, "multiphase232": 3, "uneven": 4, "serving": 5, "particles": 6,
             "water": 7, "particles10k": 8}
# beyond this many species the dense FP64 oracle (n^2 Jacobian, n^3 LU per
# setup) is out of reach of a bounded CPU sample
ORACLE_MAX_SPECIES = 4096
FP64_PEAK_NOMINAL_GFLOPS = 1250.0  # GB300 dense FP64, nominal
HBM_FALLBACK_GBS = 6800.0          # used only when the measured peaks file is absent
# DRAM bytes (read + write) per cell of one mixed-form solve launch (k_solve;
# k_arrow for particles10k), from one ncu capture of the same kernel on a
# smaller launch of the same workload (uneven: 16384 cells, 14734 + 1650 per
# group; gas72: 4096; multiphase232: 2048; particles: 512; water: 2048;
# particles10k: 19), scaled by the cells of the timed launch.  Valid only for the kernel sources whose digest
# is given: the bench reports null traffic once the kernels have changed.
DRAM_BYTES_PER_CELL = {
    "uneven": {"digest": "7ad162b3d2e196cb", "bytes_per_cell": [14963200 / 14734, 4632832 / 1650]},
    "gas72": {"digest": "7ad162b3d2e196cb", "bytes_per_cell": [4560384 / 4096]},
    "multiphase232": {"digest": "7ad162b3d2e196cb", "bytes_per_cell": [5745152 / 2048]},
    "particles": {"digest": "7ad162b3d2e196cb", "bytes_per_cell": [6214144 / 512]},
    "water": {"digest": "7ad162b3d2e196cb", "bytes_per_cell": [5969408 / 2048]},
    "particles10k": {"digest": "9df31e777d01acd0", "bytes_per_cell": [(11711516416 + 6147372544) / 19]},
}


def args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="camp", choices=["camp", "reference"])
    p.add_argument("--workload", default="uneven", choices=sorted(WORKLOADS))
    p.add_argument("--cells", type=int, default=0, help="override the workload's cell count")
    p.add_argument("--variant", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--cpb", type=int, default=0, help="cells per block (0: library default)")
    p.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--sample", type=int, default=4096, help="uneven: cells of the stratified oracle sample")
    p.add_argument("--requests", type=int, default=2000, help="serving: number of chunk requests")
    p.add_argument("--load", type=float, default=0.8, help="serving: offered load / measured capacity")
    p.add_argument("--ablation", action="store_true",
                   help="uneven: also time one queue on the 232-species superset mechanism")
    return p.parse_args()


# the sources each solve kernel and its device tables are built from (the C
# ABI, server, no-alloc entry point and FMA probe are left out): k_solve
# (cell) and k_arrow (block-arrow)
KERNEL_SOURCES = {
    "cell": ("arrow.h", "cellsolve.cuh", "devmech.h", "kernels.cuh", "launch.h", "launch_impl.cuh",
             "mech.cpp", "mech.hpp", "solve_f32.cu", "solve_f32w.cu", "solve_f64.cu", "solve_f64w.cu"),
    "arrow": ("arrow.cuh", "arrow.h", "cellsolve.cuh", "devmech.h", "launch.h", "mech.cpp", "mech.hpp",
              "solve_arrow.cu"),
}


def kernel_digest(kind="cell"):
    """Digest of one kernel's sources (the DRAM traffic table is tied to it)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2111_07436_gb300", "csrc")
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ----------------------------------------------------------------- error vs oracle
def error_vs_oracle(parts, atol, rtol, truth_cells=128):
    """GPU results against the oracle's on the sampled cells, merged over
    mechanisms.  parts: [(oracle mechanism, y0, env, dt, y_gpu, y_oracle)].
    Relative error over the species above atol in either (the parity rule's
    set), the same over values above 100 atol, the difference in units of the
    solver's tolerance rtol |y| + atol; the parity rule with every violating
    cell sent to the two-tier arbiter (tests/parity.py); and, on a seeded
    subset of each group, the error of both against the true solution (a
    tight oracle run) in the solver's tolerance units."""
    import numpy as np
    from tests import parity
    rels, tols, big_rel, eg_t, eo_t = [], [], [], [], []
    agg = {"cells": 0, "arbitrated": 0, "arbiter_pass_strict": 0, "arbiter_pass": 0, "failed": 0}
    for om, y0, env, dt, g, o in parts:
        d = np.abs(g - o)
        mask = np.maximum(np.abs(g), np.abs(o)) > atol
        rels.append(d[mask] / np.abs(o)[mask])
        big = np.abs(o) > 100 * atol
        big_rel.append(d[big] / np.abs(o)[big])
        tols.append((d / (rtol * np.abs(o) + atol)).ravel())
        rep = parity.arbiter_report(om, y0, env, dt, rtol, atol, g, o)
        agg["cells"] += rep["cells"]
        agg["arbitrated"] += rep["arbitrated"]
        agg["arbiter_pass_strict"] += rep["arbiter_pass_strict"]
        agg["arbiter_pass"] += rep["arbiter_pass"]
        agg["failed"] += len(rep["failed_cells"])
        idx = np.arange(len(g)) if len(g) <= truth_cells else \
            np.sort(np.random.default_rng(5).choice(len(g), truth_cells, replace=False))
        yt = parity.tight_solution(om, y0[idx], env[idx], dt)
        eg_t.append(parity.tol_units(g[idx], yt, rtol, atol))
        eo_t.append(parity.tol_units(o[idx], yt, rtol, atol))
    rel, tol, br = np.concatenate(rels), np.concatenate(tols), np.concatenate(big_rel)
    if rel.size == 0:
        return None
    egt, eot = np.concatenate(eg_t), np.concatenate(eo_t)
    return {"cells": agg["cells"], "max_rel": float(rel.max()), "p99_rel": float(np.percentile(rel, 99)),
            "median_rel": float(np.median(rel)), "values": int(rel.size),
            "max_rel_above_100atol": float(br.max()) if br.size else None,
            "max_in_tol_units": float(tol.max()), "p99_in_tol_units": float(np.percentile(tol, 99)),
            "arbitrated": agg["arbitrated"], "arbitrated_share": agg["arbitrated"] / max(1, agg["cells"]),
            "arbiter_pass_strict": agg["arbiter_pass_strict"], "arbiter_pass": agg["arbiter_pass"],
            "arbiter_failed": agg["failed"], "all_pass": agg["failed"] == 0,
            "vs_truth": {"cells": int(len(egt)), "unit": "max over species of |y - y_true| / (rtol |y_true| + atol)",
                         "gpu_p99": float(np.percentile(egt, 99)), "gpu_max": float(egt.max()),
                         "oracle_p99": float(np.percentile(eot, 99)), "oracle_max": float(eot.max())}}


# ----------------------------------------------------------------- cost models
def cost_models(info, st, lu_bytes, calls=1):
    """Algorithmic work of one solve from its per-cell counters st [C, 5]
    (steps, Newton iterations, setups, error-test failures, order sum):
    FP64 flops and bytes of the per-internal-step cost model
      flops = m F + (q+1)^2 n / 2 + 10 n,
      bytes = 16 (q+1) n + m (24 n + b nnzLU) + rho (2 b nnzLU + 8 R) + 24 n,
    (m Newton iterations and rho setups per step, q the mean order, F the
    per-process forcing count, b the LU element size), and the FP64 flops the
    kernel's own steps count (f evaluations, Newton updates, Nordsieck
    prediction and correction, norms)."""
    import numpy as np
    st = np.asarray(st, dtype=np.float64)
    C = len(st)
    steps, newton, jac, ordsum = st[:, 0].sum(), st[:, 1].sum(), st[:, 2].sum(), st[:, 4].sum()
    s = max(steps, 1.0)
    m, rho, q = newton / s, jac / s, ordsum / s
    n, nnz, R = info.n_species, info.nnz_lu, info.n_rxn
    model_flops = steps * (m * info.model_forcing + (q + 1) ** 2 * n / 2 + 10 * n)
    model_bytes = steps * (16 * (q + 1) * n + m * (24 * n + lu_bytes * nnz) + rho * (2 * lu_bytes * nnz + 8 * R)
                           + 24 * n)
    f_evals = newton + 2 * C * calls  # Newton iterations plus the two of each call's starting step
    counted = f_evals * info.flops_forcing + newton * 8 * n + steps * (q * (q + 1) / 2 + 2 * (q + 1) + 8) * n
    lu = jac * (info.flops_jacobian + info.flops_factor) + newton * info.flops_solve
    return {"steps": steps, "newton": newton, "setups": jac, "mean_order": q, "model_flops": model_flops,
            "model_bytes": model_bytes, "counted_fp64": counted, "lu_flops": lu}


def roofline(models, seconds, peak64, lu_dtype, traffic, kernel, per, bound="alu"):
    """The roofline object of the bench line.  bound "alu" (a cell's working
    set stays on chip): achieved = cost-model FP64 flops / time against the
    measured FP64 FMA rate, with the bytes model against the HBM peak beside
    it.  bound "hbm" (the block-arrow form, whose per-particle data lives in
    device memory): achieved = cost-model bytes / time against the measured
    HBM copy rate, with the FP64 model beside it."""
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    fl = sum(x["model_flops"] for x in models)
    by = sum(x["model_bytes"] for x in models)
    counted = sum(x["counted_fp64"] for x in models)
    lu = sum(x["lu_flops"] for x in models)
    hbm_src = f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6800 GB/s"
    bytes_model = "bytes per internal cell-step 16 (q+1) n + m (24 n + b nnzLU) + rho (2 b nnzLU + 8 R) + 24 n"
    flops_model = "FP64 flops per internal cell-step m F + (q+1)^2 n/2 + 10 n"
    fp64 = {"flops_per_launch": fl, "achieved_gflops": fl / seconds / 1e9, "peak_gflops": peak64,
            "peak_source": "measured FP64 FMA chains on this GPU (camp_probe_fma_rate)",
            "frac": fl / seconds / 1e9 / peak64, "frac_of_nominal": fl / seconds / 1e9 / FP64_PEAK_NOMINAL_GFLOPS,
            "model": flops_model}
    mem = {"bytes_per_launch": by, "achieved_gbs": by / seconds / 1e9, "peak_gbs": hbm, "peak_source": hbm_src,
           "frac": by / seconds / 1e9 / hbm, "model": bytes_model}
    if bound == "hbm":
        out = {"bound": "hbm", "unit": "GB/s", "achieved": mem["achieved_gbs"], "peak": hbm,
               "peak_source": hbm_src, "frac": mem["frac"], "model": bytes_model, "bytes_per_launch": by,
               "fp64_model": fp64}
    else:
        out = {"bound": "alu", "unit": "GFLOP/s (fp64)", "achieved": fp64["achieved_gflops"], "peak": peak64,
               "peak_source": fp64["peak_source"], "frac": fp64["frac"], "frac_of_nominal": fp64["frac_of_nominal"],
               "model": flops_model, "fp64_flops_per_launch": fl, "hbm_model": mem}
    out.update({"traffic": traffic, "traffic_unit": "DRAM bytes (read + write) per launch, from ncu",
                "kernel": kernel, "per": per,
                "fp64_counted": {"flops_per_launch": counted, "achieved": counted / seconds / 1e9,
                                 "frac": counted / seconds / 1e9 / peak64,
                                 "what": "the kernel's own FP64 steps: f evaluations, Newton updates, "
                                         "Nordsieck prediction and correction, norms"},
                "lu_flops_per_launch": lu, "lu_dtype": lu_dtype})
    return out


# ----------------------------------------------------------------- oracle timing
def oracle_sample_rate(groups, sample, dt, rtol, atol, threads):
    """Oracle cell-steps/s over a per-group sample, extrapolated group by
    group (a group's time scales by its cells over its sampled cells).
    Returns (rate, per-group (oracle mechanism, y0, env, y_oracle), seconds)."""
    import oracle
    total, wall, res = 0.0, 0.0, []
    for (mj, y, env), idx in zip(groups, sample):
        om = oracle.Mechanism(json.dumps(mj))
        t = time.perf_counter()
        yo, so, _ = om.solve(y[idx], env[idx], dt, rtol, atol, threads=threads)
        el = time.perf_counter() - t
        wall += el
        total += el * len(y) / max(1, len(idx))
        res.append((om, y[idx], env[idx], yo, so))
    n = sum(len(y) for _, y, _ in groups)
    return n / total, res, wall


def uneven_config(n_cells, groups, cloud_idx, gpus):
    from paper_2111_07436_gb300 import workloads as w
    return {"workload": f"uneven stiffness: {n_cells} cells per GPU, 50% dark, {len(cloud_idx)} "
                        "cloud cells (liquid water 0.1-1 g/m3) on the multiphase-232 mechanism, the rest on "
                        "gas-72, random order, dt 180 s",
            "cells_per_gpu": n_cells, "groups": [int(len(y)) for _, y, _ in groups],
            "species": [len(w.layout(mj).species) for mj, _, _ in groups],
            "dt_s": 180.0, "rtol": 1e-4, "atol_ppb": 1e-5,
            "parallelism": f"replicas x{gpus} (cells split, no collective)",
            "l2": "flushed between timed steps (256 MB write)"}


# ----------------------------------------------------------------- main
def main():
    a = args()
    if a.workload == "uneven":
        return bench_uneven(a)
    if a.workload == "serving" and a.impl == "camp":
        return bench_serving(a)
    return bench_single(a)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def bench_uneven(a):
    """Config 4: 131072 cells of uneven stiffness per GPU; both mechanisms in
    one camp_solve_batch call replayed from a CUDA graph, with the autotuned
    launch shapes; against the plain FP64 form, one static launch per
    mechanism per step."""
    import numpy as np
    from paper_2111_07436_gb300 import replicas, workloads as w
    rank, world, local = _dist()
    n_cells = a.cells or 131072
    dt, rtol, atol = 180.0, 1e-4, 1e-5
    groups, cloud_idx = w.uneven_batch(n_cells, seed=replicas.cell_seed(204, rank))
    config = uneven_config(n_cells, groups, cloud_idx, a.gpus)
    metric = f"cell-steps/s at rtol {rtol:g}"
    threads = os.cpu_count() or 1

    if a.impl == "reference":  # the FP64 oracle on the host cores, rank 0 only
        if rank != 0:
            return
        sample = w.stratified_sample(groups, a.sample)
        vals, wall = [], 0.0
        for _ in range(a.warmup + a.steps):
            v, _, el = oracle_sample_rate(groups, sample, dt, rtol, atol, threads)
            vals.append(v)
            wall = el
        v = statistics.mean(vals[a.warmup:])
        cpu = {"value": v, "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
               "sample": f"stratified {sum(len(s) for s in sample)} of {n_cells} cells (by mechanism and "
                         f"dark/lit, in proportion), each group's time extrapolated to all its cells; "
                         f"{threads} threads, {wall:.1f} s per step"}
        print(json.dumps({"impl": "reference", "metric": metric, "value": v, "unit": "cell-steps/s",
                          "n_gpus": 0, "steps": a.steps, "warmup": a.warmup,
                          "ms_per_step": 1e3 * n_cells / v, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                          "cpu_baseline": cpu,
                          "e2e": {"value": v, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    from paper_2111_07436_gb300 import build, camp
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())
    G = _groups_on_device(groups, dev)
    tuned = []
    for g in G:  # autotune (launch and cell shape) on a 16384-cell sample of each group
        k = min(16384, g["y0"].shape[0])
        tuned.append(g["mech"].autotune(g["y0"][:k].contiguous(), g["env"][:k].contiguous(), dt, rtol,
                                        g["atol"]) + (g["mech"].info.lanes_per_cell,))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream()
    keys = ("mech", "state", "env", "atol", "status", "workspace")

    def step(stream, stats=False):
        for g in G:
            g["state"].copy_(g["y0"])
        camp.solve_batch([dict({k: g[k] for k in keys}, stats=g["stats"] if stats else None) for g in G],
                         dt, rtol, stream=stream)

    for g in G:
        g["stats"] = torch.zeros((g["y0"].shape[0], camp.NSTATS), dtype=torch.int32, device=dev)
    with torch.cuda.stream(side):  # first call creates the fork streams outside capture
        step(side, stats=True)     # and counts the algorithmic work (untimed)
    torch.cuda.synchronize()
    counters = [g["stats"].cpu().numpy() for g in G]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        step(side)
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    with ClockSampler(dev.index) as clk:
        for i in range(a.warmup + a.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            if i >= a.warmup:
                times.append((e0, e1))
        torch.cuda.synchronize()
    ms_list = [e0.elapsed_time(e1) for e0, e1 in times]
    if dist:
        dist.barrier()
    _, t_max, value = replicas.aggregate(n_cells * a.steps, sum(ms_list) / 1e3, dist)
    ms = 1e3 * t_max / a.steps
    ok = sum(int((g["status"] == 0).sum().item()) for g in G)
    y_mixed = [g["state"].cpu().numpy() for g in G]

    # plain FP64: one static launch per mechanism per step
    plain = None
    y_plain = None
    if not a.no_plain:
        pt = []
        for i in range(1 + max(1, a.steps // 2)):
            flush.zero_()
            for g in G:
                g["state"].copy_(g["y0"])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for g in G:
                g["mech"].solve(g["state"], g["env"], dt, rtol, g["atol"], status=g["status"],
                                variant=camp.VARIANT_FP64, persistent=False, stream=stream)
            e1.record(stream)
            pt.append((e0, e1))
        torch.cuda.synchronize()
        pms = sum(e0.elapsed_time(e1) for e0, e1 in pt[1:]) / (len(pt) - 1)
        y_plain = [g["state"].cpu().numpy() for g in G]
        plain = {"value": n_cells / (pms / 1e3), "ms_per_step": pms,
                 "form": "fp64, one static launch per mechanism per step",
                 "ok_cells": sum(int((g["status"] == 0).sum().item()) for g in G)}

    # the heavier group's kernel alone: its launch duration on its stream
    gi = int(np.argmax([c[:, 1].sum() for c in counters]))
    g = G[gi]
    kt = []
    for i in range(4):
        flush.zero_()
        g["state"].copy_(g["y0"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g["mech"].solve(g["state"], g["env"], dt, rtol, g["atol"], status=g["status"],
                        variant=camp.VARIANT_MIXED, persistent=True, workspace=g["workspace"], stream=stream)
        e1.record(stream)
        kt.append((e0, e1))
    torch.cuda.synchronize()
    k_ms = sum(e0.elapsed_time(e1) for e0, e1 in kt[1:]) / (len(kt) - 1)

    # ablation: every cell in one persistent queue on the superset (232-species)
    # mechanism, the gas-only cells with dry sections (L = 0: their aqueous
    # species frozen)
    ablation = None
    if a.ablation:
        (mg, yg_, eg_), (mm, ym_, em_) = groups
        n_sec = 3 * w.layout(mm).n_sections
        ys = np.concatenate([np.concatenate([yg_, np.zeros((len(yg_), ym_.shape[1] - yg_.shape[1]))], axis=1), ym_])
        dry = np.zeros((len(eg_), n_sec))
        dry[:, 0::3], dry[:, 1::3] = w.SECTION_RADII[None, :], 1e6
        es = np.concatenate([np.concatenate([eg_, dry], axis=1), em_])
        gsup = G[1]["mech"]
        ys_d, es_d = torch.tensor(ys, device=dev), torch.tensor(es, device=dev)
        st_s = torch.empty(len(ys), dtype=torch.int32, device=dev)
        at = []
        for i in range(3):
            flush.zero_()
            yw = ys_d.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gsup.solve(yw, es_d, dt, rtol, G[1]["atol"], status=st_s, variant=camp.VARIANT_MIXED, persistent=True,
                       workspace=G[1]["workspace"], stream=stream)
            e1.record(stream)
            at.append((e0, e1))
        torch.cuda.synchronize()
        ams = min(e0.elapsed_time(e1) for e0, e1 in at[1:])
        ablation = {"superset_single_queue": {"value": n_cells / (ams / 1e3), "ms_per_step": ams,
                                              "ok_cells": int((st_s == 0).sum().item()),
                                              "form": "mixed persistent, all cells on the 232-species mechanism"}}
        del ys_d, es_d

    # end to end: the host-buffer call (pinned host arrays, copies timed)
    e2e = None
    if not a.no_e2e:
        H = []
        for (mj, y, env), g in zip(groups, G):
            H.append({"mech": g["mech"], "y0": y, "state": torch.empty(y.shape, dtype=torch.float64).pin_memory(),
                      "env": torch.from_numpy(env).pin_memory(), "atol": np.array([atol]),
                      "status": torch.zeros(len(y), dtype=torch.int32).pin_memory()})
        e2e_t = []
        for i in range(a.warmup + a.steps):
            for h in H:
                h["state"].copy_(torch.from_numpy(h["y0"]))
            t = time.perf_counter()
            camp.solve_batch_host([{k: h[k] for k in ("mech", "state", "env", "atol", "status")} for h in H],
                                  dt, rtol, stream=stream)
            if i >= a.warmup:
                e2e_t.append(time.perf_counter() - t)
        _, _, e2e_value = replicas.aggregate(n_cells * a.steps, sum(e2e_t), dist)
        e2e = {"value": e2e_value, "unit": "cell-steps/s",
               "h2d_bytes_per_step": int(sum(h["state"].numel() * 8 + h["env"].numel() * 8 + 8 for h in H)),
               "d2h_bytes_per_step": int(sum(h["state"].numel() * 8 + h["status"].numel() * 4 for h in H)),
               "call": "camp_solve_batch_host (pinned host arrays, synchronous)",
               "ok_cells": sum(int((h["status"] == 0).sum().item()) for h in H)}

    cpu = err = None
    if rank == 0 and world == 1 and not a.no_cpu:
        sample = w.stratified_sample(groups, a.sample)
        v, res, wall = oracle_sample_rate(groups, sample, dt, rtol, atol, threads)
        cpu = {"value": v, "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
               "sample": f"stratified {sum(len(s) for s in sample)} of {n_cells} cells (by mechanism and "
                         f"dark/lit, in proportion), each group's time extrapolated to all its cells; "
                         f"{threads} threads, {wall:.1f} s",
               "ok_cells": int(sum((r[4] == 0).sum() for r in res))}
        err = {"rule": "species above atol, relative to the FP64 oracle; violating cells arbitrated against a "
                       "tight oracle run (rtol 1e-10), strict per-species tier then error-control tier"}
        for name, ys in (("mixed", y_mixed), ("fp64", y_plain)):
            if ys is None:
                continue
            parts = [(om, y0s, envs, dt, ys[gi2][idx], yo)
                     for gi2, ((om, y0s, envs, yo, so), idx) in enumerate(zip(res, sample))]
            err[name] = error_vs_oracle(parts, atol, rtol)

    if rank != 0:
        return
    peak64 = camp.probe_fma_rate(True)
    models = [cost_models(g["mech"].info, c, 4) for g, c in zip(G, counters)]
    digest = kernel_digest()
    tr = DRAM_BYTES_PER_CELL.get("uneven")
    traffic = (sum(tr["bytes_per_cell"][i] * len(y) for i, (_, y, _) in enumerate(groups))
               if tr and tr["digest"] == digest else None)
    roof = roofline(models, ms / 1e3, peak64, "f32", traffic, "k_solve (two launches, one per mechanism)",
                    "step: both launches of one camp_solve_batch, CUDA events on the replay stream")
    km = cost_models(G[gi]["mech"].info, counters[gi], 4)
    roof["dominant_kernel"] = {
        "kernel": f"k_solve of the {config['species'][gi]}-species group, launched alone",
        "ms_per_launch": k_ms, "fp64_model_gflops": km["model_flops"] / k_ms / 1e6,
        "frac": km["model_flops"] / k_ms / 1e6 / peak64,
        "hbm_model_frac": km["model_bytes"] / k_ms / 1e6 / roof["hbm_model"]["peak_gbs"]}
    work = {"bdf_steps": sum(x["steps"] for x in models), "newton_iters": sum(x["newton"] for x in models),
            "lu_setups": sum(x["setups"] for x in models),
            "per_group": [{k: x[k] for k in ("steps", "newton", "setups", "mean_order")} for x in models]}
    out = {"metric": metric, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 state / f32 J+LU",
           "data": "synthetic (seeded generator shaped like the paper's gas mechanism and sectional aerosol)",
           "config": config, "form": "mixed persistent, camp_solve_batch replayed from a CUDA graph",
           "autotuned": [{"cells_per_block": t[0], "persistent": t[1], "ms": t[2], "lanes_per_cell": t[3]}
                         for t in tuned],
           "ok_cells": ok, "gpu_launches": 2 * a.steps, "work": work,
           "plain_fp64": plain, "mixed_over_plain": (value / world / plain["value"]) if plain else None,
           "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "error_vs_oracle": err,
           "kernel_digest": digest, "clocks": clk.summary()}
    if ablation:
        out["ablation"] = ablation
    print(json.dumps(out))


def bench_single(a):
    """One mechanism's workload (gas72, multiphase232, particles, water,
    small): the solve of every cell over every outer step of the workload."""
    from paper_2111_07436_gb300 import replicas, workloads as w
    rank, world, local = _dist()
    wl = w.workload(WORKLOADS[a.workload])
    if a.cells:
        wl.n_cells = a.cells
    metric = f"cell-steps/s at rtol {wl.rtol:g}"
    config = {"workload": f"{wl.mech['name']} x {wl.n_cells} cells, dt {wl.dt:g} s",
              "cells_per_gpu": wl.n_cells, "species": len(w.layout(wl.mech).species),
              "dt_s": wl.dt, "outer_steps": wl.n_outer,
              "rtol": wl.rtol, "atol_ppb": wl.atol,
              "parallelism": f"replicas x{a.gpus} (cells split, no collective)",
              "l2": "flushed between timed steps (256 MB write)"}
    wl.cell_seed = replicas.cell_seed(wl.cell_seed, rank)  # each replica solves its own cells
    threads = os.cpu_count() or 1

    def oracle_rate(seconds):
        import numpy as np
        import oracle
        om = oracle.Mechanism(wl.json())
        y0, env = wl.inputs()
        probe = min(wl.n_cells, 8 * threads)
        t = time.perf_counter()
        om.solve(y0[:probe], env[:probe], wl.dt, wl.rtol, wl.atol, threads=threads)
        per_cell = (time.perf_counter() - t) / probe
        n = int(min(wl.n_cells, max(probe, seconds / max(per_cell, 1e-9))))
        idx = np.sort(np.random.default_rng(17).choice(wl.n_cells, n, replace=False))
        t = time.perf_counter()
        y_o, st, _ = om.solve(y0[idx], env[idx], wl.dt, wl.rtol, wl.atol, threads=threads)
        el = time.perf_counter() - t
        cpu = {"value": n * wl.n_outer / el, "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
               "sample": f"{n} of {wl.n_cells} cells (seeded random), {wl.n_outer} outer step(s), "
                         f"{threads} threads, {el:.1f} s", "ok_cells": int((st == 0).sum())}
        return cpu, (om, idx, y0, env, y_o, st)

    n_species = len(w.layout(wl.mech).species)
    oracle_off = n_species > ORACLE_MAX_SPECIES and \
        f"the dense FP64 oracle needs a {n_species}^2 Jacobian ({8 * n_species ** 2 / 1e9:.0f} GB) per cell"
    if a.impl == "reference":
        if rank != 0:
            return
        if oracle_off:
            print(json.dumps({"impl": "reference", "unavailable": oracle_off}))
            return
        cpu, _ = oracle_rate(a.cpu_seconds)
        vals = [oracle_rate(a.cpu_seconds / 2)[0]["value"] for _ in range(a.warmup + a.steps)]
        v = statistics.mean(vals[a.warmup:])
        cpu["value"] = v
        print(json.dumps({"impl": "reference", "metric": metric, "value": v, "unit": "cell-steps/s",
                          "n_gpus": 0, "steps": a.steps, "warmup": a.warmup,
                          "ms_per_step": 1e3 * wl.n_cells * wl.n_outer / v, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": config, "cpu_baseline": cpu,
                          "e2e": {"value": v, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    from paper_2111_07436_gb300 import build, camp
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())
    gm = camp.Mechanism(wl.json())
    y0, env = wl.inputs()
    C = wl.n_cells
    y0_d = torch.tensor(y0, device=dev)
    env_d = torch.tensor(env, device=dev)
    state = torch.empty_like(y0_d)
    status = torch.empty(C, dtype=torch.int32, device=dev)
    atol = torch.full((1,), wl.atol, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    variant = camp.VARIANT_MIXED if a.variant == "mixed" else camp.VARIANT_FP64
    persistent = variant == camp.VARIANT_MIXED

    def run(var, pers, K, W, stats=None):
        times = []
        for i in range(W + K):
            flush.zero_()
            state.copy_(y0_d)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if wl.n_outer == 1:
                gm.solve(state, env_d, wl.dt, wl.rtol, atol, status=status, variant=var, persistent=pers,
                         cells_per_block=a.cpb, stats=stats if i == 0 else None, stream=stream)
            else:  # one bench step = every outer step of the workload, in one launch
                gm.solve_sequence(state, env_d, wl.dt, wl.n_outer, wl.rtol, atol, status=status, variant=var,
                                  persistent=pers, stats=stats if i == 0 else None, stream=stream)
            e1.record(stream)
            if i >= W:
                times.append((e0, e1))
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in times]

    # algorithmic work from one instrumented (untimed) solve of every outer step
    stats = torch.zeros((C, camp.NSTATS), dtype=torch.int32, device=dev)
    state.copy_(y0_d)
    gm.solve_sequence(state, env_d, wl.dt, wl.n_outer, wl.rtol, atol, status=status, variant=variant,
                      persistent=persistent, stats=stats, stream=stream)
    torch.cuda.synchronize()
    counters = stats.cpu().numpy()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        times = run(variant, persistent, a.steps, a.warmup)
    ok = int((status.cpu().numpy() == 0).sum())
    y_main = state.cpu().numpy()  # this form's result of the last timed step
    if dist:
        dist.barrier()
    _, t_max, value = replicas.aggregate(C * wl.n_outer * a.steps, sum(times) / 1e3, dist)
    ms = 1e3 * t_max / a.steps

    plain = y_plain = None
    if not a.no_plain and variant == camp.VARIANT_MIXED:
        pt = run(camp.VARIANT_FP64, False, max(1, a.steps // 2), 1)
        y_plain = state.cpu().numpy()
        pms = sum(pt) / len(pt)
        plain = {"value": C * wl.n_outer / (pms / 1e3), "ms_per_step": pms, "form": "fp64 static grid"}

    e2e = None
    if not a.no_e2e:
        y_h = torch.empty((C, gm.n), dtype=torch.float64).pin_memory()
        e_h = torch.tensor(env, dtype=torch.float64).pin_memory()
        st_h = None
        e2e_t = []
        for i in range(a.warmup + a.steps):
            y_h.copy_(torch.from_numpy(y0))
            torch.cuda.synchronize()
            t = time.perf_counter()
            for _ in range(wl.n_outer):
                st_h = gm.solve_host(y_h, e_h, wl.dt, wl.rtol, wl.atol, variant=variant, persistent=persistent,
                                     cells_per_block=a.cpb)
            if i >= a.warmup:
                e2e_t.append(time.perf_counter() - t)
        _, _, e2e_value = replicas.aggregate(C * wl.n_outer * a.steps, sum(e2e_t), dist)
        e2e = {"value": e2e_value, "unit": "cell-steps/s",
               "h2d_bytes_per_step": int(wl.n_outer * (y_h.numel() * 8 + e_h.numel() * 8 + 8)),
               "d2h_bytes_per_step": int(wl.n_outer * (y_h.numel() * 8 + C * 4)),
               "call": "camp_solve_host (pinned host arrays, synchronous)", "ok_cells": int((st_h == 0).sum())}

    cpu = err = None
    if oracle_off:
        cpu = {"value": None, "unit": "cell-steps/s", "kind": "oracle", "unavailable": oracle_off}
    elif rank == 0 and world == 1 and not a.no_cpu:
        cpu, (om, idx, y0s, envs, y_o, st_o) = oracle_rate(a.cpu_seconds)
        if wl.n_outer == 1:  # the oracle's sample covers one outer step
            okc = st_o == 0
            err = {"rule": "species above atol, relative to the FP64 oracle; violating cells arbitrated against a "
                           "tight oracle run (rtol 1e-10), strict per-species tier then error-control tier"}
            for name, ys in ((a.variant, y_main), ("fp64", y_plain)):
                if ys is None or (name == "fp64" and a.variant == "fp64" and ys is y_plain):
                    continue
                err[name] = error_vs_oracle([(om, y0s[idx][okc], envs[idx][okc], wl.dt, ys[idx][okc],
                                              y_o[okc])], wl.atol, wl.rtol)

    if rank != 0:
        return
    peak64 = camp.probe_fma_rate(True)
    lu_b = 4 if variant == camp.VARIANT_MIXED else 8
    models = [cost_models(gm.info, counters, lu_b, wl.n_outer)]
    arrow = bool(gm.info.block_arrow)
    digest = kernel_digest("arrow" if arrow else "cell")
    tr = DRAM_BYTES_PER_CELL.get(a.workload)
    traffic = tr["bytes_per_cell"][0] * C if tr and tr["digest"] == digest and variant == camp.VARIANT_MIXED else None
    roof = roofline(models, ms / 1e3, peak64, "f32" if lu_b == 4 else "f64", traffic,
                    "k_arrow" if arrow else "k_solve",
                    "step (one launch per outer step), CUDA events on the launch stream",
                    bound="hbm" if arrow else "alu")
    out = {"metric": metric, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 state / f32 J+LU" if variant == camp.VARIANT_MIXED else "f64",
           "data": "synthetic (seeded generator shaped like the paper's mechanisms)",
           "config": config, "form": f"{a.variant} {'persistent' if persistent else 'static'}",
           "ok_cells": ok, "gpu_launches": a.steps,
           "us_per_outer_step": 1e3 * ms / wl.n_outer,
           "work": {k: models[0][k] for k in ("steps", "newton", "setups", "mean_order")},
           "plain_fp64": plain, "mixed_over_plain": (value / world / plain["value"]) if plain else None,
           "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "error_vs_oracle": err,
           "kernel_digest": digest, "clocks": clk.summary()}
    print(json.dumps(out))


def _groups_on_device(groups, dev):
    import torch
    from paper_2111_07436_gb300 import camp
    out = []
    for mj, y, env in groups:
        gm = camp.Mechanism(json.dumps(mj))
        out.append({"mech": gm, "y0": torch.tensor(y, device=dev), "env": torch.tensor(env, device=dev),
                    "state": torch.empty(y.shape, dtype=torch.float64, device=dev),
                    "status": torch.empty(len(y), dtype=torch.int32, device=dev),
                    "atol": torch.full((1,), 1e-5, dtype=torch.float64, device=dev),
                    "workspace": camp.workspace(dev)})
    return out


def bench_serving(a):
    """A Poisson stream of chunk requests (256..65536 cells, 70% gas-72 / 30%
    multiphase-232, dt 60..600 s) through the continuous-batching server
    under an 80 GB device budget.  Reports p50/p99 latency (arrival to
    result on the host) and sustained cell-steps/s, mixed and plain FP64."""
    import numpy as np
    import torch
    from paper_2111_07436_gb300 import build, camp, workloads as w
    build.build()
    torch.cuda.set_device(0)
    reqs = w.serving_requests(a.requests)
    mechs = {"gas72": w.large_gas_mechanism(), "multiphase232": w.multiphase_mechanism()}
    gms = {k: camp.Mechanism(json.dumps(v)) for k, v in mechs.items()}
    RING = 4 * 65536
    pools = {}
    for k, mj in mechs.items():  # pinned input pools; requests take disjoint ring regions
        y, env = w.cells(mj, RING, seed=300 + len(k))
        pools[k] = {"y0": y, "y0t": torch.from_numpy(y), "state": torch.from_numpy(y.copy()).pin_memory(),
                    "env": torch.from_numpy(env).pin_memory(),
                    "status": torch.zeros(RING, dtype=torch.int32).pin_memory(), "head": 0, "busy": []}

    def region(k, n):
        p = pools[k]
        start = p["head"] if p["head"] + n <= RING else 0
        for (s0, s1) in p["busy"]:
            if start < s1 and s0 < start + n:
                return None
        p["head"] = start + n
        p["busy"].append((start, start + n))
        return start

    def run(variant, rate_cells, n_req):
        srv = camp.Server(hbm_budget_bytes=80 << 30, max_inflight=8)
        rng = np.random.default_rng(205)
        arrivals = np.cumsum(rng.exponential(1.0, n_req)) * (np.mean([r["cells"] for r in reqs[:n_req]]) / rate_cells) \
            if rate_cells else np.zeros(n_req)
        t0 = time.perf_counter()
        live, lat, done_cells = [], [], 0
        bad_cells = [0]
        for p in pools.values():
            p["busy"].clear()
            p["head"] = 0

        def reap(block):
            nonlocal done_cells
            for item in list(live):
                rid, k, s0, n, t_arr = item
                info = srv.wait(rid) if block else srv.poll(rid)
                if info is None:
                    continue
                live.remove(item)
                pools[k]["busy"].remove((s0, s0 + n))
                lat.append(time.perf_counter() - t0 - t_arr)
                done_cells += n
                assert info["rc"] == 0, info
                bad_cells[0] += int((pools[k]["status"][s0:s0 + n] != 0).sum())
                if block:
                    return

        for i, r in enumerate(reqs[:n_req]):
            while time.perf_counter() - t0 < arrivals[i]:
                reap(False)
                time.sleep(5e-5)
            k, n = r["mech"], r["cells"]
            s0 = region(k, n)
            while s0 is None:
                reap(True)
                s0 = region(k, n)
            p = pools[k]
            p["state"][s0:s0 + n].copy_(p["y0t"][s0:s0 + n])  # every request starts from fresh inputs
            rid = srv.submit(gms[k], p["state"][s0:s0 + n], p["env"][s0:s0 + n], r["dt"], 1e-4, 1e-5,
                             p["status"][s0:s0 + n], variant=variant)
            live.append((rid, k, s0, n, arrivals[i]))
        while live:
            reap(True)
        wall = time.perf_counter() - t0
        srv.close()
        lat = np.array(lat)
        return {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "cell_steps_per_s": done_cells / wall, "wall_s": wall, "requests": n_req,
                "cells": done_cells, "failed_cells": bad_cells[0]}

    def run_host_model(variant, resident, n_sets=8, cells=16384, steps=8):
        """A host model with n_sets domains of `cells` gas-72 cells, each
        stepped `steps` times (dt 180 s, the temperature drifting a little
        every step), all domains of a step submitted together: as resident
        cell sets (only env crosses the bus) or as ordinary chunks (state in
        and out every step)."""
        srv = camp.Server(hbm_budget_bytes=80 << 30, max_inflight=8)
        mj, gm = mechs["gas72"], gms["gas72"]
        doms = []
        for d in range(n_sets):
            y, env = w.cells(mj, cells, seed=400 + d)
            envs = [torch.from_numpy(env + np.array([1.0 * k] + [0.0] * (env.shape[1] - 1))).pin_memory()
                    for k in range(steps)]
            dom = {"envs": envs, "status": torch.zeros(cells, dtype=torch.int32).pin_memory()}
            if resident:
                dom["res"] = srv.resident(gm, y)
            else:
                dom["state"] = torch.from_numpy(y.copy()).pin_memory()
            doms.append(dom)
        lat = []
        t0 = time.perf_counter()
        for k in range(steps):
            rids = []
            for dom in doms:
                if resident:
                    rids.append(dom["res"].step(dom["envs"][k], 180.0, 1e-4, 1e-5, status=dom["status"],
                                                variant=variant))
                else:
                    rids.append(srv.submit(gm, dom["state"], dom["envs"][k], 180.0, 1e-4, 1e-5, dom["status"],
                                           variant=variant))
            for rid in rids:
                info = srv.wait(rid)
                assert info["rc"] == 0, info
                lat.append(info["t_done"] - info["t_submit"])
        wall = time.perf_counter() - t0
        bad = sum(int((dom["status"] != 0).sum()) for dom in doms)
        if resident:
            for dom in doms:
                dom["res"].close()
        srv.close()
        lat = np.array(lat)
        return {"cell_steps_per_s": n_sets * cells * steps / wall, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "domains": n_sets, "cells_per_domain": cells,
                "steps": steps, "bus_bytes_per_step": n_sets * cells * (8 * gms["gas72"].n_env +
                                                                      (4 if resident else 16 * gms["gas72"].n + 4)),
                "failed_cells": bad}

    host_model = {"resident": run_host_model(camp.VARIANT_MIXED, True),
                  "copying": run_host_model(camp.VARIANT_MIXED, False)}

    # capacity of each form on the same first requests, everything at t = 0
    n_cap = min(200, a.requests)
    sat = run(camp.VARIANT_MIXED, 0, n_cap)
    sat_p = run(camp.VARIANT_FP64, 0, n_cap)
    # the Poisson stream at the offered load, for each form, over every request
    mixed = run(camp.VARIANT_MIXED, a.load * sat["cell_steps_per_s"], a.requests)
    plain = run(camp.VARIANT_FP64, a.load * sat_p["cell_steps_per_s"], a.requests)
    print(json.dumps({
        "metric": "cell-steps/s at rtol 1e-4; p50/p99 chunk latency", "value": mixed["cell_steps_per_s"],
        "unit": "cell-steps/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 state / f32 J+LU", "data": "synthetic",
        "config": {"workload": f"serving: Poisson stream of {a.requests} chunks, 256..65536 cells "
                               "(log-uniform), 70% gas-72 / 30% multiphase-232, dt 60..600 s, 80 GB budget, "
                               f"offered load {a.load:g} x measured capacity", "max_inflight": 8},
        "p50_ms": mixed["p50_ms"], "p99_ms": mixed["p99_ms"], "mixed": mixed, "saturation_mixed": sat,
        "plain_fp64": plain, "saturation_plain_fp64": sat_p,
        "capacity_mixed_over_plain": sat["cell_steps_per_s"] / sat_p["cell_steps_per_s"],
        "host_model": host_model}))


if __name__ == "__main__":
    main()
