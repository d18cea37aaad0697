#!/usr/bin/env python
"""Benchmark of the batched chemistry solve: cell-steps/s at rtol 1e-4.

One step = one call of the whole hot path (rate constants, BDF + Newton +
sparse LU for every cell over one outer step) on the full workload, with the
inputs resident in HBM; a fresh copy of the initial state is taken at the
start of every step and L2 is flushed (256 MB write) between timed steps.
Default workload: 16384 cells of the 72-species / 186-process gas mechanism,
one 180 s step.  Prints one JSON line (rank 0).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--workload gas72]
    python bench.py --impl reference   # the FP64 CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
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
             "water": 7}
FP64_PEAK_NOMINAL_GFLOPS = 1250.0  # GB300 dense FP64, nominal
# DRAM bytes (read + write) per cell of one mixed-form k_solve launch, from
# one ncu capture of the same kernel on a smaller launch of the same
# workload (gas-72: 4096 cells, 4.18 MB; multiphase-232: 2048 cells,
# 5.35 MB; particles: 512 cells, 5.91 MB; water: 2048 cells, 5.56 MB): the
# inputs only, so traffic scales with the cells.  To be taken again
# whenever the kernel changes.
DRAM_BYTES_PER_CELL = {"gas72": 4.180480e6 / 4096, "multiphase232": 5.347840e6 / 2048,
                       "particles": 5.905152e6 / 512, "water": 5.557248e6 / 2048}


def args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="camp", choices=["camp", "reference"])
    p.add_argument("--workload", default="gas72", choices=sorted(WORKLOADS))
    p.add_argument("--cells", type=int, default=0, help="override the workload's cell count")
    p.add_argument("--variant", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--cpb", type=int, default=0, help="cells per block (0: library default)")
    p.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--requests", type=int, default=2000, help="serving: number of chunk requests")
    p.add_argument("--load", type=float, default=0.8, help="serving: offered load / measured capacity")
    return p.parse_args()


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


# ----------------------------------------------------------------- CPU oracle
def oracle_rate(wl, seconds, rank_seed=0):
    """Oracle cell-steps/s on this host's cores over a bounded sample of the
    workload's cells (about `seconds` of work)."""
    import numpy as np
    import oracle
    om = oracle.Mechanism(wl.json())
    y0, env = wl.inputs()
    threads = os.cpu_count() or 1
    probe = min(wl.n_cells, 8 * threads)
    t = time.perf_counter()
    om.solve(y0[:probe], env[:probe], wl.dt, wl.rtol, wl.atol, threads=threads)
    per_cell = (time.perf_counter() - t) / probe
    n = int(min(wl.n_cells, max(probe, seconds / max(per_cell, 1e-9))))
    idx = np.random.default_rng(rank_seed + 17).choice(wl.n_cells, n, replace=False)
    t = time.perf_counter()
    y_o, st, _ = om.solve(y0[idx], env[idx], wl.dt, wl.rtol, wl.atol, threads=threads)
    dt = time.perf_counter() - t
    return {"value": n * wl.n_outer / dt, "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{n} of {wl.n_cells} cells (seeded random), {wl.n_outer} outer step(s), "
                      f"{threads} threads, {dt:.1f} s", "ok_cells": int((st == 0).sum()),
            "_result": (idx, y_o, st)}


def error_vs_oracle(y_gpu, sample, rtol, atol):
    """GPU results against the oracle's on the sampled cells: relative error
    over the species above atol in either (the parity rule's set), the same
    over values above 100 atol, and the difference in units of the solver's
    tolerance rtol |y| + atol over all species."""
    import numpy as np
    idx, y_o, st = sample
    ok = st == 0
    g, o = y_gpu[idx][ok], y_o[ok]
    d = np.abs(g - o)
    mask = np.maximum(np.abs(g), np.abs(o)) > atol
    if not mask.any():
        return None
    rel = d[mask] / np.abs(o)[mask]
    big = np.abs(o) > 100 * atol
    tol = d / (rtol * np.abs(o) + atol)
    return {"max_rel": float(rel.max()), "p99_rel": float(np.percentile(rel, 99)),
            "median_rel": float(np.median(rel)), "values": int(rel.size),
            "max_rel_above_100atol": float((d[big] / np.abs(o)[big]).max()) if big.any() else None,
            "max_in_tol_units": float(tol.max()), "p99_in_tol_units": float(np.percentile(tol, 99))}


# ----------------------------------------------------------------- main
def main():
    a = args()
    if a.workload == "uneven" and a.impl == "camp":
        return bench_uneven(a)
    if a.workload == "serving" and a.impl == "camp":
        return bench_serving(a)
    from paper_2111_07436_gb300 import workloads as w
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = w.workload(WORKLOADS[a.workload])
    if a.cells:
        wl.n_cells = a.cells
    metric = f"cell-steps/s at rtol {wl.rtol:g}"
    config = {"workload": f"{wl.mech['name']} x {wl.n_cells} cells, dt {wl.dt:g} s",
              "cells_per_gpu": wl.n_cells, "species": None, "dt_s": wl.dt, "rtol": wl.rtol,
              "atol_ppb": wl.atol, "parallelism": f"replicas x{a.gpus} (cells split, no collective)",
              "l2": "flushed between timed steps (256 MB write)"}

    if a.impl == "reference":
        if rank != 0:
            return
        cpu = oracle_rate(wl, a.cpu_seconds)
        cpu.pop("_result")
        steps_t = []
        for _ in range(a.warmup + a.steps):
            r = oracle_rate(wl, a.cpu_seconds / 2)
            r.pop("_result")
            steps_t.append(r["value"])
        v = statistics.mean(steps_t[a.warmup:])
        cpu["value"] = v
        print(json.dumps({"impl": "reference", "metric": metric, "value": v, "unit": "cell-steps/s",
                          "n_gpus": 0, "steps": a.steps, "warmup": a.warmup,
                          "ms_per_step": 1e3 * wl.n_cells * wl.n_outer / v, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": config, "cpu_baseline": cpu,
                          "e2e": {"value": v, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import numpy as np
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
    config["species"] = gm.n
    from paper_2111_07436_gb300 import replicas
    wl.cell_seed = replicas.cell_seed(wl.cell_seed, rank)  # each replica solves its own cells
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
            for _ in range(wl.n_outer):  # one bench step = every outer step of the workload
                gm.solve(state, env_d, wl.dt, wl.rtol, atol, status=status, variant=var, persistent=pers,
                         cells_per_block=a.cpb, stats=stats if i == 0 else None, stream=stream)
            e1.record(stream)
            if i >= W:
                times.append((e0, e1))
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in times]

    # algorithmic work from one instrumented (untimed) solve
    stats = torch.zeros((C, camp.NSTATS), dtype=torch.int32, device=dev)
    run(variant, persistent, 0, 1, stats=stats)
    st = stats.cpu().numpy().astype(np.float64)
    ok = int((status.cpu().numpy() == 0).sum())
    inf = gm.info
    n = gm.n
    steps, newton, jac, ordsum = st[:, 0].sum(), st[:, 1].sum(), st[:, 2].sum(), st[:, 4].sum()
    qbar = ordsum / max(steps, 1)
    f_evals = newton + 2 * C  # Newton iterations plus the two of the starting step
    fp64 = f_evals * inf.flops_forcing + newton * 8 * n + steps * (qbar * (qbar + 1) / 2 + 2 * (qbar + 1) + 8) * n
    lu = jac * (inf.flops_jacobian + inf.flops_factor) + newton * inf.flops_solve
    if variant == camp.VARIANT_FP64:
        fp64 += lu

    # timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        times = run(variant, persistent, a.steps, a.warmup)
    y_main = state.cpu().numpy()  # this form's result of the last timed step
    if dist:
        dist.barrier()
    _, t_max, value = replicas.aggregate(C * wl.n_outer * a.steps, sum(times) / 1e3, dist)
    ms = 1e3 * t_max / a.steps

    # plain FP64 form, one launch per outer step, for the mixed-vs-plain ratio
    plain = None
    if not a.no_plain and variant == camp.VARIANT_MIXED:
        pt = run(camp.VARIANT_FP64, False, max(1, a.steps // 2), 1)
        y_plain = state.cpu().numpy()
        pms = sum(pt) / len(pt)
        plain = {"value": C * wl.n_outer / (pms / 1e3), "ms_per_step": pms, "form": "fp64 static grid"}

    # end to end through the host-pointer C-ABI call, pinned host buffers
    y_h = torch.empty((C, n), dtype=torch.float64).pin_memory()
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
           "ok_cells": int((st_h == 0).sum())}

    cpu = None
    err = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = oracle_rate(wl, a.cpu_seconds)
        sample = cpu.pop("_result")
        if wl.n_outer == 1:  # the oracle's sample covers one outer step
            err = {"cells": int(len(sample[0])), "rule": "species above atol, relative to the FP64 oracle",
                   a.variant: error_vs_oracle(y_main, sample, wl.rtol, wl.atol)}
            if plain is not None:
                err["fp64"] = error_vs_oracle(y_plain, sample, wl.rtol, wl.atol)

    if rank != 0:
        return
    achieved = fp64 * wl.n_outer / (ms / 1e3) / 1e9  # the counters are one outer step's
    peak64 = camp.probe_fma_rate(True)
    peak32 = camp.probe_fma_rate(False)
    roof = {"bound": "alu", "unit": "GFLOP/s (fp64)", "achieved": achieved,
            "peak": peak64, "peak_source": "measured FP64 FMA chains on this GPU (camp_probe_fma_rate)",
            "peak_nominal": FP64_PEAK_NOMINAL_GFLOPS, "peak_fp32_measured": peak32,
            "frac": achieved / peak64, "frac_of_nominal": achieved / FP64_PEAK_NOMINAL_GFLOPS,
            "traffic": (DRAM_BYTES_PER_CELL[a.workload] * C
                        if variant == camp.VARIANT_MIXED and a.workload in DRAM_BYTES_PER_CELL else None),
            "traffic_unit": "bytes per launch (ncu dram read + write, scaled by cells)",
            "kernel": "k_solve", "fp64_flops_per_launch": fp64, "lu_flops_per_launch": lu,
            "lu_dtype": "f32" if variant == camp.VARIANT_MIXED else "f64"}
    hbm = (y0.nbytes * 2 + env.nbytes + C * 4) / (ms / 1e3) / 1e9
    out = {"metric": metric, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 state / f32 J+LU" if variant == camp.VARIANT_MIXED else "f64",
           "data": "synthetic (seeded generator shaped like the paper's gas mechanism)",
           "config": config, "form": f"{a.variant} {'persistent' if persistent else 'static'}",
           "ok_cells": ok, "gpu_launches": a.steps * wl.n_outer,
           "work": {"bdf_steps": steps, "newton_iters": newton, "lu_setups": jac, "mean_order": qbar,
                    "steps_per_cell": steps / C,
                    "per_s": {k: v * wl.n_outer * world / (ms / 1e3) for k, v in
                              (("bdf_steps", steps), ("newton_iters", newton), ("lu_setups", jac))}},
           "plain_fp64": plain, "mixed_over_plain": (value / world / plain["value"]) if plain else None,
           "roofline": roof, "hbm_io_gbs": hbm, "e2e": e2e, "cpu_baseline": cpu,
           "error_vs_oracle": err, "clocks": clk.summary()}
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


def bench_uneven(a):
    """131072 cells of uneven stiffness (half dark, 10% cloud cells on the
    multiphase mechanism): both mechanisms in one camp_solve_batch call, its
    launches captured once in a CUDA graph and replayed per step, with the
    autotuned cells-per-block; against the plain FP64 form, one static launch
    per mechanism per step."""
    import torch
    from paper_2111_07436_gb300 import build, camp, workloads as w
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n_cells = a.cells or 131072
    groups, cloud_idx = w.uneven_batch(n_cells)
    G = _groups_on_device(groups, dev)
    dt, rtol = 180.0, 1e-4
    tuned = []
    for g in G:  # autotune on a 4096-cell sample of each group
        k = min(4096, g["y0"].shape[0])
        tuned.append(g["mech"].autotune(g["y0"][:k].contiguous(), g["env"][:k].contiguous(), dt, rtol,
                                        g["atol"]))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream()

    def step(stream):
        for g in G:
            g["state"].copy_(g["y0"])
        camp.solve_batch([{k: g[k] for k in ("mech", "state", "env", "atol", "status", "workspace")}
                          for g in G], dt, rtol, stream=stream)

    with torch.cuda.stream(side):  # first call creates the fork streams outside capture
        step(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        step(side)
    torch.cuda.synchronize()
    times = []
    with ClockSampler(0) as clk:
        for i in range(a.warmup + a.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            graph.replay()
            e1.record()
            times.append((e0, e1))
        torch.cuda.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in times[a.warmup:]) / a.steps
    ok = sum(int((g["status"] == 0).sum().item()) for g in G)
    # plain FP64: one static launch per mechanism per step
    pt = []
    for i in range(1 + max(1, a.steps // 2)):
        flush.zero_()
        for g in G:
            g["state"].copy_(g["y0"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for g in G:
            g["mech"].solve(g["state"], g["env"], dt, rtol, g["atol"], status=g["status"],
                            variant=camp.VARIANT_FP64, persistent=False)
        e1.record()
        pt.append((e0, e1))
    torch.cuda.synchronize()
    pms = sum(e0.elapsed_time(e1) for e0, e1 in pt[1:]) / (len(pt) - 1)
    value = n_cells / (ms / 1e3)
    print(json.dumps({
        "metric": f"cell-steps/s at rtol {rtol:g}", "value": value, "unit": "cell-steps/s", "n_gpus": 1,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 state / f32 J+LU", "data": "synthetic",
        "config": {"workload": f"uneven stiffness: {n_cells} cells, 50% dark, {len(cloud_idx)} cloud cells "
                               f"on the 232-species mechanism, the rest on the 72-species one, dt 180 s",
                   "groups": [int(g["y0"].shape[0]) for g in G],
                   "autotuned_cpb_persistent_ms": tuned, "cuda_graph": True,
                   "l2": "flushed between timed steps (256 MB write)"},
        "ok_cells": ok, "gpu_launches": 2 * a.steps,
        "plain_fp64": {"value": n_cells / (pms / 1e3), "ms_per_step": pms,
                       "form": "fp64, one static launch per mechanism"},
        "mixed_over_plain": pms / ms, "clocks": clk.summary()}))


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

    # capacity of each form on the same first requests, everything at t = 0
    n_cap = min(200, a.requests)
    sat = run(camp.VARIANT_MIXED, 0, n_cap)
    sat_p = run(camp.VARIANT_FP64, 0, n_cap)
    # the Poisson stream at the offered load, for each form
    mixed = run(camp.VARIANT_MIXED, a.load * sat["cell_steps_per_s"], a.requests)
    n_plain = min(a.requests, 400)
    plain = run(camp.VARIANT_FP64, a.load * sat_p["cell_steps_per_s"], n_plain)
    print(json.dumps({
        "metric": "cell-steps/s at rtol 1e-4; p50/p99 chunk latency", "value": mixed["cell_steps_per_s"],
        "unit": "cell-steps/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 state / f32 J+LU", "data": "synthetic",
        "config": {"workload": f"serving: Poisson stream of {a.requests} chunks, 256..65536 cells "
                               "(log-uniform), 70% gas-72 / 30% multiphase-232, dt 60..600 s, 80 GB budget, "
                               f"offered load {a.load:g} x measured capacity", "max_inflight": 8},
        "p50_ms": mixed["p50_ms"], "p99_ms": mixed["p99_ms"], "mixed": mixed, "saturation_mixed": sat,
        "plain_fp64": plain, "saturation_plain_fp64": sat_p,
        "capacity_mixed_over_plain": sat["cell_steps_per_s"] / sat_p["cell_steps_per_s"]}))


if __name__ == "__main__":
    main()
