"""Host-side logic of bench.py, on the CPU: the cost models of a solve from
its per-cell counters, the roofline object (which roof bounds the kernel),
and the DRAM traffic table that ties ncu captures to the kernel sources."""
import os
import re
import types

import numpy as np
import pytest

import bench


def _info(n=10, nnz=30, R=12, model_forcing=40, ff=50, fj=70, fa=90, fs=20):
    return types.SimpleNamespace(n_species=n, nnz_lu=nnz, n_rxn=R, model_forcing=model_forcing,
                                 flops_forcing=ff, flops_jacobian=fj, flops_factor=fa, flops_solve=fs)


def test_cost_models_by_hand():
    """Two cells: 3 + 5 steps, 6 + 10 Newton iterations, 1 + 1 setups, order
    sums 6 + 14 -> m = 2, rho = 1/4, q = 2.5 per step."""
    st = np.array([[3, 6, 1, 0, 6], [5, 10, 1, 2, 14]])
    c = bench.cost_models(_info(), st, lu_bytes=4)
    assert (c["steps"], c["newton"], c["setups"]) == (8, 16, 2)
    assert c["mean_order"] == pytest.approx(2.5)
    # flops per step: m F + (q+1)^2 n / 2 + 10 n = 2*40 + 3.5^2*10/2 + 100
    assert c["model_flops"] == pytest.approx(8 * (80 + 61.25 + 100))
    # bytes per step: 16 (q+1) n + m (24 n + b nnz) + rho (2 b nnz + 8 R) + 24 n
    per = 16 * 3.5 * 10 + 2 * (240 + 4 * 30) + 0.25 * (2 * 4 * 30 + 96) + 240
    assert c["model_bytes"] == pytest.approx(8 * per)
    # LU work: setups (J + factor) + Newton iterations (solve)
    assert c["lu_flops"] == 2 * (70 + 90) + 16 * 20
    # the kernel's own FP64 count: f evaluations (Newton + 2 per cell and call)
    f_evals = 16 + 2 * 2
    own = f_evals * 50 + 16 * 8 * 10 + 8 * (2.5 * 3.5 / 2 + 2 * 3.5 + 8) * 10
    assert c["counted_fp64"] == pytest.approx(own)


def test_cost_models_scale_with_cells():
    st = np.array([[4, 9, 2, 1, 12]] * 3)
    one = bench.cost_models(_info(), st[:1], 8)
    three = bench.cost_models(_info(), st, 8)
    for k in ("model_flops", "model_bytes", "lu_flops"):
        assert three[k] == pytest.approx(3 * one[k])


def test_roofline_bounds():
    st = np.array([[10, 20, 2, 0, 30]])
    m = [bench.cost_models(_info(), st, 4)]
    alu = bench.roofline(m, 0.5, 1000.0, "f32", None, "k_solve", "step")
    assert alu["bound"] == "alu" and alu["peak"] == 1000.0
    assert alu["achieved"] == pytest.approx(m[0]["model_flops"] / 0.5 / 1e9)
    assert alu["frac"] == pytest.approx(alu["achieved"] / 1000.0)
    assert alu["hbm_model"]["achieved_gbs"] == pytest.approx(m[0]["model_bytes"] / 0.5 / 1e9)
    hbm = bench.roofline(m, 0.5, 1000.0, "f32", 123.0, "k_arrow", "step", bound="hbm")
    assert hbm["bound"] == "hbm" and hbm["unit"] == "GB/s" and hbm["traffic"] == 123.0
    assert hbm["achieved"] == pytest.approx(alu["hbm_model"]["achieved_gbs"])
    assert hbm["frac"] == pytest.approx(hbm["achieved"] / hbm["peak"])
    assert hbm["fp64_model"]["frac"] == pytest.approx(alu["frac"])


def test_traffic_table_names_real_workloads_and_sources():
    for name, entry in bench.DRAM_BYTES_PER_CELL.items():
        assert name in bench.WORKLOADS
        assert re.fullmatch(r"[0-9a-f]{16}", entry["digest"])
        assert all(b > 0 for b in entry["bytes_per_cell"])
    assert len(bench.DRAM_BYTES_PER_CELL["uneven"]["bytes_per_cell"]) == 2  # one per mechanism group
    csrc = os.path.join(bench.ROOT, "paper_2111_07436_gb300", "csrc")
    for kind, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(csrc, f)), f
        assert re.fullmatch(r"[0-9a-f]{16}", bench.kernel_digest(kind))
    assert bench.kernel_digest("cell") != bench.kernel_digest("arrow")
