"""Opt-in warm start through the C ABI: the step size carried across
consecutive calls for the same cells (camp_solve_opts.step) against the
oracle's warm start, for both forms and both entry points."""
import json

import numpy as np
import pytest

import oracle
from paper_2111_07436_gb300 import camp, workloads as w
from tests import parity

pytestmark = pytest.mark.gpu

FORMS = [(camp.VARIANT_FP64, False), (camp.VARIANT_MIXED, True)]


@pytest.fixture(scope="module")
def gas(cuda):
    wl = w.workload(2)
    return wl, camp.Mechanism(wl.json()), oracle.Mechanism(wl.json())


@pytest.mark.parametrize("variant,persistent", FORMS, ids=["fp64", "mixed"])
def test_three_consecutive_calls_match_the_oracle(gas, variant, persistent):
    import torch
    wl, gm, om = gas
    y0, env = wl.inputs(257)
    ty, te = torch.tensor(y0, device="cuda"), torch.tensor(env, device="cuda")
    step_g = torch.zeros(len(y0), dtype=torch.float64, device="cuda")
    step_o = np.zeros(len(y0))
    stats = torch.zeros((len(y0), camp.NSTATS), dtype=torch.int32, device="cuda")
    yo = y0.copy()
    steps_warm = 0
    for call in range(3):
        y_before = yo.copy()
        st = gm.solve(ty, te, wl.dt, wl.rtol, wl.atol, variant=variant, persistent=persistent,
                      stats=stats, step=step_g)
        torch.cuda.synchronize()
        yo, so, _ = om.solve(yo, env, wl.dt, wl.rtol, wl.atol, step=step_o)
        assert (st.cpu().numpy() == 0).all() and (so == 0).all()
        parity.check(om, y_before, env, wl.dt, wl.rtol, wl.atol, ty.cpu().numpy(), yo)
        sg = step_g.cpu().numpy()
        assert (sg > 0).all() and (step_o > 0).all()
        # the same controller: carried steps agree closely for most cells
        assert np.median(np.abs(sg / step_o - 1.0)) < (1e-6 if variant == camp.VARIANT_FP64 else 0.1)
        if call > 0:
            steps_warm += stats[:, 0].sum().item()
    # cold calls over the same states take more steps
    ty2 = torch.tensor(y0, device="cuda")
    steps_cold = 0
    for call in range(3):
        gm.solve(ty2, te, wl.dt, wl.rtol, wl.atol, variant=variant, persistent=persistent, stats=stats)
        torch.cuda.synchronize()
        if call > 0:
            steps_cold += stats[:, 0].sum().item()
    assert steps_warm < steps_cold


def test_host_entry_point_and_failed_cells(gas):
    import torch
    wl, gm, om = gas
    y0, env = wl.inputs(64)
    y0[5, 3] = np.nan  # a cell that fails: status 5, step handed back as 0
    step_h = np.full(len(y0), 7.5)
    yh = y0.copy()
    st_h = gm.solve_host(yh, env, wl.dt, wl.rtol, wl.atol, step=step_h)
    ty = torch.tensor(y0, device="cuda")
    step_d = torch.full((len(y0),), 7.5, dtype=torch.float64, device="cuda")
    st_d = gm.solve(ty, torch.tensor(env, device="cuda"), wl.dt, wl.rtol, wl.atol, step=step_d)
    torch.cuda.synchronize()
    assert np.array_equal(st_h, st_d.cpu().numpy())
    assert np.array_equal(yh, ty.cpu().numpy(), equal_nan=True)
    assert np.array_equal(step_h, step_d.cpu().numpy())
    assert st_h[5] == 5 and step_h[5] == 0.0
    ok = np.arange(len(y0)) != 5
    assert (st_h[ok] == 0).all() and (step_h[ok] > 0).all()


def test_water_parameter_warm_start(cuda):
    """Warm start on the water build: three consecutive calls against the
    oracle's warm start."""
    import torch
    wl = w.workload(7)
    gm, om = camp.Mechanism(wl.json()), oracle.Mechanism(wl.json())
    y0, env = wl.inputs(129)
    ty, te = torch.tensor(y0, device="cuda"), torch.tensor(env, device="cuda")
    step_g = torch.zeros(len(y0), dtype=torch.float64, device="cuda")
    step_o = np.zeros(len(y0))
    yo = y0.copy()
    for call in range(3):
        y_before = yo.copy()
        st = gm.solve(ty, te, wl.dt, wl.rtol, wl.atol, step=step_g)
        torch.cuda.synchronize()
        yo, so, _ = om.solve(yo, env, wl.dt, wl.rtol, wl.atol, step=step_o)
        assert (st.cpu().numpy() == 0).all() and (so == 0).all()
        parity.check(om, y_before, env, wl.dt, wl.rtol, wl.atol, ty.cpu().numpy(), yo)
        assert (step_g.cpu().numpy() > 0).all()
