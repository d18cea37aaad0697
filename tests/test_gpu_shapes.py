"""Cell shapes: the same mechanism on one warp, 64 or 128 threads a cell
(camp_mech_set_lanes), in both forms, against the oracle; and the launch
autotuner's choice between the two shapes of a 129-256-species mechanism.
Each test builds its own mechanisms, since a shape change is the
mechanism's."""
import numpy as np
import pytest

import oracle
from paper_2111_07436_gb300 import camp, workloads as w
from tests import parity

pytestmark = pytest.mark.gpu

FORMS = [(camp.VARIANT_FP64, False), (camp.VARIANT_MIXED, True)]
FORM_IDS = ["fp64-static", "mixed-persistent"]


def _solve(gm, y, env, wl, variant, persistent):
    import torch
    ty = torch.tensor(y, device="cuda")
    st = gm.solve(ty, torch.tensor(env, device="cuda"), wl.dt, wl.rtol, wl.atol, variant=variant,
                  persistent=persistent)
    torch.cuda.synchronize()
    return ty.cpu().numpy(), st.cpu().numpy()


@pytest.fixture(scope="module")
def oracles(cuda):
    """The oracle's results on 67 cells of the 72-, 232- and 240-species
    workloads (the last with a water parameter)."""
    out = {}
    for k in (2, 3, 7):
        wl = w.workload(k)
        om = oracle.Mechanism(wl.json())
        y0, env = wl.inputs(67)
        yo, sto, _ = om.solve(y0, env, wl.dt, wl.rtol, wl.atol)
        assert (sto == 0).all()
        out[k] = (wl, om, y0, env, yo)
    return out


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("k,lanes", [(2, 32), (2, 64), (2, 128), (3, 32), (3, 64), (7, 32), (7, 64)])
def test_every_cell_shape_matches_the_oracle(oracles, form, k, lanes):
    wl, om, y0, env, yo = oracles[k]
    gm = camp.Mechanism(wl.json())
    gm.set_lanes(lanes)
    assert gm.info.lanes_per_cell == lanes
    yg, st = _solve(gm, y0, env, wl, *form)
    assert (st == 0).all()
    parity.check(om, y0, env, wl.dt, wl.rtol, wl.atol, yg, yo)


def test_plain_form_results_hardly_depend_on_the_shape(oracles):
    """The FP64 form on one warp and on 64 threads: the same arithmetic up
    to the order of sums, so the two agree far inside the parity rule."""
    wl, om, y0, env, yo = oracles[3]
    res = []
    for lanes in (32, 64):
        gm = camp.Mechanism(wl.json())
        gm.set_lanes(lanes)
        res.append(_solve(gm, y0, env, wl, camp.VARIANT_FP64, False)[0])
    big = np.abs(res[0]) > 100 * wl.atol
    rel = np.abs(res[0] - res[1])[big] / np.abs(res[0])[big]
    assert np.median(rel) < 1e-12 and rel.max() < 1e-6


def test_autotune_chooses_a_cell_shape(oracles):
    import torch
    wl, om, y0, env, yo = oracles[3]
    gm = camp.Mechanism(wl.json())
    assert gm.info.lanes_per_cell == 64  # the default for 193-256 species
    ys, envs = wl.inputs(512)
    ty = torch.tensor(ys, device="cuda")
    te = torch.tensor(envs, device="cuda")
    before = ty.clone()
    for _ in range(2):  # a second call starts from the shape the first chose
        cpb, pers, ms = gm.autotune(ty, te, wl.dt, wl.rtol, wl.atol)
        assert gm.info.lanes_per_cell in (32, 64) and ms > 0
        assert cpb in ((1, 2, 3, 4) if gm.info.lanes_per_cell == 32 else (1,)) and pers in (0, 1)
    assert torch.equal(ty, before)
    yg, st = _solve(gm, y0, env, wl, camp.VARIANT_MIXED, True)
    assert (st == 0).all()
    parity.check(om, y0, env, wl.dt, wl.rtol, wl.atol, yg, yo)


def test_set_lanes_refusals(cuda):
    wl = w.workload(2)
    gm = camp.Mechanism(wl.json())
    for bad in (0, 16, 96, 512):
        with pytest.raises(camp.CampError):
            gm.set_lanes(bad)
    assert gm.info.lanes_per_cell == 32  # unchanged
    big = camp.Mechanism(w.workload(6).json())  # 914 species: at most 8 a lane
    with pytest.raises(camp.CampError):
        big.set_lanes(64)
    assert big.info.lanes_per_cell == 128
