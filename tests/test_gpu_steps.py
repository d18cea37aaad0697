"""Each step of the method on the GPU against the oracle, through the C ABI:
rate constants (Table 2), forcing and Jacobian (Sect. 2.4.2), and the
static-pivot sparse LU solve of I - gamma J (Sect. 2.4.1)."""
import json

import numpy as np
import pytest

import oracle
from paper_2111_07436_gb300 import camp, workloads as w
from tests import mechs as M

pytestmark = pytest.mark.gpu

MECHS = {"small": w.small_gas_mechanism(), "gas72": w.large_gas_mechanism(),
         "multiphase232": w.multiphase_mechanism(), "variety": w.process_variety_mechanism(),
         "particles40": w.particle_resolved_mechanism(40), "water240": w.water_mechanism(),
         "water_chain": json.loads(M.water_chain_mechanism())}


def _inputs(mj, C, seed):
    y, env = w.cells(mj, C, seed=seed)
    n_gas = len(mj["species"])
    if y.shape[1] > n_gas:  # give the aqueous species non-trivial values
        y[:, n_gas:] = np.random.default_rng(seed).uniform(0.0, 1e-2, (C, y.shape[1] - n_gas))
    if mj.get("parameters"):  # electrolytes that hold a realistic amount of water
        lay = w.layout(mj)
        for e in mj["parameters"][0]["electrolytes"]:
            cols = [k for k, s in enumerate(lay.species) if s.endswith("." + e["species"])]
            y[:, cols] = np.random.default_rng(seed + 1).uniform(0.5, 5.0, (C, len(cols)))
    return y, env


@pytest.fixture(scope="module", params=sorted(MECHS))
def case(request, cuda):
    import torch
    mj = MECHS[request.param]
    text = json.dumps(mj)
    y, env = _inputs(mj, 67, seed=11)  # ragged: not a multiple of any block size
    return dict(name=request.param, gm=camp.Mechanism(text), om=oracle.Mechanism(text), y=y, env=env,
                ty=torch.tensor(y, device=cuda), tenv=torch.tensor(env, device=cuda))


def test_rate_constants(case):
    kf, kr = case["gm"].rate_constants(case["tenv"])
    kf, kr = kf.cpu().numpy(), kr.cpu().numpy()
    for c in range(len(case["y"])):
        okf, okr = case["om"].rate_constants(case["env"][c])
        np.testing.assert_allclose(kf[c], okf, rtol=1e-12, atol=0)
        np.testing.assert_allclose(kr[c], okr, rtol=1e-12, atol=0)


def test_forcing(case):
    f = case["gm"].forcing(case["ty"], case["tenv"]).cpu().numpy()
    for c in range(len(case["y"])):
        kf, kr = case["om"].rate_constants(case["env"][c])
        fo = case["om"].forcing(kf, kr, case["y"][c], case["env"][c])
        scale = np.maximum(np.abs(fo), 1e-6 * np.abs(fo).max())
        assert np.all(np.abs(f[c] - fo) <= 1e-11 * scale + 1e-300)


@pytest.mark.parametrize("variant,tol", [(camp.VARIANT_FP64, 1e-12), (camp.VARIANT_MIXED, 2e-5)])
def test_jacobian(case, variant, tol):
    gm, om = case["gm"], case["om"]
    st = gm.structure()
    J = gm.jacobian(case["ty"], case["tenv"], variant=variant).cpu().numpy()
    rows = np.repeat(np.arange(gm.n), np.diff(st["rowptr"]))
    for c in range(len(case["y"])):
        kf, kr = om.rate_constants(case["env"][c])
        Jo = om.jacobian(kf, kr, case["y"][c], case["env"][c])
        want = Jo[rows, st["colidx"]]
        scale = np.abs(Jo).max(axis=1)[rows] + 1e-300
        assert np.max(np.abs(J[c] - want) / scale) <= tol
        # nothing outside the pattern
        mask = np.ones_like(Jo, dtype=bool)
        mask[rows, st["colidx"]] = False
        assert not Jo[mask].any()


@pytest.mark.parametrize("variant,tol", [(camp.VARIANT_FP64, 1e-10), (camp.VARIANT_MIXED, 1e-4)])
@pytest.mark.parametrize("gamma", [0.1, 30.0])
def test_lu_solve(case, variant, tol, gamma):
    import torch
    gm, om = case["gm"], case["om"]
    rng = np.random.default_rng(5)
    b = rng.normal(size=case["y"].shape)
    x, st = gm.lu_solve(case["ty"], case["tenv"], gamma, torch.tensor(b, device=case["ty"].device),
                        variant=variant)
    x, st = x.cpu().numpy(), st.cpu().numpy()
    for c in range(len(case["y"])):
        kf, kr = om.rate_constants(case["env"][c])
        Jo = om.jacobian(kf, kr, case["y"][c], case["env"][c])
        Mo = np.eye(gm.n) - gamma * Jo
        xo = oracle.dense_lu_solve(Mo, b[c])
        if variant == camp.VARIANT_MIXED and st[c] != 0:
            # FP32 elimination loses the unit diagonal once gamma |J| passes
            # 1/eps32; the kernel must then report the breakdown (status 4)
            assert st[c] == 4 and gamma * np.abs(Jo).max() > 1 / np.finfo(np.float32).eps
            continue
        assert st[c] == 0
        r = np.linalg.norm(Mo @ x[c] - b[c]) / (np.linalg.norm(Mo, np.inf) * np.linalg.norm(x[c], np.inf))
        assert r <= tol
        # forward error: the fixed bound on well-conditioned matrices, else
        # the perturbation bound cond(M) u (the water mechanisms' tiny
        # liquid volumes make M ill-conditioned)
        u = 2.0 ** -53 if variant == camp.VARIANT_FP64 else 2.0 ** -24
        fwd = np.linalg.norm(x[c] - xo) / np.linalg.norm(xo)
        assert fwd <= max(tol * 1e3 * max(1.0, gamma), 10 * np.linalg.cond(Mo) * u)


def test_zero_cells_is_a_no_op(cuda):
    import torch
    gm = camp.Mechanism(json.dumps(MECHS["small"]))
    e = torch.empty((0, gm.n_env), dtype=torch.float64, device=cuda)
    kf, kr = gm.rate_constants(e)
    assert kf.shape == (0, gm.n_rxn)
