"""Several mechanisms in one call (camp_solve_batch), the launch autotuner,
and CUDA-graph replay of the batched solve -- all give the results of plain
single-mechanism solves, bit for bit, and match the oracle."""
import json

import numpy as np
import pytest

import oracle
from paper_2111_07436_gb300 import camp, workloads as w
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def groups(cuda):
    import torch
    gs, cloud = w.uneven_batch(3000, seed=44)
    out = []
    for mj, y, env in gs:
        out.append({"mj": mj, "mech": camp.Mechanism(json.dumps(mj)), "y0": y, "env_np": env,
                    "env": torch.tensor(env, device=cuda),
                    "atol": torch.full((1,), 1e-5, dtype=torch.float64, device=cuda),
                    "workspace": camp.workspace(cuda)})
    return out


def _reset(groups):
    import torch
    for g in groups:
        g["state"] = torch.tensor(g["y0"], device="cuda")
        g["status"] = torch.empty(len(g["y0"]), dtype=torch.int32, device="cuda")


def _args(groups):
    return [{k: g[k] for k in ("mech", "state", "env", "atol", "status", "workspace")} for g in groups]


def test_batch_equals_separate_solves_and_the_oracle(groups):
    import torch
    _reset(groups)
    camp.solve_batch(_args(groups), 180.0, 1e-4)
    torch.cuda.synchronize()
    got = [g["state"].cpu().numpy() for g in groups]
    for g, yb in zip(groups, got):
        ty = torch.tensor(g["y0"], device="cuda")
        st = g["mech"].solve(ty, g["env"], 180.0, 1e-4, 1e-5, persistent=True)
        torch.cuda.synchronize()
        assert np.array_equal(ty.cpu().numpy(), yb)
        assert (st.cpu().numpy() == 0).all() and (g["status"].cpu().numpy() == 0).all()
        om = oracle.Mechanism(json.dumps(g["mj"]))
        idx = np.sort(np.random.default_rng(2).choice(len(g["y0"]), 24, replace=False))
        yo, so, _ = om.solve(g["y0"][idx], g["env_np"][idx], 180.0, 1e-4, 1e-5)
        assert (so == 0).all()
        parity.check(om, g["y0"][idx], g["env_np"][idx], 180.0, 1e-4, 1e-5, yb[idx], yo)


def test_host_buffer_batch_equals_device_batch(groups):
    """camp_solve_batch_host (host arrays in and out, one synchronous call)
    gives the device-pointer batch's results bit for bit, stats included."""
    import torch
    _reset(groups)
    stats = [torch.zeros((len(g["y0"]), camp.NSTATS), dtype=torch.int32, device="cuda") for g in groups]
    args = _args(groups)
    for a_, s in zip(args, stats):
        a_["stats"] = s
    camp.solve_batch(args, 180.0, 1e-4)
    torch.cuda.synchronize()
    ref = [(g["state"].cpu().numpy(), g["status"].cpu().numpy(), s.cpu().numpy()) for g, s in zip(groups, stats)]
    for rep in range(2):  # the second call reuses the library's staging buffer
        host = [{"mech": g["mech"], "state": g["y0"].copy(), "env": g["env_np"], "atol": 1e-5,
                 "status": np.full(len(g["y0"]), -1, dtype=np.int32),
                 "stats": np.zeros((len(g["y0"]), camp.NSTATS), dtype=np.int32)} for g in groups]
        camp.solve_batch_host(host, 180.0, 1e-4)
        for h, (y, st, sts) in zip(host, ref):
            assert np.array_equal(h["state"], y)
            assert np.array_equal(h["status"], st)
            assert np.array_equal(h["stats"], sts)


def test_cloud_cells_take_more_steps(groups):
    import torch
    _reset(groups)
    stats = [torch.zeros((len(g["y0"]), camp.NSTATS), dtype=torch.int32, device="cuda") for g in groups]
    args = _args(groups)
    for a_, s in zip(args, stats):
        a_["stats"] = s
    camp.solve_batch(args, 180.0, 1e-4)
    torch.cuda.synchronize()
    gas_steps = stats[0][:, 0].float().mean().item()
    cloud_steps = stats[1][:, 0].float().mean().item()
    assert cloud_steps > gas_steps
    steps = torch.cat([s[:, 0] for s in stats]).float()
    assert steps.max().item() / max(steps.min().item(), 1) > 3  # uneven stiffness


def test_graph_replay_equals_direct_call(groups):
    import torch
    _reset(groups)
    camp.solve_batch(_args(groups), 180.0, 1e-4)
    torch.cuda.synchronize()
    ref = [g["state"].cpu().numpy() for g in groups]
    y0s = [torch.tensor(g["y0"], device="cuda") for g in groups]
    _reset(groups)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        for g, y0 in zip(groups, y0s):
            g["state"].copy_(y0)
        camp.solve_batch(_args(groups), 180.0, 1e-4, stream=side)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for g, r in zip(groups, ref):
            assert np.array_equal(g["state"].cpu().numpy(), r)


def test_autotune_picks_a_valid_launch(groups):
    import torch
    g = groups[0]
    y = torch.tensor(g["y0"][:512], device="cuda")
    e = g["env"][:512].contiguous()
    before = y.clone()
    cpb, pers, ms = g["mech"].autotune(y, e, 180.0, 1e-4, g["atol"])
    assert cpb in (1, 2, 3, 4) and pers in (0, 1) and ms > 0
    assert torch.equal(y, before)  # inputs untouched
    ta = y.clone()
    g["mech"].solve(ta, e, 180.0, 1e-4, 1e-5)  # uses the tuned defaults
    tb = y.clone()
    g["mech"].solve(tb, e, 180.0, 1e-4, 1e-5, persistent=True, cells_per_block=1)
    torch.cuda.synchronize()
    assert torch.equal(ta, tb)


def test_full_size_uneven_batch_sampled(cuda):
    """The uneven-stiffness workload at its full size (131072 cells, the
    benchmark's seeds) in the launch configuration the benchmark times:
    autotuned, both mechanisms in one camp_solve_batch call captured in a
    CUDA graph; then the plain FP64 form, one static launch per mechanism.
    A stratified sample of 4096 cells (by mechanism and dark / lit, in
    proportion) is re-solved by the oracle; every sampled cell is under the
    parity rule and the arbiter."""
    import torch
    gs, _ = w.uneven_batch(131072)
    G = []
    for mj, y, env in gs:
        G.append({"mj": mj, "mech": camp.Mechanism(json.dumps(mj)), "y0": y, "env_np": env,
                  "y0_d": torch.tensor(y, device=cuda), "env": torch.tensor(env, device=cuda),
                  "state": torch.empty(y.shape, dtype=torch.float64, device=cuda),
                  "status": torch.empty(len(y), dtype=torch.int32, device=cuda),
                  "atol": torch.full((1,), 1e-5, dtype=torch.float64, device=cuda),
                  "workspace": camp.workspace(cuda)})
    for g in G:
        k = min(4096, len(g["y0"]))
        g["mech"].autotune(g["y0_d"][:k].contiguous(), g["env"][:k].contiguous(), 180.0, 1e-4, g["atol"])
    side = torch.cuda.Stream()

    def step():
        for g in G:
            g["state"].copy_(g["y0_d"])
        camp.solve_batch([{k: g[k] for k in ("mech", "state", "env", "atol", "status", "workspace")}
                          for g in G], 180.0, 1e-4, stream=side)

    with torch.cuda.stream(side):
        step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        step()
    graph.replay()
    torch.cuda.synchronize()
    mixed = [(g["state"].cpu().numpy(), g["status"].cpu().numpy()) for g in G]
    for g in G:
        g["state"].copy_(g["y0_d"])
        g["mech"].solve(g["state"], g["env"], 180.0, 1e-4, g["atol"], status=g["status"],
                        variant=camp.VARIANT_FP64, persistent=False)
    torch.cuda.synchronize()
    plain = [(g["state"].cpu().numpy(), g["status"].cpu().numpy()) for g in G]
    sample = w.stratified_sample(gs, 4096)
    for gi, g in enumerate(G):
        assert (mixed[gi][1] == 0).all() and (plain[gi][1] == 0).all()
        idx = sample[gi]
        om = oracle.Mechanism(json.dumps(g["mj"]))
        yo, so, _ = om.solve(g["y0"][idx], g["env_np"][idx], 180.0, 1e-4, 1e-5)
        assert (so == 0).all()
        for name, (y_gpu, _) in (("mixed", mixed[gi]), ("fp64", plain[gi])):
            stats = parity.check(om, g["y0"][idx], g["env_np"][idx], 180.0, 1e-4, 1e-5, y_gpu[idx], yo)
            print(f"group {gi} ({len(idx)} sampled cells) {name}: {stats}")


def test_batch_with_a_water_parameter_mechanism(cuda):
    """A water-parameter mechanism (its own kernel build) beside a gas-only
    one in one batched call: each group equals its lone solve bit for bit."""
    import torch
    gas, water = w.large_gas_mechanism(), w.water_mechanism()
    groups = []
    for mj, C, seed in ((gas, 700, 51), (water, 300, 52)):
        y, env = w.cells(mj, C, seed=seed)
        groups.append({"mech": camp.Mechanism(json.dumps(mj)), "y0": y,
                       "env": torch.tensor(env, device=cuda),
                       "atol": torch.full((1,), 1e-5, dtype=torch.float64, device=cuda),
                       "workspace": camp.workspace(cuda)})
    _reset(groups)
    camp.solve_batch(_args(groups), 180.0, 1e-4)
    torch.cuda.synchronize()
    for g in groups:
        ty = torch.tensor(g["y0"], device="cuda")
        st = g["mech"].solve(ty, g["env"], 180.0, 1e-4, 1e-5, persistent=True)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all() and (g["status"].cpu().numpy() == 0).all()
        assert np.array_equal(ty.cpu().numpy(), g["state"].cpu().numpy())
