"""The continuous-batching request loop (camp_server_*) on the GPU: chunks of
different sizes and mechanisms submitted while others run give the same
results as lone solves and match the oracle; resident cell sets keep their
state on the device across a host's consecutive steps; the memory budget and
bounded waits behave."""
import numpy as np
import pytest

import oracle
from paper_2111_07436_gb300 import camp, workloads as w
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mechs(cuda):
    return {k: (w.workload(k), camp.Mechanism(w.workload(k).json())) for k in (2, 3)}


def _pinned(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t


def _alone(gm, y, env, dt, rtol, atol):
    import torch
    ty = torch.tensor(y, device="cuda")
    st = gm.solve(ty, torch.tensor(env, device="cuda"), dt, rtol, atol)
    torch.cuda.synchronize()
    return ty.cpu().numpy(), st.cpu().numpy()


def test_mixed_stream_equals_lone_solves(mechs):
    rng = np.random.default_rng(0)
    srv = camp.Server(hbm_budget_bytes=2 << 30, max_inflight=4)
    jobs = []
    for i in range(10):
        k = 2 if rng.random() < 0.7 else 3
        wl, gm = mechs[k]
        C = int(np.exp(rng.uniform(np.log(16), np.log(2000))))
        y, env = w.cells(wl.mech, C, seed=900 + i)
        dt = float(rng.uniform(60, 600))
        ty, te, ts = _pinned(y.copy()), _pinned(env), _pinned(np.zeros(C, dtype=np.int32))
        rid = srv.submit(gm, ty, te, dt, wl.rtol, wl.atol, ts)
        jobs.append((rid, gm, y, env, dt, wl, ty, ts))
    infos = []
    for rid, gm, y, env, dt, wl, ty, ts in jobs:
        info = srv.wait(rid)
        assert info["rc"] == 0
        infos.append(info)
        ya, sa = _alone(gm, y, env, dt, wl.rtol, wl.atol)
        assert np.array_equal(ty.numpy(), ya)
        assert np.array_equal(ts.numpy(), sa)
    srv.close()
    # later chunks were admitted while earlier ones were still running
    assert any(b["t_admit"] < a["t_done"] for a, b in zip(infos, infos[1:]))
    # a sample of every chunk against the oracle
    oms = {}
    for i, (rid, gm, y, env, dt, wl, ty, ts) in enumerate(jobs):
        om = oms.setdefault(wl.mech["name"], oracle.Mechanism(wl.json()))
        idx = np.sort(np.random.default_rng(i).choice(len(y), min(len(y), 24), replace=False))
        yo, so, _ = om.solve(y[idx], env[idx], dt, wl.rtol, wl.atol)
        assert (so == 0).all()
        parity.check(om, y[idx], env[idx], dt, wl.rtol, wl.atol, ty.numpy()[idx], yo)


def test_budget_and_bounded_wait(mechs):
    wl, gm = mechs[2]
    y, env = w.cells(wl.mech, 20000, seed=3)
    per_chunk = 20000 * (gm.n + gm.n_env) * 8 + 20000 * 4
    srv = camp.Server(hbm_budget_bytes=int(1.5 * per_chunk), max_inflight=4)
    big_y = _pinned(np.concatenate([y, y]))
    big_e = _pinned(np.concatenate([env, env]))
    big_s = _pinned(np.zeros(40000, dtype=np.int32))
    rid = srv.submit(gm, big_y, big_e, wl.dt, wl.rtol, wl.atol, big_s)  # larger than the budget
    assert srv.wait(rid)["rc"] == camp.E_BUDGET
    a = (_pinned(y.copy()), _pinned(env), _pinned(np.zeros(20000, dtype=np.int32)))
    b = (_pinned(y.copy()), _pinned(env), _pinned(np.zeros(20000, dtype=np.int32)))
    ra = srv.submit(gm, a[0], a[1], wl.dt, wl.rtol, wl.atol, a[2])
    rb = srv.submit(gm, b[0], b[1], wl.dt, wl.rtol, wl.atol, b[2])
    assert srv.wait(rb, timeout_ms=0) is None  # cannot be done yet: waits behind `a` for memory
    st = srv.stats()
    assert st["bytes_in_use"] <= int(1.5 * per_chunk)
    ia, ib = srv.wait(ra), srv.wait(rb)
    assert ia["rc"] == 0 and ib["rc"] == 0
    assert ib["t_admit"] >= ia["t_done"] - 1e-3  # budget forced b to wait for a
    assert np.array_equal(a[0].numpy(), b[0].numpy())
    srv.close()


def test_cancel_withdraws_only_pending_requests(mechs):
    wl, gm = mechs[2]
    srv = camp.Server(hbm_budget_bytes=4 << 30, max_inflight=1)
    jobs = []
    for i, C in enumerate((20000, 500, 500)):  # one slot: the last two wait behind the first
        y, env = w.cells(wl.mech, C, seed=950 + i)
        ty, te, ts = _pinned(y.copy()), _pinned(env), _pinned(np.full(C, -1, dtype=np.int32))
        jobs.append((srv.submit(gm, ty, te, wl.dt, wl.rtol, wl.atol, ts), y, ty, ts))
    assert srv.cancel(jobs[2][0])
    info = srv.wait(jobs[2][0])
    assert info["rc"] == camp.E_CANCELLED
    assert np.array_equal(jobs[2][2].numpy(), jobs[2][1]) and (jobs[2][3].numpy() == -1).all()
    for rid, y, ty, ts in jobs[:2]:
        assert srv.wait(rid)["rc"] == 0
        assert (ts.numpy() == 0).all()
    with pytest.raises(camp.CampError):  # collected: no longer known
        srv.cancel(jobs[0][0])
    srv.close()


def test_water_parameter_chunks_equal_lone_solves(mechs):
    """Chunks of a water-parameter mechanism (its own kernel build) served
    beside gas chunks give the lone solves' results bit for bit."""
    wlw = w.workload(7)
    gmw = camp.Mechanism(wlw.json())
    srv = camp.Server(hbm_budget_bytes=2 << 30, max_inflight=4)
    jobs = []
    for i, (wl, gm, C) in enumerate([(wlw, gmw, 300), (mechs[2][0], mechs[2][1], 900),
                                     (wlw, gmw, 77), (mechs[2][0], mechs[2][1], 40)]):
        y, env = w.cells(wl.mech, C, seed=950 + i)
        ty, te, ts = _pinned(y.copy()), _pinned(env), _pinned(np.zeros(C, dtype=np.int32))
        rid = srv.submit(gm, ty, te, 300.0, wl.rtol, wl.atol, ts)
        jobs.append((rid, gm, y, env, wl, ty, ts))
    for rid, gm, y, env, wl, ty, ts in jobs:
        assert srv.wait(rid)["rc"] == 0
        ya, sa = _alone(gm, y, env, 300.0, wl.rtol, wl.atol)
        assert np.array_equal(ty.numpy(), ya) and np.array_equal(ts.numpy(), sa)
        assert (sa == 0).all()
    srv.close()


def _env_for_step(env, wl, k):
    """The host model's env of step k: temperature drifts and the sun moves
    (photolysis scaled), as a host would update them between steps."""
    e = env.copy()
    e[:, 0] += 2.0 * k
    lay = w.layout(wl.mech)
    for j, kind in enumerate(lay.runtime_kind):
        if kind == "PHOTOLYSIS":
            e[:, 2 + j] *= (1.0 - 0.3 * k)
    return e


@pytest.mark.parametrize("k", [2, 3])
def test_resident_set_steps_equal_lone_solves_and_the_oracle(mechs, k):
    """A resident set stepped three times (env changing every step, a state
    write from the host between steps 2 and 3) gives, after every step, the
    lone solve of its previous state bit for bit, and matches the oracle
    integrating the same sequence."""
    wl, gm = mechs[k]
    om = oracle.Mechanism(wl.json())
    C = 300 if k == 2 else 120
    y0, env = w.cells(wl.mech, C, seed=970 + k)
    srv = camp.Server(hbm_budget_bytes=1 << 30, max_inflight=4)
    res = srv.resident(gm, y0)
    y_gpu, y_ora = y0.copy(), y0.copy()
    for step in range(3):
        if step == 2:  # the host's transport moved some air: it rewrites the state
            y_gpu = y_gpu * 1.05
            y_ora = y_ora * 1.05
            res.write(y_gpu)
        e = _env_for_step(env, wl, step)
        status = np.full(C, -1, dtype=np.int32)
        rid = res.step(e, wl.dt, wl.rtol, wl.atol, status=status)
        assert srv.wait(rid)["rc"] == 0
        y_res, st_res = res.read()
        assert (status == 0).all() and np.array_equal(st_res, status)
        ya, sa = _alone(gm, y_gpu, e, wl.dt, wl.rtol, wl.atol)
        assert np.array_equal(y_res, ya) and np.array_equal(status, sa)
        yo, so, _ = om.solve(y_ora, e, wl.dt, wl.rtol, wl.atol)
        assert (so == 0).all()
        parity.check(om, y_ora, e, wl.dt, wl.rtol, wl.atol, y_res, yo)
        y_gpu, y_ora = y_res, yo
    res.close()
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_resident_warm_start_matches_solve_with_steps_and_the_oracle(mechs):
    """A resident set created with warm_start carries each cell's step size
    on the device: its steps equal camp_solve with a step array (bit for
    bit) and the oracle's own warm start."""
    import torch
    wl, gm = mechs[2]
    om = oracle.Mechanism(wl.json())
    C = 256
    y0, env = w.cells(wl.mech, C, seed=981)
    srv = camp.Server(hbm_budget_bytes=1 << 30, max_inflight=2)
    res = srv.resident(gm, y0, warm_start=True)
    ty = torch.tensor(y0, device="cuda")
    hs_d = torch.zeros(C, dtype=torch.float64, device="cuda")
    y_ora, hs_o = y0.copy(), np.zeros(C)
    rids = [res.step(_env_for_step(env, wl, k), wl.dt, wl.rtol, wl.atol) for k in range(3)]
    # three steps queued at once run in order; compare the end state
    for rid in rids:
        assert srv.wait(rid)["rc"] == 0
    for k in range(3):
        e = _env_for_step(env, wl, k)
        st = gm.solve(ty, torch.tensor(e, device="cuda"), wl.dt, wl.rtol, wl.atol, step=hs_d)
        assert (st.cpu().numpy() == 0).all()
        y_prev = y_ora.copy()
        y_ora, so, _ = om.solve(y_ora, e, wl.dt, wl.rtol, wl.atol, step=hs_o)
        assert (so == 0).all()
    torch.cuda.synchronize()
    y_res, st_res, hs_res = res.read(with_step=True)
    assert (st_res == 0).all()
    assert np.array_equal(y_res, ty.cpu().numpy()) and np.array_equal(hs_res, hs_d.cpu().numpy())
    parity.check(om, y_prev, _env_for_step(env, wl, 2), wl.dt, wl.rtol, wl.atol, y_res, y_ora)
    res.close()
    srv.close()


def test_resident_sets_count_against_the_budget(mechs):
    wl, gm = mechs[2]
    y0, env = w.cells(wl.mech, 4000, seed=990)
    per_set = 4000 * (gm.n + gm.n_env) * 8 + 4000 * 4
    srv = camp.Server(hbm_budget_bytes=int(1.6 * per_set), max_inflight=2)
    a = srv.resident(gm, y0)
    assert srv.stats()["bytes_in_use"] >= per_set
    with pytest.raises(camp.CampError):
        srv.resident(gm, y0)  # does not fit next to the first
    # an ordinary chunk that needs more than what is left waits until the set is gone
    ty, te, ts = _pinned(y0.copy()), _pinned(env), _pinned(np.zeros(4000, dtype=np.int32))
    rid = srv.submit(gm, ty, te, wl.dt, wl.rtol, wl.atol, ts)
    assert srv.wait(rid, timeout_ms=200) is None
    a.close()
    assert srv.wait(rid)["rc"] == 0
    srv.close()
