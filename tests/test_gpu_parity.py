"""Whole solves on the GPU against the oracle, through the C ABI, for both
forms (plain FP64; mixed FP32 J/LU with FP64 state and error test), static
and persistent mappings, at small sizes in full and at the benchmark sizes on
every cell; plus the edge cases of the method.  Parity rule and arbiter:
tests/parity.py."""
import json

import numpy as np
import pytest

import oracle
from paper_2111_07436_gb300 import camp, workloads as w
from tests import parity

pytestmark = pytest.mark.gpu

FORMS = [(camp.VARIANT_FP64, False), (camp.VARIANT_MIXED, False), (camp.VARIANT_MIXED, True)]
FORM_IDS = ["fp64-static", "mixed-static", "mixed-persistent"]


def _gpu_solve(gm, y, env, dt, rtol, atol, variant, persistent, **kw):
    import torch
    ty = torch.tensor(y, device="cuda")
    te = torch.tensor(env, device="cuda")
    st = gm.solve(ty, te, dt, rtol, atol, variant=variant, persistent=persistent, **kw)
    torch.cuda.synchronize()
    return ty.cpu().numpy(), st.cpu().numpy()


@pytest.fixture(scope="module")
def mechs(cuda):
    out = {}
    for k in (1, 2, 3):
        wl = w.workload(k)
        out[k] = (wl, camp.Mechanism(wl.json()), oracle.Mechanism(wl.json()))
    return out


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_small_mechanism_one_hour(mechs, form):
    """One cell, 60 outer steps of 60 s; compared after every outer step."""
    wl, gm, om = mechs[1]
    y0, env = wl.inputs()
    yg, yo = y0.copy(), y0.copy()
    for step in range(wl.n_outer):
        yg_new, st = _gpu_solve(gm, yg, env, wl.dt, wl.rtol, wl.atol, *form)
        assert (st == 0).all()
        yo_new, sto, _ = om.solve(yo, env, wl.dt, wl.rtol, wl.atol)
        assert (sto == 0).all()
        parity.check(om, yo, env, wl.dt, wl.rtol, wl.atol, yg_new, yo_new)
        yg, yo = yg_new, yo_new


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_outer_steps_in_one_launch_equal_separate_launches(mechs, form):
    """camp_solve_sequence: the small mechanism's 60 outer steps in one
    launch write, after every step, the state 60 separate launches give (bit
    for bit); the same for 64 cells of the 72-species mechanism over three
    steps; a cell that fails stops there with its status."""
    import torch
    for k, C, n_steps in ((1, 1, 60), (2, 64, 3)):
        wl, gm, om = mechs[k]
        y0, env = wl.inputs(C)
        ty = torch.tensor(y0, device="cuda")
        traj = torch.zeros((n_steps, C, gm.n), dtype=torch.float64, device="cuda")
        st = gm.solve_sequence(ty, torch.tensor(env, device="cuda"), wl.dt, n_steps, wl.rtol, wl.atol,
                               trajectory=traj, variant=form[0], persistent=form[1])
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        traj = traj.cpu().numpy()
        yg = y0.copy()
        for j in range(n_steps):
            yg, stj = _gpu_solve(gm, yg, env, wl.dt, wl.rtol, wl.atol, *form)
            assert (stj == 0).all()
            assert np.array_equal(traj[j], yg)
        assert np.array_equal(ty.cpu().numpy(), yg)
    # a step budget too small for the first step: status 1, nothing written
    wl, gm, om = mechs[2]
    y0, env = wl.inputs(4)
    ty = torch.tensor(y0, device="cuda")
    traj = torch.full((3, 4, gm.n), -1.0, dtype=torch.float64, device="cuda")
    status = gm.solve_sequence(ty, torch.tensor(env, device="cuda"), wl.dt, 3, wl.rtol, wl.atol, trajectory=traj,
                               variant=form[0], persistent=form[1], max_steps=3)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 1).all()
    assert np.array_equal(ty.cpu().numpy(), y0) and (traj.cpu().numpy() == -1.0).all()


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("k,C", [(2, 301), (3, 67)])
def test_full_parity_small_batches(mechs, form, k, C):
    wl, gm, om = mechs[k]
    y0, env = wl.inputs(C)
    yg, st = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, *form)
    yo, sto, _ = om.solve(y0, env, wl.dt, wl.rtol, wl.atol)
    assert (st == 0).all() and (sto == 0).all()
    parity.check(om, y0, env, wl.dt, wl.rtol, wl.atol, yg, yo)


@pytest.fixture(scope="module")
def full_oracle(mechs):
    """The oracle's results on every cell of the 72- and 232-species
    workloads at their full sizes (16384 and 4096 cells), computed once."""
    out = {}
    for k in (2, 3):
        wl, gm, om = mechs[k]
        y0, env = wl.inputs()
        yo, so, _ = om.solve(y0, env, wl.dt, wl.rtol, wl.atol)
        assert (so == 0).all()
        out[k] = (y0, env, yo)
    return out


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("k", [2, 3])
def test_every_cell_at_full_size(mechs, full_oracle, form, k):
    """The full workload in one launch (16384 cells of the 72-species
    mechanism, 4096 of the 232-species one), every cell under the parity
    rule, every violating cell through the arbiter."""
    wl, gm, om = mechs[k]
    y0, env, yo = full_oracle[k]
    yg, st = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, *form)
    assert (st == 0).all()
    stats = parity.check(om, y0, env, wl.dt, wl.rtol, wl.atol, yg, yo)
    print(f"workload {k} {form}: {stats}")


def test_results_do_not_depend_on_batch_or_mapping(mechs):
    """A cell's result is bit-identical alone, in a batch, under either
    mapping and any cells-per-block."""
    wl, gm, om = mechs[2]
    y0, env = wl.inputs(200)
    ref, _ = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, camp.VARIANT_MIXED, True)
    for persistent, cpb in ((False, 1), (False, 3), (True, 2)):
        yg, _ = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, camp.VARIANT_MIXED, persistent,
                           cells_per_block=cpb)
        assert np.array_equal(yg, ref)
    alone, _ = _gpu_solve(gm, y0[17:18], env[17:18], wl.dt, wl.rtol, wl.atol, camp.VARIANT_MIXED, True)
    assert np.array_equal(alone[0], ref[17])
    shuffled = np.random.default_rng(1).permutation(200)
    ys, _ = _gpu_solve(gm, y0[shuffled], env[shuffled], wl.dt, wl.rtol, wl.atol, camp.VARIANT_MIXED, True)
    assert np.array_equal(ys, ref[shuffled])


@pytest.mark.parametrize("variant", [camp.VARIANT_FP64, camp.VARIANT_MIXED])
def test_edge_cases(mechs, variant):
    import torch
    wl, gm, om = mechs[2]
    y0, env = wl.inputs(9)
    # non-finite inputs: status 5, state untouched
    y0[2, 5] = np.nan
    env[4, 0] = np.inf
    yg, st = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, variant, False)
    assert st[2] == 5 and st[4] == 5
    assert np.isnan(yg[2, 5]) and np.array_equal(yg[4], y0[4])
    assert (st[[0, 1, 3, 5, 6, 7, 8]] == 0).all()
    # too few steps allowed: status 1, state untouched
    y1, env1 = wl.inputs(5)
    yg, st = _gpu_solve(gm, y1, env1, wl.dt, wl.rtol, wl.atol, variant, False, max_steps=3)
    assert (st == 1).all() and np.array_equal(yg, y1)
    # zero cells
    e = torch.empty((0, gm.n), dtype=torch.float64, device="cuda")
    gm.solve(e, torch.empty((0, gm.n_env), dtype=torch.float64, device="cuda"), wl.dt, wl.rtol, wl.atol,
             variant=variant)
    # per-species atol and a dark cell
    y2, env2 = wl.inputs(4)
    lay = w.layout(wl.mech)
    for k2, kind in enumerate(lay.runtime_kind):
        if kind == "PHOTOLYSIS":
            env2[0, 2 + k2] = 0.0
    atol = np.full(gm.n, wl.atol)
    atol[::3] = 1e-7
    yg, st = _gpu_solve(gm, y2, env2, wl.dt, wl.rtol, atol, variant, False)
    yo, sto, _ = om.solve(y2, env2, wl.dt, wl.rtol, atol)
    assert (st == 0).all()
    parity.check(om, y2, env2, wl.dt, wl.rtol, atol, yg, yo)


def test_dry_sections_freeze_aqueous_species(mechs):
    wl, gm, om = mechs[3]
    y0, env = wl.inputs(6)
    lay = w.layout(wl.mech)
    base = 2 + len(lay.runtime_defaults)
    env[:, base + 2::3] = 0.0  # no water anywhere
    y0[:, 72:] = 0.5
    yg, st = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, camp.VARIANT_MIXED, True)
    assert (st == 0).all()
    assert np.array_equal(yg[:, 72:], y0[:, 72:])


def test_host_entry_point_matches_device_entry_point(mechs):
    wl, gm, om = mechs[2]
    y0, env = wl.inputs(50)
    yd, std = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, camp.VARIANT_MIXED, True)
    yh = y0.copy()
    sth = gm.solve_host(yh, env, wl.dt, wl.rtol, wl.atol, variant=camp.VARIANT_MIXED, persistent=True)
    assert np.array_equal(yh, yd) and np.array_equal(sth, std)


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("variant,share", [(camp.VARIANT_FP64, 0.99), (camp.VARIANT_MIXED, 0.98)],
                         ids=["fp64", "mixed"])
def test_forms_take_the_oracles_step_sequence(mechs, full_oracle, k, variant, share):
    """The same controller: the plain form, with the oracle's FP64
    arithmetic, takes the oracle's step sequence (steps, Newton iterations,
    Jacobian setups, error-test failures) on at least 99% of the cells of
    the full workload (measured: all of them); the mixed form, whose FP32
    iteration matrix perturbs the Newton corrections, on at least 98%
    (measured: 99.7% and 99.8%).  The rest differ where a decision sits on a
    tie within that perturbation."""
    import torch
    wl, gm, om = mechs[k]
    y0, env, _ = full_oracle[k]
    C = len(y0)
    ty = torch.tensor(y0, device="cuda")
    stats = torch.zeros((C, camp.NSTATS), dtype=torch.int32, device="cuda")
    gm.solve(ty, torch.tensor(env, device="cuda"), wl.dt, wl.rtol, wl.atol, variant=variant,
             persistent=variant == camp.VARIANT_MIXED, stats=stats)
    sg = stats.cpu().numpy()
    _, _, so = om.solve(y0, env, wl.dt, wl.rtol, wl.atol)
    same = (sg[:, :4] == so[:, :4]).all(axis=1)
    print(f"workload {k} variant {variant}: identical step sequence on {same.mean():.4f} of cells")
    assert same.mean() >= share
    assert abs(sg[:, 0].mean() / so[:, 0].mean() - 1) < 0.01


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_every_process_type(form):
    """CustomH2o2, CustomOhHno3, CondensedPhaseArrhenius and SIMPOL phase
    transfer beside the other types (Table 2), over dry, hazy and cloudy
    cells."""
    mj = w.process_variety_mechanism()
    text = json.dumps(mj)
    gm, om = camp.Mechanism(text), oracle.Mechanism(text)
    y0, env = w.cells(mj, 150, seed=61)
    y1, env1 = w.cells(mj, 60, seed=62, cloud_fraction=0.5)
    y0, env = np.concatenate([y0, y1]), np.concatenate([env, env1])
    yg, st = _gpu_solve(gm, y0, env, 180.0, 1e-4, 1e-5, *form)
    yo, sto, _ = om.solve(y0, env, 180.0, 1e-4, 1e-5)
    assert (st == 0).all() and (sto == 0).all()
    parity.check(om, y0, env, 180.0, 1e-4, 1e-5, yg, yo)
    n_gas = len(mj["species"])
    assert (yo[:, n_gas:] > 0).any()  # the condensed phase takes part


@pytest.mark.parametrize("variant", [camp.VARIANT_FP64, camp.VARIANT_MIXED])
def test_atol_below_the_fp32_range(cuda, variant):
    """An error weight 1/(rtol |y| + atol) beyond FP32's range (atol 1e-40 on
    a species that starts at zero) must come out as in the oracle."""
    from tests import mechs as M
    text = M.mech(["E", "L", "A", "B"], [M.emission("E", 0.3), M.loss("L", 2e-3),
                                         M.arrhenius({"A": 1, "B": 1}, {"E": 1.0}, A=1e-12)])
    gm, om = camp.Mechanism(text), oracle.Mechanism(text)
    env = np.zeros((3, om.n_env))
    env[:, 0], env[:, 1], env[:, 2], env[:, 3] = 298.0, 1e5, 0.3, 2e-3
    y0 = np.array([[0.0, 4.0, 1.0, 2.0], [0.0, 1.0, 0.0, 0.0], [1e-3, 0.0, 5.0, 5.0]])
    atol = np.array([1e-40, 1e-5, 1e-5, 1e-5])
    yg, st = _gpu_solve(gm, y0, env, 600.0, 1e-4, atol, variant, False)
    yo, sto, _ = om.solve(y0, env, 600.0, 1e-4, atol)
    assert (st == 0).all() and (sto == 0).all()
    parity.check(om, y0, env, 600.0, 1e-4, atol, yg, yo)


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("n_particles,C", [(40, 96), (100, 12), (160, 6)])
def test_particle_resolved_cells(form, n_particles, C):
    """The particle-resolved representation: one condensed-phase instance per
    computational particle (298, 718 and 1138 species), integrated by a block
    of 64, 128 or 256 threads per cell instead of one warp."""
    mj = w.particle_resolved_mechanism(n_particles)
    text = json.dumps(mj)
    gm, om = camp.Mechanism(text), oracle.Mechanism(text)
    y0, env = w.cells(mj, C, seed=71)
    yg, st = _gpu_solve(gm, y0, env, 180.0, 1e-4, 1e-5, *form)
    yo, sto, _ = om.solve(y0, env, 180.0, 1e-4, 1e-5)
    assert (st == 0).all() and (sto == 0).all()
    parity.check(om, y0, env, 180.0, 1e-4, 1e-5, yg, yo)
    assert (yo[:, 18:] > 1e-5).sum() > C  # the particles take part


def _random_tiny_mechanisms():
    """Small random mechanisms (3-13 gas species, some with sections): dense
    blocks of 8-9 or none, few processes per species, every shape corner a
    fixed workload does not reach."""
    out = {}
    for seed in range(6):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(3, 14))
        out[f"tiny{seed}"] = w.gas_mechanism(f"tiny{seed}", n, int(rng.integers(1, n)), int(rng.integers(0, 3)),
                                             int(rng.integers(0, 3)), int(rng.integers(0, 2)),
                                             int(rng.integers(0, 2)), seed=500 + seed, max_occupancy=n)
    out["tiny_aq"] = w.add_aqueous_sections(w.gas_mechanism("t", 6, 3, 1, 1, 1, 1, seed=77, max_occupancy=8),
                                            seed=78, n_sections=2, n_phase_species=5, n_henry=2,
                                            n_split_eq=1, n_simple_eq=1)
    return out


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("name", sorted(_random_tiny_mechanisms()))
def test_random_tiny_mechanisms(form, name):
    mj = _random_tiny_mechanisms()[name]
    text = json.dumps(mj)
    gm, om = camp.Mechanism(text), oracle.Mechanism(text)
    y0, env = w.cells(mj, 40, seed=33)
    yg, st = _gpu_solve(gm, y0, env, 300.0, 1e-4, 1e-5, *form)
    yo, sto, _ = om.solve(y0, env, 300.0, 1e-4, 1e-5)
    # a cell the oracle's controller gives up on (tiny_aq has one: a section
    # with 4e-16 m^3/m^3 of water) may fail on the GPU too, with its state
    # handed back unchanged; every cell the oracle solves must succeed
    ok = sto == 0
    assert ok.mean() > 0.9 and (st[ok] == 0).all()
    assert np.array_equal(yg[st != 0], y0[st != 0])
    parity.check(om, y0[ok], env[ok], 300.0, 1e-4, 1e-5, yg[ok], yo[ok])


@pytest.fixture(scope="module")
def water_oracle():
    """The oracle on every cell of the 240-species water workload, once."""
    wl = w.workload(7)
    om = oracle.Mechanism(wl.json())
    y0, env = wl.inputs()
    yo, sto, _ = om.solve(y0, env, wl.dt, wl.rtol, wl.atol)
    assert (sto == 0).all()
    return wl, om, y0, env, yo


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_water_parameter_workload(cuda, water_oracle, form):
    """Aerosol water as a parameter of the state (Sect. 2.2.2): the
    240-species workload whose section water is held by a salt and by the
    species that Henry's-law uptake feeds.  The full workload in one launch;
    every cell (4096) under the parity rule and the arbiter."""
    wl, om, y0, env, yo = water_oracle
    gm = camp.Mechanism(wl.json())
    yg, st = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, *form)
    assert (st == 0).all()
    stats = parity.check(om, y0, env, wl.dt, wl.rtol, wl.atol, yg, yo)
    print(f"water workload {form}: {stats}")
    idx = np.random.default_rng(7).choice(wl.n_cells, 48, replace=False)
    # the water follows the state
    dL = [np.max(np.abs(om.water(env[c], yg[c]) / om.water(env[c], y0[c]) - 1)) for c in idx]
    assert max(dL) > 1e-4


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_water_parameter_every_section_type(form):
    """Henry's law, SIMPOL, aqueous equilibria and condensed-phase reactions
    in sections whose water comes from three electrolytes, two of which the
    reactions make or consume (the chain-rule Jacobian of every kind)."""
    from tests import mechs as M
    text = M.water_chain_mechanism()
    gm, om = camp.Mechanism(text), oracle.Mechanism(text)
    C = 77
    rng = np.random.default_rng(81)
    y0 = rng.uniform(0.2, 5.0, (C, om.n))
    env = np.zeros((C, om.n_env))
    env[:, 0] = rng.uniform(260.0, 310.0, C)
    env[:, 1] = rng.uniform(5e4, 1.013e5, C)
    env[:, om.m.rh_slot] = rng.uniform(0.3, 0.97, C)
    base = om.m.env_section_base
    env[:, base:base + 3] = np.column_stack([np.full(C, 2e-7), np.full(C, 1e9), np.zeros(C)])
    env[:, base + 3:base + 6] = np.column_stack([np.full(C, 1e-6), np.full(C, 1e8),
                                                 10 ** rng.uniform(-13, -11, C)])
    yg, st = _gpu_solve(gm, y0, env, 120.0, 1e-4, 1e-5, *form)
    yo, sto, _ = om.solve(y0, env, 120.0, 1e-4, 1e-5)
    # the first steps of these far-from-equilibrium cells are violent: the
    # oracle's controller gives up on one of them at rtol 1e-4 (it solves at
    # 1e-6); a cell may then fail on the GPU too, with its state unchanged
    ok = sto == 0
    assert ok.mean() > 0.95 and (st[ok] == 0).all()
    assert np.array_equal(yg[st != 0], y0[st != 0])
    parity.check(om, y0[ok], env[ok], 120.0, 1e-4, 1e-5, yg[ok], yo[ok])


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("n_particles,C", [(40, 48), (100, 8), (160, 4)])
def test_water_parameter_on_block_cells(form, n_particles, C):
    """The water builds of the block shapes (64, 128 and 256 threads per
    cell: 338, 818 and 1298 species): particles whose water is held by a
    salt and by the sulphate their chemistry makes."""
    from tests import mechs as M
    mj = M.water_particles_mechanism(n_particles)
    text = json.dumps(mj)
    gm, om = camp.Mechanism(text), oracle.Mechanism(text)
    y0, env = w.cells(mj, C, seed=73)
    yg, st = _gpu_solve(gm, y0, env, 180.0, 1e-4, 1e-5, *form)
    yo, sto, _ = om.solve(y0, env, 180.0, 1e-4, 1e-5)
    assert (st == 0).all() and (sto == 0).all()
    parity.check(om, y0, env, 180.0, 1e-4, 1e-5, yg, yo)


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_water_parameter_dry_sections(form):
    """Sections whose electrolytes hold no water take no part (the reading
    used for a section with no water in env); here every other cell has two
    such sections."""
    wl = w.workload(7)
    gm, om = camp.Mechanism(wl.json()), oracle.Mechanism(wl.json())
    y0, env = wl.inputs(96)
    lay = w.layout(wl.mech)
    for b in (0, 3):
        for e in wl.mech["parameters"][0]["electrolytes"]:
            y0[::2, lay.species.index(f"bin{b}.{e['species']}")] = 0.0
    assert om.water(env[0], y0[0])[0] == 0.0
    yg, st = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, *form)
    yo, sto, _ = om.solve(y0, env, wl.dt, wl.rtol, wl.atol)
    assert (st == 0).all() and (sto == 0).all()
    parity.check(om, y0, env, wl.dt, wl.rtol, wl.atol, yg, yo)
    dry = [lay.species.index(s) for s in lay.species if s.startswith("bin0.")]
    assert np.array_equal(yg[::2][:, dry], y0[::2][:, dry])


@pytest.mark.parametrize("variant,tol", [(camp.VARIANT_FP64, 1e-10), (camp.VARIANT_MIXED, 1e-5)],
                         ids=["fp64", "mixed"])
def test_linear_invariant_is_conserved(variant, tol):
    """With emission and loss off, the chemistry conserves an integer atom
    count per species, and BDF with Newton keeps linear invariants up to the
    Newton residual: FP64 to 1e-10 relative, the mixed form (FP32 iteration
    matrix) to 0.1 rtol."""
    wl = w.workload(3)
    lay = w.layout(wl.mech)
    gm = camp.Mechanism(wl.json())
    y0, env = wl.inputs(512)
    for k, kind in enumerate(lay.runtime_kind):
        if kind in ("EMISSION", "FIRST_ORDER_LOSS"):
            env[:, 2 + k] = 0.0
    yg, st = _gpu_solve(gm, y0, env, wl.dt, wl.rtol, wl.atol, variant, variant == camp.VARIANT_MIXED)
    assert (st == 0).all()
    w0, w1 = y0 @ lay.atoms, yg @ lay.atoms
    assert np.max(np.abs(w1 / w0 - 1)) < tol
