"""The block-arrow solve of particle-resolved cells (Sect. 2.2.3 and Table 6;
10^4 computational particles in the box model of Sect. 4.1), through the C
ABI: one cell per thread-block cluster, each particle's block eliminated
into the gas block.  Against the oracle up to 512 particles (3602 species);
at the paper's 10^4 particles (70018 species), where the dense oracle is out
of reach, the forcing against the oracle's, the exact symmetry of identical
particles against a one-particle oracle run, and agreement across launch
shapes."""
import json
import math

import numpy as np
import pytest

import oracle
from paper_2111_07436_gb300 import camp, workloads as w
from tests import parity

pytestmark = pytest.mark.gpu

VARIANTS = [camp.VARIANT_FP64, camp.VARIANT_MIXED]
VARIANT_IDS = ["fp64", "mixed"]


def _arrow(P):
    """The particle-resolved mechanism in the block-arrow form."""
    mj = w.particle_resolved_mechanism(P)
    mj["aerosol"]["solver"] = "block_arrow"
    return mj


def _solve(gm, y, env, variant, dt=180.0, **kw):
    import torch
    ty = torch.tensor(y, device="cuda")
    st = gm.solve(ty, torch.tensor(env, device="cuda"), dt, 1e-4, 1e-5, variant=variant, **kw)
    torch.cuda.synchronize()
    return ty.cpu().numpy(), st.cpu().numpy()


_ORACLE = {}


def _oracle_run(P, C):
    """The oracle on C cells of the P-particle mechanism, once per module."""
    if (P, C) not in _ORACLE:
        mj = _arrow(P)
        om = oracle.Mechanism(json.dumps(mj))
        y0, env = w.cells(mj, C, seed=71)
        yo, so, sto = om.solve(y0, env, 180.0, 1e-4, 1e-5)
        assert (so == 0).all()
        _ORACLE[(P, C)] = (mj, om, y0, env, yo, sto)
    return _ORACLE[(P, C)]


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
@pytest.mark.parametrize("P,C,cl", [(40, 48, 0), (100, 16, 0), (512, 2, 0), (512, 2, 1), (1024, 1, 1)],
                         ids=["40", "100", "512", "512-cluster1", "1024-cluster1"])
def test_block_arrow_matches_the_oracle(cuda, P, C, cl, variant):
    """Every cell under the parity rule and the arbiter; the FP64 form also
    takes the oracle's step sequence on every cell.  With one CTA (256
    threads) per cluster, 512 and 1024 particles put two and four particles
    on every thread, as the paper's 10^4 particles do on the default
    clusters."""
    import torch
    mj, om, y0, env, yo, sto = _oracle_run(P, C)
    gm = camp.Mechanism(json.dumps(mj))
    assert gm.n == 18 + 7 * P
    stats = torch.zeros((C, camp.NSTATS), dtype=torch.int32, device="cuda")
    yg, st = _solve(gm, y0, env, variant, stats=stats, cells_per_block=cl)
    assert (st == 0).all()
    stats_ = parity.check(om, y0, env, 180.0, 1e-4, 1e-5, yg, yo)
    same = (stats.cpu().numpy()[:, :4] == sto).all(axis=1)
    print(f"{P} particles, cluster {cl}, variant {variant}: {stats_}, same step sequence on {same.mean():.3f}")
    if variant == camp.VARIANT_FP64:
        assert same.all()
    assert (yo[:, 18:] > 1e-5).sum() > C  # the particles take part


def test_block_arrow_equals_itself_alone_and_in_a_batch(cuda):
    """A cell's result does not depend on the other cells of the launch."""
    mj = _arrow(200)
    gm = camp.Mechanism(json.dumps(mj))
    y0, env = w.cells(mj, 40, seed=5)
    ref, _ = _solve(gm, y0, env, camp.VARIANT_MIXED)
    alone, _ = _solve(gm, y0[7:8], env[7:8], camp.VARIANT_MIXED)
    assert np.array_equal(alone[0], ref[7])
    perm = np.random.default_rng(2).permutation(40)
    ys, _ = _solve(gm, y0[perm], env[perm], camp.VARIANT_MIXED)
    assert np.array_equal(ys, ref[perm])


def test_forcing_at_the_papers_particle_count(cuda):
    """f(y) of 10^4-particle cells (70018 species) against the oracle's
    forcing, at a state with every phase species present, to 1e-12 of each
    cell's largest rate."""
    import torch
    mj = _arrow(10000)
    gm, om = camp.Mechanism(json.dumps(mj)), oracle.Mechanism(json.dumps(mj))
    y0, env = w.cells(mj, 3, seed=9)
    y0[:, 18:] = np.random.default_rng(3).uniform(1e-3, 1.0, y0[:, 18:].shape)
    fg = gm.forcing(torch.tensor(y0, device="cuda"), torch.tensor(env, device="cuda")).cpu().numpy()
    for c in range(3):
        kf, kr = om.rate_constants(env[c])
        fo = om.forcing(kf, kr, y0[c])
        assert np.max(np.abs(fg[c] - fo)) <= 1e-12 * np.max(np.abs(fo))


def _identical_particles(P, C, seed):
    """Cells of P identical particles and the same cells as one particle
    holding all of them: the particles' number concentrations add up, and
    at any time each of the P particles holds 1/P of the one particle's
    species (the rate laws are linear in the number concentration, and the
    molarities -- hence the condensed-phase rates per unit volume -- agree)."""
    mj = _arrow(P)
    m1 = w.particle_resolved_mechanism(1)
    y1, env1 = w.cells(m1, C, seed=seed)
    lay, lay1 = w.layout(mj), w.layout(m1)
    E0 = len(lay.env) - 3 * P
    assert E0 == len(lay1.env) - 3
    env = np.zeros((C, len(lay.env)))
    env[:, :E0] = env1[:, :E0]
    r, N = env1[:, E0], env1[:, E0 + 1]
    env[:, E0::3] = r[:, None]
    env[:, E0 + 1::3] = (N / P)[:, None]
    env[:, E0 + 2::3] = ((N / P) * 4.0 / 3.0 * math.pi * r ** 3)[:, None]
    env1[:, E0 + 2] = N * 4.0 / 3.0 * math.pi * r ** 3
    y = np.zeros((C, len(lay.species)))
    y[:, :18] = y1[:, :18]
    y1[:, 18:] = np.random.default_rng(seed).uniform(0.0, 1.0, (C, 7))
    y[:, 18:] = np.tile(y1[:, 18:] / P, P)
    return mj, y, env, m1, y1, env1


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
def test_identical_particles_at_the_papers_particle_count(cuda, variant):
    """10^4 identical particles: every particle ends bit-identical to the
    others, and (gas, P x particle) matches the one-particle system's true
    solution (a tight oracle run) within the integrator's own accuracy.  The
    error of each integration is measured in its own tolerance units
    (|y - y_true| / (rtol |y_true| + atol) over its own species: a particle
    of the large system against y_true / P, the one particle against
    y_true).  The particles' error is within twice the one-particle oracle's
    error at the same tolerance or within that oracle's largest over these
    cells.  The gas species get sqrt(n / n_1) times that: the error test is a
    root mean square over all n = 70018 species, so at the acceptance
    threshold one gas species may carry sqrt(n / n_1) times the error it may
    carry among the n_1 = 25 species of the one-particle system."""
    P, C = 10000, 6
    mj, y, env, m1, y1, env1 = _identical_particles(P, C, seed=11)
    gm = camp.Mechanism(json.dumps(mj))
    yg, st = _solve(gm, y, env, variant)
    assert (st == 0).all()
    parts = yg[:, 18:].reshape(C, P, 7)
    assert (parts == parts[:, :1, :]).all()
    om1 = oracle.Mechanism(json.dumps(m1))
    yo, so, _ = om1.solve(y1, env1, 180.0, 1e-4, 1e-5)
    yt = parity.tight_solution(om1, y1, env1, 180.0)
    assert (so == 0).all()
    Eo = parity.tol_units(yo, yt, 1e-4, 1e-5)
    bound = np.maximum(2 * Eo, Eo.max())
    Eg_gas = parity.tol_units(yg[:, :18], yt[:, :18], 1e-4, 1e-5)
    Eg_part = parity.tol_units(parts[:, 0, :], yt[:, 18:] / P, 1e-4, 1e-5)
    dilution = math.sqrt(gm.n / (18 + 7))
    print(f"variant {variant}: error vs truth (tolerance units) particles {Eg_part}, gas {Eg_gas}, "
          f"one-particle oracle {Eo}, gas allowance x{dilution:.1f}")
    assert (Eg_part <= bound).all()
    assert (Eg_gas <= dilution * bound).all()


def test_launch_shapes_agree_at_the_papers_particle_count(cuda):
    """10^4-particle cells on clusters of 4, 8 and 16 CTAs (10, 5 and 2-3
    particles a thread, different orders of the particle sums): the FP64
    form's results agree to roundoff under the parity rule."""
    mj = _arrow(10000)
    gm = camp.Mechanism(json.dumps(mj))
    y0, env = w.cells(mj, 3, seed=13)
    ref, st = _solve(gm, y0, env, camp.VARIANT_FP64, cells_per_block=8)
    assert (st == 0).all()
    for cl in (4, 16):
        yg, st = _solve(gm, y0, env, camp.VARIANT_FP64, cells_per_block=cl)
        assert (st == 0).all()
        assert not parity.violations(yg, ref, 1e-5).any()
        big = np.abs(ref) > 1e-5
        assert np.max(np.abs(yg - ref)[big] / np.abs(ref)[big]) < 1e-9


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
def test_block_arrow_edge_cases_and_sequence(cuda, variant):
    """Non-finite input: status 5, state untouched; too few steps: status 1;
    two outer steps in one launch equal two launches bit for bit; warm start
    carries the step."""
    import torch
    mj = _arrow(64)
    gm = camp.Mechanism(json.dumps(mj))
    y0, env = w.cells(mj, 6, seed=17)
    y0[1, 30] = np.nan
    env[3, 0] = np.inf
    yg, st = _solve(gm, y0, env, variant)
    assert st[1] == 5 and st[3] == 5 and (st[[0, 2, 4, 5]] == 0).all()
    assert np.array_equal(yg[3], y0[3]) and np.isnan(yg[1, 30])
    y1, env1 = w.cells(mj, 3, seed=18)
    yg, st = _solve(gm, y1, env1, variant, max_steps=2)
    assert (st == 1).all() and np.array_equal(yg, y1)
    ty = torch.tensor(y1, device="cuda")
    traj = torch.zeros((2, 3, gm.n), dtype=torch.float64, device="cuda")
    st = gm.solve_sequence(ty, torch.tensor(env1, device="cuda"), 180.0, 2, 1e-4, 1e-5, trajectory=traj,
                           variant=variant)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    ya, _ = _solve(gm, y1, env1, variant)
    yb, _ = _solve(gm, ya, env1, variant)
    assert np.array_equal(traj[0].cpu().numpy(), ya) and np.array_equal(traj[1].cpu().numpy(), yb)
    hs = torch.zeros(3, dtype=torch.float64, device="cuda")
    t2 = torch.tensor(y1, device="cuda")
    gm.solve(t2, torch.tensor(env1, device="cuda"), 180.0, 1e-4, 1e-5, variant=variant, step=hs)
    torch.cuda.synchronize()
    assert (hs.cpu().numpy() > 0).all()
    om = oracle.Mechanism(json.dumps(mj))
    hso = np.zeros(3)
    om.solve(y1, env1, 180.0, 1e-4, 1e-5, step=hso)
    if variant == camp.VARIANT_FP64:  # the same step sequence, hence the same carried step
        assert np.allclose(hs.cpu().numpy(), hso, rtol=1e-9)


def test_autotune_picks_a_cluster_size(cuda):
    """camp_autotune on a block-arrow mechanism times clusters of 2, 4, 8 and
    16 CTAs; later solves with the default launch use the choice (the same
    bits as naming it)."""
    import torch
    mj = _arrow(2000)
    gm = camp.Mechanism(json.dumps(mj))
    y0, env = w.cells(mj, 12, seed=21)
    ty, te = torch.tensor(y0, device="cuda"), torch.tensor(env, device="cuda")
    cl, pers, ms = gm.autotune(ty, te, 180.0, 1e-4, 1e-5)
    assert cl in (2, 4, 8, 16) and pers == 1 and ms > 0
    assert np.array_equal(ty.cpu().numpy(), y0)  # the cells are left unchanged
    a, _ = _solve(gm, y0, env, camp.VARIANT_MIXED)
    b, _ = _solve(gm, y0, env, camp.VARIANT_MIXED, cells_per_block=cl)
    assert np.array_equal(a, b)
