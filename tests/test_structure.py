"""Integer structure (no GPU): the oracle's enumeration against brute force,
and the product's mechanism compiler against the oracle, bit for bit.

The structure is what CAMP's processes declare during initialisation
(Table 1: get_used_jacobian_elements, update_ids) plus the ordering and fill
of the sparse LU that replaces KLU (Sect. 2.4.1)."""
import json

import numpy as np
import pytest

import oracle
from oracle import structure as S
from paper_2111_07436_gb300 import workloads as w


def _mechs():
    out = {"small": w.small_gas_mechanism(), "gas72": w.large_gas_mechanism(),
           "multiphase232": w.multiphase_mechanism(), "multiphase168": w.small_multiphase_mechanism()}
    for seed in range(6):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(3, 14))
        out[f"tiny{seed}"] = w.gas_mechanism(f"tiny{seed}", n, int(rng.integers(1, n)), int(rng.integers(0, 3)),
                                             int(rng.integers(0, 3)), int(rng.integers(0, 2)),
                                             int(rng.integers(0, 2)), seed=500 + seed, max_occupancy=n)
    out["tiny_aq"] = w.add_aqueous_sections(w.gas_mechanism("t", 6, 3, 1, 1, 1, 1, seed=77, max_occupancy=8),
                                            seed=78, n_sections=2, n_phase_species=5, n_henry=2,
                                            n_split_eq=1, n_simple_eq=1)
    out["variety"] = w.process_variety_mechanism()
    out["particles40"] = w.particle_resolved_mechanism(40)
    out["variety_1sec"] = w.process_variety_mechanism(seed=9, n_sections=1)
    out["water"] = w.water_mechanism()
    tw = json.loads(json.dumps(out["tiny_aq"]))  # a water parameter over two phase species
    tw["parameters"] = [{"type": "ZSR_AEROSOL_WATER",
                         "electrolytes": [{"species": "a3", "Y": [3.0, -2.0]},
                                          {"species": "a1", "Y": [2.5, -1.0, -0.5], "low_RH": 0.4}]}]
    out["tiny_aq_water"] = tw
    from tests import mechs as M
    out["water_particles40"] = M.water_particles_mechanism(40)
    return out


MECHS = _mechs()


@pytest.mark.parametrize("name", sorted(MECHS))
def test_pattern_is_the_numeric_jacobian_support(name):
    mj = MECHS[name]
    m = oracle.Mechanism(json.dumps(mj))
    st = m.structure()
    pat = {(i, st["colidx"][q]) for i in range(m.n) for q in range(st["rowptr"][i], st["rowptr"][i + 1])}
    y, env = w.cells(mj, 1, seed=3)
    y = np.random.default_rng(1).uniform(0.5, 2.0, m.n)   # generic positive state
    if mj.get("aerosol"):
        env[0, m.m.env_section_base + 2::3] = 1e-7         # every section holds water
    kf, kr = m.rate_constants(env[0])
    J = m.jacobian(kf, kr, y, env[0])
    nz = {(i, j) for i, j in zip(*np.nonzero(J))}
    assert nz <= pat
    off = {(i, j) for (i, j) in pat if i != j}
    assert off <= nz  # generated mechanisms have no net-zero coefficients
    # the rxn map points at the right (row, column)
    rowof = np.repeat(np.arange(m.n), np.diff(st["rowptr"]))
    k = 0
    for p in m.m.processes:
        for j in S.dependence(p):
            for i in S.rows_of(p):
                q = st["rxn_map"][k]
                assert rowof[q] == i and st["colidx"][q] == j
                k += 1
    assert k == len(st["rxn_map"])


@pytest.mark.parametrize("name", sorted(MECHS))
def test_fill_is_the_numeric_lu_support(name):
    mj = MECHS[name]
    m = oracle.Mechanism(json.dumps(mj))
    st = m.structure()
    n, perm = m.n, st["perm"]
    assert sorted(perm) == list(range(n))
    A = np.zeros((n, n))
    rng = np.random.default_rng(2)
    for i in range(n):
        for q in range(st["rowptr"][i], st["rowptr"][i + 1]):
            A[i, st["colidx"][q]] = rng.uniform(0.1, 1.0)
    A[np.arange(n), np.arange(n)] = n + 1.0  # diagonally dominant: no pivoting needed
    P = A[np.ix_(perm, perm)]
    for k in range(n):  # plain Gaussian elimination without pivoting
        P[k + 1:, k] /= P[k, k]
        P[k + 1:, k + 1:] -= np.outer(P[k + 1:, k], P[k, k + 1:])
    nz = {(i, j) for i, j in zip(*np.nonzero(P))}
    lu = {(i, st["lu_colidx"][q]) for i in range(n) for q in range(st["lu_rowptr"][i], st["lu_rowptr"][i + 1])}
    assert nz == lu


@pytest.mark.parametrize("name", sorted(MECHS))
def test_ordering_is_minimum_degree(name):
    """In the symmetric fill graph, the elimination graph after k steps is the
    filled graph on the remaining vertices; each chosen vertex must have the
    smallest degree there, ties to the smallest species index."""
    mj = MECHS[name]
    m = oracle.Mechanism(json.dumps(mj))
    st = m.structure()
    n, perm = m.n, st["perm"]
    iperm = np.argsort(perm)
    G = np.zeros((n, n), dtype=bool)
    for i in range(n):
        for q in range(st["rowptr"][i], st["rowptr"][i + 1]):
            j = st["colidx"][q]
            if i != j:
                G[iperm[i], iperm[j]] = G[iperm[j], iperm[i]] = True
    for k in range(n):  # symmetric symbolic elimination
        nb = np.nonzero(G[k, k + 1:])[0] + k + 1
        G[np.ix_(nb, nb)] = True
    np.fill_diagonal(G, False)
    for k in range(n):
        rem = np.arange(k, n)
        deg = G[np.ix_(rem, rem)].sum(axis=1)
        best = min(range(len(rem)), key=lambda a: (deg[a], perm[rem[a]]))
        assert best == 0


@pytest.mark.parametrize("name", sorted(MECHS))
def test_levels_respect_dependencies(name):
    m = oracle.Mechanism(json.dumps(MECHS[name]))
    st = m.structure()
    fwd, bwd = st["level_fwd"], st["level_bwd"]
    for i in range(m.n):
        row = st["lu_colidx"][st["lu_rowptr"][i]:st["lu_rowptr"][i + 1]]
        low = [fwd[k] for k in row if k < i]
        high = [bwd[j] for j in row if j > i]
        assert fwd[i] == (max(low) + 1 if low else 0)
        assert bwd[i] == (max(high) + 1 if high else 0)


@pytest.mark.parametrize("name", sorted(MECHS))
def test_compiler_matches_oracle_bit_exact(name):
    from paper_2111_07436_gb300 import camp
    text = json.dumps(MECHS[name])
    got = camp.Mechanism(text, device=False).structure()
    want = oracle.Mechanism(text).structure()
    for key, v in want.items():
        assert np.array_equal(got[key], np.asarray(v, dtype=np.int32)), key


def test_compiler_rejects_malformed_input():
    from paper_2111_07436_gb300 import camp
    for bad in ("", "{", '{"species": []}', '{"species": [{"name": "A"}], "reactions": [{"type": "NOPE"}]}',
                '{"species": [{"name": "A"}], "reactions": [{"type": "FIRST_ORDER_LOSS", "species": "B"}]}',
                '{"species": [{"name": "A"}, {"name": "A"}], "reactions": []}'):
        with pytest.raises(camp.CampError):
            camp.Mechanism(bad, device=False)


@pytest.mark.parametrize("seed", range(8))
def test_random_water_mechanisms_compile_bit_exact(seed):
    """Random small sectional mechanisms with a water parameter over random
    electrolytes: the compiler's tables pass its own bounds checks (loading
    raises otherwise) and its structure equals the oracle's enumeration."""
    from paper_2111_07436_gb300 import camp
    rng = np.random.default_rng(600 + seed)
    n_gas = int(rng.integers(6, 10))
    mj = w.add_aqueous_sections(
        w.gas_mechanism(f"rw{seed}", n_gas, int(rng.integers(2, n_gas)), 1, 1, 1, 1, seed=700 + seed,
                        max_occupancy=3 * n_gas),
        seed=800 + seed, n_sections=int(rng.integers(1, 4)), n_phase_species=6, n_henry=2,
        n_split_eq=1, n_simple_eq=1)
    phase = [p["name"] for p in mj["phases"]["aqueous"]]
    chosen = rng.choice(phase, int(rng.integers(1, 4)), replace=False)
    mj["parameters"] = [{"type": "ZSR_AEROSOL_WATER", "electrolytes": [
        {"species": str(e), "Y": [float(rng.uniform(2, 4)), float(rng.uniform(-2, -0.5))]} for e in chosen]}]
    text = json.dumps(mj)
    got = camp.Mechanism(text, device=False).structure()
    want = oracle.Mechanism(text).structure()
    for key, v in want.items():
        assert np.array_equal(got[key], np.asarray(v, dtype=np.int32)), key
