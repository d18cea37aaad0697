"""The seeded input generator (no GPU)."""
import json

import numpy as np

from paper_2111_07436_gb300 import workloads as w


def test_deterministic():
    for k in (1, 2, 3):
        a, b = w.workload(k), w.workload(k)
        assert a.json() == b.json()
        ya, ea = a.inputs(8)
        yb, eb = b.inputs(8)
        assert np.array_equal(ya, yb) and np.array_equal(ea, eb)


def test_large_gas_mechanism_shape():
    m = w.large_gas_mechanism()
    types = [r["type"] for r in m["reactions"]]
    assert len(m["species"]) == 72 and len(types) == 186
    assert (types.count("ARRHENIUS"), types.count("TROE"), types.count("PHOTOLYSIS"),
            types.count("EMISSION"), types.count("FIRST_ORDER_LOSS")) == (112, 28, 28, 9, 9)
    occ = {s["name"]: 0 for s in m["species"]}
    for r in m["reactions"]:
        names = set(r.get("reactants", {})) | set(r.get("products", {}))
        if "species" in r:
            names.add(r["species"])
        for s in names:
            occ[s] += 1
    assert max(occ.values()) <= 12


def test_chemistry_conserves_atoms():
    for mj in (w.small_gas_mechanism(), w.multiphase_mechanism()):
        lay = w.layout(mj)
        atoms = dict(zip(lay.species, lay.atoms))
        phase_atoms = {p["name"]: p["atoms"] for p in mj.get("phases", {}).get("aqueous", [])}
        for r in mj["reactions"]:
            t = r["type"]
            if t in ("ARRHENIUS", "TROE", "PHOTOLYSIS"):
                lhs = sum(atoms[s] * c for s, c in r["reactants"].items())
                rhs = sum(atoms[s] * c for s, c in r["products"].items())
                assert abs(lhs - rhs) < 1e-12
            elif t == "AQUEOUS_REVERSIBLE":
                lhs = sum(phase_atoms[s] * c for s, c in r["reactants"].items())
                rhs = sum(phase_atoms[s] * c for s, c in r["products"].items())
                assert lhs == rhs
            elif t == "HL_PHASE_TRANSFER":
                assert atoms[r["gas"]] == phase_atoms[r["aqueous"]]


def test_multiphase_sizes_and_env():
    mj = w.multiphase_mechanism()
    lay = w.layout(mj)
    assert len(lay.species) == 232
    y, env = w.cells(mj, 16, seed=5)
    assert env.shape == (16, len(lay.env)) and (y[:, 72:] == 0).all()
    base = 2 + len(lay.runtime_defaults)
    r = env[:, base::3]
    np.testing.assert_allclose(r[0], w.SECTION_RADII)
    N, L = env[:, base + 1::3], env[:, base + 2::3]
    np.testing.assert_allclose(L, N * 4.0 / 3.0 * np.pi * r ** 3)
    assert ((N >= 1e7) & (N <= 1e10)).all()


def test_night_and_cloud_options():
    mj = w.multiphase_mechanism()
    lay = w.layout(mj)
    y, env = w.cells(mj, 2000, seed=6, night_fraction=0.5, cloud_fraction=0.1)
    jcols = [2 + k for k, kind in enumerate(lay.runtime_kind) if kind == "PHOTOLYSIS"]
    night = (env[:, jcols] == 0).all(axis=1)
    assert 0.4 < night.mean() < 0.7  # half forced dark plus SZA > 90 deg
    base = 2 + len(lay.runtime_defaults)
    lwc = env[:, base + 2::3].sum(axis=1)
    cloudy = lwc > 0
    assert 0.07 < cloudy.mean() < 0.13
    assert ((lwc[cloudy] >= 1e-7) & (lwc[cloudy] <= 1e-6 + 1e-18)).all()
    json.dumps(mj)


def test_process_variety_mechanism_holds_every_process_type():
    mj = w.process_variety_mechanism()
    types = {r["type"] for r in mj["reactions"]}
    assert types == {"ARRHENIUS", "TROE", "PHOTOLYSIS", "EMISSION", "FIRST_ORDER_LOSS",
                     "HL_PHASE_TRANSFER", "AQUEOUS_REVERSIBLE", "CUSTOM_H2O2", "CUSTOM_OH_HNO3",
                     "CONDENSED_ARRHENIUS", "SIMPOL_PHASE_TRANSFER"}
    assert json.dumps(mj) == json.dumps(w.process_variety_mechanism())
    lay = w.layout(mj)
    assert len(lay.species) == 18 + 4 * 7


def test_particle_resolved_inputs():
    mj = w.particle_resolved_mechanism(64)
    lay = w.layout(mj)
    assert len(lay.species) == 18 + 64 * 7 and lay.n_sections == 64
    y, env = w.cells(mj, 50, seed=3)
    base = 2 + len(lay.runtime_defaults)
    r, N, L = env[:, base::3], env[:, base + 1::3], env[:, base + 2::3]
    assert r.shape == (50, 64) and ((r >= 5e-9) & (r <= 1e-5)).all()
    assert 3e-8 < np.exp(np.log(r).mean()) < 3e-7               # log-normal around 0.1 um
    assert np.allclose(N, N[:, :1]) and ((N.sum(axis=1) >= 1e8) & (N.sum(axis=1) <= 1e10)).all()
    np.testing.assert_allclose(L, N * 4.0 / 3.0 * np.pi * r ** 3)
    assert (y[:, 18:] == 0).all()


def test_process_variety_isoprene_chemistry_is_table9():
    """The isoprene oxidation and SOA partitioning of the process-variety
    mechanism carry the paper's printed values (Table 9, tests/golden)."""
    from tests.golden.load import isoprene_soa_table9
    t9 = isoprene_soa_table9()
    mj = w.process_variety_mechanism()
    name = {"ISOP-P1": "ISOPP1", "ISOP-P2": "ISOPP2"}
    gas = [r for r in mj["reactions"] if r["type"] == "ARRHENIUS" and "ISOP" in r["reactants"]]
    assert len(gas) == len(t9["gas"])
    for reactants, products, A, C in t9["gas"].values():
        r = next(r for r in gas if r["reactants"] == reactants)
        assert r["products"] == {name[k]: v for k, v in products.items()}
        assert (r["A"], r["C"], r["B"], r["E"]) == (A, C, 0.0, 0.0)
    simpol = {r["gas"]: r for r in mj["reactions"] if r["type"] == "SIMPOL_PHASE_TRANSFER"}
    for g, aero, B in t9["partition"].values():
        assert simpol[name[g]]["aqueous"] == aero
        assert tuple(simpol[name[g]]["B"]) == B


def test_water_mechanism_inputs():
    mj = w.water_mechanism()
    lay = w.layout(mj)
    assert len(lay.species) == 240 and "RH" in lay.env
    y, env = w.cells(mj, 64, seed=5)
    rh = env[:, lay.env.index("RH")]
    assert ((rh >= 0.5) & (rh <= 0.95)).all()
    base = lay.env.index("bin0.r")
    assert (env[:, base + 2::3] == 0.0).all()          # all water from the electrolytes
    salt = y[:, [lay.species.index(f"bin{b}.SALT") for b in range(8)]]
    r, N = env[:, base::3], env[:, base + 1::3]
    assert np.allclose(salt / (N * r ** 3), salt[0, 0] / (N[0, 0] * r[0, 0] ** 3) *
                       (env[0, 1] / env[0, 0]) / (env[:, 1:2] / env[:, 0:1]), rtol=1e-12)
