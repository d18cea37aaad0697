"""The C ABI library builds, loads and exports every declared entry point
(no GPU: nothing here launches a kernel)."""
import ctypes
import json
import os
import re

import pytest

from paper_2111_07436_gb300 import build, camp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    text = open(os.path.join(ROOT, "include", "camp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(camp_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "camp_solve" in names and "camp_mech_load" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(declared()) <= set(camp.EXPORTS)


def test_host_only_handle_refuses_to_solve():
    from paper_2111_07436_gb300 import workloads as w
    m = camp.Mechanism(w.workload(1).json(), device=False)
    assert m.info.n_species == 8 and m.info.n_env == 7
    assert m.species_index("B") == 1 and m.species_index("nope") == -1
    L = camp.lib()
    o = camp.SolveOpts()
    L.camp_solve_opts_default(ctypes.byref(o), camp.VARIANT_MIXED)
    fake = ctypes.c_void_p(16)  # never dereferenced: the handle is rejected first
    rc = L.camp_solve(m._h, 4, fake, fake, 10.0, 1e-4, fake, 1, fake, ctypes.byref(o), None)
    assert rc == -1 and b"without device tables" in L.camp_last_error()
    rc = L.camp_solve(m._h, 4, fake, fake, -1.0, 1e-4, fake, 1, fake, ctypes.byref(o), None)
    assert rc == -1 and b"dt" in L.camp_last_error()
    rc = L.camp_solve(m._h, 4, fake, fake, 1.0, 1e-4, fake, 3, fake, ctypes.byref(o), None)
    assert rc == -1 and b"atol_len" in L.camp_last_error()
    assert L.camp_solve(m._h, 0, None, None, 1.0, 1e-4, None, 1, None, None, None) == 0
    with pytest.raises(camp.CampError):  # no device tables to rebuild
        m.set_lanes(64)
    assert m.info.lanes_per_cell == 32


def test_info_reports_the_cell_shape():
    """Lanes a cell by species count: one warp up to 192, 64 threads up to
    512, 128 up to 1024; the block-arrow form reports none."""
    from paper_2111_07436_gb300 import workloads as w
    for k, lanes in ((1, 32), (2, 32), (3, 64), (7, 64), (6, 128)):
        assert camp.Mechanism(w.workload(k).json(), device=False).info.lanes_per_cell == lanes, k
    big = camp.Mechanism(json.dumps(w.particle_resolved_mechanism(10000)), device=False)
    assert big.info.lanes_per_cell == 0


def test_info_reports_the_dense_block():
    from paper_2111_07436_gb300 import workloads as w
    inf = camp.Mechanism(w.workload(2).json(), device=False).info
    assert inf.n_species == 72 and inf.n_rxn == 186 and inf.n_env == 48
    assert 0 < inf.dense_block <= 72 and inf.nnz_lu >= inf.nnz_jac
    assert inf.smem_per_cell_fp64 > inf.smem_per_cell_mixed
    assert inf.env_rh == -1 and inf.n_electrolytes == 0


def test_info_reports_the_water_parameter():
    from paper_2111_07436_gb300 import workloads as w
    mj = w.water_mechanism()
    inf = camp.Mechanism(json.dumps(mj), device=False).info
    lay = w.layout(mj)
    assert inf.n_electrolytes == 2 and inf.env_rh == lay.env.index("RH")
    assert inf.n_env == len(lay.env)


def test_long_rows_keep_their_partial_sums_within_budget():
    """The chain-rule entries of a water parameter lengthen the gas rows that
    every particle couples to; cutting those rows into chunks must not blow
    up the per-cell partial sums (the compiler caps them per level).  Without
    the cap the 100-particle cell needed 166 KB of shared memory and the
    160-particle one did not fit."""
    from tests import mechs as M
    for n_particles, limit in ((40, 30000), (100, 60000), (160, 75000)):
        inf = camp.Mechanism(json.dumps(M.water_particles_mechanism(n_particles)), device=False).info
        assert inf.smem_per_cell_mixed < limit, (n_particles, inf.smem_per_cell_mixed)


def test_block_arrow_form_of_a_particle_resolved_mechanism():
    """A particle-resolved mechanism takes the block-arrow form when it asks
    for it or exceeds one block (2048 species): same sizes as the generic
    compile where both exist, species looked up as gas names and
    bin<p>.<name>, and a clear refusal of what the form does not keep."""
    from paper_2111_07436_gb300 import workloads as w
    mj = w.particle_resolved_mechanism(40)
    generic = camp.Mechanism(json.dumps(mj), device=False)
    ma = json.loads(json.dumps(mj))
    ma["aerosol"]["solver"] = "block_arrow"
    arrow = camp.Mechanism(json.dumps(ma), device=False)
    for k in ("n_species", "n_rxn", "n_env", "n_sections", "nnz_jac"):
        assert getattr(arrow.info, k) == getattr(generic.info, k), k
    assert arrow.info.block_arrow == 1 and generic.info.block_arrow == 0
    names = w.layout(mj).species
    for i in (0, 17, 18, 100, len(names) - 1):
        assert arrow.species_index(names[i]) == i == generic.species_index(names[i])
    assert arrow.species_index("bin40.SOA1") == -1 and arrow.species_index("binx.SOA1") == -1
    with pytest.raises(camp.CampError):
        arrow.structure()
    # the paper's 10^4 particles: beyond one block, so the block-arrow form
    big = camp.Mechanism(json.dumps(w.particle_resolved_mechanism(10000)), device=False)
    assert big.info.n_species == 18 + 7 * 10000 and big.info.block_arrow == 1
    assert big.species_index("bin9999.OLIG") == 18 + 7 * 9999 + 6
    # a water parameter is not part of the block-arrow form
    mw = json.loads(json.dumps(ma))
    mw["parameters"] = [{"type": "ZSR_AEROSOL_WATER", "electrolytes": [{"species": "SULF", "Y": [1.0]}]}]
    with pytest.raises(camp.CampError):
        camp.Mechanism(json.dumps(mw), device=False)
