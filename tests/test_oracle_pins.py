"""Pins of the FP64 oracle to facts outside it (no GPU).

Each test checks the oracle against a published constant, a closed-form
solution, a limit of a formula, an invariant or a textbook value, chosen so
that a dropped term, a wrong sign or index, or a swapped operand in
oracle/camp_oracle.c fails at least one of them.  Rate laws: CAMP paper
Table 2; forcing/Jacobian sums: Sect. 2.4.2; analytic-solution tests of
single processes: Sect. 2.5, Table 7; BDF + Newton: Sect. 2.4.1.
"""
import math

import numpy as np
import pytest

import oracle
from tests import mechs as M
from tests.golden.load import isoprene_soa_table9

# published constants (CODATA 2018)
LOSCHMIDT_CM3 = 2.686780111e19        # molec cm^-3 at 273.15 K, 101.325 kPa
MOLAR_VOLUME_STP = 22.41396954        # L mol^-1 at 273.15 K, 101.325 kPa
R_LATM = 0.082057366080960            # L atm mol^-1 K^-1
STP = (273.15, 101325.0)


def env_of(m, T, P, runtime=(), sections=()):
    e = np.zeros(m.n_env)
    e[0], e[1] = T, P
    for i, v in enumerate(runtime):
        e[2 + i] = v
    base = m.m.env_section_base
    for b, (r, N, L) in enumerate(sections):
        e[base + 3 * b: base + 3 * b + 3] = (r, N, L)
    return e


# ---------------------------------------------------------------- rate constants

def test_arrhenius_unit_conversion_uses_loschmidt_number():
    m = oracle.Mechanism(M.mech(["A", "B", "C", "D"], [
        M.arrhenius({"A": 1}, {"B": 1}, A=2.5),
        M.arrhenius({"A": 1, "B": 1}, {"C": 1}, A=1.0),
        M.arrhenius({"A": 1, "B": 1, "C": 1}, {"D": 1}, A=1.0),
    ]))
    kf, kr = m.rate_constants(env_of(m, *STP))
    mppb = LOSCHMIDT_CM3 * 1e-9
    assert kf[0] == pytest.approx(2.5, rel=1e-15)
    assert kf[1] == pytest.approx(mppb, rel=1e-9)       # the constant has 10 digits
    assert kf[2] == pytest.approx(mppb ** 2, rel=2e-9)
    assert not kr.any()


def test_arrhenius_parameter_roles():
    T = 300.0
    base = dict(A=3.0)
    m = oracle.Mechanism(M.mech(["A", "B"], [
        M.arrhenius({"A": 1}, {"B": 1}, **base, C=T * math.log(2.0)),       # exp(C/T) = 2
        M.arrhenius({"A": 1}, {"B": 1}, **base, B=1.7, D=T / 2.0),          # (T/D)^B = 2^1.7
        M.arrhenius({"A": 1}, {"B": 1}, **base, B=5.0, D=T),                # T = D: no B effect
        M.arrhenius({"A": 1}, {"B": 1}, **base, E=1e-4),                    # 1 + E P
    ]))
    P = 5e4
    kf, _ = m.rate_constants(env_of(m, T, P))
    np.testing.assert_allclose(kf, [6.0, 3.0 * 2.0 ** 1.7, 3.0, 3.0 * (1 + 1e-4 * P)], rtol=1e-14)


def test_troe_limits_and_centre():
    T, P = STP
    Mair = LOSCHMIDT_CM3
    m = oracle.Mechanism(M.mech(["A", "B", "C"], [
        M.troe({"A": 1, "B": 1}, {"C": 1}, k0_A=1e-31, kinf_A=1e3, Fc=1.0),             # low pressure
        M.troe({"A": 1, "B": 1}, {"C": 1}, k0_A=1e-10, kinf_A=2e-12, Fc=1.0),           # high pressure
        M.troe({"A": 1, "B": 1}, {"C": 1}, k0_A=3e-12 / Mair, kinf_A=3e-12, Fc=0.6),   # x = 1
        M.troe({"A": 1, "B": 1}, {"C": 1}, k0_A=10 * 3e-12 / Mair, kinf_A=3e-12, Fc=0.6, N=1.0),
        M.troe({"A": 1, "B": 1}, {"C": 1}, k0_A=10 * 3e-12 / Mair, kinf_A=3e-12, Fc=0.6, N=2.0),
    ]))
    kf, _ = m.rate_constants(env_of(m, T, P))
    k = kf / (Mair * 1e-9)  # back to cm^3 s^-1 (bimolecular)
    assert k[0] == pytest.approx(1e-31 * Mair, rel=1e-9)
    assert k[1] == pytest.approx(2e-12, rel=1e-9)
    assert k[2] == pytest.approx(0.5 * 3e-12 * 0.6, rel=1e-8)      # broadening equals Fc at the centre
    # x = 10: log10 x = 1, exponent 1/(1 + (1/N)^2)
    assert k[3] == pytest.approx(10 * 3e-12 / 11 * 0.6 ** 0.5, rel=1e-8)
    assert k[4] == pytest.approx(10 * 3e-12 / 11 * 0.6 ** 0.8, rel=1e-8)


def test_henry_equilibrium_ratio_and_mass_transfer_limits():
    # kf/kr is the equilibrium partition y_aq/y_gas = H_cc L, with the
    # dimensionless H_cc = H [M/atm] * R [L atm/mol/K] * T
    H_matm, L, T, P = 3.2e3, 2.5e-7, 298.0, 9e4
    m = oracle.Mechanism(M.mech(["G"], [M.henry("G", "a", H298=H_matm / 101325.0, C_H=2500.0,
                                                alpha=0.3, Dg=1.2e-5, MW=0.0280134)],
                                phase=["a"], sections=3))
    secs = [(1e-12, 1e9, L), (1.0, 1e2, L), (2e-6, 1e8, L)]
    kf, kr = m.rate_constants(env_of(m, T, P, sections=secs))
    np.testing.assert_allclose(kf / kr, H_matm * R_LATM * T * L, rtol=1e-8)
    # free-molecular limit (Kn >> 1): collision rate pi r^2 alpha cbar N
    cbar = 474.7 * math.sqrt(T / 298.15)  # N2 mean speed, 474.7 m/s at 298.15 K
    assert kf[0] == pytest.approx(math.pi * 1e-24 * 0.3 * cbar * 1e9, rel=2e-3)
    # continuum limit (Kn << 1): Maxwell's diffusion-limited rate 4 pi r Dg N
    assert kf[1] == pytest.approx(4 * math.pi * 1.0 * 1.2e-5 * 1e2, rel=1e-6)
    # van 't Hoff temperature dependence of H
    kf2, kr2 = m.rate_constants(env_of(m, 280.0, P, sections=secs))
    ratio = (kf2[2] / kr2[2]) / (kf[2] / kr[2])
    assert ratio == pytest.approx(math.exp(2500.0 * (1 / 280.0 - 1 / 298.0)) * 280.0 / 298.0, rel=1e-12)
    # a section without water takes no part
    kf3, kr3 = m.rate_constants(env_of(m, T, P, sections=[(1e-6, 1e8, 0.0)] * 3))
    assert not kf3.any() and not kr3.any()


def test_aqueous_constants_use_molarity_per_ppb():
    T, P = STP
    L = 1e-6
    phi = 1e-9 * (1000.0 / MOLAR_VOLUME_STP) / (1000.0 * L)  # M per ppb at STP
    m = oracle.Mechanism(M.mech(["G"], [
        M.aqrev({"a": 1}, {"b": 1}, A=40.0, kr=3.0),
        M.aqrev({"a": 1}, {"b": 1, "c": 1}, A=2e-3, kr=7.0, C=1500.0),
    ], phase=["a", "b", "c"], sections=1))
    kf, kr = m.rate_constants(env_of(m, T, P, sections=[(1e-6, 1e8, L)]))
    assert kf[0] == pytest.approx(120.0, rel=1e-14) and kr[0] == pytest.approx(3.0, rel=1e-14)
    Keq = 2e-3 * math.exp(1500.0 * (1 / T - 1 / 298.0))
    assert kf[1] == pytest.approx(Keq * 7.0, rel=1e-12)
    assert kr[1] == pytest.approx(7.0 * phi, rel=1e-9)


def test_custom_h2o2_adds_a_pressure_term():
    # k = k1 + k2 [M] (Table 2, CustomH2o2)
    T, P = STP
    mppb = LOSCHMIDT_CM3 * 1e-9
    m = oracle.Mechanism(M.mech(["H", "X"], [
        M.custom_h2o2({"H": 2}, {"X": 1}, k1_A=3e-13, k1_B=1.5, k1_C=460.0, k2_A=0.0),
        M.arrhenius({"H": 2}, {"X": 1}, A=3e-13, B=1.5, C=460.0, D=300.0),
        M.custom_h2o2({"H": 2}, {"X": 1}, k1_A=0.0, k2_A=2e-33),
        M.custom_h2o2({"H": 2}, {"X": 1}, k1_A=0.0, k2_A=2e-33, k2_C=T * math.log(2.0)),
        M.custom_h2o2({"H": 2}, {"X": 1}, k1_A=3e-13, k1_C=460.0, k2_A=2e-33, k2_C=920.0),
        M.custom_h2o2({"H": 2}, {"X": 1}, k1_A=0.0, k2_A=2e-33, k2_C=920.0),
        M.custom_h2o2({"H": 2}, {"X": 1}, k1_A=3e-13, k1_C=460.0, k2_A=0.0),
    ]))
    kf, kr = m.rate_constants(env_of(m, T, P))
    assert not kr.any()
    # without the pressure term it is the Arrhenius rate constant (D = 300 K)
    assert kf[0] == pytest.approx(kf[1], rel=1e-14)
    # the pressure term is k2 times the air number density (Loschmidt at STP)
    assert kf[2] / mppb == pytest.approx(2e-33 * LOSCHMIDT_CM3, rel=1e-9)
    assert kf[3] / kf[2] == pytest.approx(2.0, rel=1e-14)      # k2's own exp(C/T)
    assert kf[4] == pytest.approx(kf[5] + kf[6], rel=1e-14)    # the two terms add
    # (T/300)^B of the k2 term, at the same T and P
    m2 = oracle.Mechanism(M.mech(["H", "X"], [
        M.custom_h2o2({"H": 2}, {"X": 1}, k1_A=0.0, k2_A=2e-33),
        {**M.custom_h2o2({"H": 2}, {"X": 1}, k1_A=0.0, k2_A=2e-33), "k2_B": 1.0}]))
    kf2, _ = m2.rate_constants(env_of(m2, 600.0, 5e4))
    assert kf2[1] / kf2[0] == pytest.approx(2.0, rel=1e-14)


def test_custom_oh_hno3_limits():
    # k = k0 + k3[M] / (1 + k3[M]/k2) (Table 2, CustomOhHno3): linear in [M]
    # at low pressure, k0 + k2 at high pressure, k0 + k2/2 where k3[M] = k2
    T, P = STP
    Mair = LOSCHMIDT_CM3
    k0, k2 = 2.4e-14, 2.7e-17
    rx = lambda **kw: M.custom_oh_hno3({"O": 1, "N": 1}, {"X": 1}, **kw)
    m = oracle.Mechanism(M.mech(["O", "N", "X"], [
        rx(k0_A=0.0, k2_A=k2, k3_A=1e-7 * k2 / Mair),
        rx(k0_A=k0, k2_A=k2, k3_A=1e7 * k2 / Mair),
        rx(k0_A=k0, k2_A=k2, k3_A=k2 / Mair),
        rx(k0_A=k0, k2_A=k2, k3_A=0.0),
    ]))
    kf, kr = m.rate_constants(env_of(m, T, P))
    k = kf / (Mair * 1e-9)  # back to cm^3 s^-1 (bimolecular)
    assert k[0] == pytest.approx(1e-7 * k2, rel=1e-6)
    assert k[1] == pytest.approx(k0 + k2, rel=1e-6)
    assert k[2] == pytest.approx(k0 + 0.5 * k2, rel=1e-9)
    assert k[3] == pytest.approx(k0, rel=1e-9)
    assert not kr.any()


def test_condensed_arrhenius_works_in_molarity():
    # rates in M s^-1 (Table 2, CondensedPhaseArrhenius): a first-order
    # process needs no unit factor, a second-order one the molarity per ppb
    T, P = STP
    L = 1e-6
    phi = 1e-9 * (1000.0 / MOLAR_VOLUME_STP) / (1000.0 * L)  # M per ppb at STP
    m = oracle.Mechanism(M.mech(["G"], [
        M.condensed_arrhenius({"a": 1}, {"b": 1}, A=0.7),
        M.condensed_arrhenius({"a": 1, "b": 1}, {"c": 1}, A=5e3),
        M.condensed_arrhenius({"a": 2}, {"c": 0.5}, A=5e3, C=T * math.log(2.0)),
    ], phase=["a", "b", "c"], sections=2))
    kf, kr = m.rate_constants(env_of(m, T, P, sections=[(1e-6, 1e8, L), (1e-6, 1e8, 0.0)]))
    # instances: process 0 in sections 0 and 1, then process 1, then process 2
    assert kf[0] == pytest.approx(0.7, rel=1e-15)
    assert kf[2] == pytest.approx(5e3 * phi, rel=1e-9)
    assert kf[4] == pytest.approx(1e4 * phi, rel=1e-9)
    assert kf[1] == kf[3] == kf[5] == 0.0  # section 1 holds no condensed phase
    assert not kr.any()


def test_condensed_second_order_decay_in_molarity():
    # 2a -> b at k [M^-1 s^-1]: dc/dt = -2 k c^2, so 1/c = 1/c0 + 2 k t in molarity
    T, P, L = 290.0, 9.5e4, 3e-7
    k = 40.0
    m = oracle.Mechanism(M.mech(["G"], [M.condensed_arrhenius({"a": 2}, {"b": 1}, A=k)],
                                phase=["a", "b"], sections=1))
    env = env_of(m, T, P, sections=[(1e-6, 1e8, L)])
    to_M = 1e-9 * P / (8.314462618 * T) / (1000.0 * L)
    y = _integrate(m, np.array([0.0, 5.0, 0.0]), env, 100.0)
    c = 1.0 / (1.0 / (5.0 * to_M) + 2 * k * 100.0)
    assert y[1] * to_M == pytest.approx(c, rel=1e-8)
    assert y[2] == pytest.approx((5.0 - y[1]) / 2, rel=1e-10)


# SIMPOL.1 parameters of the isoprene products (Table 9, tests/golden):
# B1 [K], B2, B3 [1/K], B4; the box model's environment (Sect. 4.1)
TABLE9 = isoprene_soa_table9()
SOA_B = TABLE9["partition"]["soa1"][2]
SOA2_B = TABLE9["partition"]["soa2"][2]
BOX_T, BOX_P = TABLE9["environment"]["T"], TABLE9["environment"]["P"]


def test_simpol_partition_follows_raoults_law():
    # Reading: ideal solution of fixed molarity c_tot, so at equilibrium
    # y_g P = (c_a / c_tot) p0, i.e. y_a / y_g = c_tot R T L / p0 with the
    # SIMPOL.1 vapour pressure log10 p0 [atm] = B1/T + B2 + B3 T + B4 ln T
    T, P, L, c_tot = BOX_T, BOX_P, 4e-12, 7.0
    mt = dict(alpha=0.1, Dg=1e-5, MW=0.15)
    m = oracle.Mechanism(M.mech(["G"], [
        M.simpol("G", "a", SOA_B, c_tot=c_tot, **mt),
        M.henry("G", "a", H298=1.0, **mt),
        M.simpol("G", "a", (0.0, 0.0, 0.01, 0.0), c_tot=c_tot, **mt),
        M.simpol("G", "a", (0.0, 0.0, 0.0, 0.5), c_tot=c_tot, **mt),
        M.simpol("G", "a", SOA_B, **mt),
        M.simpol("G", "a", SOA2_B, c_tot=c_tot, **mt),
    ], phase=["a"], sections=1))
    kf, kr = m.rate_constants(env_of(m, T, P, sections=[(2e-7, 1e9, L)]))
    p0 = 10.0 ** (SOA_B[0] / T + SOA_B[1])
    assert kf[0] / kr[0] == pytest.approx(c_tot * R_LATM * T * L / p0, rel=1e-8)
    assert kf[0] == pytest.approx(kf[1], rel=1e-15)  # condensation as for Henry's law
    assert kf[2] / kr[2] == pytest.approx(c_tot * R_LATM * T * L / 10.0 ** (0.01 * T), rel=1e-8)
    assert kf[3] / kr[3] == pytest.approx(c_tot * R_LATM * T * L / T ** (0.5 * math.log(10.0)), rel=1e-8)
    # the default solvent is water, 55.5 mol per litre
    assert (kf[4] / kr[4]) / (kf[0] / kr[0]) == pytest.approx(1000.0 / 18.015 / c_tot, rel=1e-12)
    # Table 9's two products share B1 and differ by 0.4 in B2: ISOP-P1's
    # vapour pressure is 10^-0.4 of ISOP-P2's at any T, so it partitions
    # 10^0.4 = 2.51 times more strongly into the same particles
    assert (kf[0] / kr[0]) / (kf[5] / kr[5]) == pytest.approx(10.0 ** (SOA2_B[1] - SOA_B[1]), rel=1e-12)


def test_simpol_two_compartment_relaxation():
    T, P, L = BOX_T, BOX_P, 4e-12
    m = oracle.Mechanism(M.mech(["G"], [M.simpol("G", "a", SOA_B, alpha=0.1, c_tot=7.0)],
                                phase=["a"], sections=1))
    env = env_of(m, T, P, sections=[(2e-7, 1e9, L)])
    kf, kr = m.rate_constants(env)
    y0 = np.array([3.0, 0.5])
    for t in (0.3 / (kf[0] + kr[0]), 5.0 / (kf[0] + kr[0])):
        y = _integrate(m, y0, env, t)
        geq = 3.5 * kr[0] / (kf[0] + kr[0])
        assert y[0] == pytest.approx(geq + (3.0 - geq) * math.exp(-(kf[0] + kr[0]) * t), rel=1e-8)
        assert y.sum() == pytest.approx(3.5, rel=1e-12)


# ---------------------------------------------------------------- f and J

@pytest.mark.parametrize("wl_mech", ["small_gas_mechanism", "small_multiphase_mechanism",
                                     "process_variety_mechanism"])
def test_jacobian_matches_central_differences(wl_mech):
    import json
    from paper_2111_07436_gb300 import workloads as w
    mj = getattr(w, wl_mech)()
    m = oracle.Mechanism(json.dumps(mj))
    y, env = w.cells(mj, 3, seed=7)
    y[:, len(mj["species"]):] = np.random.default_rng(3).uniform(1e-3, 1.0, (3, m.n - len(mj["species"])))
    for c in range(3):
        kf, kr = m.rate_constants(env[c])
        J = m.jacobian(kf, kr, y[c])
        Jfd = np.zeros_like(J)
        for j in range(m.n):
            h = 1e-6 * max(abs(y[c, j]), 1e-3)
            yp, ym = y[c].copy(), y[c].copy()
            yp[j] += h
            ym[j] -= h
            Jfd[:, j] = (m.forcing(kf, kr, yp) - m.forcing(kf, kr, ym)) / (2 * h)
        scale = np.abs(J).max(axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(J - Jfd) / scale) < 1e-6


def test_forcing_signs_and_stoichiometry():
    m = oracle.Mechanism(M.mech(["A", "B", "C"], [
        M.arrhenius({"A": 2}, {"B": 1}, A=1.0),                 # 2A -> B, r = k A^2
        M.photolysis("B", {"C": 0.5, "A": 1.5}),
        M.emission("C", 2.0),
    ]))
    kf = np.array([0.1, 0.2, 2.0])
    kr = np.zeros(3)
    y = np.array([3.0, 5.0, 7.0])
    f = m.forcing(kf, kr, y)
    r0, r1 = 0.1 * 9.0, 0.2 * 5.0
    np.testing.assert_allclose(f, [-2 * r0 + 1.5 * r1, r0 - r1, 0.5 * r1 + 2.0], rtol=1e-15)


# ---------------------------------------------------------------- dense LU

def test_dense_lu_solve_needs_and_does_pivoting():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 40):
        A = rng.normal(size=(n, n))
        if n > 1:
            A[0, 0] = 0.0  # no static pivot order would survive this
        b = rng.normal(size=n)
        x = oracle.dense_lu_solve(A, b)
        assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(x) * n
    with pytest.raises(np.linalg.LinAlgError):
        oracle.dense_lu_solve(np.zeros((3, 3)), np.ones(3))


# ---------------------------------------------------------------- BDF coefficients

def test_bdf_coefficients_are_the_textbook_values():
    # l-vectors of the fixed-step BDF in Nordsieck form and the BDF error
    # constants 1/2, 2/9, 3/22, 12/125, 10/137
    l1, c1 = oracle.bdf_coefficients(1)
    l2, c2 = oracle.bdf_coefficients(2)
    l3, c3 = oracle.bdf_coefficients(3)
    np.testing.assert_allclose(l1, [1, 1])
    np.testing.assert_allclose(l2, [1, 1.5, 0.5])
    np.testing.assert_allclose(l3, [1, 11 / 6, 1, 1 / 6])
    cs = [oracle.bdf_coefficients(q)[1] for q in range(1, 6)]
    np.testing.assert_allclose(cs, [1 / 2, 2 / 9, 3 / 22, 12 / 125, 10 / 137], rtol=1e-15)
    # gamma = h / l_1 is the BDF-q leading coefficient beta_0 = 1 / sum_{j<=q} 1/j
    for q in range(1, 6):
        assert oracle.bdf_coefficients(q)[0][1] == pytest.approx(sum(1 / j for j in range(1, q + 1)))


def _nordsieck_from_history(vals):
    """z_m = a_m of the interpolant p(s) = sum a_m s^m through (s=-j, vals[j])."""
    q = len(vals) - 1
    V = np.array([[(-j) ** mm for mm in range(q + 1)] for j in range(q + 1)], dtype=float)
    return np.linalg.solve(V, vals)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_one_nordsieck_step_is_the_bdf_formula(q):
    """From exact history, one step equals solving sum_j (1/j) nabla^j y = h f(y)
    directly.  The correction e = y - y_pred then holds the step's own local
    error once on top of h^(q+1) y^(q+1), so c_q e = (1 + c_q) x true error."""
    k = 0.7
    m = oracle.Mechanism(M.mech(["X"], [M.loss("X")]))
    env = env_of(m, 298.0, 1e5, runtime=[k])
    cq = oracle.bdf_coefficients(q)[1]
    for h in (0.01 / k, 0.005 / k):
        past = np.array([math.exp(-k * (-j * h)) for j in range(q + 1)])  # y(t_n - j h), t_n = 0
        z = _nordsieck_from_history(past).reshape(q + 1, 1)
        zo, e, err = m.bdf_step(env, z, q, h, rtol=1e-3, atol=1e-12)
        assert err >= 0.0
        # direct BDF-q: sum_{j=1..q} (1/j) nabla^j y_{n+1} = -k h y_{n+1}
        # values v[0] = y_{n+1} (unknown), v[i] = past[i-1]
        coef_new = sum(1.0 / j for j in range(1, q + 1)) + k * h
        rhs = 0.0
        for j in range(1, q + 1):
            for i in range(1, j + 1):
                rhs -= (1.0 / j) * math.comb(j, i) * (-1) ** i * past[i - 1]
        y_bdf = rhs / coef_new
        assert zo[0, 0] == pytest.approx(y_bdf, rel=1e-12)
        assert zo[1, 0] == pytest.approx(-k * h * y_bdf, rel=1e-10)  # z_1 = h f(y_{n+1})
        true_err = abs(zo[0, 0] - math.exp(-k * h))
        assert cq * abs(e[0]) == pytest.approx((1 + cq) * true_err, rel=0.05)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_error_estimate_tracks_local_error_along_a_run(q):
    """After many fixed-(h, q) steps the history is the method's own, and the
    estimate c_q e matches the true local error of the next step (the error
    of one step taken from exact values of the local solution) within 10%."""
    k = 0.7
    m = oracle.Mechanism(M.mech(["X"], [M.loss("X")]))
    env = env_of(m, 298.0, 1e5, runtime=[k])
    cq = oracle.bdf_coefficients(q)[1]
    h = 0.01 / k
    z = _nordsieck_from_history(np.array([math.exp(k * j * h) for j in range(q + 1)])).reshape(q + 1, 1)
    for _ in range(40):
        z, e, err = m.bdf_step(env, z, q, h, rtol=1e-3, atol=1e-12)
        assert err >= 0.0
    yn = z[0, 0]
    _, e_run, _ = m.bdf_step(env, z, q, h, rtol=1e-3, atol=1e-12)
    zl = _nordsieck_from_history(np.array([yn * math.exp(k * j * h) for j in range(q + 1)])).reshape(q + 1, 1)
    zl_out, _, _ = m.bdf_step(env, zl, q, h, rtol=1e-3, atol=1e-12)
    local_err = abs(zl_out[0, 0] - yn * math.exp(-k * h))
    assert cq * abs(e_run[0]) == pytest.approx(local_err, rel=0.1)


# ---------------------------------------------------------------- analytic solutions

def _integrate(m, y0, env, dt, rtol=1e-10, atol=1e-14):
    y, s, st = m.integrate(y0, env, dt, rtol, atol)
    assert s == 0
    return y


def test_first_order_chain_bateman():
    """A -> B -> C photolysis (the embedded sub-case of the small mechanism)."""
    import json
    from paper_2111_07436_gb300 import workloads as w
    mj = w.small_gas_mechanism()
    m = oracle.Mechanism(json.dumps(mj))
    lay = w.layout(mj)
    y0, env = w.cells(mj, 1, seed=201, T=298.0, P=101300.0, sza=False)
    y0, env = y0[0], env[0]
    k1, k2 = env[2], env[3]  # the two chain photolysis rates
    A0, B0, C0 = y0[:3]

    def exact(t):
        A = A0 * math.exp(-k1 * t)
        B = B0 * math.exp(-k2 * t) + A0 * k1 / (k2 - k1) * (math.exp(-k1 * t) - math.exp(-k2 * t))
        return np.array([A, B, A0 + B0 + C0 - A - B])

    for rtol, tol in ((1e-10, 1e-8), (1e-4, 1e-3)):
        y = y0.copy()
        for step in range(60):
            y = _integrate(m, y, env, 60.0, rtol=rtol, atol=1e-5 if rtol > 1e-6 else 1e-14)
            if step in (0, 59):
                np.testing.assert_allclose(y[:3], exact(60.0 * (step + 1)), rtol=tol)
    assert lay.species[:3] == ["A", "B", "C"]


def test_warm_start_keeps_the_analytic_solution_and_saves_steps():
    """Opt-in warm start: the step size carried across consecutive calls.
    Whatever the carried value, the A -> B -> C chain stays on its Bateman
    solution; carried from the previous call it takes fewer steps over 60
    consecutive calls than cold starts do."""
    import json
    from paper_2111_07436_gb300 import workloads as w
    mj = w.small_gas_mechanism()
    m = oracle.Mechanism(json.dumps(mj))
    y0, env = w.cells(mj, 1, seed=201, T=298.0, P=101300.0, sza=False)
    y0, env = y0[0], env[0]
    k1, k2 = env[2], env[3]
    A0, B0, C0 = y0[:3]
    t = 60.0
    A = A0 * math.exp(-k1 * t)
    B = B0 * math.exp(-k2 * t) + A0 * k1 / (k2 - k1) * (math.exp(-k1 * t) - math.exp(-k2 * t))
    for h in (1e-6, 1.0, 1e4):
        step = np.array([h])
        y, s, _ = m.integrate(y0, env, t, 1e-10, 1e-14, step=step)
        assert s == 0 and 0.0 < step[0] <= 10.0 * t
        np.testing.assert_allclose(y[:3], [A, B, A0 + B0 + C0 - A - B], rtol=1e-8)
    # 60 consecutive calls of 60 s: warm chains take fewer steps than cold
    # ones, and their global error stays proportional to rtol within the
    # bound of the tolerance-proportionality pin (100 rtol)
    T = 3600.0
    A = A0 * math.exp(-k1 * T)
    B = B0 * math.exp(-k2 * T) + A0 * k1 / (k2 - k1) * (math.exp(-k1 * T) - math.exp(-k2 * T))
    exact = np.array([A, B, A0 + B0 + C0 - A - B])
    for rtol in (1e-4, 1e-6):
        totals = []
        for warm in (False, True):
            y, step, n = y0.copy(), np.array([0.0]), 0
            for _ in range(60):
                y, s, st = m.integrate(y, env, 60.0, rtol, 1e-5 * rtol / 1e-4,
                                       step=step if warm else None)
                assert s == 0
                n += st[0]
            totals.append(n)
            np.testing.assert_allclose(y[:3], exact, rtol=100 * rtol)
        assert totals[1] < totals[0]
    # a failed cell hands back 0 (the next call starts cold)
    step = np.array([5.0])
    _, s, _ = m.integrate(y0, env, 1e4, 1e-8, 1e-12, max_steps=3, step=step)
    assert s == 1 and step[0] == 0.0


def test_reversible_pair_relaxes_to_equilibrium():
    kfw, kbw = 0.3, 0.05  # A <-> B with K_eq kr = 0.3, kr = 0.05 (linear in ppb)
    m = oracle.Mechanism(M.mech(["G"], [M.aqrev({"a": 1}, {"b": 1}, A=kfw / kbw, kr=kbw)],
                                phase=["a", "b"], sections=1))
    env = env_of(m, 298.0, 1e5, sections=[(1e-6, 1e8, 1e-6)])
    y0 = np.array([0.0, 10.0, 2.0])
    for t in (1.0, 10.0, 100.0):
        y = _integrate(m, y0, env, t)
        Aeq = 12.0 * kbw / (kfw + kbw)
        A = Aeq + (10.0 - Aeq) * math.exp(-(kfw + kbw) * t)
        assert y[1] == pytest.approx(A, rel=1e-8)
        assert y[1] + y[2] == pytest.approx(12.0, rel=1e-12)


def test_second_order_self_reaction():
    T, P = STP
    A_k = 2e-12
    m = oracle.Mechanism(M.mech(["A", "B"], [M.arrhenius({"A": 2}, {"B": 1}, A=A_k)]))
    env = env_of(m, T, P)
    kp = A_k * LOSCHMIDT_CM3 * 1e-9  # ppb^-1 s^-1
    y = _integrate(m, np.array([50.0, 0.0]), env, 600.0)
    Aexact = 1.0 / (1.0 / 50.0 + 2 * kp * 600.0)  # dA/dt = -2 k A^2
    assert y[0] == pytest.approx(Aexact, rel=1e-8)
    assert y[1] == pytest.approx((50.0 - Aexact) / 2, rel=1e-8)


def test_emission_and_loss():
    m = oracle.Mechanism(M.mech(["E", "L"], [M.emission("E"), M.loss("L")]))
    env = env_of(m, 298.0, 1e5, runtime=[0.37, 2e-3])
    y = _integrate(m, np.array([1.0, 4.0]), env, 900.0)
    assert y[0] == pytest.approx(1.0 + 0.37 * 900.0, rel=1e-13)  # BDF is exact on linear growth
    assert y[1] == pytest.approx(4.0 * math.exp(-2e-3 * 900.0), rel=1e-8)


def test_henry_two_compartment_relaxation():
    m = oracle.Mechanism(M.mech(["G"], [M.henry("G", "a", H298=1e4 / 101325.0, alpha=0.1)],
                                phase=["a"], sections=1))
    env = env_of(m, 298.0, 1e5, sections=[(5e-6, 1e8, 5e-8)])
    kf, kr = m.rate_constants(env)
    y0 = np.array([20.0, 0.0])
    for t in (0.5 / (kf[0] + kr[0]), 3.0 / (kf[0] + kr[0]), 50.0 / (kf[0] + kr[0])):
        y = _integrate(m, y0, env, t)
        geq = 20.0 * kr[0] / (kf[0] + kr[0])
        g = geq + (20.0 - geq) * math.exp(-(kf[0] + kr[0]) * t)
        assert y[0] == pytest.approx(g, rel=1e-8)
        assert y.sum() == pytest.approx(20.0, rel=1e-12)
    # at equilibrium the partition is Henry's law: y_aq / y_g = H R T L
    assert y[1] / y[0] == pytest.approx(1e4 * R_LATM * 298.0 * 5e-8, rel=1e-6)


def test_aqueous_dissociation_reaches_keq_in_molarity():
    T, P, L = 290.0, 9.5e4, 3e-7
    Keq, kr = 5e-3, 20.0
    m = oracle.Mechanism(M.mech(["G"], [M.aqrev({"a": 1}, {"b": 1, "c": 1}, A=Keq, kr=kr)],
                                phase=["a", "b", "c"], sections=1))
    env = env_of(m, T, P, sections=[(1e-6, 1e8, L)])
    y = _integrate(m, np.array([0.0, 5.0, 0.0, 0.0]), env, 5e3)
    air_mol_per_m3 = P / (8.314462618 * T)
    to_M = 1e-9 * air_mol_per_m3 / (1000.0 * L)
    ca, cb, cc = y[1] * to_M, y[2] * to_M, y[3] * to_M
    assert cb * cc / ca == pytest.approx(Keq, rel=1e-6)
    assert y[1] + y[2] == pytest.approx(5.0, rel=1e-12)  # a -> b conserves the 'a' moiety


def test_linear_invariant_is_conserved_on_the_multiphase_workload():
    import json
    from paper_2111_07436_gb300 import workloads as w
    mj = w.multiphase_mechanism()
    lay = w.layout(mj)
    m = oracle.Mechanism(json.dumps(mj))
    y0, env = w.cells(mj, 4, seed=9)
    for k, kind in enumerate(lay.runtime_kind):  # switch off sources and sinks
        if kind in ("EMISSION", "FIRST_ORDER_LOSS"):
            env[:, 2 + k] = 0.0
    y, st, _ = m.solve(y0, env, 300.0, 1e-4, 1e-5, threads=4)
    assert (st == 0).all()
    w0, w1 = y0 @ lay.atoms, y @ lay.atoms
    np.testing.assert_allclose(w1, w0, rtol=1e-10)


def test_tolerance_proportionality():
    """Global error on y' = -k y over five e-folds stays within 100 x rtol and
    shrinks as rtol does (an error-per-step BDF; SciPy's BDF lands at 3-30 x
    rtol on the same problem)."""
    m = oracle.Mechanism(M.mech(["X"], [M.loss("X")]))
    env = env_of(m, 298.0, 1e5, runtime=[0.05])
    errs = {}
    for rtol in (1e-3, 1e-5, 1e-7, 1e-9):
        y, s, _ = m.integrate(np.array([1.0]), env, 100.0, rtol, 1e-20)
        assert s == 0
        errs[rtol] = abs(y[0] - math.exp(-5.0)) / math.exp(-5.0)
        assert errs[rtol] <= 100 * rtol
    assert errs[1e-3] > 100 * errs[1e-7] > 0


# ---------------------------------------------------------------- statuses

def test_status_codes():
    m = oracle.Mechanism(M.mech(["X"], [M.loss("X")]))
    env = env_of(m, 298.0, 1e5, runtime=[0.05])
    y, s, _ = m.integrate(np.array([np.nan]), env, 10.0, 1e-4, 1e-5)
    assert s == 5
    bad = env.copy()
    bad[0] = np.inf
    assert m.integrate(np.array([1.0]), bad, 10.0, 1e-4, 1e-5)[1] == 5
    y, s, st = m.integrate(np.array([1.0]), env, 1e4, 1e-8, 1e-12, max_steps=3)
    assert s == 1 and y[0] == 1.0 and st[0] == 3


# ---------------------------------------------------------------- accuracy

def test_rate_constants_match_50_digit_evaluation():
    """The oracle's FP64 rate constants against the same expressions in
    50-digit arithmetic (every Arrhenius parameter active, Troe with N != 1,
    the custom types, the Henry partition H_cc L and K_eq(T))."""
    pytest.importorskip("mpmath")
    from tests import highprec
    m = oracle.Mechanism(highprec.mechanism())
    for T, P, L in highprec.CONDITIONS:
        kf, kr = m.rate_constants(env_of(m, T, P, sections=[(1e-6, 1e8, L)]))
        for k, kind, exact in highprec.constants(T, P, L):
            got = kf[k] if kind == "kf" else kf[k] / kr[k]
            assert abs(got / float(exact) - 1) < 1e-14, (k, kind, T)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_fixed_order_global_error_slope(q):
    """Order of accuracy: BDF-q at a fixed step from exact starting history
    integrates y' = -y to t = 1 with a global error O(h^q), so halving h
    divides the error by 2^q."""
    m = oracle.Mechanism(M.mech(["X"], [M.loss("X")]))
    env = env_of(m, 298.0, 1e5, runtime=[1.0])
    errs = []
    for n_steps in (16, 32, 64):
        h = 1.0 / n_steps
        z = np.array([[(-h) ** j / math.factorial(j)] for j in range(q + 1)])  # exact Nordsieck
        for _ in range(n_steps):
            z, _, err = m.bdf_step(env, z, q, h, 1e-12, 1e-20)
            assert err >= 0.0
        errs.append(abs(z[0, 0] - math.exp(-1.0)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(s - q) < 0.35 for s in slopes), (q, slopes, errs)
