"""Pins of the oracle's ZSR aerosol-water parameter (no GPU).

CAMP paper Sect. 2.2.2: a Parameter is computed from the state, the processes
use its value, and the solver's Jacobian is the processes' partial
derivatives plus, by the chain rule, their partial derivatives with respect
to the parameters times the parameters' partial derivatives with respect to
the state.  Table 4, ZSRAerosolWater: W = sum_i 1000 M_i / (MW_i m_i(a_w)),
m_i the molality of electrolyte i alone in water at water activity a_w
(Zdanovskii-Stokes-Robinson: each electrolyte holds the water of its binary
solution at the same activity).  Molality fits of the Jacobson et al. (1996)
form, sqrt(m) = sum_j Y_j a_w^j; the paper prints none, so the fits here are
made up.

The pins: the binary-solution limit and the additivity that define the ZSR
rule; central differences of the forcing against the chain-rule Jacobian;
closed-form solutions of transfer and equilibria whose liquid volume is the
water of the state's electrolytes.
"""
import json
import math

import numpy as np
import pytest

import oracle
from tests import mechs as M

MOLAR_VOLUME_STP = 22.41396954        # L mol^-1 at 273.15 K, 101.325 kPa (CODATA; 10 digits)
R_LATM = 0.082057366080960            # L atm mol^-1 K^-1
STP = (273.15, 101325.0)
AIR_STP = 1000.0 / MOLAR_VOLUME_STP   # mol of air per m^3 at STP
RHO_W = 1000.0                        # kg m^-3


def env_w(m, T, P, RH, sections, runtime=()):
    e = np.zeros(m.n_env)
    e[0], e[1] = T, P
    for i, v in enumerate(runtime):
        e[2 + i] = v
    e[m.m.rh_slot] = RH
    base = m.m.env_section_base
    for b, (r, N, L) in enumerate(sections):
        e[base + 3 * b: base + 3 * b + 3] = (r, N, L)
    return e


def molality(Y, aw, low=0.0):
    aw = max(aw, low)
    return sum(c * aw ** j for j, c in enumerate(Y)) ** 2


Y1 = (3.1, -2.2, -0.3)        # sqrt(m) falls from 3.1 at a_w = 0 to 0.6 at a_w = 1
Y2 = (2.4, -1.1)
SEC = (1e-6, 1e8)             # radius, number: the volume test needs no transfer


def test_binary_solution_limit_and_zsr_additivity():
    T, P = STP
    m = oracle.Mechanism(M.mech(["G"], [], phase=["E1", "E2", "X"], sections=2,
                                water=[("E1", Y1, 0.0), ("E2", Y2, 0.6)]))
    i = {s: k for k, s in enumerate(m.m.species)}

    def water_kg(y, RH, Lenv=(0.0, 0.0)):
        L = m.water(env_w(m, T, P, RH, [(*SEC, Lenv[0]), (*SEC, Lenv[1])]), y)
        return (L - np.asarray(Lenv)) * RHO_W

    for RH in (0.8, 0.3):                    # 0.3 is below E2's fit: m2 held at a_w = 0.6
        y1 = np.zeros(m.n); y1[i["bin0.E1"]] = 3.0
        y2 = np.zeros(m.n); y2[i["bin0.E2"]] = 5.0
        W1, W2 = water_kg(y1, RH)[0], water_kg(y2, RH)[0]
        # alone in its section, each electrolyte makes its binary solution:
        # moles over kg of water is the fitted molality at the activity
        assert 3e-9 * AIR_STP / W1 == pytest.approx(molality(Y1, RH), rel=1e-9)
        assert 5e-9 * AIR_STP / W2 == pytest.approx(molality(Y2, RH, 0.6), rel=1e-9)
        # ZSR: the mixture holds the sum of the binary solutions' water
        assert water_kg(y1 + y2, RH)[0] == pytest.approx(W1 + W2, rel=1e-14)
    # water belongs to the section the electrolytes are in; L_env adds
    y = np.zeros(m.n); y[i["bin1.E1"]] = 2.0; y[i["bin1.X"]] = 7.0
    L = m.water(env_w(m, T, P, 0.8, [(*SEC, 4e-12), (*SEC, 3e-12)]), y)
    assert L[0] == 4e-12
    assert (L[1] - 3e-12) * RHO_W == pytest.approx(2e-9 * AIR_STP / molality(Y1, 0.8), rel=1e-9)
    # a fit without a positive molality holds no water
    m0 = oracle.Mechanism(M.mech(["G"], [], phase=["E"], sections=1, water=[("E", (1.0, -1.0), 0.0)]))
    assert m0.water(env_w(m0, T, P, 1.0, [(*SEC, 5e-12)]), np.array([0.0, 4.0]))[0] == 5e-12


def test_chain_rule_jacobian_matches_central_differences():
    m = oracle.Mechanism(M.water_chain_mechanism(Y1, Y2))
    i = {s: k for k, s in enumerate(m.m.species)}
    rng = np.random.default_rng(11)
    for trial in range(3):
        env = env_w(m, 285.0 + 10 * trial, 9e4, 0.55 + 0.1 * trial,
                    [(2e-7, 1e9, 0.0), (1e-6, 1e8, 2e-12)])
        y = rng.uniform(0.5, 2.0, m.n)
        kf, kr = m.rate_constants(env)
        J = m.jacobian(kf, kr, y, env)
        Jfd = np.zeros_like(J)
        for j in range(m.n):
            h = 1e-6 * abs(y[j])
            yp, ym = y.copy(), y.copy()
            yp[j] += h
            ym[j] -= h
            Jfd[:, j] = (m.forcing(kf, kr, yp, env) - m.forcing(kf, kr, ym, env)) / (2 * h)
        scale = np.abs(J).max(axis=1, keepdims=True) + 1e-300  # the inert salt rows are 0
        assert np.max(np.abs(J - Jfd) / scale) < 1e-6
        # the inert salt enters f only through the water: its column is the
        # chain-rule term alone, and it is not small
        for b in (0, 1):
            col = J[:, i[f"bin{b}.S"]]
            assert np.abs(col[i[f"bin{b}.A"]]) > 1e-3 * scale[i[f"bin{b}.A"], 0]
            assert col[i[f"bin{b}.S"]] == 0.0 and col[i["G2"]] != 0.0


def test_uptake_into_its_own_water_relaxes_exponentially():
    """Gas G dissolves into species A, the only electrolyte, with no other
    water: L = w y_A, so the evaporation term k_c y_A / (H_cc w y_A) is the
    constant k_c / (H_cc w) and y_G relaxes to 1 / (H_cc w) at rate k_c."""
    T, P = STP
    H_matm, RH = 6e8, 0.75
    m = oracle.Mechanism(M.mech(["G"], [M.henry("G", "A", H298=H_matm / 101325.0, alpha=0.3)],
                                phase=["A"], sections=1, water=[("A", Y1, 0.0)]))
    env = env_w(m, T, P, RH, [(1e-6, 1e9, 0.0)])
    kc = m.rate_constants(env)[0][0]
    w = 1e-9 * AIR_STP / molality(Y1, RH) / RHO_W      # m^3 of water per ppb of A
    ystar = 1.0 / (H_matm * R_LATM * T * w)
    y0 = np.array([20.0, 1.0])
    assert 1.0 < ystar < 20.0
    for t in (0.5 / kc, 3.0 / kc):
        y, s, _ = m.integrate(y0, env, t, 1e-10, 1e-14)
        assert s == 0
        assert y[0] == pytest.approx(ystar + (20.0 - ystar) * math.exp(-kc * t), rel=1e-8)
        assert y.sum() == pytest.approx(21.0, rel=1e-12)


def test_aqueous_equilibria_in_the_water_of_an_inert_salt():
    """a <-> b + c and 2 d <-> e settle at their K_eq in molarity, with the
    molarity per ppb set by the salt's water plus L_env."""
    T, P, RH = STP[0], STP[1], 0.65
    K1, K2 = 4e-3, 30.0
    m = oracle.Mechanism(M.mech(["G"], [
        M.aqrev({"a": 1}, {"b": 1, "c": 1}, A=K1, kr=50.0),
        M.aqrev({"d": 2}, {"e": 1}, A=K2, kr=2.0),
    ], phase=["S", "a", "b", "c", "d", "e"], sections=1, water=[("S", Y2, 0.0)]))
    Lenv = 1e-12
    env = env_w(m, T, P, RH, [(1e-6, 1e8, Lenv)])
    y0 = np.array([0.0, 2.0, 5.0, 0.0, 0.0, 3.0, 0.0])
    y, s, _ = m.integrate(y0, env, 2e4, 1e-10, 1e-16)
    assert s == 0
    L = Lenv + 2e-9 * AIR_STP / molality(Y2, RH) / RHO_W
    to_M = 1e-9 * AIR_STP / (RHO_W * L)
    ca, cb, cc, cd, ce = (y[k] * to_M for k in (2, 3, 4, 5, 6))
    assert cb * cc / ca == pytest.approx(K1, rel=1e-6)
    assert ce / cd ** 2 == pytest.approx(K2, rel=1e-6)
    assert y[1] == 2.0                                  # the salt is inert


def test_condensed_second_order_decay_in_the_water_of_an_inert_salt():
    # 2a -> b at k [M^-1 s^-1]: 1/c = 1/c0 + 2 k t in molarity, c = y / (1000 L)
    # mol per ppb, L the salt's water
    T, P, RH, k = STP[0], STP[1], 0.9, 1e-3   # 2 k t c0 ~ 1.5: c depends on the water
    m = oracle.Mechanism(M.mech(["G"], [M.condensed_arrhenius({"a": 2}, {"b": 1}, A=k)],
                                phase=["S", "a", "b"], sections=1, water=[("S", Y1, 0.0)]))
    env = env_w(m, T, P, RH, [(1e-6, 1e8, 0.0)])
    y, s, _ = m.integrate(np.array([0.0, 0.5, 5.0, 0.0]), env, 100.0, 1e-10, 1e-14)
    assert s == 0
    L = 0.5e-9 * AIR_STP / molality(Y1, RH) / RHO_W
    to_M = 1e-9 * AIR_STP / (RHO_W * L)
    c = 1.0 / (1.0 / (5.0 * to_M) + 2 * k * 100.0)
    assert y[2] * to_M == pytest.approx(c, rel=1e-8)


def test_inert_water_equals_the_same_volume_given_in_env():
    """With an inert salt as the only electrolyte, the liquid volume never
    changes, so a whole solve of the process-variety mechanism matches the
    same mechanism with that volume given in env."""
    from paper_2111_07436_gb300 import workloads as w
    base = w.process_variety_mechanism(seed=9, n_sections=2)
    mw = json.loads(json.dumps(base))
    mw["phases"]["aqueous"].append({"name": "S", "atoms": 1})
    mw["parameters"] = [{"type": "ZSR_AEROSOL_WATER", "electrolytes": [{"species": "S", "Y": list(Y1)}]}]
    mp = json.loads(json.dumps(mw))
    del mp["parameters"]
    om_w, om_p = oracle.Mechanism(json.dumps(mw)), oracle.Mechanism(json.dumps(mp))
    y, env = w.cells(mw, 4, seed=31)
    i = {s: k for k, s in enumerate(om_w.m.species)}
    for b in range(2):
        y[:, i[f"bin{b}.S"]] = [0.3, 1.0, 3.0, 10.0]
    env_p = np.delete(env, om_w.m.rh_slot, axis=1)
    for c in range(4):
        env_p[c, om_p.m.env_section_base + 2::3] = om_w.water(env[c], y[c])
    yw, sw, _ = om_w.solve(y, env, 60.0, 1e-9, 1e-12, threads=2)
    yp, sp, _ = om_p.solve(y, env_p, 60.0, 1e-9, 1e-12, threads=2)
    assert (sw == 0).all() and (sp == 0).all()
    np.testing.assert_allclose(yw, yp, rtol=1e-6, atol=1e-9)


def test_a_section_without_water_takes_no_part():
    """Reading: like a section with no water in env, a section whose
    electrolytes hold no water (and L_env = 0) takes no part; the cell still
    solves, equal to the same cell with that section's particles removed."""
    T, P = STP
    m = oracle.Mechanism(M.mech(["G"], [
        M.henry("G", "A", H298=3e3 / 101325.0, alpha=0.2),
        M.aqrev({"A": 1}, {"B": 1, "C": 1}, A=1e-3, kr=10.0),
        M.condensed_arrhenius({"B": 1}, {"C": 1}, A=0.05),
    ], phase=["S", "A", "B", "C"], sections=2, water=[("S", Y1, 0.0)]))
    y0 = np.array([10.0, 2.0, 0.0, 0.5, 0.0, 0.0, 0.3, 0.2, 0.1])  # section 1: no salt
    dry = env_w(m, T, P, 0.8, [(1e-6, 1e8, 0.0), (1e-6, 1e8, 0.0)])
    gone = env_w(m, T, P, 0.8, [(1e-6, 1e8, 0.0), (1e-6, 0.0, 0.0)])  # no particles
    assert m.water(dry, y0)[1] == 0.0
    y1, s1, _ = m.integrate(y0, dry, 300.0, 1e-10, 1e-14)
    y2, s2, _ = m.integrate(y0, gone, 300.0, 1e-10, 1e-14)
    assert s1 == 0 and s2 == 0
    np.testing.assert_allclose(y1, y2, rtol=1e-9, atol=1e-14)
    assert (y1[5:] == y0[5:]).all() and y1[2] != y0[2]   # section 1 frozen, section 0 active
