"""Rate constants of Table 2 evaluated in 50-digit arithmetic (mpmath), for
the accuracy pins of the FP64 oracle and of the GPU's rate constants.  The
unit factors are those of the ppb state: [M] = P / (k_B T) 1e-6 cm^-3 and a
gas reaction of molecularity n carries (1e-9 [M])^(n-1)."""
import json

from tests import mechs as M

KB = "1.380649e-23"
NA = "6.02214076e23"


def mechanism():
    """One process of each kind whose constant has a closed form, with every
    parameter active (B, D, E of Arrhenius; N != 1 of Troe)."""
    return M.mech(["A", "B", "C", "D"], [
        M.arrhenius({"A": 1, "B": 1}, {"C": 1}, A=3.3e-12, B=-1.7, C=-1234.5, D=287.0, E=2.1e-6),
        M.troe({"A": 1, "B": 1}, {"C": 1}, k0_A=2.2e-30, kinf_A=1.4e-11, k0_B=-3.1, k0_C=150.0,
               kinf_B=-0.4, kinf_C=-80.0, Fc=0.45, N=1.3),
        M.custom_h2o2({"A": 2}, {"B": 1}, k1_A=3.1e-13, k2_A=2.1e-33, k1_C=460.0, k2_C=920.0),
        M.custom_oh_hno3({"A": 1, "D": 1}, {"B": 1}, k0_A=2.4e-14, k2_A=2.7e-17, k3_A=6.5e-34,
                         k0_C=460.0, k2_C=2199.0, k3_C=1335.0),
        M.henry("D", "a", H298=3.7e3 / 101325.0, C_H=2400.0, alpha=0.3, Dg=1.1e-5, MW=0.046),
        M.aqrev({"a": 1}, {"b": 1}, A=0.037, kr=4.2, C=1750.0),
    ], phase=["a", "b"], sections=1)


def constants(T, P, L):
    """[(process index, kind, exact value)]: kind 'kf' for a forward constant,
    'ratio' for kf / kr."""
    import mpmath as mp
    mp.mp.dps = 50
    T, P, L = mp.mpf(T), mp.mpf(P), mp.mpf(L)
    kB, R = mp.mpf(KB), mp.mpf(KB) * mp.mpf(NA)
    Mair = P / (kB * T) * mp.mpf("1e-6")
    mppb = Mair * mp.mpf("1e-9")
    e = mp.e

    def arr300(A, B, C):
        return mp.mpf(A) * e ** (mp.mpf(C) / T) * (T / 300) ** mp.mpf(B)

    out = []
    k = mp.mpf("3.3e-12") * e ** (mp.mpf("-1234.5") / T) * (T / mp.mpf("287.0")) ** mp.mpf("-1.7") \
        * (1 + mp.mpf("2.1e-6") * P)
    out.append((0, "kf", k * mppb))
    k0, ki = arr300("2.2e-30", "-3.1", "150.0"), arr300("1.4e-11", "-0.4", "-80.0")
    x = k0 * Mair / ki
    lg = mp.log10(x) / mp.mpf("1.3")
    out.append((1, "kf", k0 * Mair / (1 + x) * mp.mpf("0.45") ** (1 / (1 + lg * lg)) * mppb))
    out.append((2, "kf", (arr300("3.1e-13", 0, "460.0") + arr300("2.1e-33", 0, "920.0") * Mair) * mppb))
    k3M = arr300("6.5e-34", 0, "1335.0") * Mair
    out.append((3, "kf", (arr300("2.4e-14", 0, "460.0") + k3M / (1 + k3M / arr300("2.7e-17", 0, "2199.0")))
                * mppb))
    H = mp.mpf("3.7e3") / mp.mpf("101325.0") * e ** (mp.mpf("2400.0") * (1 / T - 1 / mp.mpf(298)))
    out.append((4, "ratio", 1000 * H * R * T * L))
    out.append((5, "ratio", mp.mpf("0.037") * e ** (mp.mpf("1750.0") * (1 / T - 1 / mp.mpf(298)))))
    return out


CONDITIONS = [(298.15, 101325.0, 3e-7), (231.7, 2.35e4, 1e-10), (309.2, 9.1e4, 4.4e-6)]
