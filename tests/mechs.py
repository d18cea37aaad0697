"""Tiny hand-written mechanisms for the pin tests (JSON-able dicts)."""
import json


def mech(species, reactions, phase=None, sections=0, atoms=None, water=None):
    """water: [(phase species, [Y_0, ...], low_RH), ...] -> a ZSR aerosol-water
    parameter over those electrolytes."""
    d = {"name": "test",
         "species": [{"name": s, "atoms": (atoms or {}).get(s, 1)} for s in species],
         "reactions": reactions}
    if phase is not None:
        d["phases"] = {"aqueous": [{"name": p, "atoms": 1} for p in phase]}
        d["aerosol"] = {"phase": "aqueous", "sections": sections}
    if water:
        d["parameters"] = [{"type": "ZSR_AEROSOL_WATER",
                            "electrolytes": [{"species": e, "Y": list(Y), "low_RH": lo}
                                             for e, Y, lo in water]}]
    return json.dumps(d)


def arrhenius(reactants, products, A, B=0.0, C=0.0, D=300.0, E=0.0):
    return {"type": "ARRHENIUS", "reactants": reactants, "products": products,
            "A": A, "B": B, "C": C, "D": D, "E": E}


def troe(reactants, products, k0_A, kinf_A, k0_B=0.0, k0_C=0.0, kinf_B=0.0, kinf_C=0.0, Fc=0.6, N=1.0):
    return {"type": "TROE", "reactants": reactants, "products": products,
            "k0_A": k0_A, "k0_B": k0_B, "k0_C": k0_C, "kinf_A": kinf_A, "kinf_B": kinf_B,
            "kinf_C": kinf_C, "Fc": Fc, "N": N}


def photolysis(x, products, value=1e-3):
    return {"type": "PHOTOLYSIS", "reactants": {x: 1}, "products": products, "value": value}


def emission(x, value=1e-3):
    return {"type": "EMISSION", "species": x, "value": value}


def loss(x, value=1e-3):
    return {"type": "FIRST_ORDER_LOSS", "species": x, "value": value}


def henry(gas, aq, H298, C_H=0.0, alpha=0.5, Dg=1e-5, MW=0.05):
    return {"type": "HL_PHASE_TRANSFER", "gas": gas, "aqueous": aq, "H298": H298, "C_H": C_H,
            "alpha": alpha, "Dg": Dg, "MW": MW}


def aqrev(reactants, products, A, kr, C=0.0):
    return {"type": "AQUEOUS_REVERSIBLE", "reactants": reactants, "products": products,
            "A": A, "C": C, "kr": kr}


def custom_h2o2(reactants, products, k1_A, k2_A, k1_B=0.0, k1_C=0.0, k2_B=0.0, k2_C=0.0):
    return {"type": "CUSTOM_H2O2", "reactants": reactants, "products": products,
            "k1_A": k1_A, "k1_B": k1_B, "k1_C": k1_C, "k2_A": k2_A, "k2_B": k2_B, "k2_C": k2_C}


def custom_oh_hno3(reactants, products, k0_A, k2_A, k3_A, k0_C=0.0, k2_C=0.0, k3_C=0.0):
    return {"type": "CUSTOM_OH_HNO3", "reactants": reactants, "products": products,
            "k0_A": k0_A, "k0_C": k0_C, "k2_A": k2_A, "k2_C": k2_C, "k3_A": k3_A, "k3_C": k3_C}


def condensed_arrhenius(reactants, products, A, B=0.0, C=0.0, D=300.0, E=0.0):
    return {"type": "CONDENSED_ARRHENIUS", "reactants": reactants, "products": products,
            "A": A, "B": B, "C": C, "D": D, "E": E}


def simpol(gas, aq, B, alpha=0.5, Dg=1e-5, MW=0.05, c_tot=None):
    d = {"type": "SIMPOL_PHASE_TRANSFER", "gas": gas, "aqueous": aq, "B": list(B),
         "alpha": alpha, "Dg": Dg, "MW": MW}
    if c_tot is not None:
        d["c_tot"] = c_tot
    return d



def water_chain_mechanism(Y1=(3.1, -2.2, -0.3), Y2=(2.4, -1.1)):
    """Every section process type over two sections with a ZSR water
    parameter whose electrolytes take part in them (an inert salt S, the
    dissociation product C and the condensation product E)."""
    return mech(["G1", "G2"], [
        henry("G1", "A", H298=2e3 / 101325.0, C_H=1000.0, alpha=0.2),
        simpol("G2", "B", (2.5e3, -9.0, 0.0, 0.0)),
        aqrev({"A": 1}, {"C": 1, "D": 1}, A=3e-2, kr=5.0),        # L^-1 on kr
        aqrev({"B": 2}, {"E": 1}, A=4.0, kr=0.3),                 # L^-1 on kf
        condensed_arrhenius({"A": 1, "C": 1}, {"E": 1}, A=2e2),   # L^-1 on kf
        condensed_arrhenius({"D": 1}, {"B": 1}, A=0.1),           # first order: no L
    ], phase=["A", "B", "C", "D", "E", "S"], sections=2,
        water=[("S", Y1, 0.0), ("C", Y2, 0.3), ("E", (2.0, -0.5, -0.5), 0.2)])


def water_particles_mechanism(n_particles):
    """The particle-resolved mechanism with an inert salt in every particle
    and a ZSR water parameter over the salt and the sulphate that the
    particles' H2O2 + HSO3 chemistry makes (made-up molality fits)."""
    from paper_2111_07436_gb300 import workloads as w
    mj = w.particle_resolved_mechanism(n_particles)
    mj["phases"]["aqueous"].append({"name": "SALT", "atoms": 1})
    mj["parameters"] = [{"type": "ZSR_AEROSOL_WATER", "electrolytes": [
        {"species": "SALT", "Y": [3.3, -2.6, 0.1], "low_RH": 0.45},
        {"species": "SULF", "Y": [6.0, -4.5], "low_RH": 0.45}]}]
    return mj
