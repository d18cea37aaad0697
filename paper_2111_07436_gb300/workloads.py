"""Seeded synthetic workloads: mechanism descriptions and per-cell inputs.

This module only *describes inputs*: which species and reactions a mechanism
has, their parameters, and the initial state and environment of each grid
cell.  It holds none of the solver's arithmetic (no rate laws, no forcing, no
integration) and imports nothing from the CUDA path or from the oracle, so both
sides can draw identical inputs from it.

The mechanisms are shaped like the workloads of the CAMP paper (Sect. 4: a
CB05-like gas mechanism of ~50-70 species with ~150-190 reactions, Sect. 3.1;
an 8-section aerosol with one aqueous phase per section, Sect. 4.1) but the
numbers are drawn from seeded distributions, because the paper's mechanism
files are not part of the paper text.

Mechanism JSON schema (our own; the paper's example files exist only as
figures, Sect. 2.3):

    {"name": str,
     "species": [{"name": str, "atoms": int}, ...],          # gas phase
     "phases": {"aqueous": [{"name": str, "atoms": int}, ...]},
     "aerosol": {"phase": "aqueous", "sections": 8,           # optional
                 "representation": "particles"},   # optional: instances are
                                                   # computational particles
     "reactions": [ {"type": ..., ...}, ... ]}

Reaction types and their fields (units follow Table 2 of the paper):
    ARRHENIUS          reactants{name:int}, products{name:float}, A, B, C, D, E
                       (C = -Ea/k_B in K; D in K; E in Pa^-1)
    TROE               reactants, products, k0_A, k0_B, k0_C, kinf_A, kinf_B,
                       kinf_C, Fc, N
    PHOTOLYSIS         reactants{X:1}, products; "value" = default J [s^-1]
    EMISSION           species; "value" = default rate [ppb s^-1]
    FIRST_ORDER_LOSS   species; "value" = default rate constant [s^-1]
    HL_PHASE_TRANSFER  gas, aqueous, H298 [M Pa^-1], C_H [K], alpha,
                       Dg [m^2 s^-1], MW [kg mol^-1]      (one per section)
    AQUEOUS_REVERSIBLE reactants{name:int}, products{name:int}, A (K_eq at
                       298 K, M^(np-nr)), C [K], kr [M^(1-np) s^-1]
    CUSTOM_H2O2        reactants, products, k1_A, k1_B, k1_C, k2_A, k2_B, k2_C
                       (k = k1 + k2 [M], each A exp(C/T) (T/300)^B)
    CUSTOM_OH_HNO3     reactants, products, k0_*, k2_*, k3_* as above
                       (k = k0 + k3[M] / (1 + k3[M]/k2))
    CONDENSED_ARRHENIUS reactants{name:int}, products{name:float} (phase
                       species), A [M^(1-nr) s^-1], B, C, D, E as ARRHENIUS
                                                          (one per section)
    SIMPOL_PHASE_TRANSFER gas, aqueous, B [B1 (K), B2, B3 (K^-1), B4]
                       (log10 p0/atm = B1/T + B2 + B3 T + B4 ln T), alpha,
                       Dg, MW, c_tot [M] (condensed-phase total molarity,
                       default that of water)               (one per section)

Parameters (optional; Sect. 2.2.2 and Table 4 of the paper):
    "parameters": [{"type": "ZSR_AEROSOL_WATER",
                    "electrolytes": [{"species": phase species name,
                                      "Y": [Y_0, ..., Y_k] (k < 8),
                                      "low_RH": lowest water activity of
                                                the fit (default 0)}, ...]}]
    The water of every section by the ZSR rule, W = sum_i 1000 M_i /
    (MW_i m_i(a_w)), with molality fits sqrt(m_i) = sum_j Y_j a_w^j
    (Jacobson et al. 1996 form) at a_w = relative humidity.  The section's
    liquid volume becomes L_b = L_env,b + W_b(y) / 1000 kg m^-3.

Per-cell environment vector (the solver reads only this; "value" fields are
the defaults a host model would copy in):
    [T (K), P (Pa), one entry per PHOTOLYSIS / EMISSION / FIRST_ORDER_LOSS
     reaction in declaration order, RH (0..1; only with a water parameter),
     then per section b: r_b (m), N_b (m^-3), L_b (m^3 water per m^3 air;
     with a water parameter the part its electrolytes do not hold)]

State: every species, gas and aqueous, in ppb-equivalent of air (mole ratio
x 1e9).  Species order: gas species in declaration order, then for section
b = 0..nb-1 the phase species in declaration order, named "bin<b>.<name>".
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass

import numpy as np

RUNTIME_TYPES = ("PHOTOLYSIS", "EMISSION", "FIRST_ORDER_LOSS")
SECTION_TYPES = ("HL_PHASE_TRANSFER", "AQUEOUS_REVERSIBLE", "CONDENSED_ARRHENIUS",
                 "SIMPOL_PHASE_TRANSFER")


def _logu(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


# --------------------------------------------------------------------------
# gas-phase mechanisms
# --------------------------------------------------------------------------

class _Occupancy:
    """Draws species so that none takes part in more than `cap` reactions."""

    def __init__(self, names, cap, rng):
        self.names = list(names)
        self.count = {s: 0 for s in self.names}
        self.cap = cap
        self.rng = rng

    def pick(self, k, exclude=()):
        pool = [s for s in self.names if self.count[s] < self.cap and s not in exclude]
        if len(pool) < k:
            raise RuntimeError("species occupancy cap too tight for this mechanism")
        wts = np.array([self.cap - self.count[s] for s in pool], dtype=float)
        idx = self.rng.choice(len(pool), size=k, replace=False, p=wts / wts.sum())
        out = [pool[i] for i in idx]
        for s in out:
            self.count[s] += 1
        return out


def _yields(reactant_atoms, products, atoms):
    """Product yields that conserve the single integer 'atom' count."""
    m = len(products)
    return {p: reactant_atoms / (m * atoms[p]) for p in products}


def gas_mechanism(name, n_species, n_arrhenius, n_troe, n_photolysis, n_emission,
                  n_loss, seed, max_occupancy=12, loss_value=None, prefix="S"):
    """A random gas mechanism with the given reaction counts.

    Rate parameters follow the distributions of the synthetic workloads:
    photolysis J log-uniform 1e-6..1e-2 s^-1; bimolecular Arrhenius A
    log-uniform 1e-14..1e-10 cm^3 s^-1 and C uniform -2000..500 K; Troe k0
    ~1e-30 cm^6 s^-1 and kinf ~1e-11 cm^3 s^-1 with Fc = 0.6, N = 1;
    emission log-uniform 1e-6..1e-3 ppb/s; loss log-uniform 1e-6..1e-4 s^-1.
    Every chemical reaction conserves one integer 'atom' count per species.
    """
    rng = np.random.default_rng(seed)
    names = [f"{prefix}{i}" for i in range(n_species)]
    atoms = {s: int(rng.integers(1, 5)) for s in names}
    occ = _Occupancy(names, max_occupancy, rng)
    rxns = []
    for _ in range(n_arrhenius):
        a, b = occ.pick(2)
        n_prod = int(rng.integers(1, 4))
        prods = occ.pick(n_prod, exclude=(a, b))
        rxns.append({"type": "ARRHENIUS", "reactants": {a: 1, b: 1},
                     "products": _yields(atoms[a] + atoms[b], prods, atoms),
                     "A": float(_logu(rng, 1e-14, 1e-10)), "B": 0.0,
                     "C": float(rng.uniform(-2000.0, 500.0)), "D": 300.0, "E": 0.0})
    for _ in range(n_troe):
        a, b = occ.pick(2)
        (c,) = occ.pick(1, exclude=(a, b))
        rxns.append({"type": "TROE", "reactants": {a: 1, b: 1},
                     "products": _yields(atoms[a] + atoms[b], [c], atoms),
                     "k0_A": float(1e-30 * _logu(rng, 0.5, 2.0)),
                     "k0_B": float(rng.uniform(-4.0, -2.0)), "k0_C": 0.0,
                     "kinf_A": float(1e-11 * _logu(rng, 0.5, 2.0)),
                     "kinf_B": float(rng.uniform(-1.0, 0.0)), "kinf_C": 0.0,
                     "Fc": 0.6, "N": 1.0})
    for _ in range(n_photolysis):
        (x,) = occ.pick(1)
        n_prod = int(rng.integers(1, 4))
        prods = occ.pick(n_prod, exclude=(x,))
        rxns.append({"type": "PHOTOLYSIS", "reactants": {x: 1},
                     "products": _yields(atoms[x], prods, atoms),
                     "value": float(_logu(rng, 1e-6, 1e-2))})
    for s in occ.pick(n_emission):
        rxns.append({"type": "EMISSION", "species": s,
                     "value": float(_logu(rng, 1e-6, 1e-3))})
    for s in occ.pick(n_loss):
        v = loss_value if loss_value is not None else float(_logu(rng, 1e-6, 1e-4))
        rxns.append({"type": "FIRST_ORDER_LOSS", "species": s, "value": v})
    return {"name": name,
            "species": [{"name": s, "atoms": atoms[s]} for s in names],
            "reactions": rxns}


def small_gas_mechanism(seed=101):
    """8 species, 12 reactions: 4 photolysis, 6 Arrhenius, 1 Troe, 1 loss.

    Species A, B, C form an isolated photolysis chain A -> B -> C (an analytic
    sub-case: two first-order steps, Bateman solution); the other five species
    carry the remaining 10 reactions.  The loss rate is fixed at 1e-5 s^-1.
    """
    rng = np.random.default_rng(seed)
    others = [f"X{i}" for i in range(5)]
    atoms = {"A": 1, "B": 1, "C": 1}
    atoms.update({s: int(rng.integers(1, 5)) for s in others})
    rxns = [
        {"type": "PHOTOLYSIS", "reactants": {"A": 1}, "products": {"B": 1.0},
         "value": float(_logu(rng, 1e-6, 1e-2))},
        {"type": "PHOTOLYSIS", "reactants": {"B": 1}, "products": {"C": 1.0},
         "value": float(_logu(rng, 1e-6, 1e-2))},
    ]
    sub = gas_mechanism("x", 5, 6, 1, 2, 0, 1, seed=seed + 1000, max_occupancy=12,
                        loss_value=1e-5, prefix="X")
    for s in sub["species"]:
        atoms[s["name"]] = s["atoms"]
    # photolysis first so the four photolysis reactions are adjacent
    order = {"PHOTOLYSIS": 0, "ARRHENIUS": 1, "TROE": 2, "FIRST_ORDER_LOSS": 3}
    rxns += sorted(sub["reactions"], key=lambda r: order[r["type"]])
    names = ["A", "B", "C"] + others
    return {"name": "small-gas-8x12",
            "species": [{"name": s, "atoms": atoms[s]} for s in names],
            "reactions": rxns}


def large_gas_mechanism(seed=102):
    """72 species, 186 reactions: 112 Arrhenius, 28 Troe, 28 photolysis,
    9 emission, 9 first-order loss; each species in at most 12 reactions."""
    return gas_mechanism("gas-72x186", 72, 112, 28, 28, 9, 9, seed=seed)


def add_aqueous_sections(gas, seed=103, n_sections=8, n_phase_species=20, n_henry=10,
                         n_split_eq=4, n_simple_eq=2):
    """Append an aqueous phase instanced in every aerosol section.

    `n_henry` gas species get Henry's-law transfer into phase species a0..a9
    (kH log-uniform 1e-2..1e5 M/atm, given to the mechanism in M/Pa; C_H
    uniform 2000..6000 K; accommodation uniform 0.01..1; Dg = 1e-5 m^2/s times
    uniform 0.5..2; MW uniform 30..150 g/mol).  Aqueous reversible equilibria
    (K_eq log-uniform 1e-8..1e2, C = 0, kr log-uniform 1e-2..1e4) turn a
    transferred species into one or two of the remaining phase species, each
    used once, conserving the atom count.
    """
    rng = np.random.default_rng(seed)
    mech = json.loads(json.dumps(gas))
    gas_atoms = {s["name"]: s["atoms"] for s in mech["species"]}
    gas_names = [s["name"] for s in mech["species"]]
    henry_gas = [gas_names[i] for i in sorted(rng.choice(len(gas_names), n_henry, replace=False))]
    ph = [f"a{i}" for i in range(n_phase_species)]
    atoms = {}
    rxns = []
    for i, g in enumerate(henry_gas):
        atoms[ph[i]] = gas_atoms[g]
        rxns.append({"type": "HL_PHASE_TRANSFER", "gas": g, "aqueous": ph[i],
                     "H298": float(_logu(rng, 1e-2, 1e5)) / 101325.0,
                     "C_H": float(rng.uniform(2000.0, 6000.0)),
                     "alpha": float(rng.uniform(0.01, 1.0)),
                     "Dg": float(1e-5 * rng.uniform(0.5, 2.0)),
                     "MW": float(rng.uniform(30.0, 150.0)) * 1e-3})
    free = ph[n_henry:]
    heavy = [p for p in ph[:n_henry] if atoms[p] >= 2]
    light = [p for p in ph[:n_henry] if p not in heavy]
    rng.shuffle(heavy)
    rng.shuffle(light)
    n_split = min(n_split_eq, len(heavy))
    n_simple = n_split_eq + n_simple_eq - n_split
    reactants = heavy[:n_split] + (light + heavy[n_split:])[:n_simple]
    for k, a in enumerate(reactants):
        if k < n_split:
            b, c = free.pop(0), free.pop(0)
            atoms[b] = int(rng.integers(1, atoms[a]))
            atoms[c] = atoms[a] - atoms[b]
            prods = {b: 1, c: 1}
        else:
            b = free.pop(0)
            atoms[b] = atoms[a]
            prods = {b: 1}
        rxns.append({"type": "AQUEOUS_REVERSIBLE", "reactants": {a: 1}, "products": prods,
                     "A": float(_logu(rng, 1e-8, 1e2)), "C": 0.0,
                     "kr": float(_logu(rng, 1e-2, 1e4))})
    for p in free:
        atoms[p] = 1
    mech["name"] = gas["name"] + f"+aq{n_sections}x{n_phase_species}"
    mech["phases"] = {"aqueous": [{"name": p, "atoms": atoms[p]} for p in ph]}
    mech["aerosol"] = {"phase": "aqueous", "sections": n_sections}
    mech["reactions"] = mech["reactions"] + rxns
    return mech


def multiphase_mechanism(seed=103):
    """72 gas species + 8 sections x 20 aqueous species = 232 species,
    186 + 8*(10 + 6) = 314 reaction instances."""
    return add_aqueous_sections(large_gas_mechanism(), seed=seed)


def small_multiphase_mechanism(seed=104):
    """8 gas species + 8 sections x 20 aqueous species = 168 species."""
    return add_aqueous_sections(small_gas_mechanism(), seed=seed, n_henry=5,
                                n_split_eq=2, n_simple_eq=1)


def process_variety_mechanism(seed=106, n_sections=4):
    """Every process type of Table 2 that this solver implements, in one
    mechanism: the 8-species gas mechanism plus an HOx/NOy/isoprene block
    (CUSTOM_H2O2 for HO2 + HO2, CUSTOM_OH_HNO3 for OH + HNO3, the isoprene
    oxidation of Table 9 with its rate constants and yields) and a condensed
    phase per section with Henry's-law uptake of H2O2 and SO2, SIMPOL.1
    partitioning of the two isoprene products (Table 9's B parameters),
    condensed-phase Arrhenius chemistry and one aqueous equilibrium.
    Parameters the paper does not print are drawn here (custom rate
    constants near their usual magnitudes; transfer parameters as in
    add_aqueous_sections)."""
    rng = np.random.default_rng(seed)
    mech = json.loads(json.dumps(small_gas_mechanism()))
    extra = ["HO2", "H2O2", "OH", "HNO3", "NO3", "O3", "ISOP", "ISOPP1", "ISOPP2", "SO2"]
    mech["species"] += [{"name": s, "atoms": 1} for s in extra]

    def arr(A, C):
        return {"A": float(A), "B": 0.0, "C": float(C), "D": 300.0, "E": 0.0}

    def drawn(prefix, A, C):  # A exp(C/T) around a usual magnitude
        return {f"{prefix}_A": float(A * _logu(rng, 0.5, 2.0)), f"{prefix}_B": 0.0,
                f"{prefix}_C": float(C + rng.uniform(-100.0, 100.0))}

    rx = mech["reactions"]
    rx += [
        {"type": "CUSTOM_H2O2", "reactants": {"HO2": 2}, "products": {"H2O2": 1.0},
         **drawn("k1", 3e-13, 460.0), **drawn("k2", 2e-33, 920.0)},
        {"type": "CUSTOM_OH_HNO3", "reactants": {"OH": 1, "HNO3": 1}, "products": {"NO3": 1.0},
         **drawn("k0", 2.4e-14, 460.0), **drawn("k2", 2.7e-17, 2199.0), **drawn("k3", 6.5e-34, 1335.0)},
        {"type": "PHOTOLYSIS", "reactants": {"H2O2": 1}, "products": {"OH": 2.0},
         "value": float(_logu(rng, 1e-6, 1e-5))},
        {"type": "PHOTOLYSIS", "reactants": {"NO3": 1}, "products": {"HNO3": 1.0},
         "value": float(_logu(rng, 1e-3, 1e-1))},
        {"type": "ARRHENIUS", "reactants": {"OH": 1, "O3": 1}, "products": {"HO2": 1.0},
         **arr(1.7e-12, -940.0)},
        # isoprene oxidation, Table 9 (mass-based yields)
        {"type": "ARRHENIUS", "reactants": {"ISOP": 1, "OH": 1}, "products": {"ISOPP1": 0.192},
         **arr(2.54e-11, 407.6)},
        {"type": "ARRHENIUS", "reactants": {"ISOP": 1, "O3": 1}, "products": {"ISOPP2": 0.215},
         **arr(7.86e-15, -1912.0)},
        {"type": "EMISSION", "species": "ISOP", "value": float(_logu(rng, 1e-4, 1e-3))},
        {"type": "EMISSION", "species": "O3", "value": float(_logu(rng, 1e-4, 1e-3))},
        {"type": "FIRST_ORDER_LOSS", "species": "HNO3", "value": float(_logu(rng, 1e-5, 1e-4))},
    ]
    ph = ["H2O2aq", "SO2aq", "HSO3", "SULF", "SOA1", "SOA2", "OLIG"]

    def transfer():
        return {"alpha": float(rng.uniform(0.01, 1.0)), "Dg": float(1e-5 * rng.uniform(0.5, 2.0)),
                "MW": float(rng.uniform(30.0, 150.0)) * 1e-3}

    rx += [
        {"type": "HL_PHASE_TRANSFER", "gas": "H2O2", "aqueous": "H2O2aq",
         "H298": float(_logu(rng, 1e4, 1e5)) / 101325.0, "C_H": float(rng.uniform(2000.0, 6000.0)),
         **transfer()},
        {"type": "HL_PHASE_TRANSFER", "gas": "SO2", "aqueous": "SO2aq",
         "H298": float(_logu(rng, 1e2, 1e3)) / 101325.0, "C_H": float(rng.uniform(2000.0, 6000.0)),
         **transfer()},
        {"type": "SIMPOL_PHASE_TRANSFER", "gas": "ISOPP1", "aqueous": "SOA1",
         "B": [3.81e3, -2.13e1, 0.0, 0.0], **transfer()},
        {"type": "SIMPOL_PHASE_TRANSFER", "gas": "ISOPP2", "aqueous": "SOA2",
         "B": [3.81e3, -2.09e1, 0.0, 0.0], **transfer()},
        {"type": "AQUEOUS_REVERSIBLE", "reactants": {"SO2aq": 1}, "products": {"HSO3": 1},
         "A": float(_logu(rng, 1e-2, 1e1)), "C": 0.0, "kr": float(_logu(rng, 1e-1, 1e2))},
        {"type": "CONDENSED_ARRHENIUS", "reactants": {"H2O2aq": 1, "HSO3": 1},
         "products": {"SULF": 1.0}, "A": float(_logu(rng, 1e5, 1e7)), "B": 0.0,
         "C": float(rng.uniform(-4000.0, -3000.0)), "D": 300.0, "E": 0.0},
        {"type": "CONDENSED_ARRHENIUS", "reactants": {"SOA1": 1}, "products": {"OLIG": 1.0},
         "A": float(_logu(rng, 1e-5, 1e-3)), "B": 0.0, "C": 0.0, "D": 300.0, "E": 0.0},
    ]
    mech["name"] = f"process-variety-{len(mech['species'])}+aq{n_sections}x{len(ph)}"
    mech["phases"] = {"aqueous": [{"name": p, "atoms": 1} for p in ph]}
    mech["aerosol"] = {"phase": "aqueous", "sections": n_sections}
    return mech


def particle_resolved_mechanism(n_particles=128, seed=106):
    """The process-variety mechanism with its condensed phase instanced once
    per computational particle (the particle-resolved SingleParticle
    representation, Sect. 2.2.3 and Table 6; the paper's box model used 10^4
    particles, Sect. 4.1): the same instance expansion as the sections, with
    many more instances, so the Jacobian is block-arrow (particle blocks coupled to the gas species
    they exchange with).  18 gas species + 7 per particle."""
    mech = process_variety_mechanism(seed=seed, n_sections=n_particles)
    mech["name"] = f"particle-resolved-{n_particles}x7+gas18"
    mech["aerosol"]["representation"] = "particles"
    return mech


def water_mechanism(seed=107, n_sections=8):
    """The 232-species multiphase mechanism with its aerosol water as a
    parameter (Sect. 2.2.2; Table 4, ZSRAerosolWater): one more phase species,
    an inert salt (the sections' dry particle volume, per cell), and a ZSR
    water parameter over two electrolytes -- the
    salt and the aqueous species that the first Henry's-law transfer feeds,
    so that the water, and with it every section rate that depends on the
    liquid volume, follows the state.  72 gas + 8 x 21 phase species = 240.
    The paper prints no molality fits, so each electrolyte gets a synthetic
    fit of the Jacobson et al. (1996) form sqrt(m) = Y0 + Y1 a_w + Y2 a_w^2:
    molality log-uniform 4..12 mol/kg at a_w = 0.5 and 0.5..2 at 0.95 for
    the salt, ten times that for the fed species (it holds a tenth of the
    salt's water per mole), joined linearly in sqrt(m) plus a small
    curvature, held below a_w = 0.5."""
    rng = np.random.default_rng(seed)
    mech = multiphase_mechanism()
    mech["phases"]["aqueous"].append({"name": "SALT", "atoms": 1})
    hl = [r for r in mech["reactions"] if r["type"] == "HL_PHASE_TRANSFER"]
    electrolytes = []
    for name, scale in (("SALT", 1.0), (hl[0]["aqueous"], 10.0)):
        s05 = math.sqrt(scale * float(_logu(rng, 4.0, 12.0)))
        s95 = math.sqrt(scale * float(_logu(rng, 0.5, 2.0)))
        kappa = float(rng.uniform(-0.5, 0.5))
        slope = (s95 - s05) / 0.45
        # s05 + slope (a - 0.5) + kappa (a - 0.5)(a - 0.95), expanded in a
        Y = [s05 - 0.5 * slope + kappa * 0.475, slope - 1.45 * kappa, kappa]
        electrolytes.append({"species": name, "Y": Y, "low_RH": 0.5})
    mech["parameters"] = [{"type": "ZSR_AEROSOL_WATER", "electrolytes": electrolytes}]
    mech["name"] = f"multiphase-water-{len(mech['species']) + n_sections * 21}"
    return mech


# --------------------------------------------------------------------------
# layout helpers (interface description only)
# --------------------------------------------------------------------------

@dataclass
class Layout:
    species: list          # full species names in state order
    atoms: np.ndarray      # integer atom count per species
    env: list              # env entry names in order
    runtime_defaults: list  # default value per runtime entry
    runtime_kind: list     # reaction type per runtime entry
    n_sections: int


def layout(mech) -> Layout:
    species = [s["name"] for s in mech["species"]]
    atoms = [s["atoms"] for s in mech["species"]]
    nsec = mech.get("aerosol", {}).get("sections", 0)
    if nsec:
        phase = mech["phases"][mech["aerosol"]["phase"]]
        for b in range(nsec):
            species += [f"bin{b}.{p['name']}" for p in phase]
            atoms += [p["atoms"] for p in phase]
    env = ["T", "P"]
    defaults, kinds = [], []
    for i, r in enumerate(mech["reactions"]):
        if r["type"] in RUNTIME_TYPES:
            env.append(f"{r['type'].lower()}[{i}]")
            defaults.append(float(r["value"]))
            kinds.append(r["type"])
    if mech.get("parameters"):
        env.append("RH")
    for b in range(nsec):
        env += [f"bin{b}.r", f"bin{b}.N", f"bin{b}.L"]
    return Layout(species, np.array(atoms, dtype=np.int64), env, defaults, kinds, nsec)


# --------------------------------------------------------------------------
# per-cell inputs
# --------------------------------------------------------------------------

SECTION_RADII = np.logspace(math.log10(1e-8), math.log10(1e-5), 8)  # m, 0.01..10 um


def cells(mech, n_cells, seed, T=None, P=None, sza=True, night_fraction=None,
          cloud_fraction=0.0, y_range=(1e-3, 1e2)):
    """Initial state [n_cells, n_species] (ppb) and env [n_cells, n_env].

    T uniform 220..310 K and P uniform 2e4..1.013e5 Pa unless fixed; the
    photolysis entries are the mechanism defaults times max(cos SZA, 0) with
    SZA uniform 0..100 deg (or unscaled when sza=False).  Gas species start
    log-uniform in y_range ppb, aqueous species at 0.  Sections: radii
    log-spaced 0.01..10 um, N log-uniform 1e1..1e4 cm^-3, water volume
    L = N * 4/3 pi r^3.  With night_fraction, that share of cells gets J = 0.
    With cloud_fraction, that share of cells holds cloud water: a liquid water
    content uniform 0.1..1 g/m^3 spread over the sections in proportion to
    N r^3; the other cells of a sectional mechanism then hold no water (L = 0).
    A particle-resolved mechanism (aerosol "representation": "particles")
    gets per cell and particle a radius log-normal around 0.1 um (geometric
    standard deviation 1.8, within 5 nm..10 um), the cell's number
    concentration (log-uniform 1e2..1e4 cm^-3) shared evenly by its
    computational particles, and L = N 4/3 pi r^3.
    """
    rng = np.random.default_rng(seed)
    lay = layout(mech)
    n = len(lay.species)
    n_gas = len(mech["species"])
    y = np.zeros((n_cells, n))
    y[:, :n_gas] = _logu(rng, y_range[0], y_range[1], (n_cells, n_gas))
    env = np.zeros((n_cells, len(lay.env)))
    env[:, 0] = T if T is not None else rng.uniform(220.0, 310.0, n_cells)
    env[:, 1] = P if P is not None else rng.uniform(2e4, 1.013e5, n_cells)
    if sza:
        mu = np.maximum(np.cos(np.deg2rad(rng.uniform(0.0, 100.0, n_cells))), 0.0)
    else:
        mu = np.ones(n_cells)
    if night_fraction is not None:
        night = rng.random(n_cells) < night_fraction
        mu = np.where(night, 0.0, mu)
    for k, (d, kind) in enumerate(zip(lay.runtime_defaults, lay.runtime_kind)):
        env[:, 2 + k] = d * (mu if kind == "PHOTOLYSIS" else 1.0)
    base = 2 + len(lay.runtime_defaults)
    water = bool(mech.get("parameters"))
    if water:  # relative humidity, and the electrolytes that hold the water
        env[:, base] = rng.uniform(0.5, 0.95, n_cells)
        base += 1
    if lay.n_sections and mech["aerosol"].get("representation") == "particles":
        P = lay.n_sections
        r = np.clip(np.exp(rng.normal(math.log(1e-7), math.log(1.8), (n_cells, P))), 5e-9, 1e-5)
        N = np.repeat(_logu(rng, 1e8, 1e10, (n_cells, 1)) / P, P, axis=1)
        L = N * (4.0 / 3.0) * math.pi * r ** 3
    elif lay.n_sections:
        r = SECTION_RADII[: lay.n_sections]
        N = _logu(rng, 1e1, 1e4, (n_cells, lay.n_sections)) * 1e6
        L = N * (4.0 / 3.0) * math.pi * r[None, :] ** 3
        if cloud_fraction > 0.0:
            cloudy = rng.random(n_cells) < cloud_fraction
            lwc = rng.uniform(0.1, 1.0, n_cells) * 1e-6  # m^3 water / m^3 air
            share = N * r[None, :] ** 3
            share = share / share.sum(axis=1, keepdims=True)
            L = np.where(cloudy[:, None], lwc[:, None] * share, 0.0)
        r = np.broadcast_to(r[None, :], (n_cells, lay.n_sections))
    if water:
        # all section water comes from the electrolytes: L_env = 0.  Each
        # section's dry particles, N 4/3 pi r^3 per m^3 of air, are salt of
        # 13400 mol m^-3 (1770 kg m^-3 at 0.132 kg mol^-1, ammonium-sulphate
        # like); the other electrolytes start at 1% of the salt
        L = np.zeros_like(L)
        idx = {s: i for i, s in enumerate(lay.species)}
        air = env[:, 1] / (8.314462618 * env[:, 0])  # mol air per m^3
        for b in range(lay.n_sections):
            salt = N[:, b] * (4.0 / 3.0) * math.pi * r[:, b] ** 3 * 13400.0 / air * 1e9
            for e in mech["parameters"][0]["electrolytes"]:
                name = f"bin{b}.{e['species']}"
                y[:, idx[name]] = salt if e["species"] == "SALT" else 0.01 * salt
    if lay.n_sections:
        for b in range(lay.n_sections):
            env[:, base + 3 * b] = r[:, b]
            env[:, base + 3 * b + 1] = N[:, b]
            env[:, base + 3 * b + 2] = L[:, b]
    return y, env


# --------------------------------------------------------------------------
# the five benchmark workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    mech: dict
    n_cells: int
    dt: float
    n_outer: int
    rtol: float
    atol: float
    cell_seed: int
    cell_kwargs: dict

    def json(self):
        return json.dumps(self.mech)

    def inputs(self, n_cells=None):
        return cells(self.mech, self.n_cells if n_cells is None else n_cells,
                     self.cell_seed, **self.cell_kwargs)


def uneven_batch(n_cells=131072, seed=204, cloud_fraction=0.1, night_fraction=0.5):
    """Cells of uneven stiffness: half dark (J = 0), and a `cloud_fraction`
    share carrying the aqueous sections with cloud water (liquid water
    content uniform 0.1..1 g/m^3 spread over the sections in proportion to
    N r^3); the rest are gas-only cells of the 72-species mechanism.
    Returns [(mechanism, y0, env), ...] for the gas and cloud groups and the
    seeded random cell order they were drawn in."""
    rng = np.random.default_rng(seed)
    cloudy = rng.random(n_cells) < cloud_fraction
    n_cloud = int(cloudy.sum())
    gas, mp = large_gas_mechanism(), multiphase_mechanism()
    yg, eg = cells(gas, n_cells - n_cloud, seed + 1, night_fraction=night_fraction)
    ym, em = cells(mp, n_cloud, seed + 2, night_fraction=night_fraction, cloud_fraction=1.0)
    return [(gas, yg, eg), (mp, ym, em)], np.flatnonzero(cloudy)


def dark_cells(mech, env):
    """Boolean [cells]: cells whose photolysis rates are all zero (night,
    or the sun below the horizon)."""
    lay = layout(mech)
    ks = [2 + k for k, kind in enumerate(lay.runtime_kind) if kind == "PHOTOLYSIS"]
    return (env[:, ks] == 0.0).all(axis=1) if ks else np.zeros(len(env), dtype=bool)


def stratified_sample(groups, n, seed=17):
    """A seeded random sample of about n cells of an uneven batch (the
    [(mechanism, y0, env), ...] of uneven_batch), stratified by group and by
    dark / lit cells, each stratum's share in proportion to its size (at
    least one cell of every non-empty stratum).  Returns one sorted index
    array per group; a timing over group g's sample extrapolates to the
    whole group by len(group) / len(sample)."""
    rng = np.random.default_rng(seed)
    total = sum(len(y) for _, y, _ in groups)
    out = []
    for mj, y, env in groups:
        dark = dark_cells(mj, env)
        picks = []
        for mask in (dark, ~dark):
            idx = np.flatnonzero(mask)
            if len(idx) == 0:
                continue
            k = min(len(idx), max(1, int(round(n * len(idx) / total))))
            picks.append(rng.choice(idx, k, replace=False))
        out.append(np.sort(np.concatenate(picks)) if picks else np.zeros(0, dtype=np.int64))
    return out


def serving_requests(n_requests=2000, seed=205, gas_share=0.7, cells_lo=256, cells_hi=65536,
                     dt_lo=60.0, dt_hi=600.0):
    """A stream of chunk requests: size log-uniform in [cells_lo, cells_hi],
    mechanism gas-72 with probability gas_share else multiphase-232, step
    uniform in [dt_lo, dt_hi] s, inputs seeded per request.  Arrival times
    are drawn by the caller (Poisson at a chosen rate)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_requests):
        out.append({"cells": int(np.exp(rng.uniform(math.log(cells_lo), math.log(cells_hi)))),
                    "mech": "gas72" if rng.random() < gas_share else "multiphase232",
                    "dt": float(rng.uniform(dt_lo, dt_hi)), "seed": 10_000 + i})
    return out


def workload(k: int) -> Workload:
    """k = 1..3: the single-mechanism workloads (sizes in the docstrings);
    k = 6: the particle-resolved workload; k = 7: the water-parameter
    workload; k = 8: particle-resolved cells at the paper's 10^4
    computational particles (70018 species; the block-arrow solve)."""
    if k == 1:
        return Workload("small-gas 1 cell, 60 x 60 s", small_gas_mechanism(), 1, 60.0, 60,
                        1e-4, 1e-5, 201, dict(T=298.0, P=101300.0, sza=False))
    if k == 2:
        return Workload("gas-72x186 16384 cells, 180 s", large_gas_mechanism(), 16384, 180.0, 1,
                        1e-4, 1e-5, 202, {})
    if k == 3:
        return Workload("multiphase-232 4096 cells, 300 s", multiphase_mechanism(), 4096, 300.0, 1,
                        1e-4, 1e-5, 203, {})
    if k == 6:  # the particle-resolved shape (a row beyond the five configurations)
        return Workload("particle-resolved 128 particles (914 species) 2048 cells, 180 s",
                        particle_resolved_mechanism(128), 2048, 180.0, 1, 1e-4, 1e-5, 206, {})
    if k == 7:  # aerosol water as a parameter of the state
        return Workload("multiphase-water-240 (ZSR water parameter) 4096 cells, 300 s",
                        water_mechanism(), 4096, 300.0, 1, 1e-4, 1e-5, 207, {})
    if k == 8:  # the paper's particle count (Sect. 4.1)
        return Workload("particle-resolved 10^4 particles (70018 species) 152 cells, 180 s",
                        particle_resolved_mechanism(10000), 152, 180.0, 1, 1e-4, 1e-5, 208, {})
    raise ValueError(k)
