"""Oracle side: read a mechanism JSON text into the oracle's own arrays.

TEST INFRASTRUCTURE ONLY -- imported by tests, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py; the product path never imports it.

Mechanism semantics (CAMP paper Sect. 2.2.1, Table 2; Sect. 2.2.3 for the
aerosol phase instances): every process declared on an aerosol phase is
applied to each instance of that phase, here one instance per section, so the
process list is the declaration order with each section process expanded
over sections 0..nb-1 in place.
"""
from __future__ import annotations

import ctypes
import json
from dataclasses import dataclass, field

KB = 1.380649e-23

TYPE_CODE = {"ARRHENIUS": 0, "TROE": 1, "PHOTOLYSIS": 2, "EMISSION": 3,
             "FIRST_ORDER_LOSS": 4, "HL_PHASE_TRANSFER": 5, "AQUEOUS_REVERSIBLE": 6,
             "CUSTOM_H2O2": 7, "CUSTOM_OH_HNO3": 8, "CONDENSED_ARRHENIUS": 9,
             "SIMPOL_PHASE_TRANSFER": 10}
RUNTIME = ("PHOTOLYSIS", "EMISSION", "FIRST_ORDER_LOSS")
SECTIONED = ("HL_PHASE_TRANSFER", "AQUEOUS_REVERSIBLE", "CONDENSED_ARRHENIUS",
             "SIMPOL_PHASE_TRANSFER")
REVERSIBLE = ("HL_PHASE_TRANSFER", "AQUEOUS_REVERSIBLE", "SIMPOL_PHASE_TRANSFER")
WATER_MOLARITY = 1000.0 / 18.015  # mol L^-1, default total molarity of a condensed phase
MAXSP = 4


class OmRxn(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int),
                ("n_react", ctypes.c_int),
                ("react", ctypes.c_int * MAXSP),
                ("rstoich", ctypes.c_int * MAXSP),
                ("n_prod", ctypes.c_int),
                ("prod", ctypes.c_int * MAXSP),
                ("yield_", ctypes.c_double * MAXSP),
                ("env_slot", ctypes.c_int),
                ("section", ctypes.c_int),
                ("p", ctypes.c_double * 10)]


ZSR_NY = 8  # coefficients of one molality fit


class OmMech(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int),
                ("n_rxn", ctypes.c_int),
                ("n_env", ctypes.c_int),
                ("n_sections", ctypes.c_int),
                ("env_section_base", ctypes.c_int),
                ("rxn", ctypes.POINTER(OmRxn)),
                ("rh_slot", ctypes.c_int),
                ("n_zsr", ctypes.c_int),
                ("zsr_species", ctypes.POINTER(ctypes.c_int)),
                ("zsr_Y", ctypes.POINTER(ctypes.c_double)),
                ("zsr_low", ctypes.POINTER(ctypes.c_double))]


@dataclass
class Process:
    """One process instance: reactants/products as (species index, coefficient)."""
    type: str
    reactants: list            # [(idx, int stoich)] distinct, declaration order
    products: list             # [(idx, float yield)] distinct, declaration order
    params: list
    env_slot: int = -1
    section: int = -1

    @property
    def reversible(self):
        return self.type in REVERSIBLE


@dataclass
class Mechanism:
    species: list
    index: dict
    processes: list
    n_env: int
    n_sections: int
    env_section_base: int
    raw: dict = field(repr=False, default=None)
    # ZSR aerosol-water parameter (Sect. 2.2.2, Table 4): env slot of the
    # relative humidity (-1: none) and per electrolyte (phase species name,
    # fit coefficients Y_j of sqrt(m) = sum_j Y_j a_w^j, lowest a_w of the fit)
    rh_slot: int = -1
    electrolytes: list = field(default_factory=list)

    @property
    def n(self):
        return len(self.species)


def _merge(pairs):
    out, seen = [], {}
    for idx, c in pairs:
        if idx in seen:
            out[seen[idx]] = (idx, out[seen[idx]][1] + c)
        else:
            seen[idx] = len(out)
            out.append((idx, c))
    return out


def parse(text) -> Mechanism:
    d = json.loads(text) if isinstance(text, (str, bytes)) else text
    species = [s["name"] for s in d["species"]]
    nsec = 0
    phase = []
    if "aerosol" in d:
        nsec = int(d["aerosol"]["sections"])
        phase = [p["name"] for p in d["phases"][d["aerosol"]["phase"]]]
        for b in range(nsec):
            species += [f"bin{b}.{p}" for p in phase]
    index = {s: i for i, s in enumerate(species)}
    if len(index) != len(species):
        raise ValueError("duplicate species name")
    n_runtime = sum(1 for r in d["reactions"] if r["type"] in RUNTIME)
    electrolytes = []
    for par in d.get("parameters", []):
        if par["type"] != "ZSR_AEROSOL_WATER":
            raise ValueError(f"unknown parameter type {par['type']}")
        if electrolytes or not nsec:
            raise ValueError("one water parameter, on a mechanism with aerosol sections")
        for e in par["electrolytes"]:
            Y = [float(v) for v in e["Y"]]
            if not 1 <= len(Y) <= ZSR_NY or e["species"] not in phase:
                raise ValueError("bad electrolyte")
            electrolytes.append((e["species"], Y + [0.0] * (ZSR_NY - len(Y)),
                                 float(e.get("low_RH", 0.0))))
        if not electrolytes:
            raise ValueError("a water parameter needs electrolytes")
    rh_slot = 2 + n_runtime if electrolytes else -1
    base = 2 + n_runtime + (1 if electrolytes else 0)
    procs = []
    slot = 2
    for r in d["reactions"]:
        t = r["type"]
        if t not in TYPE_CODE:
            raise ValueError(f"unknown reaction type {t}")
        if t in SECTIONED:
            for b in range(nsec):
                def sp(name, b=b):
                    return index[f"bin{b}.{name}"]
                if t == "HL_PHASE_TRANSFER":
                    procs.append(Process(t, [(index[r["gas"]], 1)], [(sp(r["aqueous"]), 1.0)],
                                         [r["H298"], r["C_H"], r["alpha"], r["Dg"], r["MW"]],
                                         section=b))
                elif t == "SIMPOL_PHASE_TRANSFER":
                    B = list(r["B"]) + [0.0] * (4 - len(r["B"]))
                    procs.append(Process(t, [(index[r["gas"]], 1)], [(sp(r["aqueous"]), 1.0)],
                                         B[:4] + [r["alpha"], r["Dg"], r["MW"],
                                                  r.get("c_tot", WATER_MOLARITY)],
                                         section=b))
                elif t == "CONDENSED_ARRHENIUS":
                    rs = _merge([(sp(k), int(v)) for k, v in r["reactants"].items()])
                    ps = _merge([(sp(k), float(v)) for k, v in r.get("products", {}).items()])
                    C = r["C"] if "C" in r else -r.get("Ea", 0.0) / KB
                    procs.append(Process(t, rs, ps, [r["A"], r.get("B", 0.0), C, r.get("D", 300.0),
                                                     r.get("E", 0.0)], section=b))
                else:
                    rs = _merge([(sp(k), int(v)) for k, v in r["reactants"].items()])
                    ps = _merge([(sp(k), float(int(v))) for k, v in r["products"].items()])
                    procs.append(Process(t, rs, ps, [r["A"], r.get("C", 0.0), r["kr"]], section=b))
            continue
        if t == "EMISSION":
            procs.append(Process(t, [], [(index[r["species"]], 1.0)], [], env_slot=slot))
        elif t == "FIRST_ORDER_LOSS":
            procs.append(Process(t, [(index[r["species"]], 1)], [], [], env_slot=slot))
        else:
            rs = _merge([(index[k], int(v)) for k, v in r["reactants"].items()])
            ps = _merge([(index[k], float(v)) for k, v in r.get("products", {}).items()])
            if t == "ARRHENIUS":
                C = r["C"] if "C" in r else -r.get("Ea", 0.0) / KB
                params = [r["A"], r.get("B", 0.0), C, r.get("D", 300.0), r.get("E", 0.0)]
            elif t == "TROE":
                params = [r["k0_A"], r.get("k0_B", 0.0), r.get("k0_C", 0.0),
                          r["kinf_A"], r.get("kinf_B", 0.0), r.get("kinf_C", 0.0),
                          r.get("Fc", 0.6), r.get("N", 1.0)]
            elif t == "CUSTOM_H2O2":
                params = [r[f"k{i}_{c}"] if c == "A" else r.get(f"k{i}_{c}", 0.0)
                          for i in (1, 2) for c in "ABC"]
            elif t == "CUSTOM_OH_HNO3":
                params = [r[f"k{i}_{c}"] if c == "A" else r.get(f"k{i}_{c}", 0.0)
                          for i in (0, 2, 3) for c in "ABC"]
            else:  # PHOTOLYSIS
                params = []
            procs.append(Process(t, rs, ps, params,
                                 env_slot=slot if t in RUNTIME else -1))
        if t in RUNTIME:
            slot += 1
    for p in procs:
        if p.type in ("AQUEOUS_REVERSIBLE", "CONDENSED_ARRHENIUS") and not p.reactants:
            raise ValueError("a condensed-phase reaction needs reactants")
        if p.type == "AQUEOUS_REVERSIBLE" and not p.products:
            raise ValueError("a reversible aqueous reaction needs products")
    return Mechanism(species, index, procs, base + 3 * nsec, nsec, base, d, rh_slot, electrolytes)


def water_powers(p: Process):
    """Powers of 1/L in (kf, kr) of a section process when the liquid volume is
    a parameter: a side with f concentration factors carries L^-(f-1) (molarity
    y phi, phi ~ 1/L, one division by phi back to ppb s^-1); the evaporation
    constant of the phase-transfer types carries L^-1."""
    nr = sum(s for _, s in p.reactants)
    np_ = sum(int(y) for _, y in p.products)
    if p.type in ("HL_PHASE_TRANSFER", "SIMPOL_PHASE_TRANSFER"):
        return 0, 1
    if p.type == "AQUEOUS_REVERSIBLE":
        return nr - 1, np_ - 1
    if p.type == "CONDENSED_ARRHENIUS":
        return nr - 1, 0
    return 0, 0


def to_ctypes(m: Mechanism):
    """Build the C arrays; returns (OmMech, keepalive)."""
    arr = (OmRxn * max(1, len(m.processes)))()
    for k, p in enumerate(m.processes):
        r = arr[k]
        r.type = TYPE_CODE[p.type]
        if len(p.reactants) > MAXSP or len(p.products) > MAXSP:
            raise ValueError("too many species in one process")
        r.n_react = len(p.reactants)
        for i, (idx, s) in enumerate(p.reactants):
            r.react[i] = idx
            r.rstoich[i] = s
        r.n_prod = len(p.products)
        for i, (idx, y) in enumerate(p.products):
            r.prod[i] = idx
            r.yield_[i] = y
        r.env_slot = p.env_slot
        r.section = p.section
        for i, v in enumerate(p.params):
            r.p[i] = v
    ne = len(m.electrolytes)
    sp = (ctypes.c_int * max(1, m.n_sections * ne))()
    Y = (ctypes.c_double * max(1, ne * ZSR_NY))()
    low = (ctypes.c_double * max(1, ne))()
    for e, (name, coef, lo) in enumerate(m.electrolytes):
        for b in range(m.n_sections):
            sp[b * ne + e] = m.index[f"bin{b}.{name}"]
        for j, v in enumerate(coef):
            Y[e * ZSR_NY + j] = v
        low[e] = lo
    cm = OmMech(m.n, len(m.processes), m.n_env, m.n_sections, m.env_section_base,
                ctypes.cast(arr, ctypes.POINTER(OmRxn)), m.rh_slot, ne,
                ctypes.cast(sp, ctypes.POINTER(ctypes.c_int)),
                ctypes.cast(Y, ctypes.POINTER(ctypes.c_double)),
                ctypes.cast(low, ctypes.POINTER(ctypes.c_double)))
    return cm, (arr, sp, Y, low)
