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


class OmMech(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int),
                ("n_rxn", ctypes.c_int),
                ("n_env", ctypes.c_int),
                ("n_sections", ctypes.c_int),
                ("env_section_base", ctypes.c_int),
                ("rxn", ctypes.POINTER(OmRxn))]


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
    base = 2 + n_runtime
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
    return Mechanism(species, index, procs, base + 3 * nsec, nsec, base, d)


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
    cm = OmMech(m.n, len(m.processes), m.n_env, m.n_sections, m.env_section_base,
                ctypes.cast(arr, ctypes.POINTER(OmRxn)))
    return cm, arr
