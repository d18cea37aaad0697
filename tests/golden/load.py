"""Readers for the fixtures in this folder (values printed in the CAMP paper,
each file citing where)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def isoprene_soa_table9():
    """{'gas': {name: (reactants, products, A, C)}, 'partition': {name:
    (gas, aerosol, (B1, B2, B3, B4))}, 'environment': {'T': .., 'P': ..}}."""
    out = {"gas": {}, "partition": {}, "environment": {}}
    with open(os.path.join(HERE, "isoprene_soa_table9.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            kind, name, *rest = line
            if kind == "gas":
                reactants = {s: 1 for s in rest[0].split("+")}
                y, p = rest[1].split("*")
                out["gas"][name] = (reactants, {p: float(y)}, float(rest[2]), float(rest[3]))
            elif kind == "partition":
                out["partition"][name] = (rest[0], rest[1], tuple(float(v) for v in rest[2:6]))
            elif kind == "environment":
                for kv in rest:
                    k, v = kv.split("=")
                    out["environment"][k] = float(v)
    return out
