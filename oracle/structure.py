"""Oracle side: the integer structure of a mechanism, enumerated directly.

TEST INFRASTRUCTURE ONLY.  Recomputes, with plain Python sets and loops, the
integer work that the product's mechanism compiler does once per mechanism
(CAMP paper Table 1, get_used_jacobian_elements and update_ids):

  pattern   every (i, j) with d f_i / d y_j possibly non-zero, plus the
            diagonal: the rows R_k u P_k times the species D_k that appear in
            r_k (D_k = R_k, or R_k u P_k for reversible processes); with a
            ZSR water parameter (Sect. 2.2.2) also the rows R_k u P_k of every
            section process whose constants carry a power of 1/L, times the
            electrolytes of its section (the chain-rule term J_p P_y)
  rxn_map   for each process k, each j in D_k, each i in R_k u P_k (all in
            declaration order, reactants before products, each species once):
            the CSR position of (i, j)
  perm      exact minimum-degree elimination order on pattern u pattern^T
            (ties: smallest species index; eliminating a node joins its
            neighbours into a clique)
  lu        fill pattern of the permuted matrix under elimination without
            pivoting, rows and columns in permuted numbering
  levels    factor/forward level of row i: 1 + max level of rows k < i with
            (i, k) in lu (0 if none); backward level mirrors it over k > i
"""
from __future__ import annotations

from .mech import Mechanism, water_powers


def _ordered_unique(seq):
    out = []
    for s in seq:
        if s not in out:
            out.append(s)
    return out


def dependence(p):
    """Species whose values enter the process rate r_k."""
    d = [i for i, _ in p.reactants]
    if p.reversible:
        d += [i for i, _ in p.products]
    return _ordered_unique(d)


def rows_of(p):
    return _ordered_unique([i for i, _ in p.reactants] + [i for i, _ in p.products])


def pattern(m: Mechanism):
    s = {(i, i) for i in range(m.n)}
    for p in m.processes:
        for j in dependence(p):
            for i in rows_of(p):
                s.add((i, j))
        if m.electrolytes and p.section >= 0 and any(water_powers(p)):
            for name, _, _ in m.electrolytes:
                j = m.index[f"bin{p.section}.{name}"]
                for i in rows_of(p):
                    s.add((i, j))
    return s


def csr(pat, n):
    rows = [[] for _ in range(n)]
    for i, j in pat:
        rows[i].append(j)
    rowptr, colidx = [0], []
    for r in rows:
        colidx += sorted(r)
        rowptr.append(len(colidx))
    return rowptr, colidx


def rxn_map(m: Mechanism, rowptr, colidx):
    pos = {}
    for i in range(m.n):
        for q in range(rowptr[i], rowptr[i + 1]):
            pos[(i, colidx[q])] = q
    out = []
    for p in m.processes:
        for j in dependence(p):
            for i in rows_of(p):
                out.append(pos[(i, j)])
    return out


def min_degree(pat, n):
    adj = [set() for _ in range(n)]
    for i, j in pat:
        if i != j:
            adj[i].add(j)
            adj[j].add(i)
    alive = set(range(n))
    perm = []
    while alive:
        v = min(alive, key=lambda a: (len(adj[a]), a))
        perm.append(v)
        nb = adj[v]
        for a in nb:
            adj[a] |= nb
            adj[a].discard(a)
            adj[a].discard(v)
        alive.discard(v)
        adj[v] = set()
    return perm


def symbolic_lu(pat, perm, n):
    iperm = [0] * n
    for k, v in enumerate(perm):
        iperm[v] = k
    row = [set() for _ in range(n)]
    col = [set() for _ in range(n)]
    for i, j in pat:
        a, b = iperm[i], iperm[j]
        row[a].add(b)
        col[b].add(a)
    for k in range(n):
        lower = [i for i in col[k] if i > k]
        upper = [j for j in row[k] if j > k]
        for i in lower:
            for j in upper:
                if j not in row[i]:
                    row[i].add(j)
                    col[j].add(i)
    rowptr, colidx = [0], []
    for i in range(n):
        colidx += sorted(row[i])
        rowptr.append(len(colidx))
    return rowptr, colidx


def levels(lu_rowptr, lu_colidx, n):
    fwd = [0] * n
    for i in range(n):
        ks = [k for k in lu_colidx[lu_rowptr[i]:lu_rowptr[i + 1]] if k < i]
        fwd[i] = 1 + max(fwd[k] for k in ks) if ks else 0
    bwd = [0] * n
    for i in range(n - 1, -1, -1):
        js = [j for j in lu_colidx[lu_rowptr[i]:lu_rowptr[i + 1]] if j > i]
        bwd[i] = 1 + max(bwd[j] for j in js) if js else 0
    return fwd, bwd


def structure(m: Mechanism):
    """All integer arrays, as plain Python lists, keyed like the C ABI export."""
    pat = pattern(m)
    rowptr, colidx = csr(pat, m.n)
    rmap = rxn_map(m, rowptr, colidx)
    perm = min_degree(pat, m.n)
    lu_rowptr, lu_colidx = symbolic_lu(pat, perm, m.n)
    fwd, bwd = levels(lu_rowptr, lu_colidx, m.n)
    return {"rowptr": rowptr, "colidx": colidx, "rxn_map": rmap, "perm": perm,
            "lu_rowptr": lu_rowptr, "lu_colidx": lu_colidx,
            "level_fwd": fwd, "level_bwd": bwd}
