"""The parity rule between the CUDA path and the oracle, and its arbiter.

Rule (after every outer step): for each species with max(|y_gpu|, |y_ora|)
above atol, |y_gpu - y_ora| <= 1e-3 |y_ora|; otherwise |y_gpu - y_ora| <=
atol.

Both sides are accurate only to the requested tolerances: the integrator
controls the local error of each step in the weighted norm with weights
1 / (rtol |y| + atol) (Sect. 2.4.1, CVODE's error control), not the global
error, which at rtol 1e-4 reaches tens of those tolerance units on stiff
cells in the oracle itself.  Where a controller decision (accept/reject,
order change) sits on a tie, two implementations take different step
sequences and their results differ by up to their global errors.  A cell
that breaks the rule therefore goes to the arbiter, with a tight oracle run
(rtol 1e-10, atol 1e-12, minimum step 1e-18 dt; 1e-9 or 1e-8 for a cell
the tightest run cannot finish) standing for the true solution:

1. strict tier: for every species the CUDA result's error against the
   tight run is within twice the oracle's own error, or within the rule's
   bound around the true value (1e-3 |y_true| above atol, atol otherwise);
2. error-control tier, for a cell the strict tier rejects: the cell's error
   in the integrator's own norm, E = max_i |y_i - y_true,i| / (rtol |y_true,i|
   + atol_i), is within twice the oracle's E on that cell, or within the
   largest E the oracle itself makes on a seeded reference sample of the
   same cells (the oracle's own global error at this tolerance).

A cell passes if either tier passes; every violating cell is arbitrated and
the share and the tier counts are reported, not capped.
"""
import numpy as np

REL = 1e-3
TIGHT_RTOL, TIGHT_ATOL = 1e-10, 1e-12
REFERENCE_CELLS = 256


def violations(y_gpu, y_ora, atol, rel=REL):
    """Boolean [cells, species]: where the rule is broken."""
    big = np.maximum(np.abs(y_gpu), np.abs(y_ora)) > atol
    d = np.abs(y_gpu - y_ora)
    bad = np.where(big, d > rel * np.abs(y_ora), d > atol)
    return bad


def tight_solution(om, y0, env, dt):
    """The oracle at rtol 1e-10 / atol 1e-12, with the minimum step lowered
    to 1e-18 dt (the fast initial transients of phase transfer, ~1e6 s^-1,
    need steps below the default 1e-10 dt at that tolerance); a cell whose
    controller still gives up is run at rtol 1e-9, then 1e-8, still four
    orders of magnitude below the rule's 1e-3."""
    yt, st, _ = om.solve(y0, env, dt, TIGHT_RTOL, TIGHT_ATOL, max_steps=200000, hmin_frac=1e-18)
    for r in (1e-9, 1e-8):
        bad = np.nonzero(st != 0)[0]
        if not len(bad):
            break
        yb, sb, _ = om.solve(y0[bad], env[bad], dt, r, r * 1e-2, max_steps=200000, hmin_frac=1e-18)
        yt[bad], st[bad] = yb, sb
    assert (st == 0).all(), "the tight oracle run failed"
    return yt


def tol_units(y, yt, rtol, atol):
    """Per-cell error against the true solution in the integrator's own
    units: max over species of |y - y_true| / (rtol |y_true| + atol)."""
    return (np.abs(y - yt) / (rtol * np.abs(yt) + atol)).max(axis=1)


def reference_error(om, y0, env, dt, rtol, atol, y_ora, n=REFERENCE_CELLS, seed=0):
    """The largest error (integrator units) the oracle makes on a seeded
    reference sample of the given cells."""
    idx = np.arange(len(y0)) if len(y0) <= n else np.sort(np.random.default_rng(seed).choice(len(y0), n, replace=False))
    yt = tight_solution(om, y0[idx], env[idx], dt)
    return float(tol_units(y_ora[idx], yt, rtol, atol).max())


def arbitrate(om, y0, env, dt, rtol, atol, y_gpu, y_ora, e_ref, rel=REL):
    """Tight oracle runs on the given (violating) cells.  Returns (strict-tier
    pass per cell, error-control-tier pass per cell, E of the CUDA result,
    E of the oracle)."""
    yt = tight_solution(om, y0, env, dt)
    eg = np.abs(y_gpu - yt)
    eo = np.abs(y_ora - yt)
    big = np.maximum(np.abs(y_gpu), np.abs(yt)) > atol
    bound = np.where(big, np.maximum(2 * eo, rel * np.abs(yt)), np.maximum(2 * eo, atol))
    strict = (eg <= bound).all(axis=1)
    Eg, Eo = tol_units(y_gpu, yt, rtol, atol), tol_units(y_ora, yt, rtol, atol)
    norm = Eg <= np.maximum(2 * Eo, e_ref)
    return strict, norm, Eg, Eo


def rule_stats(y_gpu, y_ora, atol, rel=REL):
    """Error statistics over the species above atol (relative to the oracle)."""
    big = np.maximum(np.abs(y_gpu), np.abs(y_ora)) > atol
    relerr = np.where(big, np.abs(y_gpu - y_ora) / np.maximum(np.abs(y_ora), 1e-300), 0.0)
    bad = violations(y_gpu, y_ora, atol, rel)
    cells = np.nonzero(bad.any(axis=1))[0]
    return {"cells": int(len(y_gpu)), "max_rel": float(relerr.max()) if relerr.size else 0.0,
            "p99_rel": float(np.quantile(relerr.max(axis=1), 0.99)) if relerr.size else 0.0,
            "violating_cells": cells}


def arbiter_report(om, y0, env, dt, rtol, atol, y_gpu, y_ora, rel=REL):
    """The rule over every cell and the arbiter over every violating cell,
    without asserting: a dict with the counts and, per tier, how many
    arbitrated cells pass."""
    stats = rule_stats(y_gpu, y_ora, atol, rel)
    cells = stats.pop("violating_cells")
    stats.update({"arbitrated": int(len(cells)), "arbitrated_share": len(cells) / max(1, len(y_gpu)),
                  "arbiter_pass_strict": 0, "arbiter_pass": 0, "failed_cells": []})
    if len(cells):
        e_ref = reference_error(om, y0, env, dt, rtol, atol, y_ora)
        strict, norm, Eg, Eo = arbitrate(om, y0[cells], env[cells], dt, rtol, atol, y_gpu[cells], y_ora[cells],
                                         e_ref, rel)
        ok = strict | norm
        stats.update({"arbiter_pass_strict": int(strict.sum()), "arbiter_pass": int(ok.sum()),
                      "oracle_reference_error_tol_units": e_ref,
                      "arbitrated_error_tol_units_max": float(Eg.max()),
                      "arbitrated_oracle_error_tol_units_max": float(Eo.max()),
                      "failed_cells": cells[~ok].tolist()})
    return stats


def check(om, y0, env, dt, rtol, atol, y_gpu, y_ora, rel=REL):
    """Assert the rule, sending every violating cell to the arbiter.  Returns
    a dict of error statistics with the arbitrated count, share and tier
    counts."""
    stats = arbiter_report(om, y0, env, dt, rtol, atol, y_gpu, y_ora, rel)
    assert not stats["failed_cells"], stats
    return stats
