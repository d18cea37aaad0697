"""The parity rule between the CUDA path and the oracle, and its arbiter.

Rule (after every outer step): for each species with max(|y_gpu|, |y_ora|)
above atol, |y_gpu - y_ora| <= 1e-3 |y_ora|; otherwise |y_gpu - y_ora| <=
atol.  Both sides are accurate only to the requested tolerances, and near
ties of the step controller (accept/reject, order change) the two may take
different step sequences.  A cell that breaks the rule goes to the arbiter: a
tight oracle run (rtol 1e-10, atol 1e-12) stands for the true solution, and
the CUDA result passes if its error against it is within max(2 x the
oracle's own error, 1e-3 relative + atol) for every species.
"""
import numpy as np

REL = 1e-3


def violations(y_gpu, y_ora, atol, rel=REL):
    big = np.maximum(np.abs(y_gpu), np.abs(y_ora)) > atol
    d = np.abs(y_gpu - y_ora)
    bad = np.where(big, d > rel * np.abs(y_ora), d > atol)
    return bad


def check(om, y0, env, dt, rtol, atol, y_gpu, y_ora, rel=REL, max_arbitrated=0.05):
    """Assert the rule, sending violating cells to the arbiter.  Returns a
    dict of error statistics."""
    bad = violations(y_gpu, y_ora, atol, rel)
    cells = np.nonzero(bad.any(axis=1))[0]
    big = np.maximum(np.abs(y_gpu), np.abs(y_ora)) > atol
    relerr = np.where(big, np.abs(y_gpu - y_ora) / np.maximum(np.abs(y_ora), 1e-300), 0.0)
    stats = {"cells": len(y0), "max_rel": float(relerr.max()) if relerr.size else 0.0,
             "p99_rel": float(np.quantile(relerr.max(axis=1), 0.99)) if relerr.size else 0.0,
             "arbitrated": int(len(cells))}
    assert len(cells) <= max(1, int(max_arbitrated * len(y0))), stats
    if len(cells):
        yt, st, _ = om.solve(y0[cells], env[cells], dt, 1e-10, 1e-12, max_steps=200000)
        assert (st == 0).all()
        eg = np.abs(y_gpu[cells] - yt)
        eo = np.abs(y_ora[cells] - yt)
        ok = eg <= np.maximum(2 * eo, rel * np.abs(yt) + atol)
        assert ok.all(), {"cells": cells.tolist(), **stats}
    return stats
