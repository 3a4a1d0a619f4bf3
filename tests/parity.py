"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and the
FP64 oracle on the same seeded inputs, and compare what is gauge invariant."""
from __future__ import annotations

import numpy as np

from oracle import epwi_oracle as O


def gpu_run(sysm, grid, T, mu, eta, emin, emax, precision="fp64", ctx=None, **kw):
    from paper_2306_16493_gb300 import epwi
    own = ctx is None
    if own:
        ctx = epwi.Context(precision=precision, **kw)
        ctx.setup(sysm)
    else:
        ctx.set_precision(precision)
    ctx.eigs(grid)
    ns, npairs = ctx.scatter_rates(T, mu, eta, emin, emax)
    k, b, r = ctx.rates()
    sig = ctx.conductivity() if ns > 0 else np.zeros((3, 3))
    out = dict(ik=k.astype(np.int64), n=b.astype(np.int64), inv_tau=r, sigma=sig,
               n_pairs=npairs, stats=ctx.stats(), ctx=ctx)
    return out


def oracle_run(gr: O.Grids, T, mu, eta, emin, emax, k_subset=None):
    res = O.serta(gr, T, mu, eta, emin, emax, k_subset=k_subset)
    if len(res["ik"]):
        v = gr.velocities(res["ik"], res["n"])
        res["sigma"] = O.conductivity(gr.sys.volume, gr.nk, v, res["inv_tau"],
                                      gr.eps[res["ik"], res["n"]], mu, T)
    else:
        res["sigma"] = np.zeros((3, 3))
    return res


def group_sums(ik, n, vals, eps, tol=1e-6):
    """Sums of vals over groups of states at the same k whose energies differ by < tol
    (only such sums are gauge invariant inside degenerate subspaces)."""
    out = {}
    order = np.lexsort((n, ik))
    ik, n, vals = ik[order], n[order], vals[order]
    i = 0
    while i < len(ik):
        j = i + 1
        while j < len(ik) and ik[j] == ik[i] and abs(eps[ik[j], n[j]] - eps[ik[j - 1], n[j - 1]]) < tol:
            j += 1
        out[(int(ik[i]), int(n[i]))] = vals[i:j].sum()
        i = j
    return out


def compare_rates(gpu, ora, eps, rtol):
    """Relative error of 1/tau over degenerate groups; returns (max_rel, n_compared)."""
    assert np.array_equal(np.sort(gpu["ik"] * 1000 + gpu["n"]), np.sort(ora["ik"] * 1000 + ora["n"]))
    gs = group_sums(gpu["ik"], gpu["n"], gpu["inv_tau"], eps)
    os_ = group_sums(ora["ik"], ora["n"], ora["inv_tau"], eps)
    assert gs.keys() == os_.keys()
    scale = max(abs(v) for v in os_.values()) if os_ else 1.0
    worst = 0.0
    for key, ref in os_.items():
        err = abs(gs[key] - ref) / max(abs(ref), 1e-12 * scale)
        worst = max(worst, err)
    return worst, len(os_)


def rel_frob(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
