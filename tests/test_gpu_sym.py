"""Symmetry-reduced k grids (Sec. III A) on the GPU: with the 48 operations of the fcc point
group, epwi_scatter_rates computes the sieve and 1/tau only for one representative per star of
window k-points and gives every member its representative's rates.  On the symmetrised Al-like
crystal the states, 1/tau (per degenerate group) and sigma equal those of the full-grid run and
of the full-grid oracle; the work drops by about the order of the group."""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import epwi, synth
from tests.parity import compare_rates, gpu_run, oracle_run, rel_frob

pytestmark = pytest.mark.gpu
T = 300.0


def _kops(s):
    return synth.kpoint_ops(synth.point_group(s.lattice))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("N", [8, 12])
def test_reduced_rates_equal_the_full_grid(prec, tol, N):
    s = synth.al_like_sym_system()
    grid = (N, N, N)
    gr = O.Grids(s, grid)
    mu = gr.band_centre()
    lo, hi, eta = mu - 0.4, mu + 0.4, 0.04
    full = gpu_run(s, grid, T, mu, eta, lo, hi, precision=prec)
    ctx = epwi.Context(precision=prec)
    ctx.setup(s)
    ctx.set_symmetry(_kops(s))
    red = gpu_run(s, grid, T, mu, eta, lo, hi, precision=prec, ctx=ctx)
    st = red["stats"]
    assert np.array_equal(red["ik"], full["ik"]) and np.array_equal(red["n"], full["n"])
    assert 0 < st["sym_kpoints"] < st["n_kpoints"] and st["sym_states"] < st["n_states"]
    assert red["n_pairs"] < full["n_pairs"] / 8                 # computed pairs: representatives only
    err, n = compare_rates(red, full, gr.eps, tol)
    assert n > 0 and err <= tol, err
    assert rel_frob(red["sigma"], full["sigma"]) <= tol
    if prec == "fp64":
        ora = oracle_run(gr, T, mu, eta, lo, hi)
        err, _ = compare_rates(red, ora, gr.eps, tol)
        assert err <= tol, err
        assert rel_frob(red["sigma"], ora["sigma"]) <= tol
    with pytest.raises(epwi.EpwiError):                         # sieve lists are per representative
        ctx.sieve()
    with pytest.raises(epwi.EpwiError):                         # the iteration couples all k-points
        ctx.ibte(T, mu, eta, lo, hi, max_iter=2, tol=0.0)
    ctx.set_symmetry(None)                                      # off again: the full run
    again = gpu_run(s, grid, T, mu, eta, lo, hi, precision=prec, ctx=ctx)
    assert again["n_pairs"] == full["n_pairs"] and np.array_equal(again["inv_tau"], full["inv_tau"])
    ctx.close()
    full["ctx"].close()


def test_symmetry_is_checked():
    s = synth.al_like_ws_system()                  # the same lattice, not symmetrised
    ctx = epwi.Context()
    ctx.setup(s)
    ctx.set_symmetry(_kops(s))
    ctx.eigs(6)
    lo, hi = ctx.band_range()
    mu = 0.5 * (lo + hi)
    with pytest.raises(epwi.EpwiError) as e:       # eps(K k) != eps(k)
        ctx.scatter_rates(T, mu, 0.05, mu - 0.3, mu + 0.3)
    assert e.value.status == 1                     # EPWI_EINVAL
    ctx.eigs((6, 6, 4))
    with pytest.raises(epwi.EpwiError):            # not an N x N x N grid
        ctx.scatter_rates(T, mu, 0.05, mu - 0.3, mu + 0.3)
    with pytest.raises(epwi.EpwiError):            # not a group: one rotation without its powers
        ctx.set_symmetry(_kops(s)[[0, 5]] if not np.array_equal(_kops(s)[0], np.eye(3)) else _kops(s)[[1, 5]])
    ctx.close()
