"""GPU parity of the fp32 mode: FP32 Re->k, the Rp->q sum factorised over the axes of the R_p
cube (per plane block, per q1 run, per pair), FP32 rotations and delta terms, FP64 sums per
state.  Compared with the FP64 oracle on cubic and non-cubic grids (ragged plane blocks and
runs), with the FP64 GPU path, across k-point chunking and repeated runs, and at the 48^3
benchmark configuration on sampled k-points.

1/tau is compared per degenerate group with the error relative to that group's own rate
(tests.parity.compare_rates), sigma in Frobenius norm."""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import epwi, synth
from tests.parity import compare_rates, gpu_run, oracle_run, rel_frob

pytestmark = pytest.mark.gpu
T = 300.0
TOL = 1e-5          # FP32 interpolation and delta terms, FP64 sums
SIGMA_TOL = 1e-5


def _rates(system, grid, mu, eta, lo, hi, precision="fp32", chunk=0):
    ctx = epwi.Context(precision=precision, device=0, kpoint_chunk=chunk)
    ctx.setup(system)
    ctx.eigs(grid)
    ns, npairs = ctx.scatter_rates(T, mu, eta, lo, hi)
    k, b, r = ctx.rates()
    ctx.close()
    o = np.lexsort((b, k))
    return k[o], b[o], r[o], npairs


@pytest.mark.parametrize("name,grid,half,eta", [
    ("tiny", (6, 6, 6), None, 0.05),
    ("tiny", (3, 4, 5), None, 0.05),
    ("al_like", (10, 10, 10), 0.3, 0.05),
    ("al_like", (12, 7, 9), 0.3, 0.05),
    ("al_like", (6, 18, 17), 0.3, 0.04),
    ("al_like_ws", (10, 10, 10), 0.3, 0.05),     # genuine Wigner-Seitz R-set, not a cube
    ("al_like_ws", (9, 20, 15), 0.3, 0.04),      # ... two plane blocks, ragged
    ("si_like", (6, 5, 4), None, 0.05),          # W = 8, 6 modes, 7^3: q2 groups
    ("al_like", (64, 5, 6), 0.3, 0.05),          # >= 64 points on axis 1: the sieve's segment pruning
])
def test_fp32_matches_the_oracle(name, grid, half, eta):
    s = getattr(synth, f"{name}_system")()
    gr = O.Grids(s, grid)
    mu = gr.band_centre()
    lo, hi = (-1e9, 1e9) if half is None else (mu - half, mu + half)
    ref = oracle_run(gr, T, mu, eta, lo, hi)
    out = gpu_run(s, grid, T, mu, eta, lo, hi, precision="fp32")
    assert out["n_pairs"] == ref["n_pairs"]
    err, n = compare_rates(out, ref, gr.eps, TOL)
    assert n > 0 and err <= TOL, err
    assert rel_frob(out["sigma"], ref["sigma"]) <= SIGMA_TOL
    out["ctx"].close()


def test_fp32_against_fp64_gpu_and_determinism():
    s = synth.al_like_system()
    gr = O.Grids(s, (16, 16, 16))
    mu = gr.band_centre()
    args = (s, (16, 16, 16), mu, 0.03, mu - 0.3, mu + 0.3)
    a = _rates(*args, precision="fp64")
    b = _rates(*args)
    c = _rates(*args, chunk=37)
    d = _rates(*args)
    assert np.abs(a[2] - b[2]).max() <= TOL * a[2].max()
    assert np.array_equal(b[2], c[2]) and np.array_equal(b[2], d[2])


@pytest.mark.parametrize("name,grid,half", [("al_like", (14, 9, 40), 0.3), ("si_like", (8, 8, 8), None),
                                             ("al_like", (66, 4, 5), 0.3)])
def test_sieve_without_mask_gives_the_same_rates(monkeypatch, name, grid, half):
    """When the decision mask does not fit (forced with EPWI_SIEVE_MASK_MAX_BYTES=0) the pair
    lists are rebuilt per chunk by the sieve kernel's fill mode: the pair counts and the rates
    (FP64 and fp32, several chunks) are bitwise those of the mask path."""
    s = getattr(synth, f"{name}_system")()
    gr = O.Grids(s, grid)
    mu = gr.band_centre()
    lo, hi = (-1e9, 1e9) if half is None else (mu - half, mu + half)
    for prec in ("fp64", "fp32"):
        monkeypatch.delenv("EPWI_SIEVE_MASK_MAX_BYTES", raising=False)
        a = gpu_run(s, grid, T, mu, 0.03, lo, hi, precision=prec, kpoint_chunk=5)
        monkeypatch.setenv("EPWI_SIEVE_MASK_MAX_BYTES", "0")
        b = gpu_run(s, grid, T, mu, 0.03, lo, hi, precision=prec, kpoint_chunk=5)
        assert a["n_pairs"] == b["n_pairs"] > 0
        assert np.array_equal(a["inv_tau"], b["inv_tau"]) and np.array_equal(a["sigma"], b["sigma"])
        a["ctx"].close()
        b["ctx"].close()
    ref = oracle_run(gr, T, mu, 0.03, lo, hi)
    assert b["n_pairs"] == ref["n_pairs"]


def test_al_like_48_sampled_fp32():
    """The benchmark configuration in the benchmark's precision: Al-like 48^3, window +-0.3 eV
    around the band centre, eta = 20 meV, default k-point chunking (as the benchmark launches it).  Eight sampled window
    k-points are recomputed by the oracle (all their q); the full sigma is compared with the
    FP64 GPU path on the same grid."""
    s = synth.al_like_system()
    N, eta = 48, 0.02
    ctx = epwi.Context(precision="fp32")
    ctx.setup(s)
    ctx.eigs(N)
    lo, hi = ctx.band_range()
    mu = 0.5 * (lo + hi)
    out = gpu_run(s, (N, N, N), T, mu, eta, mu - 0.3, mu + 0.3, precision="fp32", ctx=ctx)
    gr = O.Grids(s, (N, N, N))
    kp, cnt = ctx.sieve()
    pick = kp[np.random.default_rng(29).choice(len(kp), 8, replace=False)]
    ora = oracle_run(gr, T, mu, eta, mu - 0.3, mu + 0.3, k_subset=pick)
    sel = np.isin(out["ik"], pick)
    sub = dict(ik=out["ik"][sel], n=out["n"][sel], inv_tau=out["inv_tau"][sel])
    err, n = compare_rates(sub, ora, gr.eps, TOL)
    assert n >= 8 and err <= TOL, err
    assert [int(x) for x in cnt[np.searchsorted(kp, pick)]] == [ora["pairs_per_k"][int(k)] for k in pick]
    ref64 = gpu_run(s, (N, N, N), T, mu, eta, mu - 0.3, mu + 0.3, precision="fp64", ctx=ctx)
    err64, _ = compare_rates(out, ref64, gr.eps, TOL)
    assert err64 <= TOL, err64
    assert rel_frob(out["sigma"], ref64["sigma"]) <= SIGMA_TOL
    ctx.close()


def test_si_like_mobility_fp32():
    """The Si-like semiconductor (W = 8 with 4 valence and 4 conduction Wannier functions,
    6 modes, 7^3 R-sets) at 12^3: mu from n_c = 1e18 cm^-3, window [CBM, CBM + 0.25 eV],
    eta = 10 meV; 1/tau per degenerate group and the mobility tensor against the oracle."""
    s = synth.si_like_system()
    N, eta, n_c = 12, 0.01, 1e18
    gr = O.Grids(s, (N, N, N))
    vbm, cbm = gr.band_edges(4)
    mu = O.find_mu(gr.eps[:, 4:], gr.nk, s.volume, n_c, T)
    out = gpu_run(s, (N, N, N), T, mu, eta, cbm, cbm + 0.25, precision="fp32")
    ora = oracle_run(gr, T, mu, eta, cbm, cbm + 0.25)
    assert out["n_pairs"] == ora["n_pairs"]
    err, n = compare_rates(out, ora, gr.eps, TOL)
    assert n > 0 and err <= TOL, err
    assert rel_frob(out["ctx"].mobility(n_c), O.mobility(ora["sigma"], n_c)) <= SIGMA_TOL
    out["ctx"].close()


def test_fp32_refuses_what_it_does_not_serve():
    ctx = epwi.Context(precision="fp32", device=0)
    ctx.setup(synth.batch_system(13)[0])          # nw = 24: no fp32 kernel of that shape
    ctx.eigs((3, 3, 4))
    with pytest.raises(epwi.EpwiError):
        ctx.scatter_rates(T, 0.0, 0.05, -1e9, 1e9)
    ctx.close()
    ctx = epwi.Context(precision="fp32", device=0)
    ctx.setup(synth.tiny_system())
    ctx.eigs(4)
    with pytest.raises(epwi.EpwiError):           # per-pair |g|^2 of arbitrary pairs
        ctx.g2(np.array([0, 1], np.int32), np.array([3, 5], np.int32), 0, 2)
    ctx.close()
