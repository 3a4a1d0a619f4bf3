"""Split-precision Rp->q path on the tcgen05 tensor cores vs the FP64 oracle.

Stated tolerances (relative): |g|^2 <= 1e-5 norm-wise per batch of pairs, 1/tau <= 1e-4 per
degenerate group, sigma and mobility <= 1e-4 in Frobenius norm.  fp16x3 and tf32x3 keep ~22
mantissa bits per operand and meet all three: they are the split modes that meet the stated
tolerances.  bf16x3 keeps ~16 bits (two 8-bit bf16 terms per operand) and does NOT meet the
stated |g|^2 bound; it is kept as a measured comparison mode, and its |g|^2 test records the
1e-4 it reaches so that a regression shows (its 1/tau and sigma still meet 1e-4)."""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import synth
from tests import models as M
from tests.parity import compare_rates, gpu_run, oracle_run, rel_frob

pytestmark = pytest.mark.gpu
G2_TOL = {"fp16x3": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-4}   # bf16x3: not the stated 1e-5 (see above)
RATE_TOL = 1e-4
MODES = ["fp16x3", "tf32x3", "bf16x3"]


@pytest.fixture(scope="module")
def epwi():
    from paper_2306_16493_gb300 import epwi as E
    return E


@pytest.mark.parametrize("prec", MODES)
@pytest.mark.parametrize("make,N", [(synth.al_like_system, 8), (synth.si_like_system, 6)])
def test_g2_norm_error(epwi, prec, make, N):
    s = make()
    ctx = epwi.Context(precision=prec)
    ctx.setup(s)
    ctx.eigs(N)
    gr = O.Grids(s, (N, N, N))
    rng = np.random.default_rng(21)
    ik = rng.integers(0, gr.nk, 300)
    iq = rng.integers(0, gr.nk, 300)
    got = ctx.g2(ik, iq, 0, s.nw)                                  # [p, n, nu, m]
    ref = np.empty_like(got)
    for p in range(len(ik)):
        ikq = O.kq_index(int(ik[p]), np.array([iq[p]]), gr.ngrid)[0]
        g = O.g_matrix(s, gr.frac[ik[p]], gr.frac[iq[p]][None], gr.V[ik[p]], gr.V[ikq][None],
                       gr.u[iq[p]][None])[0]
        ref[p] = np.where(gr.keep[iq[p]][:, None, None], np.abs(g) ** 2, 0.0).transpose(2, 0, 1)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < G2_TOL[prec], (prec, err)
    ctx.close()


@pytest.mark.parametrize("prec", MODES)
def test_tiny_rates_sigma(epwi, prec):
    s = synth.tiny_system()
    N, T, eta = 8, 300.0, 0.05
    gr = O.Grids(s, (N, N, N))
    mu = gr.band_centre()
    out = gpu_run(s, (N, N, N), T, mu, eta, -1e9, 1e9, precision=prec)
    ora = oracle_run(gr, T, mu, eta, -1e9, 1e9)
    err, n = compare_rates(out, ora, gr.eps, RATE_TOL)
    assert n == 4 * N ** 3 and err < RATE_TOL, err
    assert rel_frob(out["sigma"], ora["sigma"]) < RATE_TOL
    assert out["n_pairs"] == ora["n_pairs"]
    out["ctx"].close()


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_tb_dp_closed_form_split(epwi, prec):
    tb = M.tb_dp_system()
    N, T, eta, mu = 10, 300.0, 0.05, 0.1
    gr = O.Grids(tb, (N, N, N))
    out = gpu_run(tb, (N, N, N), T, mu, eta, -np.inf, np.inf, precision=prec)
    ora = oracle_run(gr, T, mu, eta, -np.inf, np.inf)
    err, n = compare_rates(out, ora, gr.eps, RATE_TOL)
    assert err < RATE_TOL, err
    out["ctx"].close()


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_al_like_12_split(epwi, prec):
    s = synth.al_like_system()
    N, T, eta = 12, 300.0, 0.02
    gr = O.Grids(s, (N, N, N))
    mu = gr.band_centre()
    out = gpu_run(s, (N, N, N), T, mu, eta, mu - 0.3, mu + 0.3, precision=prec)
    ora = oracle_run(gr, T, mu, eta, mu - 0.3, mu + 0.3)
    err, n = compare_rates(out, ora, gr.eps, RATE_TOL)
    assert err < RATE_TOL, err
    assert rel_frob(out["sigma"], ora["sigma"]) < RATE_TOL
    out["ctx"].close()


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_wigner_seitz_rset_split(epwi, prec):
    """A genuine Wigner-Seitz R_p set (93 vectors, not a cube) through the split-precision path,
    which embeds it in its bounding 7^3 cube with zero weights: 1/tau and sigma against the
    oracle on a ragged grid."""
    s = synth.al_like_ws_system()
    N, T, eta = (10, 9, 11), 300.0, 0.04
    gr = O.Grids(s, N)
    mu = gr.band_centre()
    out = gpu_run(s, N, T, mu, eta, mu - 0.3, mu + 0.3, precision=prec)
    ora = oracle_run(gr, T, mu, eta, mu - 0.3, mu + 0.3)
    assert out["n_pairs"] == ora["n_pairs"]
    err, n = compare_rates(out, ora, gr.eps, RATE_TOL)
    assert n > 0 and err < RATE_TOL, err
    assert rel_frob(out["sigma"], ora["sigma"]) < RATE_TOL
    out["ctx"].close()


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_si_like_mobility_split(epwi, prec):
    s = synth.si_like_system()
    N, T, eta, n_c = 12, 300.0, 0.01, 1e18
    gr = O.Grids(s, (N, N, N))
    vbm, cbm = gr.band_edges(4)
    mu = O.find_mu(gr.eps[:, 4:], gr.nk, s.volume, n_c, T)
    out = gpu_run(s, (N, N, N), T, mu, eta, cbm, cbm + 0.25, precision=prec)
    ora = oracle_run(gr, T, mu, eta, cbm, cbm + 0.25)
    err, n = compare_rates(out, ora, gr.eps, RATE_TOL)
    assert n > 0 and err < RATE_TOL, err
    mob = out["ctx"].mobility(n_c)
    assert rel_frob(mob, O.mobility(ora["sigma"], n_c)) < RATE_TOL
    out["ctx"].close()


def test_al_like_48_sampled_split(epwi):
    """48^3 Al-like workload in the bench configuration (fp16x3); sampled k-points recomputed
    by the oracle; the full sigma is compared with the GPU FP64 path."""
    s = synth.al_like_system()
    N, T, eta = 48, 300.0, 0.02
    ctx = epwi.Context(precision="fp16x3")
    ctx.setup(s)
    ctx.eigs(N)
    lo, hi = ctx.band_range()
    mu = 0.5 * (lo + hi)
    out = gpu_run(s, (N, N, N), T, mu, eta, mu - 0.3, mu + 0.3, precision="fp16x3", ctx=ctx)
    gr = O.Grids(s, (N, N, N))
    kp, cnt = ctx.sieve()
    pick = kp[np.random.default_rng(13).choice(len(kp), 6, replace=False)]
    ora = oracle_run(gr, T, mu, eta, mu - 0.3, mu + 0.3, k_subset=pick)
    sel = np.isin(out["ik"], pick)
    sub = dict(ik=out["ik"][sel], n=out["n"][sel], inv_tau=out["inv_tau"][sel])
    err, _ = compare_rates(sub, ora, gr.eps, RATE_TOL)
    assert err < RATE_TOL, err
    ref64 = gpu_run(s, (N, N, N), T, mu, eta, mu - 0.3, mu + 0.3, precision="fp64", ctx=ctx)
    assert rel_frob(out["sigma"], ref64["sigma"]) < RATE_TOL
    ctx.close()


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3"])
@pytest.mark.parametrize("make,N", [(synth.al_like_system, (10, 10, 10)),
                                    (synth.si_like_system, (6, 5, 4)),
                                    (synth.tiny_system, (7, 7, 7))])
def test_gathered_and_generated_phase_operands_agree(epwi, prec, make, N):
    """The precomputed split phase rows gathered into shared memory give the rates of the
    per-tile generation into TMEM: the same operand bits, so agreement to FP32 summation
    order (<= 1e-6), and both meet the FP64 oracle bound."""
    s = make()
    gr = O.Grids(s, N)
    mu = gr.band_centre()
    T, eta = 300.0, 0.05
    lo, hi = (mu - 0.5, mu + 0.5) if s.nw <= 4 else (-np.inf, np.inf)
    res = {}
    for mode in (0, 1):
        res[mode] = gpu_run(s, N, T, mu, eta, lo, hi, precision=prec, tc_a_operand=mode)
    a, b = res[0]["inv_tau"], res[1]["inv_tau"]
    assert np.array_equal(res[0]["ik"], res[1]["ik"]) and np.array_equal(res[0]["n"], res[1]["n"])
    assert np.allclose(a, b, rtol=1e-6, atol=1e-6 * np.abs(b).max())
    ora = oracle_run(gr, T, mu, eta, lo, hi)
    err, n = compare_rates(res[0], ora, gr.eps, RATE_TOL)
    assert n > 0 and err < RATE_TOL, err
    for r in res.values():
        r["ctx"].close()
