"""Pins of the oracle's iterative BTE (Sec. II C, iteration equation) and of the transport
coefficients formed from the mean free paths F, against facts fixed outside the code under
test:
  * with every band in the window, each row of Gamma sums to the SERTA rate 1/tau (Eq. 10),
    the pinned SERTA oracle;
  * the converged iteration is the solution of the linear BTE v = F/tau - Gamma F, obtained
    by a direct sparse solve;
  * isotropic scattering (one band, dispersionless modes, local coupling): the in-scattering
    sum vanishes on an inversion-symmetric grid, so F = v tau and sigma equals the SERTA
    sigma (a textbook result);
  * single entries of Gamma evaluated by brute force from the definition, with the k + q
    bookkeeping done in fractional coordinates;
  * transport from F = v tau reproduces the pinned SERTA transport coefficients.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import synth

T = 300.0


@pytest.fixture(scope="module")
def tiny5():
    return O.Grids(synth.tiny_system(), (5, 5, 5))


def test_einstein_system_has_the_closed_form_band():
    s = synth.einstein_system()
    gr = O.Grids(s, (6, 6, 6))
    expect = -2 * 0.5 * np.cos(2 * np.pi * gr.frac).sum(axis=1)
    assert np.allclose(gr.eps[:, 0], expect, atol=1e-13)
    assert np.allclose(gr.hw, gr.hw[0, 0], rtol=1e-12)            # dispersionless modes


def test_rows_of_gamma_sum_to_the_serta_rates(tiny5):
    gr = tiny5
    mu, eta = gr.band_centre(), 0.05
    res = O.ibte(gr, T, mu, eta, -1e9, 1e9, max_iter=1)
    ref = O.serta(gr, T, mu, eta, -1e9, 1e9)
    assert np.array_equal(res["ik"], ref["ik"]) and np.array_equal(res["n"], ref["n"])
    rows = np.asarray(res["A"].sum(axis=1)).ravel()
    assert np.allclose(rows, ref["inv_tau"], rtol=1e-12, atol=0)
    assert np.allclose(res["inv_tau"], ref["inv_tau"], rtol=1e-12, atol=0)


def test_converged_iteration_solves_the_linear_bte():
    gr = O.Grids(synth.tiny_system(), (6, 6, 6))
    mu, eta = gr.band_centre(), 0.05
    # window +-0.3 eV: states near its edges lose final states, so the slowest mode of
    # tau Gamma (the number-conserving one) has |lambda| ~ 0.995 and the iteration converges
    res = O.ibte(gr, T, mu, eta, mu - 0.3, mu + 0.3, max_iter=20000, tol=1e-14)
    assert res["iters"] < 20000
    ok = res["inv_tau"] > 0
    idx = np.nonzero(ok)[0]
    A = res["A"][idx][:, idx]
    v = gr.velocities(res["ik"], res["n"])[idx]
    M = sp.diags(res["inv_tau"][idx]) - A
    F = np.stack([spla.spsolve(M.tocsc(), v[:, a]) for a in range(3)], axis=1)
    scale = np.abs(F).max()
    assert np.abs(res["F"][idx] - F).max() <= 1e-9 * scale
    # the in-scattering term matters here: F differs from F^0 = v tau
    assert np.abs(res["F"] - res["F0"]).max() > 1e-3 * scale


def test_isotropic_scattering_leaves_sigma_at_its_serta_value():
    s = synth.einstein_system()
    gr = O.Grids(s, (8, 8, 8))
    mu, eta = 0.3, 0.08
    res = O.ibte(gr, T, mu, eta, mu - 0.5, mu + 0.5, max_iter=50, tol=1e-14)
    assert res["A"].nnz > 1000                                     # in-scattering is present
    v = gr.velocities(res["ik"], res["n"])
    e = gr.eps[res["ik"], res["n"]]
    sig_F, S_F, k_F = O.transport_from_F(s.volume, gr.nk, v, res["F"], e, mu, T)
    sig, S, k = O.transport_coefficients(s.volume, gr.nk, v, res["inv_tau"], e, mu, T)
    assert np.abs(sig_F - sig).max() <= 1e-10 * np.abs(sig).max()
    assert np.abs(S_F - S).max() <= 1e-9 * np.abs(S).max()
    assert np.abs(res["F"] - res["F0"]).max() <= 1e-10 * np.abs(res["F0"]).max()


def test_gamma_entries_by_brute_force():
    s = synth.tiny_system()
    gr = O.Grids(s, (4, 4, 4))
    mu, eta, c = gr.band_centre(), 0.05, 6.0
    res = O.ibte(gr, T, mu, eta, mu - 1.0, mu + 1.0, max_iter=1)
    A = res["A"].tocoo()
    rng = np.random.default_rng(5)
    picks = rng.choice(A.nnz, size=min(25, A.nnz), replace=False)
    pref = 2.0 * math.pi / O.HBAR_EVS / gr.nk
    for p in picks:
        i, j, val = A.row[p], A.col[p], A.data[p]
        k, n = res["ik"][i], res["n"][i]
        kp, m = res["ik"][j], res["n"][j]
        dq = np.mod(gr.frac[kp] - gr.frac[k] + 1e-9, 1.0) - 1e-9
        iq = int(np.nonzero(np.abs(gr.frac - dq).max(axis=1) < 1e-9)[0][0])
        g = O.g_matrix(s, gr.frac[k], gr.frac[iq][None], gr.V[k][:, [n]], gr.V[kp][None],
                       gr.u[iq][None])[0, :, m, 0]                 # [nu]
        total = 0.0
        for nu in range(s.nm):
            if not gr.keep[iq, nu]:
                continue
            w = gr.hw[iq, nu]
            N = 1.0 / math.expm1(w / (O.KB_EVK * T))
            fm = 1.0 / (math.exp((gr.eps[kp, m] - mu) / (O.KB_EVK * T)) + 1.0)
            en, em = gr.eps[k, n], gr.eps[kp, m]
            d = lambda x: (math.exp(-(x / eta) ** 2) / (math.sqrt(math.pi) * eta)
                           if abs(x) <= c * eta else 0.0)
            total += abs(g[nu]) ** 2 * ((N + fm) * d(en + w - em) + (1 + N - fm) * d(en - w - em))
        assert val == pytest.approx(pref * total, rel=1e-11)


def test_transport_from_vtau_is_the_serta_transport(tiny5):
    gr = tiny5
    mu, eta = gr.band_centre(), 0.05
    ref = O.serta(gr, T, mu, eta, mu - 0.5, mu + 0.5)
    v = gr.velocities(ref["ik"], ref["n"])
    e = gr.eps[ref["ik"], ref["n"]]
    tau = np.where(ref["inv_tau"] > 0, 1.0 / np.maximum(ref["inv_tau"], 1e-300), 0.0)
    a = O.transport_from_F(gr.sys.volume, gr.nk, v, tau[:, None] * v, e, mu, T)
    b = O.transport_coefficients(gr.sys.volume, gr.nk, v, ref["inv_tau"], e, mu, T)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-12 * np.abs(y).max())


def test_time_reversal_inputs_cancel_the_number_mode_drive():
    """With real H(R) and g, eps(-k) = eps(k) and v(-k) = -v(k) on the Gamma-centred grid, so
    sum f(1-f) v over the window vanishes and the iteration converges quickly; with the
    complex inputs it does not vanish."""
    base = synth.al_like_system()
    for sysm, zero in ((synth.time_reversal_symmetric(base), True), (base, False)):
        gr = O.Grids(sysm, (8, 8, 8))
        mu = gr.band_centre()
        ik, n = gr.window_states(mu - 0.3, mu + 0.3)
        v = gr.velocities(ik, n)
        f = O.fermi(gr.eps[ik, n], mu, T)
        w = (f * (1 - f))[:, None]
        drive = np.abs((w * v).sum(axis=0)).max() / np.abs(w * v).sum(axis=0).max()
        assert (drive < 1e-12) == zero
    gr = O.Grids(synth.time_reversal_symmetric(base), (8, 8, 8))
    mu = gr.band_centre()
    res = O.ibte(gr, T, mu, 0.05, mu - 0.3, mu + 0.3, max_iter=500, tol=1e-10)
    assert res["iters"] < 200
