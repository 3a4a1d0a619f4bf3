"""GPU FP64 path vs the FP64 oracle, element by element on seeded inputs (bar:
1e-10 relative on 1/tau degenerate-group sums and on sigma)."""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import synth
from tests import models as M
from tests.parity import compare_rates, gpu_run, oracle_run, rel_frob

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def epwi():
    from paper_2306_16493_gb300 import epwi as E
    return E


def _proj_err(Va, Vb, ea, tol=1e-6):
    """max |P_a - P_b| over non-degenerate eigenvector projectors |v><v|."""
    worst = 0.0
    nb = ea.shape[1]
    for n in range(nb):
        nd = np.ones(len(ea), bool)
        if n > 0:
            nd &= np.abs(ea[:, n] - ea[:, n - 1]) > tol
        if n < nb - 1:
            nd &= np.abs(ea[:, n + 1] - ea[:, n]) > tol
        pa = np.einsum("ki,kj->kij", Va[nd, :, n], Va[nd, :, n].conj())
        pb = np.einsum("ki,kj->kij", Vb[nd, :, n], Vb[nd, :, n].conj())
        if nd.any():
            worst = max(worst, np.abs(pa - pb).max())
    return worst


@pytest.mark.parametrize("make,N", [(synth.tiny_system, 8), (synth.al_like_system, 10),
                                    (synth.si_like_system, 6),
                                    (lambda: synth.batch_system(10)[0], 5),    # nw 16, 12 modes
                                    (lambda: synth.batch_system(15)[0], 5)])   # nw 24, 18 modes
def test_eigs_parity(epwi, make, N):
    s = make()
    ctx = epwi.Context()
    ctx.setup(s)
    ctx.eigs((N, N, N))
    e, V, v = ctx.bands()
    w, u = ctx.phonons()
    gr = O.Grids(s, (N, N, N))
    scale = np.abs(gr.eps).max()
    assert np.abs(e - gr.eps).max() < 1e-12 * scale
    assert _proj_err(V, gr.V, gr.eps) < 1e-10
    vo = O.velocities(s, gr.frac, gr.V)
    # velocities of non-degenerate states
    nd = np.ones_like(gr.eps, bool)
    nd[:, 1:] &= np.diff(gr.eps, axis=1) > 1e-6
    nd[:, :-1] &= np.diff(gr.eps, axis=1) > 1e-6
    assert np.abs(v[nd] - vo[nd]).max() < 1e-10 * np.abs(vo).max()
    keep = gr.keep
    assert np.abs(w[keep] - gr.hw[keep]).max() < 1e-12 * gr.hw.max()
    assert np.abs(w[~keep]).max() < 1e-4
    assert _proj_err(u / np.maximum(np.linalg.norm(u, axis=1, keepdims=True), 1e-300),
                     gr.u / np.maximum(np.linalg.norm(gr.u, axis=1, keepdims=True), 1e-300),
                     np.where(keep, gr.hw, -1e3 * np.arange(gr.hw.shape[1]))) < 1e-9
    ctx.close()


def test_large_matrices_rates_parity(epwi):
    """nw = 24 and 18 modes (the warp-per-matrix eigensolver and the generic FP64 kernels):
    1/tau and sigma vs the oracle at 1e-10 on a non-cubic grid."""
    s = synth.batch_system(15)[0]
    grid = (3, 4, 5)
    gr = O.Grids(s, grid)
    mu = gr.band_centre()
    T, eta = 300.0, 0.05
    out = gpu_run(s, grid, T, mu, eta, mu - 1.0, mu + 1.0)
    ora = oracle_run(gr, T, mu, eta, mu - 1.0, mu + 1.0)
    err, n = compare_rates(out, ora, gr.eps, TOL)
    assert n > 0 and err < TOL, err
    assert rel_frob(out["sigma"], ora["sigma"]) < TOL
    out["ctx"].close()


def test_tb_dp_closed_form_through_gpu(epwi):
    """TB + axial springs + deformation potential: GPU 1/tau vs the analytic grid sum."""
    tb = M.tb_dp_system()
    N, T, eta, c, mu = 10, 300.0, 0.05, 6.0, 0.1
    out = gpu_run(tb, (N, N, N), T, mu, eta, -np.inf, np.inf)
    gr = O.Grids(tb, (N, N, N))
    ora = oracle_run(gr, T, mu, eta, -np.inf, np.inf)
    err, n = compare_rates(out, ora, gr.eps, TOL)
    assert n == N ** 3 and err < TOL, err
    out["ctx"].close()


def test_tiny_full_parity(epwi):
    s = synth.tiny_system()
    N, T, eta = 8, 300.0, 0.05
    gr = O.Grids(s, (N, N, N))
    mu = gr.band_centre()
    out = gpu_run(s, (N, N, N), T, mu, eta, -1e9, 1e9)
    ora = oracle_run(gr, T, mu, eta, -1e9, 1e9)
    err, n = compare_rates(out, ora, gr.eps, TOL)
    assert n == 4 * N ** 3 and err < TOL, err
    assert rel_frob(out["sigma"], ora["sigma"]) < TOL
    assert out["n_pairs"] == ora["n_pairs"]
    kp, cnt = out["ctx"].sieve()
    assert np.array_equal(cnt, [ora["pairs_per_k"][int(k)] for k in kp])
    out["ctx"].close()


def test_al_like_window_parity_ragged_grid(epwi):
    """Wigner-Seitz weights, +-0.3 eV window, a non-cubic grid (lcm 60, ragged tiles)."""
    s = synth.al_like_system()
    grid, T, eta = (6, 5, 4), 300.0, 0.02
    gr = O.Grids(s, grid)
    mu = gr.band_centre()
    out = gpu_run(s, grid, T, mu, eta, mu - 0.3, mu + 0.3)
    ora = oracle_run(gr, T, mu, eta, mu - 0.3, mu + 0.3)
    err, n = compare_rates(out, ora, gr.eps, TOL)
    assert n > 0 and err < TOL, err
    assert rel_frob(out["sigma"], ora["sigma"]) < TOL
    assert out["n_pairs"] == ora["n_pairs"]
    out["ctx"].close()


def test_al_like_12_parity_and_chunking(epwi):
    s = synth.al_like_system()
    N, T, eta = 12, 300.0, 0.02
    gr = O.Grids(s, (N, N, N))
    mu = gr.band_centre()
    out = gpu_run(s, (N, N, N), T, mu, eta, mu - 0.3, mu + 0.3)
    ora = oracle_run(gr, T, mu, eta, mu - 0.3, mu + 0.3)
    err, n = compare_rates(out, ora, gr.eps, TOL)
    assert err < TOL, err
    assert rel_frob(out["sigma"], ora["sigma"]) < TOL
    # the same run in chunks of 7 k-points is bitwise identical (fixed-order reductions)
    out2 = gpu_run(s, (N, N, N), T, mu, eta, mu - 0.3, mu + 0.3, kpoint_chunk=7)
    assert out2["stats"]["n_chunks"] > 1
    assert np.array_equal(out2["inv_tau"], out["inv_tau"])
    assert np.array_equal(out2["sigma"], out["sigma"])
    out["ctx"].close()
    out2["ctx"].close()


def test_si_like_mu_and_mobility_parity(epwi):
    s = synth.si_like_system()
    N, T, eta, n_c = 12, 300.0, 0.01, 1e18
    gr = O.Grids(s, (N, N, N))
    vbm, cbm = gr.band_edges(4)
    mu_o = O.find_mu(gr.eps[:, 4:], gr.nk, s.volume, n_c, T)
    ctx = epwi.Context()
    ctx.setup(s)
    ctx.eigs(N)
    v2, c2 = ctx.band_edges(4)
    assert abs(v2 - vbm) < 1e-12 and abs(c2 - cbm) < 1e-12
    mu_g = ctx.find_mu(T, n_c, 4)
    assert abs(mu_g - mu_o) < 1e-11
    assert ctx.carrier_density(T, mu_g, 4) == pytest.approx(n_c, rel=1e-12)
    out = gpu_run(s, (N, N, N), T, mu_o, eta, cbm, cbm + 0.25, ctx=ctx)
    ora = oracle_run(gr, T, mu_o, eta, cbm, cbm + 0.25)
    err, n = compare_rates(out, ora, gr.eps, TOL)
    assert n > 0 and err < TOL, err
    mob = ctx.mobility(n_c)
    mob_o = O.mobility(ora["sigma"], n_c)
    assert rel_frob(mob, mob_o) < TOL
    ctx.close()


def test_g2_parity_fp64(epwi):
    s = synth.al_like_system()
    N = 8
    ctx = epwi.Context()
    ctx.setup(s)
    ctx.eigs(N)
    gr = O.Grids(s, (N, N, N))
    rng = np.random.default_rng(11)
    ik = rng.integers(0, gr.nk, 40)
    iq = rng.integers(0, gr.nk, 40)
    got = ctx.g2(ik, iq, 0, s.nw)                                   # [p, n, nu, m]
    for p in range(len(ik)):
        ikq = O.kq_index(int(ik[p]), np.array([iq[p]]), gr.ngrid)[0]
        g = O.g_matrix(s, gr.frac[ik[p]], gr.frac[iq[p]][None], gr.V[ik[p]], gr.V[ikq][None],
                       gr.u[iq[p]][None])[0]                        # [nu, m, n]
        ref = np.where(gr.keep[iq[p]][:, None, None], np.abs(g) ** 2, 0.0)
        assert np.allclose(got[p].transpose(1, 2, 0), ref, rtol=TOL, atol=TOL * ref.max() + 1e-300)
    ctx.close()


def test_al_like_48_sampled_parity(epwi):
    """The 48^3 Al-like workload in the bench launch configuration; a sample of k-points is
    recomputed one by one by the oracle."""
    s = synth.al_like_system()
    N, T, eta = 48, 300.0, 0.02
    out_ctx = epwi.Context()
    out_ctx.setup(s)
    out_ctx.eigs(N)
    lo, hi = out_ctx.band_range()
    mu = 0.5 * (lo + hi)
    out = gpu_run(s, (N, N, N), T, mu, eta, mu - 0.3, mu + 0.3, ctx=out_ctx)
    gr = O.Grids(s, (N, N, N))
    assert abs(mu - gr.band_centre()) < 1e-12
    kp, cnt = out_ctx.sieve()
    pick = kp[np.random.default_rng(12).choice(len(kp), 6, replace=False)]
    ora = oracle_run(gr, T, mu, eta, mu - 0.3, mu + 0.3, k_subset=pick)
    sel = np.isin(out["ik"], pick)
    sub = dict(ik=out["ik"][sel], n=out["n"][sel], inv_tau=out["inv_tau"][sel])
    err, n = compare_rates(sub, ora, gr.eps, TOL)
    assert err < TOL, err
    for k in pick:
        assert cnt[list(kp).index(k)] == ora["pairs_per_k"][int(k)]
    sig = out["sigma"]
    assert np.allclose(sig, sig.T, rtol=1e-13) and np.linalg.eigvalsh(sig).min() > 0
    out_ctx.close()


def test_edge_cases(epwi):
    s = synth.tiny_system()
    ctx = epwi.Context()
    with pytest.raises(epwi.EpwiError) as e:
        ctx.eigs(4)
    assert e.value.status == 4                                      # ESTATE before setup
    ctx.setup(s)
    with pytest.raises(epwi.EpwiError) as e:
        ctx.scatter_rates(300, 0, 0.05, -1, 1)
    assert e.value.status == 4                                      # ESTATE before eigs
    ctx.eigs(1)                                                     # single Gamma point
    ns, npairs = ctx.scatter_rates(300.0, 0.0, 0.05, -1e9, 1e9)
    assert ns == 4 and npairs == 0                                  # all modes dropped at Gamma
    assert np.all(ctx.rates()[2] == 0)
    assert np.all(ctx.conductivity() == 0)
    ctx.eigs(4)
    ns, npairs = ctx.scatter_rates(300.0, 0.0, 0.05, 100.0, 101.0)  # empty window
    assert ns == 0 and npairs == 0
    bad = synth.tiny_system()
    bad.H = bad.H.copy()
    bad.H[0, 0, 1] += 0.1                                           # break Hermiticity
    with pytest.raises(epwi.EpwiError) as e:
        ctx.setup(bad)
    assert e.value.status == 1
    with pytest.raises(epwi.EpwiError):
        ctx.eigs((4, 4, 0))
    ctx.close()


@pytest.mark.parametrize("which", ["tiny", "si"])
def test_seebeck_and_kappa_parity(epwi, which):
    """sigma, Seebeck and kappa_e (Eqs. 12-14) from the GPU moments vs the oracle: 1e-10."""
    T = 300.0
    if which == "tiny":
        s = synth.tiny_system(1)
        N, eta = 8, 0.05
        gr = O.Grids(s, (N,) * 3)
        mu = gr.band_centre()
        lo, hi = -np.inf, np.inf
    else:
        s = synth.si_like_system(3)
        N, eta = 12, 0.01
        gr = O.Grids(s, (N,) * 3)
        cbm = gr.eps[:, s.n_valence].min()
        mu = O.find_mu(gr.eps[:, s.n_valence:], gr.nk, s.volume, 1e18, T)
        lo, hi = cbm, cbm + 0.25
    out = gpu_run(s, (N,) * 3, T, mu, eta, lo, hi)
    sig, S, kap = out["ctx"].transport()
    ora = oracle_run(gr, T, mu, eta, lo, hi)
    v = gr.velocities(ora["ik"], ora["n"])
    sr, Sr, kr = O.transport_coefficients(s.volume, gr.nk, v, ora["inv_tau"],
                                          gr.eps[ora["ik"], ora["n"]], mu, T)
    assert rel_frob(sig, sr) < TOL
    assert rel_frob(S, Sr) < TOL and rel_frob(kap, kr) < TOL
    if which == "si":
        assert (np.diag(S) < 0).all()          # electrons: negative thermopower
    out["ctx"].close()
