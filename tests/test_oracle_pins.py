"""Pins of the FP64 CPU oracle against closed forms, invariants and brute force.

Each test checks the oracle against something other than itself: an analytic model, a
library routine used for a different purpose, a symmetry of the physics, or a direct
loop over the defining sums.  A dropped term, a wrong sign, index or unit, or a
transposed operand anywhere in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import synth
from tests import models as M


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_system()


@pytest.fixture(scope="module")
def tb():
    return M.tb_dp_system()


# ------------------------------------------------------------------ inputs / invariants
@pytest.mark.parametrize("make", [synth.tiny_system, synth.al_like_system])
def test_hermitian_inputs(make):
    s = make()
    mi = [list(map(tuple, s.Re.tolist())).index(tuple((-r).tolist())) for r in s.Re]
    assert np.abs(s.H - np.conj(np.transpose(s.H[mi], (0, 2, 1)))).max() < 1e-15
    assert np.abs(s.Phi - np.transpose(s.Phi[mi], (0, 2, 1))).max() < 1e-15


def test_hamiltonian_k_hermitian(tiny):
    k = np.random.default_rng(0).random((7, 3))
    Hk = O.hamiltonian_k(tiny, k)
    assert np.abs(Hk - np.conj(np.transpose(Hk, (0, 2, 1)))).max() < 1e-13


@pytest.mark.parametrize("make", [synth.tiny_system, synth.al_like_system, synth.si_like_system])
def test_acoustic_sum_rule(make):
    s = make()
    hw, u, keep = O.phonons(s, np.zeros((1, 3)))
    assert np.abs(hw[0, :3]).max() < 1e-7          # three acoustic modes vanish at Gamma
    assert not keep[0, :3].any()
    q = np.random.default_rng(1).random((50, 3))
    hw, _, _ = O.phonons(s, q)
    assert hw.min() > -1e-9                         # spring models: D(q) positive semidefinite


def test_semiconductor_gap_at_gamma():
    s = synth.si_like_system()
    eps, _ = O.bands(s, np.zeros((1, 3)))
    assert abs(eps[0, 3] - 0.0) < 1e-12 and abs(eps[0, 4] - 1.1) < 1e-12
    k = np.random.default_rng(2).random((200, 3))
    e, _ = O.bands(s, k)
    assert e[:, :4].max() <= 1e-12 and e[:, 4:].min() >= 1.1 - 1e-12


# ------------------------------------------------------------------ closed-form models
def test_tight_binding_closed_form(tb):
    k = np.random.default_rng(3).random((40, 3))
    eps, V = O.bands(tb, k)
    assert np.allclose(eps[:, 0], M.tb_eps(k), rtol=0, atol=1e-13)
    v = O.velocities(tb, k, V)
    assert np.allclose(v[:, 0, :], M.tb_vel(k), rtol=1e-12, atol=1e-6)


def test_spring_closed_form(tb):
    q = np.random.default_rng(4).random((40, 3))
    hw, u, keep = O.phonons(tb, q)
    assert np.allclose(np.sort(hw, 1), np.sort(M.spring_hw(q), 1), rtol=1e-12, atol=1e-15)
    # u = (hbar^2 / (2 M hbar omega))^{1/2} e with e a unit vector per axis
    amp = np.sqrt(M.C_EV / (2.0 * 20.0 * hw))
    assert np.allclose(np.linalg.norm(u, axis=1), amp, rtol=1e-12)


def test_deformation_potential_g2_closed_form(tb):
    rng = np.random.default_rng(5)
    k = rng.random(3)
    q = rng.random((30, 3))
    eps_k, Vk = O.bands(tb, k[None])
    kq = (k[None] + q) % 1.0
    _, Vkq = O.bands(tb, kq)
    _, u, keep = O.phonons(tb, q)
    g = O.g_matrix(tb, k, q, Vk[0], Vkq, u)           # [q, nu, m, n]
    hw, _, _ = O.phonons(tb, q)
    # modes are the Cartesian axes; match each mode to its axis by energy
    g2 = np.abs(g[:, :, 0, 0]) ** 2
    ref = M.dp_g2(q)
    ref_hw = M.spring_hw(q)
    for iq in range(len(q)):
        for nu in range(3):
            ax = np.argmin(np.abs(ref_hw[iq] - hw[iq, nu]))
            assert g2[iq, nu] == pytest.approx(ref[iq, ax], rel=1e-11, abs=1e-20)


def test_inv_tau_closed_form_grid_sum(tb):
    """Full SERTA pipeline on the TB+DP model against the analytic grid sum of Eq. 10."""
    N = 10
    T, eta, c = 300.0, 0.05, 6.0
    gr = O.Grids(tb, (N, N, N))
    mu = 0.1
    res = O.serta(gr, T, mu, eta, -np.inf, np.inf, c=c)
    frac = gr.frac
    e_all = M.tb_eps(frac)
    hw_all = M.spring_hw(frac)                         # [q, axis]
    g2_all = M.dp_g2(frac)
    kT = O.KB_EVK * T
    ref = np.zeros(len(frac))
    grid = O.grid_indices((N, N, N))
    for ik in range(len(frac)):
        ikq = O.flat_index((grid[ik] + grid) % N, (N, N, N))
        ek, ekq = e_all[ik], e_all[ikq]
        for ax in range(3):
            w = hw_all[:, ax]
            ok = w >= 1e-4
            wn = np.where(ok, w, 1.0)
            Nb = 1.0 / (np.exp(wn / kT) - 1.0)
            f = 1.0 / (np.exp((ekq - mu) / kT) + 1.0)

            def dl(x):
                return np.where(np.abs(x) <= c * eta,
                                np.exp(-(x / eta) ** 2) / (math.sqrt(math.pi) * eta), 0.0)
            term = g2_all[:, ax] * ((Nb + f) * dl(ek + w - ekq) + (1 + Nb - f) * dl(ek - w - ekq))
            ref[ik] += np.where(ok, term, 0.0).sum()
    ref *= 2 * math.pi / O.HBAR_EVS / len(frac)
    got = np.zeros(len(frac))
    got[res["ik"]] = res["inv_tau"]
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-9 * ref.max())


# ------------------------------------------------------------------ brute force
def test_g_bruteforce_tiny(tiny):
    """Direct quadruple sum of Eq. 7 (no factorisation) vs the bracketed evaluation."""
    rng = np.random.default_rng(6)
    k = rng.random(3)
    q = rng.random((3, 3))
    _, Vk = O.bands(tiny, k[None])
    _, Vkq = O.bands(tiny, (k[None] + q) % 1.0)
    _, u, _ = O.phonons(tiny, q)
    got = O.g_matrix(tiny, k, q, Vk[0], Vkq, u)
    nw, nm = tiny.nw, tiny.nm
    for iq in range(len(q)):
        ref = np.zeros((nm, nw, nw), complex)          # [nu, m, n]
        for ie, Re in enumerate(tiny.Re):
            for ip, Rp in enumerate(tiny.Rp):
                ph = np.exp(2j * np.pi * (k @ Re + q[iq] @ Rp)) * tiny.we[ie] * tiny.wp[ip]
                for mu_ in range(nm):
                    for nu in range(nm):
                        # sum_ij U_mi(k+q) U^dag_jn(k) g^mu_ij u_mu,nu with U = V^dag
                        Ukq = Vkq[iq].conj().T
                        Udk = Vk[0]
                        ref[nu] += ph * u[iq, mu_, nu] * (Ukq @ tiny.g[ie, ip, mu_] @ Udk)
        assert np.allclose(got[iq], ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_g_bruteforce_weighted_rsets():
    """Direct double sum over (Re, Rp) with Wigner-Seitz weights (Al-like 5^3 sets)."""
    s = synth.al_like_system()
    rng = np.random.default_rng(16)
    k = rng.random(3)
    q = rng.random((2, 3))
    _, Vk = O.bands(s, k[None])
    _, Vkq = O.bands(s, (k[None] + q) % 1.0)
    _, u, _ = O.phonons(s, q)
    got = O.g_matrix(s, k, q, Vk[0], Vkq, u)
    for iq in range(len(q)):
        ph = (np.exp(2j * np.pi * (s.Re @ k))[:, None] * np.exp(2j * np.pi * (s.Rp @ q[iq]))[None, :]
              * s.we[:, None] * s.wp[None, :])
        G = np.einsum("ab,abmij->mij", ph, s.g)                 # all Re, Rp at once
        ref = np.einsum("mi,lij,jn,lv->vmn", Vkq[iq].conj().T, G, Vk[0], u[iq])
        assert np.allclose(got[iq], ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_sieve_bruteforce(tiny):
    gr = O.Grids(tiny, (4, 4, 4))
    eta, c = 0.02, 6.0
    for ik in (0, 5, 37):
        nsel = np.array([1, 2])
        got = O.sieve_k(gr, ik, nsel, eta, c)
        ref = []
        g3 = O.grid_indices(gr.ngrid)
        for iq in range(gr.nk):
            ikq = O.flat_index((g3[ik] + g3[iq]) % 4, gr.ngrid)
            hit = False
            for n in nsel:
                for m in range(tiny.nw):
                    for nu in range(tiny.nm):
                        if not gr.keep[iq, nu]:
                            continue
                        for s in (1, -1):
                            if abs(gr.eps[ik, n] + s * gr.hw[iq, nu] - gr.eps[ikq, m]) <= c * eta:
                                hit = True
            if hit:
                ref.append(iq)
        assert list(got) == ref


# ------------------------------------------------------------------ gauge invariance
def test_gauge_invariance_g2(tiny):
    rng = np.random.default_rng(7)
    k = rng.random(3)
    q = rng.random((5, 3))
    _, Vk = O.bands(tiny, k[None])
    _, Vkq = O.bands(tiny, (k[None] + q) % 1.0)
    _, u, _ = O.phonons(tiny, q)
    g0 = np.abs(O.g_matrix(tiny, k, q, Vk[0], Vkq, u)) ** 2
    ph_k = np.exp(1j * rng.random(tiny.nw) * 6.3)
    ph_kq = np.exp(1j * rng.random((5, 1, tiny.nw)) * 6.3)
    ph_q = np.exp(1j * rng.random((5, 1, tiny.nm)) * 6.3)
    g1 = np.abs(O.g_matrix(tiny, k, q, Vk[0] * ph_k, Vkq * ph_kq, u * ph_q)) ** 2
    assert np.allclose(g0, g1, rtol=1e-13, atol=1e-14 * g0.max())


# ------------------------------------------------------------------ velocities
def test_velocity_finite_difference():
    s = synth.al_like_system()
    rng = np.random.default_rng(8)
    k = rng.random((5, 3))
    eps, V = O.bands(s, k)
    v = O.velocities(s, k, V)
    h = 1e-5                                           # 1/A
    for a in range(3):
        dk = np.zeros(3)
        dk[a] = h
        kp = k + s.lattice @ dk / (2 * np.pi)          # k_frac shift for a Cartesian step
        km = k - s.lattice @ dk / (2 * np.pi)
        ep, _ = O.bands(s, kp)
        em, _ = O.bands(s, km)
        fd = (ep - em) / (2 * h) / O.HBAR_EVS * 1e-10  # m/s
        assert np.allclose(v[:, :, a], fd, rtol=1e-6, atol=1e-4 * np.abs(fd).max())


# ------------------------------------------------------------------ delta, occupations
def test_gaussian_delta_normalisation():
    eta, c = 0.02, 6.0
    val, _ = scipy.integrate.quad(lambda x: float(O.delta_gauss(x, eta, c)), -c * eta, c * eta,
                                  points=[0.0], epsabs=1e-14)
    assert val == pytest.approx(scipy.special.erf(c), rel=1e-12)
    assert float(O.delta_gauss(c * eta * 1.0001, eta, c)) == 0.0


def test_occupations():
    T = 300.0
    kT = O.KB_EVK * T
    assert float(O.fermi(0.7, 0.7, T)) == pytest.approx(0.5, rel=1e-15)
    x = np.linspace(-40, 40, 81) * kT
    f = O.fermi(x, 0.0, T)
    assert np.allclose(f + O.fermi(-x, 0.0, T), 1.0, atol=1e-15)
    w = np.linspace(0.001, 0.1, 20)
    Nb = O.bose(w, T)
    assert np.allclose((Nb + 1.0) / Nb, np.exp(w / kT), rtol=1e-12)   # detailed balance
    assert np.isfinite(O.fermi(np.array([-1e3, 1e3]), 0.0, 10.0)).all()


# ------------------------------------------------------------------ 1/tau invariances
def test_inv_tau_order_and_batching_invariant(tiny):
    gr = O.Grids(tiny, (6, 6, 6))
    T, mu, eta = 300.0, gr.band_centre(), 0.05
    ik = 17
    bands_n = np.arange(tiny.nw)
    q = O.sieve_k(gr, ik, bands_n, eta)
    r0, _ = O.inv_tau_k(gr, ik, bands_n, T, mu, eta, q_list=q)
    perm = np.random.default_rng(9).permutation(q)
    r1, _ = O.inv_tau_k(gr, ik, bands_n, T, mu, eta, q_list=perm)
    ra, _ = O.inv_tau_k(gr, ik, bands_n, T, mu, eta, q_list=perm[: len(q) // 3])
    rb, _ = O.inv_tau_k(gr, ik, bands_n, T, mu, eta, q_list=perm[len(q) // 3:])
    assert np.allclose(r0, r1, rtol=1e-13)
    assert np.allclose(r0, ra + rb, rtol=1e-13)
    assert (r0 >= 0).all()
    # pairs outside the sieve contribute exactly zero
    rall, _ = O.inv_tau_k(gr, ik, bands_n, T, mu, eta, q_list=np.arange(gr.nk))
    assert np.allclose(r0, rall, rtol=1e-14)


# ------------------------------------------------------------------ transport
def _boltzmann_tb(N, T, mu, t=0.5, a=3.0):
    tb = M.tb_dp_system(a=a, t=t, eps0=0.0)
    gr = O.Grids(tb, (N, N, N))
    return tb, gr


def test_conductivity_drude_bessel_identity():
    """Nondegenerate 1-band TB with constant tau: the grid sums are trapezoidal rules of
    periodic integrands, so n and sigma equal modified-Bessel closed forms:
    n = (2/V) e^{beta(mu)} I0(z)^3 and sigma_xx = n e^2 tau (2ta/hbar)^2 (I1(z)/z)/I0(z)/kT,
    z = 2 t / kT."""
    N, T, t, a = 48, 300.0, 0.5, 3.0
    mu = -6 * t - 0.6                                  # 0.6 eV below the band bottom
    tb, gr = _boltzmann_tb(N, T, mu, t, a)
    kT = O.KB_EVK * T
    z = 2 * t / kT
    tau = 1e-14
    ik = np.arange(gr.nk)
    v = gr.velocities(ik, np.zeros(gr.nk, int))
    sig = O.conductivity(tb.volume, gr.nk, v, np.full(gr.nk, 1 / tau), gr.eps[:, 0], mu, T)
    n_cm3 = O.carrier_density(gr.eps[:, :1], gr.nk, tb.volume, mu, T)
    i0 = scipy.special.ive(0, z)                       # e^{-z} I0(z)
    i1 = scipy.special.ive(1, z)
    # e^{beta mu} prod_a sum_k e^{2 beta t cos} = e^{beta mu} (N I0(z))^3 per grid of N^3
    n_ref = 2.0 / (tb.volume * 1e-24) * math.exp((mu + 6 * t) / kT) * i0 ** 3
    assert n_cm3 == pytest.approx(n_ref, rel=1e-8)
    vel2 = (2 * t * a * 1e-10 / O.HBAR_EVS) ** 2 * (i1 / z) / i0     # <v_x^2> (m/s)^2
    sxx_ref = n_ref * 1e6 * O.E_CHARGE ** 2 * tau * vel2 / (kT * O.E_CHARGE)
    assert sig[0, 0] == pytest.approx(sxx_ref, rel=1e-7)
    assert np.allclose(np.diag(sig), sig[0, 0], rtol=1e-10)
    assert np.abs(sig - np.diag(np.diag(sig))).max() < 1e-12 * sig[0, 0]
    mob = O.mobility(sig, n_cm3)
    assert mob[0, 0] == pytest.approx(O.E_CHARGE * tau * vel2 / (kT * O.E_CHARGE) * 1e4, rel=1e-7)


def test_find_mu_boltzmann_closed_form():
    N, T, t, a = 48, 300.0, 0.5, 3.0                  # N >> z: trapezoid rule is exact
    tb, gr = _boltzmann_tb(N, T, 0.0, t, a)
    kT = O.KB_EVK * T
    z = 2 * t / kT
    n_target = 1e12                                    # mu ~0.5 eV below the band: Boltzmann
    mu = O.find_mu(gr.eps[:, :1], gr.nk, tb.volume, n_target, T)
    n = O.carrier_density(gr.eps[:, :1], gr.nk, tb.volume, mu, T)
    assert n == pytest.approx(n_target, rel=1e-12)
    i0 = scipy.special.ive(0, z)
    mu_ref = -6 * t + kT * math.log(n_target * tb.volume * 1e-24 / (2.0 * i0 ** 3))
    assert mu == pytest.approx(mu_ref, abs=1e-9)


def test_conductivity_symmetric_psd(tiny):
    gr = O.Grids(tiny, (6, 6, 6))
    T, mu, eta = 300.0, gr.band_centre(), 0.05
    res = O.serta(gr, T, mu, eta, -np.inf, np.inf)
    v = gr.velocities(res["ik"], res["n"])
    sig = O.conductivity(tiny.volume, gr.nk, v, res["inv_tau"], gr.eps[res["ik"], res["n"]], mu, T)
    assert np.allclose(sig, sig.T, rtol=1e-14, atol=0)
    assert np.linalg.eigvalsh(sig).min() > -1e-12 * np.trace(sig)


# ------------------------------------------------------------------ Seebeck and kappa_e
def _parabolic_states(n, kmax, m_eff=1.0):
    """States of an isotropic parabolic band eps = hbar^2 k^2 / 2m sampled on a uniform cubic
    k-mesh (|k_a| <= kmax, 1/A), with v = hbar k / m in m/s."""
    k1 = np.linspace(-kmax, kmax, n)
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    k = np.stack([kx.ravel(), ky.ravel(), kz.ravel()], -1)                  # 1/A
    hb2_2m = O.HBAR_JS ** 2 / (2 * m_eff * 9.1093837015e-31) / O.E_CHARGE * 1e20   # eV A^2
    eps = hb2_2m * (k ** 2).sum(1)
    v = O.HBAR_JS * k * 1e10 / (m_eff * 9.1093837015e-31)                   # m/s
    return eps, v


def test_seebeck_nondegenerate_parabolic_band():
    """Boltzmann statistics, constant tau, parabolic band: S = -(k_B/e)(5/2 - eta),
    eta = mu / k_B T (band edge at 0)."""
    T = 300.0
    kT = O.KB_EVK * T
    eps, v = _parabolic_states(121, 0.35)
    assert eps.max() > 25 * kT                   # the mesh covers the thermal tail
    for eta in (-4.0, -6.0):
        mu = eta * kT
        sig, S, kap = O.transport_coefficients(10.0, len(eps), v, np.full(len(eps), 1e13), eps, mu, T)
        ref = -(O.KB_EVK) * (2.5 - eta)          # k_B / e in V/K equals k_B in eV/K
        assert abs(S[0, 0] / ref - 1) < 1e-2, (S[0, 0], ref)
        assert abs(S[1, 1] / S[0, 0] - 1) < 1e-6 and abs(S[0, 1]) < 1e-6 * abs(S[0, 0])


def test_wiedemann_franz_degenerate_parabolic_band():
    """Degenerate electrons, constant tau: kappa_e / (sigma T) -> L0 = (pi^2/3)(k_B/e)^2 with
    Sommerfeld corrections O((k_B T / E_F)^2); the thermopower is Mott's -(pi^2/2)(k_B/e)
    (k_B T / E_F) for sigma(E) ~ E^{3/2}."""
    T, EF = 300.0, 1.0
    kT = O.KB_EVK * T
    eps, v = _parabolic_states(161, 0.62)
    sel = np.abs(eps - EF) < 20 * kT
    eps, v = eps[sel], v[sel]
    sig, S, kap = O.transport_coefficients(10.0, 1000, v, np.full(len(eps), 1e14), eps, EF, T)
    L0 = np.pi ** 2 / 3 * O.KB_EVK ** 2
    assert abs(kap[0, 0] / (sig[0, 0] * T) / L0 - 1) < 2e-2
    mott = -(np.pi ** 2 / 2) * O.KB_EVK * kT / EF
    assert abs(S[0, 0] / mott - 1) < 5e-2, (S[0, 0], mott)


def test_oracle_matches_stored_golden_values():
    """Regression pin: the oracle reproduces tests/golden/tiny_6_serta.txt (written by
    tests/golden/make_golden.py from the oracle) to 1e-9 on degenerate-group sums of 1/tau and
    on the transport tensors (headroom for platform eigensolver rounding)."""
    import os
    from tests.parity import group_sums
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_6_serta.txt")
    rows, meta = [], {}
    for line in open(path):
        if line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] in ("mu", "n_pairs", "sigma", "seebeck", "kappa_e"):
            meta[parts[0]] = np.array([float(x) for x in parts[1:]])
        else:
            rows.append((int(parts[0]), int(parts[1]), float(parts[2])))
    s = synth.tiny_system(1)
    gr = O.Grids(s, (6, 6, 6))
    mu = gr.band_centre()
    assert abs(mu - meta["mu"][0]) < 1e-12
    T, eta = 300.0, 0.05
    r = O.serta(gr, T, mu, eta, -np.inf, np.inf)
    assert r["n_pairs"] == int(meta["n_pairs"][0])
    ik = np.array([x[0] for x in rows])
    n = np.array([x[1] for x in rows])
    ref = group_sums(ik, n, np.array([x[2] for x in rows]), gr.eps)
    got = group_sums(r["ik"], r["n"], r["inv_tau"], gr.eps)
    assert ref.keys() == got.keys()
    assert max(abs(got[k] - v) / abs(v) for k, v in ref.items()) < 1e-9
    v = gr.velocities(r["ik"], r["n"])
    sig, S, kap = O.transport_coefficients(s.volume, gr.nk, v, r["inv_tau"], gr.eps[r["ik"], r["n"]], mu, T)
    for name, t in (("sigma", sig), ("seebeck", S), ("kappa_e", kap)):
        assert np.linalg.norm(t.ravel() - meta[name]) <= 1e-9 * np.linalg.norm(meta[name]), name


def test_serta_rates_are_invariant_on_the_stars_of_a_symmetric_crystal():
    """Pins the symmetry reduction (Sec. III A): on the crystal symmetrised under the fcc point
    group, the oracle's full-grid 1/tau_n(K k) equals 1/tau_n(k) for all 48 k-space operations
    K (degenerate-group sums), and sigma of the cubic crystal is isotropic."""
    s = synth.al_like_sym_system()
    N, T, eta = 6, 300.0, 0.05
    gr = O.Grids(s, (N, N, N))
    mu = gr.band_centre()
    r = O.serta(gr, T, mu, eta, mu - 0.5, mu + 0.5)
    rate = {(int(k), int(n)): v for k, n, v in zip(r["ik"], r["n"], r["inv_tau"])}
    idx = O.grid_indices((N, N, N))
    worst = 0.0
    for K in synth.kpoint_ops(synth.point_group(s.lattice)):
        j = O.flat_index((idx @ K.T) % N, (N, N, N))
        for (k, n), v in rate.items():
            worst = max(worst, abs(rate[(int(j[k]), n)] - v) / v)
    assert worst < 1e-10
    v = gr.velocities(r["ik"], r["n"])
    sig = O.conductivity(s.volume, gr.nk, v, r["inv_tau"], gr.eps[r["ik"], r["n"]], mu, T)
    assert np.allclose(sig, np.trace(sig) / 3 * np.eye(3), rtol=0, atol=1e-10 * np.abs(sig).max())
