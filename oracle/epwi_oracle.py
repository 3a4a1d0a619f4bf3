"""Plain FP64 CPU oracle for the EPWI transport hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.
It shares no code with the CUDA path; the one common dependency is the seeded input
generator ``paper_2306_16493_gb300.synth``, which holds none of the method's arithmetic.

Everything is computed one k-point at a time in the paper's order, in float64/complex128,
with numpy library primitives (matmul, einsum, exp, Hermitian eigensolver) as steps and
no blocking or fusion beyond what the equations state:

* H(k) = sum_R w_R e^{i k.R} H(R), diagonalised H(k) V = V diag(eps)      (Sec. II B, Eq. 4)
* D(q) = sum_R w_R Phi(R) e^{i q.R} / sqrt(m m), D e = omega^2 e          (Sec. II B, Eqs. 5-6)
* g^nu_mn(k,q) = sum U_mi(k+q) U^dag_jn(k) e^{i(k.Re+q.Rp)} g^mu_ij(Re,Rp) u_mu,nu(q),
  u = (hbar / 2 m omega)^{1/2} e, evaluated in the bracket order
  {U(k+q)[(g P^el U^dag(k)) P^ph]} u(q)                                  (Sec. II B Eq. 7; Sec. III C Eq. 16)
* SERTA 1/tau_nk with Gaussian delta functions                           (Sec. II C, Eq. 10)
* sigma, mobility                                                        (Sec. II C, Eqs. 12, 15)
* iterative BTE for the mean free paths F                                (Sec. II C, iteration eq.)
* effective-process sieve by energy conservation                         (Sec. III A)

Equation numbers count the numbered displays of the paper in order (Eq. 1 is the
el-ph Hamiltonian).  Readings of points the paper leaves open:
U = V^dagger (rows of U are eigenvectors), so U_mi(k+q) = conj(V_im(k+q)) and
U^dag_jn(k) = V_jn(k); the lattice-vector weights w_R multiply every Fourier sum;
1/tau carries 1/N_q; delta_eta(x) = exp(-(x/eta)^2)/(sqrt(pi) eta) for |x| <= c eta, else 0;
omega_{-q} = omega_q; modes with hbar omega < omega_min (or omega^2 < 0) are dropped;
sigma = (2 e^2/(N_k V)) sum v_a v_b tau f(1-f)/(k_B T); states with 1/tau = 0 are left out of
sigma; the sieve keeps (k,q) when some n in the window, m, nu and sign satisfy
|eps_nk +/- omega - eps_m,k+q| <= c eta.
"""
from __future__ import annotations

import math

import numpy as np

# CODATA 2018
HBAR_EVS = 6.582119569e-16          # eV s
HBAR_JS = 1.054571817e-34           # J s
KB_EVK = 8.617333262e-5             # eV / K
E_CHARGE = 1.602176634e-19          # C
AMU_KG = 1.66053906660e-27          # kg
#: hbar^2 / (amu A^2) in eV: (hbar omega)^2 [eV^2] = lambda [eV/A^2/amu] * this
HBAR2_AMU_A2 = HBAR_JS ** 2 / (AMU_KG * 1e-20) / E_CHARGE


# ----------------------------------------------------------------------------- grids
def grid_indices(ngrid) -> np.ndarray:
    """Gamma-centred grid, integer coordinates (i1, i2, i3), i3 fastest (Sec. III E: integer
    grid indices rather than float coordinates)."""
    n1, n2, n3 = ngrid
    a = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    return a.reshape(-1, 3)


def grid_frac(ngrid) -> np.ndarray:
    return grid_indices(ngrid) / np.asarray(ngrid, float)


def flat_index(idx3, ngrid) -> np.ndarray:
    n1, n2, n3 = ngrid
    return (idx3[..., 0] * n2 + idx3[..., 1]) * n3 + idx3[..., 2]


def kq_index(ik: int, iq: np.ndarray, ngrid) -> np.ndarray:
    """Grid index of k+q (component-wise modulo the grid)."""
    g = grid_indices(ngrid)
    s = (g[ik][None, :] + g[iq]) % np.asarray(ngrid)
    return flat_index(s, ngrid)


def phases(frac: np.ndarray, R: np.ndarray) -> np.ndarray:
    """e^{i k.R} = e^{2 pi i k_frac . n_R}, shape [nk, nR]."""
    return np.exp(2j * np.pi * (frac @ R.T.astype(float)))


# --------------------------------------------------------------------- electrons
def hamiltonian_k(sysm, kfrac) -> np.ndarray:
    """H(k) = sum_R w_R e^{i k.R} H(R)   (Sec. II B, Eq. 4)."""
    P = phases(np.atleast_2d(kfrac), sysm.Re) * sysm.we[None, :]
    return np.einsum("kr,rij->kij", P, sysm.H)


def bands(sysm, kfrac):
    """Eigenvalues (ascending, eV) and eigenvectors V (columns) of H(k)."""
    Hk = hamiltonian_k(sysm, kfrac)
    eps, V = np.linalg.eigh(Hk)
    return eps, V


def velocities(sysm, kfrac, V) -> np.ndarray:
    """Band velocities in m/s: v_n = (1/hbar) Re[V^dag dH/dk V]_nn with
    dH/dk_a = sum_R w_R i R_a e^{i k.R} H(R) (Sec. III A: velocities in preprocessing)."""
    Rc = sysm.Re @ sysm.lattice                                    # A
    P = phases(np.atleast_2d(kfrac), sysm.Re) * sysm.we[None, :]
    out = np.empty(V.shape[:2] + (3,))
    for a in range(3):
        dH = np.einsum("kr,rij->kij", 1j * Rc[None, :, a] * P, sysm.H)
        m = np.einsum("kin,kij,kjn->kn", V.conj(), dH, V)
        out[:, :, a] = m.real / HBAR_EVS * 1e-10
    return out


# ----------------------------------------------------------------------- phonons
def dynmat_q(sysm, qfrac) -> np.ndarray:
    """D(q) = sum_R w_R Phi(R) e^{i q.R} / sqrt(m_a m_b)   (Sec. II B, Eq. 5)."""
    P = phases(np.atleast_2d(qfrac), sysm.Rp) * sysm.wp[None, :]
    m = np.repeat(sysm.mass, 3)
    D = np.einsum("qr,rab->qab", P, sysm.Phi.astype(complex))
    return D / np.sqrt(np.outer(m, m))[None]


def phonons(sysm, qfrac, omega_min=1e-4):
    """Mode energies hbar*omega (eV), displacement vectors u (A) and the keep mask.

    D e = omega^2 e (Sec. II B, Eq. 6); u_{mu nu} = (hbar / 2 m_mu omega_nu)^{1/2} e_{mu nu}
    (Sec. II B, after Eq. 7).  Modes with omega^2 < 0 or hbar*omega < omega_min are dropped.
    """
    lam, e = np.linalg.eigh(dynmat_q(sysm, qfrac))
    hw = np.sign(lam) * np.sqrt(np.abs(lam) * HBAR2_AMU_A2)
    keep = hw >= omega_min
    m = np.repeat(sysm.mass, 3)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(keep, np.sqrt(HBAR2_AMU_A2 / (2.0 * np.abs(hw))), 0.0)
    u = e * amp[:, None, :] / np.sqrt(m)[None, :, None]
    return hw, u, keep


# -------------------------------------------------------------- el-ph interpolation
def g_wannier_k(sysm, kfrac) -> np.ndarray:
    """g P^el: sum_Re w_e e^{i k.Re} g(Re, Rp), shape [nRp, nm, nw, nw] (Eq. 16, inner bracket)."""
    P = phases(np.atleast_2d(kfrac), sysm.Re)[0] * sysm.we
    return np.tensordot(P, sysm.g, axes=(0, 0))


def g_matrix(sysm, kfrac, qfrac, Vk, Vkq, u) -> np.ndarray:
    """g^nu_mn(k, q) for one k and a batch of q (Sec. II B Eq. 7, bracket order of Eq. 16).

    Vk: [nw, nsel] eigenvector columns of the initial states n at k.
    Vkq: [nq, nw, nw] eigenvectors at k+q; u: [nq, nm, nm] phonon displacements at q.
    Returns g[nq, nu, m, n] in eV.
    """
    gk = g_wannier_k(sysm, kfrac)                                  # [Rp, mu, i, j]
    ghat = np.einsum("rmij,jn->rmin", gk, Vk)                      # (g P^el) U^dag(k)
    Pp = phases(np.atleast_2d(qfrac), sysm.Rp) * sysm.wp[None, :]
    G = np.tensordot(Pp, ghat, axes=(1, 0))                        # ... P^ph(q): [q, mu, i, n]
    gq = np.einsum("qim,qlin->qlmn", Vkq.conj(), G)                # U(k+q) [...]: [q, mu, m, n]
    return np.einsum("qlmn,qlv->qvmn", gq, u)                      # {...} u(q): [q, nu, m, n]


# ------------------------------------------------------------------ occupations etc.
def fermi(e, mu, T):
    x = (np.asarray(e, float) - mu) / (KB_EVK * T)
    ex = np.exp(-np.abs(x))
    return np.where(x > 0, ex / (1.0 + ex), 1.0 / (1.0 + ex))


def bose(w, T):
    return 1.0 / np.expm1(np.asarray(w, float) / (KB_EVK * T))


def delta_gauss(x, eta, c=6.0):
    """delta_eta(x) = exp(-(x/eta)^2) / (sqrt(pi) eta) on |x| <= c eta (Gaussian broadening
    eta of Sec. IV A)."""
    x = np.asarray(x, float)
    return np.where(np.abs(x) <= c * eta, np.exp(-(x / eta) ** 2) / (math.sqrt(math.pi) * eta), 0.0)


# ---------------------------------------------------------------------- the workload
class Grids:
    """Electron and phonon quantities on the full Gamma-centred grid (preprocessing)."""

    def __init__(self, sysm, ngrid, omega_min=1e-4):
        self.sys = sysm
        self.ngrid = tuple(int(x) for x in ngrid)
        self.frac = grid_frac(self.ngrid)
        self.nk = len(self.frac)
        self.eps, self.V = bands(sysm, self.frac)
        self.hw, self.u, self.keep = phonons(sysm, self.frac, omega_min)

    def band_centre(self) -> float:
        return 0.5 * (self.eps.min() + self.eps.max())

    def band_edges(self, n_valence):
        return self.eps[:, n_valence - 1].max(), self.eps[:, n_valence].min()

    def window_states(self, emin, emax):
        ik, n = np.nonzero((self.eps >= emin) & (self.eps <= emax))
        return ik.astype(np.int64), n.astype(np.int64)

    def velocities(self, ik, n):
        v = velocities(self.sys, self.frac[ik], self.V[ik])
        return v[np.arange(len(ik)), n]


def sieve_k(gr: Grids, ik: int, bands_n, eta, c=6.0):
    """Effective-process sieve for one k (Sec. III A): sorted q indices for which some n in
    ``bands_n``, m, kept mode nu and sign satisfy |eps_nk +/- omega - eps_m,k+q| <= c eta."""
    iq = np.arange(gr.nk)
    ikq = kq_index(ik, iq, gr.ngrid)
    en = gr.eps[ik, bands_n]                                       # [nsel]
    em = gr.eps[ikq]                                               # [q, m]
    w = gr.hw                                                      # [q, nu]
    ok = np.zeros(gr.nk, bool)
    for s in (1.0, -1.0):
        x = en[None, :, None, None] + s * w[:, None, None, :] - em[:, None, :, None]
        hit = (np.abs(x) <= c * eta) & gr.keep[:, None, None, :]
        ok |= hit.any(axis=(1, 2, 3))
    return iq[ok]


def pair_terms_full_k(gr: Grids, ik: int, bands_n, T, mu, eta, c, q_list) -> np.ndarray:
    """The summand of Eq. 10 for one k, resolved in q, mode and final band:
    t[q, nu, m, n] = |g^nu_mn(k,q)|^2 [(N + f_m) delta(x+) + (1 + N - f_m) delta(x-)] in eV
    (Sec. II C, Eq. 10), for the q in ``q_list`` and the initial bands ``bands_n``."""
    bands_n = np.asarray(bands_n)
    q_list = np.asarray(q_list, dtype=np.int64)
    if len(q_list) == 0:
        return np.zeros((0, gr.hw.shape[1], gr.eps.shape[1], len(bands_n)))
    ikq = kq_index(ik, q_list, gr.ngrid)
    g = g_matrix(gr.sys, gr.frac[ik], gr.frac[q_list], gr.V[ik][:, bands_n],
                 gr.V[ikq], gr.u[q_list])                          # [q, nu, m, n]
    g2 = np.abs(g) ** 2
    w = gr.hw[q_list]                                              # [q, nu]
    keep = gr.keep[q_list]
    N = np.where(keep, bose(np.where(keep, w, 1.0), T), 0.0)
    fm = fermi(gr.eps[ikq], mu, T)                                 # [q, m]
    en = gr.eps[ik, bands_n]
    x_abs = en[None, None, None, :] + w[:, :, None, None] - gr.eps[ikq][:, None, :, None]
    x_emi = en[None, None, None, :] - w[:, :, None, None] - gr.eps[ikq][:, None, :, None]
    occ_abs = N[:, :, None, None] + fm[:, None, :, None]
    occ_emi = 1.0 + N[:, :, None, None] - fm[:, None, :, None]
    term = g2 * (occ_abs * delta_gauss(x_abs, eta, c) + occ_emi * delta_gauss(x_emi, eta, c))
    return term * keep[:, :, None, None]


def pair_terms_k(gr: Grids, ik: int, bands_n, T, mu, eta, c, q_list) -> np.ndarray:
    """The summand of Eq. 10 for one k before the q and mode sums:
    t[q, nu, n] = sum_m |g^nu_mn(k,q)|^2 [(N + f) delta(x+) + (1 + N - f) delta(x-)] in eV."""
    return pair_terms_full_k(gr, ik, bands_n, T, mu, eta, c, q_list).sum(axis=2)


def inv_tau_k(gr: Grids, ik: int, bands_n, T, mu, eta, c=6.0, q_list=None, q_weights=None):
    """SERTA scattering rates 1/tau_nk (s^-1) for the states n in ``bands_n`` at k
    (Sec. II C, Eq. 10, with 1/N_q and Gaussian delta).  Returns (rates, n_pairs).

    With ``q_weights`` the q sum is the weighted sum sum_q w_q t(q) over ``q_list`` (an
    importance-sampling estimate of the full sum when w_q = count_q / (S p(q)))."""
    bands_n = np.asarray(bands_n)
    if q_list is None:
        q_list = sieve_k(gr, ik, bands_n, eta, c)
    rates = np.zeros(len(bands_n))
    if len(q_list) == 0:
        return rates, 0
    t = pair_terms_k(gr, ik, bands_n, T, mu, eta, c, q_list)       # [q, nu, n]
    if q_weights is not None:
        t = t * np.asarray(q_weights, float)[:, None, None]
    rates = t.sum(axis=(0, 1)) * (2.0 * math.pi / HBAR_EVS) / gr.nk
    return rates, len(q_list)


def serta(gr: Grids, T, mu, eta, emin, emax, c=6.0, k_subset=None):
    """1/tau for every state in the window [emin, emax] (or for the k-points in ``k_subset``).

    Returns dict(ik, n, inv_tau, pairs_per_k: {ik: count}, n_pairs)."""
    ik_all, n_all = gr.window_states(emin, emax)
    kpts = np.unique(ik_all)
    if k_subset is not None:
        kpts = np.intersect1d(kpts, np.asarray(k_subset))
    out_ik, out_n, out_r, pairs = [], [], [], {}
    for ik in kpts:
        nsel = n_all[ik_all == ik]
        r, npair = inv_tau_k(gr, int(ik), nsel, T, mu, eta, c)
        out_ik.append(np.full(len(nsel), ik))
        out_n.append(nsel)
        out_r.append(r)
        pairs[int(ik)] = npair
    cat = (lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt))
    return dict(ik=cat(out_ik, np.int64), n=cat(out_n, np.int64), inv_tau=cat(out_r, float),
                pairs_per_k=pairs, n_pairs=int(sum(pairs.values())))


# ----------------------------------------------------------------------- transport
def conductivity(volume_A3, nk, v, inv_tau, eps, mu, T) -> np.ndarray:
    """sigma_ab = (2 e^2 / (N_k V)) sum v_a v_b tau f(1-f)/(k_B T) in S/m (Sec. II C, Eq. 12
    with F = F^0 = v tau; states with 1/tau = 0 excluded)."""
    ok = inv_tau > 0
    tau = np.where(ok, 1.0 / np.where(ok, inv_tau, 1.0), 0.0)
    f = fermi(eps, mu, T)
    w = tau * f * (1.0 - f)
    kT_J = KB_EVK * T * E_CHARGE
    s = np.einsum("s,sa,sb->ab", w, v, v)
    return 2.0 * E_CHARGE ** 2 / (nk * volume_A3 * 1e-30 * kT_J) * s


def transport_coefficients(volume_A3, nk, v, inv_tau, eps, mu, T):
    """sigma (S/m), Seebeck S (V/K) and electronic thermal conductivity kappa_e (W/(m K)) from
    the zeroth, first and second energy moments of the SERTA sum (Sec. II C, Eqs. 12-14, with
    F = F^0 = v tau):
        sigma        = (2 q^2 / (N_k V)) sum v v tau (-df/de),
        nu = sigma S = (2 q / (T V N_k)) sum (e - mu) v v tau (-df/de),   q = -e (electrons),
        kappa_0      = (2 / (T V N_k)) sum (e - mu)^2 v v tau (-df/de),
        S = sigma^-1 nu,  kappa_e = kappa_0 - T nu sigma^-1 nu
    (the tensor form of kappa_0 - T sigma S^2).  States with 1/tau = 0 are left out."""
    ok = inv_tau > 0
    tau = np.where(ok, 1.0 / np.where(ok, inv_tau, 1.0), 0.0)
    f = fermi(eps, mu, T)
    kT_J = KB_EVK * T * E_CHARGE
    w = tau * f * (1.0 - f) / kT_J                                    # tau (-df/de), s / J
    de_J = (np.asarray(eps, float) - mu) * E_CHARGE                    # e - mu in J
    vol = nk * volume_A3 * 1e-30
    m0 = np.einsum("s,sa,sb->ab", w, v, v)
    m1 = np.einsum("s,sa,sb->ab", w * de_J, v, v)
    m2 = np.einsum("s,sa,sb->ab", w * de_J ** 2, v, v)
    sigma = 2.0 * E_CHARGE ** 2 / vol * m0
    nu = 2.0 * (-E_CHARGE) / (T * vol) * m1
    kappa0 = 2.0 / (T * vol) * m2
    seebeck = np.linalg.solve(sigma, nu)
    kappa_e = kappa0 - T * nu @ seebeck
    return sigma, seebeck, kappa_e


# ------------------------------------------------------------------- iterative BTE
def ibte(gr: Grids, T, mu, eta, emin, emax, c=6.0, max_iter=200, tol=1e-12):
    """Iterative solution of the linearised BTE for the mean free paths F (Sec. II C, the
    iteration equation after Eq. 10):

        F^0_nk = v_nk tau_nk,
        F^{i+1}_nk = F^0_nk + tau_nk sum_{q p m} (Gamma^+ + Gamma^-)_{nk -> m k+q} F^i_{m k+q}.

    The paper's Gamma are the equilibrium transition rates with f_nk (1 - f_nk) divided out.
    By detailed balance, f_n (1 - f_m) N = f_n (1 - f_n) (N + f_m) on the absorption shell and
    f_n (1 - f_m)(1 + N) = f_n (1 - f_n)(1 + N - f_m) on the emission shell, so Gamma^+ and
    Gamma^- are exactly the two terms of the SERTA summand of Eq. 10 for the final state
    (m, k+q) and mode p, and 1/tau_nk is the sum of Gamma over all final states.

    The states are those of the energy window (the order of ``serta``).  Final states outside
    the window keep their share of 1/tau but carry F = 0 in the in-scattering sum.  The
    iteration stops when max |F^{i+1} - F^i| <= tol max |F^{i+1}| or after ``max_iter``
    applications.  Returns dict(ik, n, inv_tau, A (CSR, s^-1, rows = initial states, columns =
    final states), F0, F, iters)."""
    import scipy.sparse as sp

    ik_all, n_all = gr.window_states(emin, emax)
    ns = len(ik_all)
    pos = -np.ones(gr.eps.shape, np.int64)
    pos[ik_all, n_all] = np.arange(ns)
    pref = 2.0 * math.pi / HBAR_EVS / gr.nk
    inv_tau = np.zeros(ns)
    rows, cols, vals = [], [], []
    for ik in np.unique(ik_all):
        nsel = n_all[ik_all == ik]
        q = sieve_k(gr, int(ik), nsel, eta, c)
        if len(q) == 0:
            continue
        t = pair_terms_full_k(gr, int(ik), nsel, T, mu, eta, c, q).sum(axis=1) * pref   # [q, m, n]
        i_rows = pos[ik, nsel]
        inv_tau[i_rows] = t.sum(axis=(0, 1))
        j = pos[kq_index(int(ik), q, gr.ngrid)]                     # [q, m] final-state index
        qi, m = np.nonzero(j >= 0)
        for a, r in enumerate(i_rows):
            rows.append(np.full(len(qi), r))
            cols.append(j[qi, m])
            vals.append(t[qi, m, a])
    cat = (lambda x, dt: np.concatenate(x).astype(dt) if x else np.zeros(0, dt))
    A = sp.csr_matrix((cat(vals, float), (cat(rows, np.int64), cat(cols, np.int64))), shape=(ns, ns))
    v = gr.velocities(ik_all, n_all)
    ok = inv_tau > 0
    tau = np.where(ok, 1.0 / np.where(ok, inv_tau, 1.0), 0.0)
    F0 = tau[:, None] * v
    F = F0.copy()
    iters = 0
    for iters in range(1, max_iter + 1):
        Fn = F0 + tau[:, None] * (A @ F)
        change = np.abs(Fn - F).max() if ns else 0.0
        scale = np.abs(Fn).max() if ns else 0.0
        F = Fn
        if change <= tol * scale:
            break
    return dict(ik=ik_all, n=n_all, inv_tau=inv_tau, A=A, F0=F0, F=F, iters=iters)


def transport_from_F(volume_A3, nk, v, F, eps, mu, T):
    """sigma, Seebeck S and kappa_e from the mean free paths F (Sec. II C, Eqs. 12-14):
        m_p[a, b] = sum (e - mu)^p v_a F_b (-df/de),
        sigma = (2 e^2 / (N_k V)) m_0,  nu = sigma S = (2 (-e) / (T V N_k)) m_1,
        kappa_0 = (2 / (T V N_k)) m_2,  S = sigma^-1 nu,  kappa_e = kappa_0 - T nu sigma^-1 nu.
    With F = v tau this is ``transport_coefficients``."""
    f = fermi(eps, mu, T)
    kT_J = KB_EVK * T * E_CHARGE
    w = f * (1.0 - f) / kT_J
    de_J = (np.asarray(eps, float) - mu) * E_CHARGE
    vol = nk * volume_A3 * 1e-30
    m0 = np.einsum("s,sa,sb->ab", w, v, F)
    m1 = np.einsum("s,sa,sb->ab", w * de_J, v, F)
    m2 = np.einsum("s,sa,sb->ab", w * de_J ** 2, v, F)
    sigma = 2.0 * E_CHARGE ** 2 / vol * m0
    nu = 2.0 * (-E_CHARGE) / (T * vol) * m1
    kappa0 = 2.0 / (T * vol) * m2
    seebeck = np.linalg.solve(sigma, nu)
    kappa_e = kappa0 - T * nu @ seebeck
    return sigma, seebeck, kappa_e


def carrier_density(eps_cb, nk, volume_A3, mu, T) -> float:
    """Conduction electrons per cm^3: (2 / (N_k V)) sum_{n >= n_v, k} f(eps_nk)."""
    return 2.0 * fermi(eps_cb, mu, T).sum() / (nk * volume_A3 * 1e-24)


def find_mu(eps_cb, nk, volume_A3, n_cm3, T, rtol=1e-13):
    """Chemical potential by bisection on the monotone n(mu) (Sec. III A: chemical potential
    at the given doping and temperature)."""
    lo, hi = float(eps_cb.min()) - 3.0, float(eps_cb.max()) + 3.0
    mid = 0.5 * (lo + hi)
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        n = carrier_density(eps_cb, nk, volume_A3, mid, T)
        if abs(n - n_cm3) <= rtol * n_cm3 or hi - lo <= 1e-15:
            break
        if n < n_cm3:
            lo = mid
        else:
            hi = mid
    return mid


def mobility(sigma, n_cm3) -> np.ndarray:
    """mu_ab = sigma_ab / (n e) in cm^2/(V s) (Sec. II C, Eq. 15)."""
    return sigma / (n_cm3 * 1e6 * E_CHARGE) * 1e4
