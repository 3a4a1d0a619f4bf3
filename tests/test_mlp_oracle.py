"""Pins of the learned-proposal oracle (oracle/mlp_oracle.py) against finite differences,
closed forms and invariants.  CPU only."""
import math

import numpy as np
import pytest

from oracle import epwi_oracle as O
from oracle import mlp_oracle as M
from paper_2306_16493_gb300 import synth


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, M.N_PARAM)


def test_param_layout():
    assert M.N_PARAM == 128 * 9 + 128 + 2 * (128 * 128 + 128) + 128 + 1
    p = _params(0)
    assert np.array_equal(M.pack(M.unpack(p)), p)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(2)
    X = rng.normal(0, 1, (7, M.D_IN))
    Y = rng.normal(0, 1, 7)
    _, g = M.loss_grad(p, X, Y)
    idx = np.concatenate([rng.choice(M.N_PARAM, 200, replace=False), [M.N_PARAM - 1]])
    h = 1e-6
    for i in idx:
        e = np.zeros(M.N_PARAM)
        e[i] = h
        fd = (M.loss_grad(p + e, X, Y)[0] - M.loss_grad(p - e, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_silu_derivative_and_values():
    z = np.linspace(-8, 8, 33)
    assert np.allclose(M.silu(z), z / (1 + np.exp(-z)), rtol=1e-14, atol=1e-300)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    assert np.allclose(M.dsilu(z), fd, rtol=1e-8, atol=1e-10)


def test_adam_first_step_is_signed_lr():
    """On its first step Adam moves every parameter by -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, m, v = M.adam_step(w, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(w1 - w, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_round_bf16():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 1 + 2 ** -7, 3.0e38], np.float32)
    r = M.round_bf16(x)
    assert list(r[:5]) == [1.0, 1.0, 1 + 2 ** -6, -2.5, 1 + 2 ** -7]
    assert np.isfinite(r[5])


def test_features_hand_values():
    X = M.features((4, 6, 8), ik=[0, (3 * 6 + 5) * 8 + 4], iq=[(2 * 6 + 3) * 8 + 1, 0],
                   e_rel=[0.05, -0.125], n=[1, 3], nu=[0, 5], W=8, Nm=6)
    # k = (0,0,0); q = (2/4, 3/6, 1/8) -> centred (-1/2, -1/2, 1/8) -> doubled
    assert np.allclose(X[0], [0, 0, 0, -1, -1, 0.25, 0.2, 1 / 8, 0], atol=0)
    # k = (3/4, 5/6, 4/8) -> (-1/4, -1/6, -1/2) -> doubled
    assert np.allclose(X[1], [-0.5, -1 / 3, -1, 0, 0, 0, -0.5, 3 / 8, 5 / 6], rtol=1e-7)


@pytest.mark.parametrize("ngrid,s", [((8, 8, 8), 2), ((12, 6, 9), 3), ((6, 6, 6), 1)])
def test_cells_partition_grid(ngrid, s):
    nq = int(np.prod(ngrid))
    c = M.cell_of(np.arange(nq), ngrid, s)
    counts = np.bincount(c)
    assert len(counts) == nq // s ** 3 and np.all(counts == s ** 3)
    cen = M.cell_centres(ngrid, s)
    assert np.array_equal(M.cell_of(cen, ngrid, s), np.arange(nq // s ** 3))
    # every fine point is within s//2 grid steps (periodically) of its cell centre
    n1, n2, n3 = ngrid
    q = np.arange(nq)
    qc = cen[c]
    for div, mod, n in ((n2 * n3, None, n1), (n3, n2, n2), (1, n3, n3)):
        a = q // div if mod is None else (q // div) % mod
        b = qc // div if mod is None else (qc // div) % mod
        d = (a - b) % n
        d = np.minimum(d, n - d)
        assert d.max() <= s // 2


def test_p_mix_normalised():
    rng = np.random.default_rng(4)
    ngrid, s = (8, 8, 8), 2
    probs = rng.dirichlet(np.ones(64), size=3)
    p = M.p_mix(np.arange(512), ngrid, s, 0.1, probs)
    assert abs(p.sum() - 1.0) < 1e-13 and p.min() >= 0.1 / 512


def _tiny_state():
    sysm = synth.tiny_system(1)
    gr = O.Grids(sysm, (6, 6, 6))
    mu = gr.band_centre()
    ik, n = gr.window_states(mu - 0.3, mu + 0.3)
    return gr, mu, int(ik[0]), int(n[0])


def test_perfect_proposal_has_zero_variance():
    """With p(q) = t(q) / sum t the weighted sum equals the full sum for ANY draw."""
    gr, mu, ik, n = _tiny_state()
    eta, T = 0.05, 300.0
    q_all = O.sieve_k(gr, ik, [n], eta)
    t = O.pair_terms_k(gr, ik, [n], T, mu, eta, 6.0, q_all)[:, :, 0].sum(1)
    pos = t > 0
    q_all, t = q_all[pos], t[pos]
    p = t / t.sum()
    full, _ = O.inv_tau_k(gr, ik, [n], T, mu, eta)
    rng = np.random.default_rng(5)
    for S in (1, 17, 1000):
        draw = rng.choice(len(q_all), size=S, p=p)
        uq, cnt = np.unique(draw, return_counts=True)
        w = cnt / (S * p[uq])
        est, _ = O.inv_tau_k(gr, ik, [n], T, mu, eta, q_list=q_all[uq], q_weights=w)
        assert abs(est[0] - full[0]) <= 1e-12 * full[0]


def test_uniform_importance_sampling_is_unbiased():
    """Uniform draws over the whole q grid: the mean of 40 independent estimates lies within
    4 standard errors of the full sum."""
    gr, mu, ik, n = _tiny_state()
    eta, T = 0.05, 300.0
    full, _ = O.inv_tau_k(gr, ik, [n], T, mu, eta)
    q_all = np.arange(gr.nk)
    t_all = O.pair_terms_k(gr, ik, [n], T, mu, eta, 6.0, q_all)[:, :, 0].sum(1)
    rng = np.random.default_rng(6)
    S, est = 200, []
    for _ in range(40):
        draw = rng.integers(0, gr.nk, S)
        uq, cnt = np.unique(draw, return_counts=True)
        w = cnt / (S * (1.0 / gr.nk))
        r, _ = O.inv_tau_k(gr, ik, [n], T, mu, eta, q_list=uq, q_weights=w)
        est.append(r[0])
        # the weighted sum of the oracle equals the plain per-sample average
        direct = (t_all[draw] * gr.nk).mean() * (2 * math.pi / O.HBAR_EVS) / gr.nk
        assert abs(r[0] - direct) <= 1e-12 * abs(direct) + 1e-300
    est = np.asarray(est)
    se = est.std(ddof=1) / math.sqrt(len(est))
    assert abs(est.mean() - full[0]) <= 4 * se
