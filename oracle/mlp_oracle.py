"""Plain FP64 CPU oracle for the learned q-proposal and the importance-sampled 1/tau.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the oracle legs of
``bench.py`` may import this module.  It shares no code with the CUDA path.

The paper has no learned component.  What this oracle checks is an estimator of the q sum in
the SERTA rate (Sec. II C, Eq. 10):

    1/tau_nk = (2 pi / hbar) (1/N_q) sum_{q, nu} t_nu(k, q, n),

with t the summand of Eq. 10 (``epwi_oracle.pair_terms_k``).  Drawing S grid points q_s from a
proposal p(q) that is positive wherever t is, (1/S) sum_s t(q_s) / p(q_s) has expectation
sum_q t(q).  Repeated draws are merged: a distinct q drawn c_q times gets the weight
w_q = c_q / (S p(q)).

The proposal is built from a multilayer perceptron 9 -> 128 -> 128 -> 128 -> 1 with SiLU
activations, z * sigmoid(z), on the hidden layers.  Its inputs, in this order, are:
  * the fractional coordinates of k, each mapped to [-1/2, 1/2) and then doubled;
  * the same for q;
  * (eps_nk - mu) / 0.25 eV;
  * the band index n / W;
  * the mode index nu / N_m.
Its output estimates log t, in the normalised form (log(t + floor) - mean) / std of the
training targets.  The network is trained by least squares, L = (1/2B) sum (yhat - y)^2.

The q grid is divided into cells of s^3 points, where the stride s divides each N_a.  Cell c
holds the fine indices s c - floor(s/2) ... s c - floor(s/2) + s - 1 (mod N); its centre is the
fine point s c.  For a state (k, n) the network is evaluated at every cell centre and mode,
giving the cell probability
    P_n(c) = sum_nu exp(a yhat) / sum_{c', nu} exp(a yhat),
where a is the std of the training targets.  The proposal for a state is
    p_n(q) = alpha / N_q + (1 - alpha) P_n(cell(q)) / s^3.
The alpha / N_q term keeps p positive everywhere, so the estimate stays unbiased.  All window
bands of one k share one draw, from the band mixture p(q) = (1/n_win) sum_n p_n(q); the
weights of that draw are unbiased for every band.
"""
from __future__ import annotations

import numpy as np

D_IN = 9
HID = 128
E_SCALE = 0.25                       # eV, scale of the energy feature
#: parameter blocks in storage order: name -> shape
SHAPES = (("W1", (HID, D_IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("w4", (HID,)), ("b4", (1,)))
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat) -> dict:
    flat = np.asarray(flat, np.float64)
    assert flat.size == N_PARAM
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = flat[o:o + n].reshape(shp)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SHAPES])


def round_bf16(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


# ------------------------------------------------------------------------- features
def centred_frac(i, n) -> np.ndarray:
    """i / n mapped to [-1/2, 1/2)."""
    i = np.asarray(i, np.int64)
    return np.where(2 * i < n, i / n, i / n - 1.0)


def features(ngrid, ik, iq, e_rel, n, nu, W, Nm) -> np.ndarray:
    """Network inputs (float32) for the samples (k index, q index, eps_nk - mu, n, nu)."""
    n1, n2, n3 = ngrid
    ik = np.asarray(ik, np.int64)
    iq = np.asarray(iq, np.int64)
    cols = []
    for idx in (ik, iq):
        i1, i2, i3 = idx // (n2 * n3), (idx // n3) % n2, idx % n3
        cols += [2.0 * centred_frac(i1, n1), 2.0 * centred_frac(i2, n2), 2.0 * centred_frac(i3, n3)]
    cols.append(np.asarray(e_rel, float) / E_SCALE + 0 * ik)
    cols.append(np.asarray(n, float) / W + 0 * ik)
    cols.append(np.asarray(nu, float) / Nm + 0 * ik)
    return np.stack(cols, -1).astype(np.float32)


# -------------------------------------------------------------------------- network
def sigmoid(z):
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(flat, X):
    """yhat[B] and the pre-activations of the three hidden layers."""
    p = unpack(flat)
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = silu(z3)
    y = h3 @ p["w4"] + p["b4"][0]
    return y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def loss_grad(flat, X, Y):
    """L = (1/2B) sum (yhat - y)^2 and dL/dparams (flat, storage order), by the chain rule
    taken layer by layer from the output back."""
    p = unpack(flat)
    yhat, c = forward(flat, X)
    B = len(yhat)
    r = yhat - np.asarray(Y, np.float64)
    loss = 0.5 * np.dot(r, r) / B
    dy = r / B                                         # dL/dyhat
    g = {"w4": c["h3"].T @ dy, "b4": np.array([dy.sum()])}
    dz3 = np.outer(dy, p["w4"]) * dsilu(c["z3"])
    g["W3"] = dz3.T @ c["h2"]
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * dsilu(c["z2"])
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * dsilu(c["z1"])
    g["W1"] = dz1.T @ c["X"]
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def adam_step(flat, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); step counts from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------------- proposal
def cell_of(iq, ngrid, s) -> np.ndarray:
    """Flat cell index of the fine q indices for stride s."""
    n1, n2, n3 = ngrid
    iq = np.asarray(iq, np.int64)
    i = (iq // (n2 * n3), (iq // n3) % n2, iq % n3)
    c = [((ia + s // 2) % na) // s for ia, na in zip(i, ngrid)]
    return (c[0] * (n2 // s) + c[1]) * (n3 // s) + c[2]


def cell_centres(ngrid, s) -> np.ndarray:
    """Fine flat index of every cell centre, in cell order."""
    n1, n2, n3 = ngrid
    c1, c2, c3 = np.meshgrid(np.arange(n1 // s), np.arange(n2 // s), np.arange(n3 // s),
                             indexing="ij")
    return ((s * c1 * n2 + s * c2) * n3 + s * c3).reshape(-1)


def cell_probs(scores) -> np.ndarray:
    """P(c) from scores[c, nu] (already multiplied by the output scale a)."""
    s = np.asarray(scores, np.float64)
    m = s.max()
    e = np.exp(s - m).sum(axis=1)
    return e / e.sum()


def p_mix(iq, ngrid, s, alpha, probs) -> np.ndarray:
    """Band-mixture proposal probability of the fine q indices; ``probs`` is [n_win][cells]."""
    nq = int(np.prod(ngrid))
    c = cell_of(iq, ngrid, s)
    probs = np.asarray(probs, np.float64)
    pn = alpha / nq + (1.0 - alpha) * probs[:, c] / s ** 3
    return pn.mean(axis=0)
