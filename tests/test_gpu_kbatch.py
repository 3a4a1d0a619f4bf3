"""The k-batch ordering (Sec. III C, Table 3: Rp->q once per q, Re->k per pair) computes the
same SERTA rates as the q-batch ordering: parity with the FP64 oracle and with the FP64 q-batch
path, on the tiny crystal, the Al-like metal (ragged q buckets) and the Si-like shapes (8 bands,
6 modes)."""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import epwi, synth

pytestmark = pytest.mark.gpu
T = 300.0


def _rates(system, grid, mu, eta, lo, hi, ordering, precision="fp64"):
    ctx = epwi.Context(precision=precision, device=0, ordering=ordering)
    ctx.setup(system)
    ctx.eigs(grid)
    ns, npairs = ctx.scatter_rates(T, mu, eta, lo, hi)
    k, b, r = ctx.rates()
    st = ctx.stats()
    ctx.close()
    o = np.lexsort((b, k))
    return k[o], b[o], r[o], npairs, st


@pytest.mark.parametrize("name,grid,half,eta", [("tiny", (6, 6, 6), None, 0.05),
                                                ("al_like", (8, 8, 8), 0.3, 0.05),
                                                ("si_like", (4, 4, 4), None, 0.05)])
def test_kbatch_matches_the_oracle(name, grid, half, eta):
    s = getattr(synth, f"{name}_system")()
    gr = O.Grids(s, grid)
    if name == "si_like":
        cbm = gr.eps[:, s.n_valence].min()
        mu, lo, hi = cbm - 0.2, cbm, cbm + 0.5
    else:
        mu = gr.band_centre()
        lo, hi = (-1e9, 1e9) if half is None else (mu - half, mu + half)
    ref = O.serta(gr, T, mu, eta, lo, hi)
    k, b, r, npairs, st = _rates(s, grid, mu, eta, lo, hi, "k-batch")
    assert np.array_equal(k, ref["ik"]) and np.array_equal(b, ref["n"])
    assert npairs == ref["n_pairs"]
    assert np.abs(r - ref["inv_tau"]).max() <= 1e-10 * ref["inv_tau"].max()


def test_kbatch_equals_qbatch_fp64():
    s = synth.al_like_system()
    gr = O.Grids(s, (10, 10, 10))
    mu = gr.band_centre()
    a = _rates(s, (10, 10, 10), mu, 0.05, mu - 0.3, mu + 0.3, "q-batch")
    b = _rates(s, (10, 10, 10), mu, 0.05, mu - 0.3, mu + 0.3, "k-batch")
    assert np.array_equal(a[0], b[0]) and a[3] == b[3]
    assert np.abs(a[2] - b[2]).max() <= 1e-12 * a[2].max()
    # per-pair volumes: k-batch n_Re N_m W^2, q-batch n_Rp N_m W n_k
    assert b[4]["scatter_flops"] > a[4]["scatter_flops"]


def test_kbatch_is_fp64_only():
    ctx = epwi.Context(precision="fp16x3", device=0, ordering="k-batch")
    ctx.setup(synth.tiny_system())
    ctx.eigs(4)
    with pytest.raises(epwi.EpwiError):
        ctx.scatter_rates(T, 0.0, 0.05, -1e9, 1e9)
    ctx.close()
