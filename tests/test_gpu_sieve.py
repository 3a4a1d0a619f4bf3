"""GPU parity of the energy-conservation sieve (Sec. III A) for the compiled shapes (4 bands
with 3 modes, 8 bands with 6 modes): the pair count of every window k-point against the
oracle's sieve, in both the mask form and the fill form (the form used when the decision mask
does not fit).

The kernel decides most candidates from the distance between the window energies at k and the
energies at k+q, against hbar omega_max(q) + c eta with a rounding margin, and sends the rest
to the per-mode FP32 test and its FP64 re-check.  The cases cover both regimes: a smearing
whose c eta exceeds every phonon energy (nearly every decision from the distance), and a
narrow smearing (c eta below the top phonon energies) where the per-mode test decides for
many q."""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import epwi, synth

pytestmark = pytest.mark.gpu
T = 300.0


def _window(name, gr):
    if name == "si_like":
        _, cbm = gr.band_edges(4)
        return cbm, cbm + 0.25
    mu = gr.band_centre()
    return mu - 0.3, mu + 0.3


@pytest.mark.parametrize("name,grid,eta", [
    ("al_like", (10, 10, 10), 0.02),      # c eta = 0.12 eV above every phonon energy
    ("al_like", (10, 10, 10), 0.004),     # c eta = 0.024 eV: the per-mode test for many q
    ("al_like", (12, 7, 9), 0.006),       # ragged plane blocks
    ("si_like", (10, 10, 10), 0.01),
    ("si_like", (9, 10, 11), 0.004),
])
@pytest.mark.parametrize("mask", [True, False])
def test_sieve_counts_match_the_oracle(monkeypatch, name, grid, eta, mask):
    s = getattr(synth, f"{name}_system")()
    gr = O.Grids(s, grid)
    lo, hi = _window(name, gr)
    mu = 0.5 * (lo + hi)
    if mask:
        monkeypatch.delenv("EPWI_SIEVE_MASK_MAX_BYTES", raising=False)
    else:
        monkeypatch.setenv("EPWI_SIEVE_MASK_MAX_BYTES", "0")
    ctx = epwi.Context(precision="fp64", device=0, kpoint_chunk=7)
    ctx.setup(s)
    ctx.eigs(grid)
    ctx.scatter_rates(T, mu, eta, lo, hi)
    kp, cnt = ctx.sieve()
    ctx.close()
    ik_all, n_all = gr.window_states(lo, hi)
    want_k = np.unique(ik_all)
    assert np.array_equal(np.sort(kp), want_k) and len(kp) > 0
    for k, c in zip(kp, cnt):
        nsel = n_all[ik_all == k]
        assert int(c) == len(O.sieve_k(gr, int(k), nsel, eta)), int(k)
