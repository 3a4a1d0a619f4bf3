"""Batched uneven systems (one graph, one persistent kernel) against the oracle and against
each system's FP64 GPU path: 1/tau per degenerate group and sigma per system within the
mixed-precision bound (1e-4), bitwise-identical replays, and tile-shape independence."""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import synth
from tests.parity import compare_rates, oracle_run, rel_frob

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def epwi():
    from paper_2306_16493_gb300 import epwi as E
    return E


# (system, grid): W in {4, 8, 16, 24}, modes in {3, 6, 12, 18}, R-sets of 27, 125 and 343
# vectors, a non-cubic grid among them
CASES = [
    (lambda: synth.tiny_system(1), (5, 5, 5)),
    (lambda: synth.batch_system(5)[0], (4, 4, 4)),      # nat 2, nw 8, 343 R
    (lambda: synth.batch_system(10)[0], (4, 4, 4)),     # nat 4, nw 16, 125 R
    (lambda: synth.batch_system(15)[0], (3, 4, 5)),     # nat 6, nw 24, 27 R
    (lambda: synth.batch_system(13)[0], (4, 4, 4)),     # nat 2, nw 24, 125 R
]
T, ETA = 300.0, 0.05


@pytest.fixture(scope="module")
def batch_setup(epwi):
    systems = [make() for make, _ in CASES]
    grids = [g for _, g in CASES]
    grs = [O.Grids(s, g) for s, g in zip(systems, grids)]
    mu = np.array([gr.band_centre() for gr in grs])
    b = epwi.Batch()
    b.setup(systems, grids)
    return b, systems, grids, grs, mu


def test_batch_vs_oracle_and_fp64(epwi, batch_setup):
    b, systems, grids, grs, mu = batch_setup
    lo, hi = mu - 1.0, mu + 1.0
    npairs = b.plan(T, mu, ETA, lo, hi, autotune=True)
    assert npairs > 0
    sig = b.run()
    st = b.stats()
    assert st["n_systems"] == len(systems) and st["n_items"] > 0 and st["runs"] == 1
    for s, (sysm, grid, gr) in enumerate(zip(systems, grids, grs)):
        k, n, r = b.rates(s)
        gpu = dict(ik=k.astype(np.int64), n=n.astype(np.int64), inv_tau=r)
        if sysm.nw <= 8 or len(sysm.Re) <= 125:
            ora = oracle_run(gr, T, mu[s], ETA, lo[s], hi[s])
            worst, ng = compare_rates(gpu, ora, gr.eps, TOL)
            assert ng > 0 and worst <= TOL, (s, worst)
            assert rel_frob(sig[s], ora["sigma"]) <= TOL, s
        # the same system through the single-system FP64 path
        ctx = epwi.Context()
        ctx.setup(sysm)
        ctx.eigs(grid)
        ctx.scatter_rates(T, mu[s], ETA, lo[s], hi[s])
        kf, nf, rf = ctx.rates()
        ref = dict(ik=kf.astype(np.int64), n=nf.astype(np.int64), inv_tau=rf)
        worst, _ = compare_rates(gpu, ref, gr.eps, TOL)
        assert worst <= TOL, (s, worst)
        assert rel_frob(sig[s], ctx.conductivity()) <= TOL, s
        mt, kc, src = b.tile(s)
        assert mt >= 1 and kc >= 1 and src in (1, 2)


def test_batch_replay_is_bitwise_identical(epwi, batch_setup):
    b, systems, grids, grs, mu = batch_setup
    b.plan(T, mu, ETA, mu - 1.0, mu + 1.0, autotune=False)
    s1 = b.run()
    r1 = [b.rates(s)[2].copy() for s in range(len(systems))]
    s2 = b.run()
    assert np.array_equal(s1, s2)
    for s in range(len(systems)):
        assert np.array_equal(r1[s], b.rates(s)[2])
    assert b.stats()["runs"] >= 2


def test_batch_tile_shapes_agree(epwi, batch_setup):
    """Two forced tile shapes per system give the same rates up to FP32 summation order."""
    b, systems, grids, grs, mu = batch_setup
    out = []
    for mt, kc in ((8, 8), (4, 4)):
        for s in range(len(systems)):
            b.set_tile(s, mt, kc)
        b.plan(T, mu, ETA, mu - 1.0, mu + 1.0, autotune=False)
        for s in range(len(systems)):
            assert b.tile(s) == (mt, kc, 3)
        b.run()
        out.append([b.rates(s)[2].copy() for s in range(len(systems))])
    for s in range(len(systems)):
        a, c = out[0][s], out[1][s]
        assert np.allclose(a, c, rtol=1e-5, atol=1e-9 * np.abs(c).max()), s
    for s in range(len(systems)):
        b.set_tile(s, 0, 0)
