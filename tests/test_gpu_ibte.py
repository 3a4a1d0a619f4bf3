"""GPU parity of the iterative BTE (Sec. II C, iteration equation) against the FP64 oracle.

The CUDA path stores Gamma during the interpolation (FP64 blocks on the FP64 path, FP32 on
the split paths) and runs one deterministic step kernel per iteration.  Cases:
  * FP64: 1/tau, F after a fixed number of steps, the converged F and the transport tensors
    from F, on the tiny crystal (6^3) and the Al-like crystal (10^3, ragged pair lists, also
    in a split precision);
  * split precisions and the sum-factorised fp32 mode: the same after a fixed number of
    steps, within 1e-4;
  * 16 bands in the window (two register groups of the step kernel);
  * k-point chunking and repeated runs give bitwise identical F; max_iter = 0 gives v tau.
"""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import epwi, synth

pytestmark = pytest.mark.gpu

T = 300.0
SPLIT = tuple(getattr(epwi, "SPLIT_MODES", ()))


def _case(system, grid, half_window, eta):
    gr = O.Grids(system, grid)
    mu = gr.band_centre() if system.name != "einstein" else 0.3
    return gr, mu, mu - half_window, mu + half_window, eta


def _run(system, grid, mu, emin, emax, eta, max_iter, tol, precision="fp64", chunk=0):
    ctx = epwi.Context(precision=precision, device=0, kpoint_chunk=chunk)
    ctx.setup(system)
    ctx.eigs(grid)
    it, ch = ctx.ibte(T, mu, eta, emin, emax, max_iter=max_iter, tol=tol)
    k, b, r = ctx.rates()
    F = ctx.mfp()
    tr = ctx.ibte_transport()
    serta_tr = ctx.transport()
    st = ctx.ibte_stats()
    ctx.close()
    return dict(k=k, b=b, r=r, F=F, tr=tr, serta=serta_tr, it=it, ch=ch, st=st)


def _ordered(res, ref):
    order = np.lexsort((res["b"], res["k"]))
    assert np.array_equal(res["k"][order], ref["ik"]) and np.array_equal(res["b"][order], ref["n"])
    return order


@pytest.fixture(scope="module")
def tiny6():
    s = synth.tiny_system()
    gr, mu, lo, hi, eta = _case(s, (6, 6, 6), 0.3, 0.05)
    return s, gr, mu, lo, hi, eta


@pytest.mark.parametrize("steps", [0, 1, 25])
def test_fp64_fixed_steps_match_the_oracle(tiny6, steps):
    s, gr, mu, lo, hi, eta = tiny6
    ref = O.ibte(gr, T, mu, eta, lo, hi, max_iter=steps, tol=0.0)
    res = _run(s, (6, 6, 6), mu, lo, hi, eta, steps, 0.0)
    o = _ordered(res, ref)
    assert res["it"] == steps
    assert np.abs(res["r"][o] - ref["inv_tau"]).max() <= 1e-10 * ref["inv_tau"].max()
    assert np.abs(res["F"][o] - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()
    if steps == 0:
        assert np.array_equal(ref["F"], ref["F0"])


def test_fp64_converged_mfp_and_transport(tiny6):
    s, gr, mu, lo, hi, eta = tiny6
    ref = O.ibte(gr, T, mu, eta, lo, hi, max_iter=20000, tol=1e-12)
    res = _run(s, (6, 6, 6), mu, lo, hi, eta, 20000, 1e-12)
    o = _ordered(res, ref)
    assert abs(res["it"] - ref["iters"]) <= 2 and res["ch"] <= 1e-12
    assert np.abs(res["F"][o] - ref["F"]).max() <= 1e-8 * np.abs(ref["F"]).max()
    v = gr.velocities(ref["ik"], ref["n"])
    e = gr.eps[ref["ik"], ref["n"]]
    want = O.transport_from_F(s.volume, gr.nk, v, ref["F"], e, mu, T)
    for got, exp in zip(res["tr"], want):
        assert np.abs(got - exp).max() <= 1e-8 * np.abs(exp).max()
    # the iteration changes sigma against SERTA on this crystal
    assert np.abs(res["tr"][0] - res["serta"][0]).max() > 1e-3 * np.abs(res["serta"][0]).max()


@pytest.mark.parametrize("precision", ("fp64", "fp32") + SPLIT[:1])
def test_al_like_ragged_pairs(precision):
    s = synth.al_like_system()
    gr, mu, lo, hi, eta = _case(s, (10, 10, 10), 0.3, 0.05)
    ref = O.ibte(gr, T, mu, eta, lo, hi, max_iter=8, tol=0.0)
    res = _run(s, (10, 10, 10), mu, lo, hi, eta, 8, 0.0, precision=precision)
    o = _ordered(res, ref)
    tol = 1e-10 if precision == "fp64" else 1e-4
    assert np.abs(res["r"][o] - ref["inv_tau"]).max() <= tol * ref["inv_tau"].max()
    assert np.abs(res["F"][o] - ref["F"]).max() <= tol * np.abs(ref["F"]).max()
    assert res["st"]["n_pairs"] == O.serta(gr, T, mu, eta, lo, hi)["n_pairs"]
    # one stored value per (pair, n in window(k), m in window(k+q)): at least the nonzeros
    assert res["st"]["n_entries"] >= ref["A"].nnz
    # the step's index: a column word per entry and an offset per k-point
    nkp = len(np.unique(res["k"]))
    assert res["st"]["index_bytes"] == 4 * res["st"]["n_entries"] + 8 * (nkp + 1)


@pytest.mark.parametrize("precision", SPLIT + ("fp32",))
def test_split_precision_fixed_steps(tiny6, precision):
    s, gr, mu, lo, hi, eta = tiny6
    ref = O.ibte(gr, T, mu, eta, lo, hi, max_iter=10, tol=0.0)
    res = _run(s, (6, 6, 6), mu, lo, hi, eta, 10, 0.0, precision=precision)
    o = _ordered(res, ref)
    assert res["st"]["entry_bytes"] == 4
    assert np.abs(res["r"][o] - ref["inv_tau"]).max() <= 1e-4 * ref["inv_tau"].max()
    assert np.abs(res["F"][o] - ref["F"]).max() <= 1e-4 * np.abs(ref["F"]).max()
    v = gr.velocities(ref["ik"], ref["n"])
    e = gr.eps[ref["ik"], ref["n"]]
    sig = O.transport_from_F(s.volume, gr.nk, v, ref["F"], e, mu, T)[0]
    assert np.abs(res["tr"][0] - sig).max() <= 1e-4 * np.abs(sig).max()


def test_fp64_windows_wider_than_one_band_group():
    """16 Wannier functions, window over every band: up to 16 states per k-point, two
    register groups of 8 bands in the step kernel."""
    s, _ = synth.batch_system(8)
    assert s.nw == 16
    gr = O.Grids(s, (4, 4, 4))
    mu, eta = gr.band_centre(), 0.1
    lo, hi = -1e9, 1e9
    ref = O.ibte(gr, T, mu, eta, lo, hi, max_iter=6, tol=0.0)
    res = _run(s, (4, 4, 4), mu, lo, hi, eta, 6, 0.0)
    o = _ordered(res, ref)
    assert np.abs(res["r"][o] - ref["inv_tau"]).max() <= 1e-10 * ref["inv_tau"].max()
    assert np.abs(res["F"][o] - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()


def test_chunking_and_repeat_are_bitwise_identical(tiny6):
    s, gr, mu, lo, hi, eta = tiny6
    a = _run(s, (6, 6, 6), mu, lo, hi, eta, 12, 0.0)
    b = _run(s, (6, 6, 6), mu, lo, hi, eta, 12, 0.0, chunk=7)
    c = _run(s, (6, 6, 6), mu, lo, hi, eta, 12, 0.0)
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["F"], c["F"])
    assert np.array_equal(a["r"], b["r"])


def test_fp64_time_reversal_symmetric_metal_converges_to_the_oracle():
    """Real H(R) and g: the drive of the number-conserving mode vanishes and the iteration
    converges in tens of steps; converged F and sigma match the oracle."""
    s = synth.time_reversal_symmetric(synth.al_like_system())
    gr, mu, lo, hi, eta = _case(s, (10, 10, 10), 0.3, 0.05)
    ref = O.ibte(gr, T, mu, eta, lo, hi, max_iter=500, tol=1e-11)
    assert ref["iters"] < 200
    res = _run(s, (10, 10, 10), mu, lo, hi, eta, 500, 1e-11)
    o = _ordered(res, ref)
    assert abs(res["it"] - ref["iters"]) <= 1
    assert np.abs(res["F"][o] - ref["F"]).max() <= 1e-9 * np.abs(ref["F"]).max()
    v = gr.velocities(ref["ik"], ref["n"])
    e = gr.eps[ref["ik"], ref["n"]]
    sig = O.transport_from_F(s.volume, gr.nk, v, ref["F"], e, mu, T)[0]
    assert np.abs(res["tr"][0] - sig).max() <= 1e-9 * np.abs(sig).max()


def test_fp32_long_warp_ranges_match_fp64():
    """Al-like 40^3 with a +-0.5 eV window: each warp's Gamma range is longer than the staged
    step's shared ring (2048 entries), so the ring wraps within a warp's range.  Eight fixed
    steps of the fp32 mode against the FP64 path (itself pinned to the oracle on smaller
    grids)."""
    s = synth.al_like_system()
    grid = (40, 40, 40)
    ctx = epwi.Context(precision="fp64", device=0)
    ctx.setup(s)
    ctx.eigs(grid)
    lo, hi = ctx.band_range()
    ctx.close()
    mu, eta = 0.5 * (lo + hi), 0.02
    ref = _run(s, grid, mu, mu - 0.5, mu + 0.5, eta, 8, 0.0, precision="fp64")
    res = _run(s, grid, mu, mu - 0.5, mu + 0.5, eta, 8, 0.0, precision="fp32")
    assert np.array_equal(res["k"], ref["k"]) and np.array_equal(res["b"], ref["b"])
    assert res["st"]["n_pairs"] == ref["st"]["n_pairs"]
    nkp = len(np.unique(res["k"]))
    assert res["st"]["n_entries"] / (8 * nkp) > 2048
    assert np.abs(res["r"] - ref["r"]).max() <= 1e-4 * ref["r"].max()
    assert np.abs(res["F"] - ref["F"]).max() <= 1e-4 * np.abs(ref["F"]).max()
