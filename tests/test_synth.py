"""The seeded input generator: the chunked, threaded draw of large complex-normal arrays gives
exactly the values of the sequential SplitMix64 + Box-Muller stream, and the Wigner-Seitz
R-sets are complete sets of supercell representatives."""
import itertools

import numpy as np
import pytest

from paper_2306_16493_gb300 import synth
from paper_2306_16493_gb300.synth import SplitMix64


def test_chunked_complex_normal_is_the_sequential_stream():
    for n in ((1 << 21) + 7, 3 * (1 << 21)):
        a, b = SplitMix64(2024), SplitMix64(2024)
        a.uniform(5)
        b.uniform(5)
        z = b.normal(2 * n)
        ref = (0.5 / np.sqrt(2.0)) * (z[0::2] + 1j * z[1::2])
        got = a.complex_normal((n,), sigma=0.5)
        assert np.array_equal(got, ref)
        assert a.state == b.state
        assert np.array_equal(a.uniform(3), b.uniform(3))


def test_splitmix64_reference_values():
    """First outputs of SplitMix64 seeded with 0 (the published generator's known sequence)."""
    r = SplitMix64(0)
    assert [int(x) for x in r.next_u64(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                               0x06C45D188009454F]


@pytest.mark.parametrize("cell,nsc", [(synth.fcc_cell(4.05)[0], 2), (synth.fcc_cell(4.05)[0], 4),
                                      (synth.diamond_cell(5.43)[0], 3), (np.diag([3.0, 3.5, 4.2]), 3)])
def test_wigner_seitz_set_is_a_weighted_set_of_supercell_representatives(cell, nsc):
    """Every residue class of Z^3 mod nsc carries total weight 1 (boundary vectors share it
    with their equivalent images), so sum(w) = nsc^3 and sum_R w e^{2 pi i m.n / nsc} =
    nsc^3 delta_{m = 0 mod nsc}; the set is closed under R -> -R with equal weights, and every
    member is no farther from the origin than any of its supercell images."""
    n, w = synth.ws_rset(cell, nsc)
    assert w.sum() == pytest.approx(nsc ** 3, abs=1e-12)
    cls = {}
    for v, x in zip(map(tuple, np.mod(n, nsc)), w):
        cls[v] = cls.get(v, 0.0) + x
    assert len(cls) == nsc ** 3 and all(abs(x - 1.0) < 1e-12 for x in cls.values())
    lut = {tuple(v): x for v, x in zip(n.tolist(), w)}
    assert all(lut.get(tuple((-np.array(v)).tolist())) == x for v, x in lut.items())
    for m in itertools.product(range(nsc), repeat=3):
        f = (w * np.exp(2j * np.pi * (n @ np.array(m)) / nsc)).sum()
        assert abs(f - (nsc ** 3 if m == (0, 0, 0) else 0.0)) < 1e-9
    R = n @ cell
    for t in itertools.product((-1, 0, 1), repeat=3):
        img = R + nsc * (np.array(t) @ cell)
        assert np.all(np.linalg.norm(R, axis=1) <= np.linalg.norm(img, axis=1) + 1e-9)


def test_point_group_and_symmetric_crystal():
    """The fcc point group in lattice coordinates has 48 operations and is closed; the
    symmetrised Al-like crystal has eps(K k) = eps(k) and omega(K q) = omega(q) on a grid for
    every k-space operation K = M^-T, while the crystal before symmetrisation does not (so the
    check can fail)."""
    from oracle import epwi_oracle as O
    lat = synth.fcc_cell(4.05)[0]
    ops = synth.point_group(lat)
    assert len(ops) == 48
    keys = {tuple(M.ravel()) for M in ops}
    assert all(tuple((A @ B).ravel()) in keys for A in ops for B in ops)
    K = synth.kpoint_ops(ops)
    N = 6
    idx = O.grid_indices((N, N, N))

    def worst(sysm):
        gr = O.Grids(sysm, (N, N, N))
        e = 0.0
        for k in K:
            j = O.flat_index((idx @ k.T) % N, (N, N, N))
            e = max(e, np.abs(gr.eps[j] - gr.eps).max(), np.abs(gr.hw[j] - gr.hw).max())
        return e
    assert worst(synth.al_like_sym_system()) < 1e-12
    assert worst(synth.al_like_ws_system()) > 1e-3
