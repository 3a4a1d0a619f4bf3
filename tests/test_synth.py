"""The seeded input generator: the chunked, threaded draw of large complex-normal arrays gives
exactly the values of the sequential SplitMix64 + Box-Muller stream."""
import numpy as np

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
