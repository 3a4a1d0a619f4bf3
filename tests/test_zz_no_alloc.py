"""The allocation-free conductivity entry point (for callers that cannot call cudaMalloc:
a framework owning all device memory through its own pool, or a service that must not
allocate after start-up) against the regular epwi_conductivity, on two calls in a row.

Collected last on purpose (file name), so a run that stops at the first failure has already
run every other test."""
import numpy as np
import pytest

from oracle import epwi_oracle as O
from paper_2306_16493_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_conductivity_noalloc_matches_context_path():
    torch = pytest.importorskip("torch")
    from paper_2306_16493_gb300 import epwi
    s = synth.al_like_system()
    N, T, eta = 12, 300.0, 0.02
    ctx = epwi.Context()
    ctx.setup(s)
    ctx.eigs(N)
    lo, hi = ctx.band_range()
    mu = 0.5 * (lo + hi)
    ns, _ = ctx.scatter_rates(T, mu, eta, mu - 0.3, mu + 0.3)
    assert ns > 0
    sigma_ref = ctx.conductivity()
    k, b, r = ctx.rates()
    eps, _, vel = ctx.bands()
    dev = torch.device("cuda", 0)
    eps_s = torch.tensor(eps[k, b], dtype=torch.float64, device=dev)
    vel_s = torch.tensor(np.ascontiguousarray(vel[k, b]), dtype=torch.float64, device=dev)
    rate_s = torch.tensor(r, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):                      # two calls in a row share the scratch array
        out = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
        epwi.epwi_conductivity_noalloc(ns, eps_s.data_ptr(), vel_s.data_ptr(), rate_s.data_ptr(),
                                       mu, T, s.volume, N ** 3, stream.cuda_stream, out.data_ptr())
        stream.synchronize()
        sig = out.cpu().numpy().reshape(3, 3)
        assert np.linalg.norm(sig - sigma_ref) <= TOL * np.linalg.norm(sigma_ref)
    with pytest.raises(epwi.EpwiError) as e:   # beyond the scratch capacity
        epwi.epwi_conductivity_noalloc(4096 * 1024 + 1, eps_s.data_ptr(), vel_s.data_ptr(),
                                       rate_s.data_ptr(), mu, T, s.volume, N ** 3,
                                       stream.cuda_stream, out.data_ptr())
    assert e.value.status == 8
    ctx.close()
