"""The short-latency reciprocal and reciprocal square root of the small factorisations (an FP32
estimate refined by two Newton-Raphson steps in FP64) against CUDA's correctly rounded 1/x and
1/sqrt(x), over the whole normal range, both signs (reciprocal), and the edge cases that take
the IEEE path (zero, subnormal, huge, infinite)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_fast_rcp_and_rsqrt_within_a_few_ulp(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    g = np.random.default_rng(0)
    mant = g.uniform(1.0, 2.0, 200000)
    expo = g.integers(-1018, 1019, 200000)
    x = np.ldexp(mant, expo)
    x = np.concatenate([x, -x[:50000], [1.0, 2.0, 0.5, 3.0, 1e-300, 1e300, np.nextafter(2.0, 0.0)]])
    xd = torch.from_numpy(x).cuda()
    rcp, rsq = P.rhosvd_selftest_fastmath(xd)
    ref_rcp = (1.0 / xd).cpu().numpy()
    rcp = rcp.cpu().numpy()
    ulp = np.spacing(np.abs(ref_rcp))
    assert np.max(np.abs(rcp - ref_rcp) / ulp) <= 4
    pos = x > 0
    ref_rsq = torch.rsqrt(xd[torch.from_numpy(pos).cuda()]).cpu().numpy()
    rsq = rsq.cpu().numpy()[pos]
    assert np.max(np.abs(rsq - ref_rsq) / np.spacing(ref_rsq)) <= 4


def test_fast_helpers_edge_cases_take_the_ieee_path(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    x = np.array([0.0, -0.0, 5e-324, 2.2250738585072014e-308, 1.7976931348623157e308, np.inf, -np.inf, 4.0])
    rcp, rsq = P.rhosvd_selftest_fastmath(torch.from_numpy(x).cuda())
    rcp = rcp.cpu().numpy()
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ref = 1.0 / x
    assert np.array_equal(np.isinf(rcp), np.isinf(ref)) and np.allclose(rcp[np.isfinite(ref)], ref[np.isfinite(ref)],
                                                                         rtol=4e-16, atol=0)
    assert rsq.cpu().numpy()[-1] == 0.5
