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


def test_bit_conversions_match_exact_arithmetic(rhosvd_cuda):
    """The epilogues' conversions built from the bits (no FP64 instruction) against numpy's exact
    ones: rh is x truncated to a float (toward zero) and |rh + rl - x| <= max(2^-48 |x|, 2^-120) on
    FP32's normal range (both zero below it); f 2^e exactly as a double wherever the result is a normal double,
    FP32 subnormals included; 2^e as a float (subnormal from 2^-149, zero below, infinity above)."""
    P = rhosvd_cuda
    import torch
    g = np.random.default_rng(11)
    n = 400000
    x = np.ldexp(g.uniform(1.0, 2.0, n), g.integers(-140, 128, n)) * g.choice([-1.0, 1.0], n)
    x[:10] = [0.0, -0.0, 1.0, -1.0, 2.0 ** -126, 2.0 ** -127, 1.5, np.nextafter(2.0, 0.0), 3.0, 2.0 ** -149]
    f = (np.ldexp(g.uniform(1.0, 2.0, n), g.integers(-149, 128, n)) * g.choice([-1.0, 1.0], n)).astype(np.float32)
    f[:6] = np.array([0.0, -0.0, 1e-45, -3e-40, 1.0, 3.4e38], dtype=np.float32)
    e = g.integers(-300, 300, n).astype(np.int32)
    e[:6] = [0, 5, 100, -20, -1200, 3]
    rh, rl, fd, p2 = P.rhosvd_selftest_bits(torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda(),
                                            torch.from_numpy(e).cuda())
    rh, rl, fd, p2 = rh.cpu().numpy(), rl.cpu().numpy(), fd.cpu().numpy(), p2.cpu().numpy()
    # split
    big = np.abs(x) >= 2.0 ** -126
    E = np.frexp(np.where(big, np.abs(x), 1.0))[1] - 1                # |x| in [2^E, 2^(E+1))
    rh_ref = np.copysign(np.ldexp(np.trunc(np.ldexp(np.abs(x), 23 - E)), E - 23), x)
    assert np.array_equal(rh[big].astype(np.float64), rh_ref[big])
    err = np.abs(rh[big].astype(np.float64) + rl[big].astype(np.float64) - x[big])
    # (below 2^-97 the rest underflows FP32's range: an absolute error under 2^-120 there)
    assert np.all(err <= np.maximum(2.0 ** -48 * np.abs(x[big]), 2.0 ** -120))
    assert np.all(rh[~big] == 0.0) and np.all(rl[~big] == 0.0)
    # f 2^e
    ref = np.ldexp(f.astype(np.float64), e)
    normal = (np.abs(ref) >= 2.0 ** -1022) & np.isfinite(ref)
    assert np.array_equal(fd[normal], ref[normal])
    assert np.all(fd[(f == 0)] == 0.0)
    # 2^e as a float
    with np.errstate(over="ignore"):
        p2_ref = np.ldexp(np.float32(1.0), e).astype(np.float32)
    assert np.array_equal(p2, p2_ref)
