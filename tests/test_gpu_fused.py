"""The fused Hadamard-product reduction (rhosvd_c2t_hadamard) against the stored product
(rhosvd_cp_hadamard, then rhosvd_c2t) and against the CPU oracle.

The fused path forms column nu = i + Ra j of the product as a_i .* b_j (one FP64 multiply an
entry) and its weight as xa_i xb_j, exactly the values rhosvd_cp_hadamard stores, and everything
after the normalisation is the same code on the same numbers: the outputs are bit-identical.
Against the oracle (RHOSVD of the oracle's stored product) the plain-form tolerances of the
parity tests hold."""
import numpy as np
import pytest

import oracle
import workloads
from tests import tensor_utils as tu

pytestmark = pytest.mark.gpu


def _dev(P, cp, ld_pad=0):
    import torch
    U = []
    for u in cp.U:
        n, R = u.shape
        buf = torch.zeros(R, n + ld_pad, dtype=torch.float64, device="cuda")
        buf[:, :n] = torch.from_numpy(np.ascontiguousarray(u.T)).cuda()
        U.append(buf.t()[:n])
    return U, torch.from_numpy(np.ascontiguousarray(cp.xi)).cuda()


def _same(P, a, b):
    import torch
    ia, ib = a.info(), b.info()
    for f in ("status", "kept"):
        assert getattr(ia, f) == getattr(ib, f), f
    for f in ("r", "k", "direct"):
        assert list(getattr(ia, f)) == list(getattr(ib, f)), f
    for f in ("xi_norm",):
        assert getattr(ia, f) == getattr(ib, f)
    for f in ("total", "resid", "tail"):
        assert list(getattr(ia, f)) == list(getattr(ib, f)), f
    r = list(ia.r)
    assert torch.equal(a.beta[: r[0] * r[1] * r[2]], b.beta[: r[0] * r[1] * r[2]])
    for l in range(3):
        assert torch.equal(a.Z[l], b.Z[l])
    assert torch.equal(a.sigma, b.sigma)
    if a.V is not None:
        for l in range(3):
            assert torch.equal(a.V[l][: r[l]], b.V[l][: r[l]])
    if a.xi_out is not None:
        assert torch.equal(a.xi_out, b.xi_out)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,Ra,Rb,eps,ld_pad", [(200, 12, 10, 1e-8, 0), (96, 7, 1, 1e-6, 3), (300, 20, 25, 1e-7, 0)])
def test_fused_is_bit_identical(rhosvd_cuda, prec, n, Ra, Rb, eps, ld_pad):
    P = rhosvd_cuda
    A = workloads.gaussian_sum(n, Ra, 11)
    B = workloads.gaussian_sum(n, Rb, 12)
    Ua, xa = _dev(P, A, ld_pad)
    Ub, xb = _dev(P, B)
    kw = dict(eps=eps, r_max=64, oversample=32, seed=77, precision=prec, with_V=True, with_xi=True)
    f = P.rhosvd_c2t_hadamard(Ua, xa, Ub, xb, **kw)
    Uc, xc = P.rhosvd_cp_hadamard(Ua, xa, Ub, xb)
    s = P.rhosvd_c2t(Uc, xc, **kw)
    _same(P, f, s)


def test_fused_full_size_bit_identical(rhosvd_cuda):
    """The hadamard_n1024_R64x64 workload at eps = 1e-7 in the mixed form, r_max 160."""
    P = rhosvd_cuda
    A, B = workloads.hartree_like_factors(1024, 64, 64, (0, 1))
    Ua, xa = _dev(P, A)
    Ub, xb = _dev(P, B)
    kw = dict(eps=1e-7, r_max=160, oversample=32, seed=12345, precision=1)
    f = P.rhosvd_c2t_hadamard(Ua, xa, Ub, xb, **kw)
    Uc, xc = P.rhosvd_cp_hadamard(Ua, xa, Ub, xb)
    s = P.rhosvd_c2t(Uc, xc, **kw)
    _same(P, f, s)


def test_fused_against_oracle(rhosvd_cuda):
    P = rhosvd_cuda
    A = workloads.gaussian_sum(64, 9, 21)
    B = workloads.gaussian_sum(64, 8, 22)
    Ua, xa = _dev(P, A)
    Ub, xb = _dev(P, B)
    g = P.rhosvd_c2t_hadamard(Ua, xa, Ub, xb, eps=1e-8, r_max=64)
    info = g.info()
    r = [info.r[l] for l in range(3)]
    Uo, xo = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    o = oracle.c2t(Uo, xo, eps=1e-8)
    beta = g.beta[: r[0] * r[1] * r[2]].cpu().numpy().reshape(r, order="F")
    Z = [g.Z[l][:, : r[l]].cpu().numpy() for l in range(3)]
    assert info.status == 0
    assert all(abs(r[l] - o["ranks"][l]) <= 1 for l in range(3))
    assert tu.tucker_rel_diff(beta, Z, o["beta"], o["Z"]) <= 1e-6


def test_fused_empty_factor(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    A = workloads.gaussian_sum(40, 5, 1)
    Ua, xa = _dev(P, A)
    Ue = [torch.zeros(40, 0, dtype=torch.float64, device="cuda") for _ in range(3)]
    g = P.rhosvd_c2t_hadamard(Ua, xa, Ue, torch.zeros(0, dtype=torch.float64, device="cuda"), eps=1e-6, r_max=8)
    info = g.info()
    assert info.status == 0 and list(info.r) == [0, 0, 0]
