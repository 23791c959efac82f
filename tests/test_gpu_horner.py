"""GPU parity of the Horner-scheme polynomial of a canonical tensor (rhosvd_cp_horner) and of the
direct cube P (.) P (.) P (two rhosvd_cp_hadamard calls and one C2C), against the CPU oracle
(oracle/horner.py) and against the polynomial evaluated entry by entry on the full tensor.

Tolerances.  Each reduction (RHOSVD with eps_t, then T2C with eps_c) changes its input X_k by at
most 4 (eps_t + eps_c) ||X_k||_F on these positive-weight inputs (the oracle pins hold the same
bar), and Y_0 - P(A) = sum_k A^k (.) E_k, so ||Y_0 - P(A)||_F <= sum_k max|A|^k 4 (eps_t + eps_c)
||X_k||_F, with X_k the exact partial polynomials; the GPU and the oracle each meet it, hence differ
by at most twice that.  Tucker ranks per step: equal, or one apart at a threshold tie."""
import numpy as np
import pytest

import workloads
from oracle import horner as oh
from oracle import t2c as ot
from numpy.polynomial import polynomial as npoly

pytestmark = pytest.mark.gpu


def _dev(P, U, xi):
    import torch
    return [P.to_device_factor(u) for u in U], torch.from_numpy(np.ascontiguousarray(xi)).cuda()


def _full_gpu(res):
    R = res.R
    return ot.full_from_cp([res.U[l][:, :R].cpu().numpy() for l in range(3)], res.xi[:R].cpu().numpy())


def _bound(A, coeffs, eps_t, eps_c):
    c = np.asarray(coeffs, dtype=np.float64)
    n = oh.degree(c)
    amax = np.abs(A).max()
    Y = c[n] * np.ones_like(A)
    b = 0.0
    for k in range(n - 1, -1, -1):
        Y = A * Y + c[k]
        b += amax ** k * 4 * (eps_t + eps_c) * np.linalg.norm(Y)
    return b


def _ranks_close(gs, os_):
    assert len(gs) == len(os_)
    for g, o in zip(gs, os_):
        assert g["k"] == o["k"] and g["status"] == 0
        assert all(abs(a - b) <= 1 for a, b in zip(g["r"], o["ranks"])), (g, o)


@pytest.mark.parametrize("coeffs,eps", [([0.5, -1.0, 2.0, 0.3], 1e-8), ([0, 0, 0, 1], 1e-6),
                                        ([1.0, 0.0, -0.5, 0.0, 0.25], 1e-7), ([3.0, 2.0], 1e-10)])
def test_horner_matches_polynomial_and_oracle(rhosvd_cuda, coeffs, eps):
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(24, 5, 3, b=3.0, centre_box=1.5, a_range=(0.3, 2.0))
    A = ot.full_from_cp(cp.U, cp.xi)
    eps_t, eps_c = eps, eps / 10
    U, x = _dev(P, cp.U, cp.xi)
    res = P.rhosvd_cp_horner(U, x, coeffs, eps_t, eps_c, R_max=600, r_max=24)
    ref = npoly.polyval(A, np.asarray(coeffs, dtype=np.float64))
    bnd = _bound(A, coeffs, eps_t, eps_c)
    Yg = _full_gpu(res)
    o = oh.horner(cp.U, cp.xi, coeffs, eps_t, eps_c)
    Yo = ot.full_from_cp(o["U"], o["xi"])
    tiny = 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(Yg - ref) <= bnd + tiny
    assert np.linalg.norm(Yo - ref) <= bnd + tiny
    assert np.linalg.norm(Yg - Yo) <= 2 * bnd + tiny
    _ranks_close(res.steps, o["steps"])
    assert len(res.steps) == oh.degree(coeffs)


def test_horner_exact_and_degenerate(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    cp = workloads.gaussian_sum(16, 3, 4, b=3.0, centre_box=1.5, a_range=(0.3, 2.0))
    A = ot.full_from_cp(cp.U, cp.xi)
    U, x = _dev(P, cp.U, cp.xi)
    c = [0.25, -0.5, 1.5]
    res = P.rhosvd_cp_horner(U, x, c, 0.0, 0.0, R_max=400, r_max=16)
    ref = npoly.polyval(A, c)
    assert np.abs(_full_gpu(res) - ref).max() <= 1e-11 * np.abs(ref).max()
    z = P.rhosvd_cp_horner(U, x, [0.0, 0.0, 0.0], 1e-6, 1e-6, R_max=4)
    assert z.R == 0 and z.steps == []
    k = P.rhosvd_cp_horner(U, x, [2.5, 0.0], 1e-6, 1e-6, R_max=4)
    assert k.R == 1 and float(k.xi[0]) == 2.5
    assert all(bool(torch.all(k.U[l][:, 0] == 1.0)) for l in range(3))
    # a zero reference tensor: P(0) = a_0
    U0 = [torch.zeros_like(u) for u in U]
    y = P.rhosvd_cp_horner(U0, x, [1.5, 2.0, 3.0], 1e-8, 1e-8, R_max=32, r_max=16)
    assert np.abs(_full_gpu(y) - 1.5).max() <= 1e-14


def test_horner_rank_overflow_is_reported(rhosvd_cuda):
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(24, 6, 5, b=3.0, centre_box=1.5, a_range=(0.3, 2.0))
    U, x = _dev(P, cp.U, cp.xi)
    with pytest.raises(P.RhosvdError) as e:
        P.rhosvd_cp_horner(U, x, [0.1, 0.2, 0.3, 0.4], 1e-10, 1e-10, R_max=8, r_max=24)
    assert e.value.code == P.RHOSVD_ERR_RANK_OVERFLOW
    assert e.value.steps and e.value.steps[-1]["status"] == P.RHOSVD_ERR_RANK_OVERFLOW


@pytest.mark.parametrize("long_range", [False, True])
def test_newton_cube_full_size(rhosvd_cuda, long_range):
    """P^(3) = P (.) P (.) P of the sinc Newton kernel at n = 257, eps = 1e-5 (Sec. 5): directly (rank
    19^3 = 6859, or 10^3 for the long-range part) and by the Horner scheme; the error measured on
    the full 257^3 tensor, the ranks against the oracle's."""
    P = rhosvd_cuda
    import torch
    cp = workloads.newton_kernel(long_range=long_range)
    eps_t = eps_c = 1e-5
    U, x = _dev(P, cp.U, cp.xi)
    U2, x2 = P.rhosvd_cp_hadamard(U, x, U, x)
    U3, x3 = P.rhosvd_cp_hadamard(U2, x2, U, x)
    can, tk = P.rhosvd_c2c(U3, x3, eps_t, eps_c, R_max=2000, r_max=64)
    R, st = can.rank()
    assert st == 0 and tk.info().status == 0
    od = oh.power_direct(cp.U, cp.xi, 3, eps_t, eps_c)
    info = tk.info()
    assert all(abs(info.r[l] - od["tucker"]["ranks"][l]) <= 1 for l in range(3))
    assert abs(R - od["R"]) <= max(3, od["R"] // 20)
    Ad = [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in cp.U]
    xd = torch.from_numpy(cp.xi).cuda()
    full = torch.einsum("k,ik,jk,mk->ijm", xd, *Ad)
    cube = full ** 3
    Yd = torch.einsum("k,ik,jk,mk->ijm", can.xi[:R], *[can.U[l][:, :R] for l in range(3)])
    nrm = float(torch.linalg.norm(cube))
    assert float(torch.linalg.norm(Yd - cube)) <= 4 * (eps_t + eps_c) * nrm
    h = P.rhosvd_cp_horner(U, x, [0, 0, 0, 1], eps_t, eps_c, R_max=2000, r_max=64)
    Yh = torch.einsum("k,ik,jk,mk->ijm", h.xi[: h.R], *[h.U[l][:, : h.R] for l in range(3)])
    amax = float(full.abs().max())
    bnd = 4 * (eps_t + eps_c) * (amax ** 2 * float(torch.linalg.norm(full)) + amax * float(torch.linalg.norm(full ** 2))
                                  + nrm)
    assert float(torch.linalg.norm(Yh - cube)) <= bnd
    oh_ = oh.horner(cp.U, cp.xi, [0, 0, 0, 1], eps_t, eps_c)
    _ranks_close(h.steps, oh_["steps"])


@pytest.mark.parametrize("coeffs", [[0.5, -1.0, 2.0], [0.0, 0.0, 1.0]])
def test_horner_exact_with_rank_deficient_cores(rhosvd_cuda, coeffs):
    """n = 20 with every Tucker rank at n after the second product: the cores carry singular values
    at rounding level, which T2C must treat as zero (else its re-orthonormalised left vectors are
    noise and the C2C is off by O(1))."""
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(20, 4, 2, b=3.0, centre_box=1.5, a_range=(0.3, 2.0))
    U, x = _dev(P, cp.U, cp.xi)
    res = P.rhosvd_cp_horner(U, x, coeffs, 0.0, 0.0, R_max=400, r_max=20)
    ref = npoly.polyval(ot.full_from_cp(cp.U, cp.xi), np.asarray(coeffs, dtype=np.float64))
    assert np.abs(_full_gpu(res) - ref).max() <= 1e-12 * np.abs(ref).max()
