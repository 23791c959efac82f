"""GPU parity of the mixed-precision form (tcgen05 tensor cores with exact 8-bit digit planes)
against the CPU oracle, with the plain-form tolerances, and against the plain FP64 GPU form.

The mixed form reproduces FP64 products to about 2^-40 of sum |a||b| (2^-31 for the core
contraction), so it must meet every plain-form bar: Tucker <= 1e-6 vs the oracle, equal
ranks (+-1 only at a tie), the sigma bound, tau_gpu >= tau_oracle and tau^2 <= eps^2 total.
Against the plain GPU form (same sketch) the Tucker tensors agree to 1e-7 (core digits: 2^-31)."""
import numpy as np
import pytest

import oracle
import workloads
from tests import tensor_utils as tu
from tests.test_gpu_parity import check_case, run_gpu

pytestmark = pytest.mark.gpu
MIXED = 1


def test_mixed_gauss_n128_R200_direct(rhosvd_cuda):
    cp = workloads.gaussian_sum(128, 200, 0)
    g, o, d = check_case(rhosvd_cuda, cp.U, cp.xi, 1e-6, r_max=128, precision=MIXED)
    assert g["ranks"] == o["ranks"] and d < 1e-7


def test_mixed_sketch_ragged(rhosvd_cuda):
    cp = workloads.gaussian_sum(300, 700, 3)
    g, o, d = check_case(rhosvd_cuda, cp.U, cp.xi, 1e-6, r_max=128, oversample=32, precision=MIXED)
    assert g["info"].direct[0] == 0 and d is not None


def test_mixed_hadamard_then_reduce(rhosvd_cuda):
    A = workloads.gaussian_sum(256, 24, 0)
    B = workloads.gaussian_sum(256, 20, 1)
    Uo, xo = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    check_case(rhosvd_cuda, Uo, xo, 1e-7, r_max=160, oversample=32, precision=MIXED)


def test_mixed_newton_long_range(rhosvd_cuda):
    cp = workloads.newton_long_range_sum(n=320, N=40, seed=0)
    check_case(rhosvd_cuda, cp.U, cp.xi, 1e-6, r_max=64, oversample=32, precision=MIXED)


def test_mixed_fixed_ranks_and_edges(rhosvd_cuda):
    cp = workloads.gaussian_sum(200, 300, 9)
    g, o, d = check_case(rhosvd_cuda, cp.U, cp.xi, 1e-6, r_max=64, oversample=96, ranks=(5, 12, 30),
                         precision=MIXED)
    assert g["ranks"] == [5, 12, 30]
    g0 = np.random.default_rng(11)
    U = [g0.standard_normal((n, 1)) for n in (70, 300, 5)]
    g, o, d = check_case(rhosvd_cuda, U, np.array([2.5]), 1e-12, r_max=8, precision=MIXED)
    assert g["ranks"] == [1, 1, 1]


@pytest.mark.parametrize("case", ["gauss", "hadamard"])
def test_mixed_matches_plain_gpu(rhosvd_cuda, case):
    """Same input, same sketch seed: the two GPU forms agree on ranks and Tucker tensors.  Their
    tails are each an exact measurement of ||U - Z V|| for their own sketch; the pivoted
    CholeskyQR may keep one column more or less in one form, so the tails are checked against
    the optimum (the oracle's SVD tail at that rank) and the eps rule, not against each other."""
    if case == "gauss":
        cp = workloads.gaussian_sum(400, 500, 14)
        U, xi, eps, rmax = cp.U, cp.xi, 1e-6, 128
    else:
        A = workloads.gaussian_sum(320, 30, 2)
        B = workloads.gaussian_sum(320, 28, 3)
        U, xi = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
        eps, rmax = 1e-7, 192
    a = run_gpu(rhosvd_cuda, U, xi, eps, r_max=rmax, seed=5, precision=0)
    b = run_gpu(rhosvd_cuda, U, xi, eps, r_max=rmax, seed=5, precision=MIXED)
    assert a["info"].status == 0 and b["info"].status == 0
    assert a["ranks"] == b["ranks"]
    assert tu.tucker_rel_diff(b["beta"], b["Z"], a["beta"], a["Z"]) < 1e-7
    o = oracle.c2t(U, xi, eps=eps, ranks=tuple(a["ranks"]))
    for g in (a, b):
        for l in range(3):
            total = g["info"].total[l]
            assert g["info"].tail[l] >= o["tails"][l] * (1 - 1e-9) - 1e-13 * total ** 0.5
            assert g["info"].tail[l] ** 2 <= eps * eps * total * (1 + 1e-9)


def test_mixed_rank_one_exact(rhosvd_cuda):
    """One canonical term: the normalised side matrices are single unit columns, so sigma_1 = 1
    and V = Z^T U = +-1 exactly, and nothing lies outside Z.  In the mixed form every one of
    these passes through digit-plane products of one-signed data over K = n, the case where
    inexact FP32 accumulation would lose bits in proportion to K."""
    P = rhosvd_cuda
    g0 = np.random.default_rng(11)
    U = [np.abs(g0.standard_normal((n, 1))) + 0.1 for n in (70, 300, 5)]
    g = run_gpu(P, U, np.array([2.5]), 1e-12, r_max=8, precision=MIXED)
    assert g["info"].status == 0, P.rhosvd_strerror(g["info"].status)
    assert g["ranks"] == [1, 1, 1]
    for l in range(3):
        assert abs(g["sigma"][l][0] - 1.0) <= 1e-13, (l, g["sigma"][l][0])
        assert abs(abs(g["V"][l][0, 0]) - 1.0) <= 1e-13, (l, g["V"][l][0, 0])
        assert g["info"].resid[l] <= 1e-26, (l, g["info"].resid[l])
        u = U[l][:, 0] / np.linalg.norm(U[l][:, 0])
        assert abs(abs(g["Z"][l][:, 0] @ u) - 1.0) <= 1e-14
