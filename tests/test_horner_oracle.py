"""Pins of the Horner-polynomial oracle (oracle/horner.py) against things other than itself: the
polynomial evaluated entry by entry on the full tensor (numpy's polyval), the closed-form rank of a
polynomial of a rank-one tensor, the per-step reduction errors measured on full tensors (with the
true coefficient a_k of each Horner step), and the direct cube P (.) P (.) P of Sec. 5."""
import numpy as np
import pytest

import workloads
from oracle import horner as oh
from oracle import t2c as ot
from numpy.polynomial import polynomial as npoly


def _small(n=8, R=3, seed=0):
    cp = workloads.gaussian_sum(n, R, seed, b=3.0, centre_box=1.5, a_range=(0.3, 2.0))
    return cp.U, cp.xi


@pytest.mark.parametrize("coeffs", [[0.5, -1.0, 2.0], [0, 0, 0, 1], [1.0, 0.0, -0.5, 0.0, 0.25], [3.0, 2.0],
                                    [0.0, 1.0, 0.0]])
def test_exact_reductions_give_the_polynomial(coeffs):
    U, xi = _small()
    A = ot.full_from_cp(U, xi)
    res = oh.horner(U, xi, coeffs, 0.0, 0.0)
    Y = ot.full_from_cp(res["U"], res["xi"])
    ref = npoly.polyval(A, np.asarray(coeffs, dtype=np.float64))
    assert np.abs(Y - ref).max() <= 1e-11 * max(np.abs(ref).max(), 1.0)
    assert len(res["steps"]) == oh.degree(coeffs)


def test_degenerate_polynomials():
    U, xi = _small()
    z = oh.horner(U, xi, [0.0, 0.0], 1e-6, 1e-6)
    assert z["R"] == 0 and z["steps"] == []
    c = oh.horner(U, xi, [2.5, 0.0, 0.0], 1e-6, 1e-6)
    assert c["R"] == 1 and c["xi"][0] == 2.5 and all(np.all(u == 1.0) for u in c["U"])


def test_rank_one_reference_tensor():
    # A = u (x) v (x) w: Y_k is a polynomial of degree n - k in A, sum_m c_m u^m (x) v^m (x) w^m
    # (powers entrywise), so every mode of it lies in span{1, u, .., u^(n-k)}: Tucker rank n-k+1,
    # and T2C's canonical rank is at most r3 min(r1, r2)
    g = np.random.default_rng(3)
    U = [np.asfortranarray(g.uniform(0.2, 1.0, (10, 1))) for _ in range(3)]
    xi = np.array([1.3])
    coeffs = [0.7, -0.4, 1.1, 0.3]
    res = oh.horner(U, xi, coeffs, 1e-12, 1e-12)
    n = len(coeffs) - 1
    for st in res["steps"]:
        assert st["ranks"] == [n - st["k"] + 1] * 3, st
        assert st["R"] <= (n - st["k"] + 1) ** 2
    A = ot.full_from_cp(U, xi)
    assert np.abs(ot.full_from_cp(res["U"], res["xi"]) - npoly.polyval(A, coeffs)).max() <= 1e-10


def test_steps_are_faithful_reductions():
    # E_k = Y_k - (A (.) Y_{k+1} + a_k I) on full tensors, with a_k taken from the polynomial: each
    # is a small relative error, and Y_0 - P(A) = sum_k A^k (.) E_k bounds the result.
    U, xi = _small(n=12, R=4, seed=1)
    A = ot.full_from_cp(U, xi)
    coeffs = [0.3, 1.0, -0.8, 0.5]
    eps_t, eps_c = 1e-5, 1e-6
    res = oh.horner(U, xi, coeffs, eps_t, eps_c, keep_steps=True)
    amax = np.abs(A).max()
    Yprev = coeffs[-1] * np.ones_like(A)
    bound = 0.0
    for st in res["steps"]:
        k = st["k"]
        Xk = A * Yprev + coeffs[k]
        Yk = ot.full_from_cp(st["U"], st["xi"])
        Ek = np.linalg.norm(Yk - Xk)
        assert Ek <= 4 * (eps_t + eps_c) * np.linalg.norm(Xk), (k, Ek)
        bound += amax ** k * Ek
        Yprev = Yk
    err = np.linalg.norm(ot.full_from_cp(res["U"], res["xi"]) - npoly.polyval(A, coeffs))
    assert err <= bound * (1 + 1e-9) + 1e-13 * np.linalg.norm(A)
    assert [st["k"] for st in res["steps"]] == [2, 1, 0]


def test_cube_direct_and_by_horner():
    cp = workloads.newton_kernel(n=17, b=4.0, M=3, h=0.8)
    A = ot.full_from_cp(cp.U, cp.xi)
    ref = A ** 3
    eps_t, eps_c = 1e-7, 1e-8
    d = oh.power_direct(cp.U, cp.xi, 3, eps_t, eps_c)
    assert d["R_in"] == cp.R ** 3
    h = oh.horner(cp.U, cp.xi, [0, 0, 0, 1], eps_t, eps_c)
    for Y in (ot.full_from_cp(d["U_can"], d["xi_can"]), ot.full_from_cp(h["U"], h["xi"])):
        assert np.linalg.norm(Y - ref) <= 1e-5 * np.linalg.norm(ref)
