"""Pins of the CPU oracle to things other than itself: LAPACK, closed forms, hand-worked
rank rules, brute force on the full tensor, and the paper's bounds (Thm. 2.3, Cor. 2.4)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads
from tests import tensor_utils as tu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- building blocks

def test_col_norm_exact_and_scaled():
    assert oracle.col_norm(np.array([3.0, 4.0])) == 5.0
    t = 2.0 ** -1060                      # subnormal range: squares would underflow
    assert oracle.col_norm(np.array([3 * t, 4 * t])) == 5 * t
    big = np.array([3e200, 4e200])        # squares would overflow
    assert abs(oracle.col_norm(big) / 5e200 - 1) < 1e-15
    assert oracle.col_norm(np.zeros(7)) == 0.0


@pytest.mark.parametrize("m,n,grade", [(40, 40, 0), (60, 25, 0), (33, 33, 12), (80, 17, 8), (1, 1, 0)])
def test_jacobi_matches_lapack(m, n, grade):
    g = np.random.default_rng(m * 100 + n)
    A = g.standard_normal((m, n))
    if grade:                              # graded columns: singular values over `grade` decades
        A = A * np.logspace(0, -grade, n)[None, :]
    sig, Z = oracle.jacobi_left(A)
    s_ref = np.linalg.svd(A, compute_uv=False)
    big = s_ref > 1e-9 * s_ref[0]
    assert np.all(np.abs(sig[big] - s_ref[big]) <= 1e-12 * s_ref[big] + 1e-15 * s_ref[0])
    assert np.all(np.diff(sig) <= 0)
    # orthonormal left vectors and A^T z_i = sigma_i v_i (row norms of Z^T A are sigma)
    q = int(big.sum())
    assert np.allclose(Z[:, :q].T @ Z[:, :q], np.eye(q), atol=1e-12)
    assert np.allclose(np.linalg.norm(Z[:, :q].T @ A, axis=1), sig[:q], rtol=1e-11, atol=1e-14 * sig[0])


def test_jacobi_rank_deficient_resolvable_part():
    """Numerically zero columns (norm <= m u ||A||_F) are left alone; the resolvable singular
    values still match LAPACK and the rest stay at the noise level."""
    g = np.random.default_rng(17)
    A = (g.standard_normal((100, 15)) * np.logspace(0, -6, 15)) @ g.standard_normal((15, 40))
    sig, Z = oracle.jacobi_left(A)
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(sig[:15], s_ref[:15], rtol=1e-10)
    assert np.all(sig[15:] <= 1e-13 * sig[0])
    assert np.allclose(Z[:, :15].T @ Z[:, :15], np.eye(15), atol=1e-11)


def test_householder_r_factor():
    g = np.random.default_rng(7)
    A = g.standard_normal((50, 20))
    Rf = oracle.householder_r(A)
    assert np.allclose(np.tril(Rf, -1), 0.0)
    assert np.allclose(Rf.T @ Rf, A.T @ A, rtol=1e-13, atol=1e-12)
    Rl = np.linalg.qr(A, mode="r")
    assert np.allclose(np.abs(np.diag(Rf)), np.abs(np.diag(Rl)), rtol=1e-12)


@pytest.mark.parametrize("n,R", [(30, 90), (45, 12), (20, 20)])
def test_side_svd_both_branches(n, R):
    g = np.random.default_rng(n + R)
    U = g.standard_normal((n, R))
    sig, Z = oracle.side_svd(U)
    u, s, _ = np.linalg.svd(U, full_matrices=False)
    assert sig.shape[0] == min(n, R)
    assert np.allclose(sig, s, rtol=1e-12, atol=1e-14 * s[0])
    # same left singular subspaces for each (simple) singular value: |z_i . u_i| = 1
    assert np.allclose(np.abs(np.sum(Z * u, axis=0)), 1.0, atol=1e-9)


def test_eps_rank_golden():
    with open(os.path.join(GOLDEN, "eps_rank_cases.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        assert oracle.eps_rank(np.array(c["sigma"]), c["eps"]) == c["r"], c


def test_normalize_and_drop_zero_terms():
    g = np.random.default_rng(3)
    U = [g.random((9, 6)) + 0.1 for _ in range(3)]
    U[1][:, 2] = 0.0                       # term 2 is the zero tensor
    U[2][:, 4] *= 2.0 ** -1000             # tiny but nonzero column: must be kept
    xi = g.standard_normal(6)
    Un, xin, norms, keep = oracle.normalize(U, xi)
    assert keep.tolist() == [1, 1, 0, 1, 1, 1]
    assert xin[2] == 0.0 and np.all(Un[0][:, 2] == 0) and np.all(Un[2][:, 2] == 0)
    for l in range(3):
        for nu in [0, 1, 3, 4, 5]:
            assert abs(np.linalg.norm(Un[l][:, nu]) - 1.0) < 1e-15
            assert np.allclose(Un[l][:, nu] * norms[l, nu], U[l][:, nu], rtol=1e-15, atol=0)
    for nu in [0, 1, 3, 4, 5]:
        assert math.isclose(xin[nu], xi[nu] * np.prod(norms[:, nu]), rel_tol=1e-15)


# ---------------------------------------------------------------- RHOSVD special cases

def _rel_err_vs_full(out, A):
    T = tu.tucker_full(out["beta"], out["Z"])
    return np.linalg.norm(A - T) / np.linalg.norm(A)


def test_rank_one_exact():
    g = np.random.default_rng(11)
    a, b, c = (g.standard_normal(n) for n in (13, 17, 19))
    xi = np.array([2.5])
    U = [a[:, None], b[:, None], c[:, None]]
    out = oracle.c2t(U, xi, eps=1e-12)
    assert out["ranks"] == [1, 1, 1]
    na, nb, nc = (np.linalg.norm(v) for v in (a, b, c))
    for Zl, v, nv in zip(out["Z"], (a, b, c), (na, nb, nc)):
        assert abs(abs(Zl[:, 0] @ v) / nv - 1.0) < 1e-15
    assert math.isclose(abs(out["beta"][0, 0, 0]), 2.5 * na * nb * nc, rel_tol=1e-14)
    assert _rel_err_vs_full(out, tu.full_from_cp(U, xi)) < 1e-15


def test_separable_exact_low_rank():
    g = np.random.default_rng(5)
    n, R, s = 18, 40, (3, 5, 2)
    U = [g.standard_normal((n, s[l])) @ g.standard_normal((s[l], R)) for l in range(3)]
    xi = g.standard_normal(R)
    out = oracle.c2t(U, xi, eps=1e-10)
    assert out["ranks"] == list(s)
    assert _rel_err_vs_full(out, tu.full_from_cp(U, xi)) < 1e-12


def test_identical_mode_columns_give_rank_one():
    g = np.random.default_rng(9)
    n, R = 16, 30
    col = g.random(n) + 0.1
    U = [np.repeat(col[:, None], R, axis=1), g.random((n, R)), g.random((n, R))]
    xi = g.random(R) + 0.1
    out = oracle.c2t(U, xi, eps=1e-8)
    assert out["ranks"][0] == 1
    assert math.isclose(out["sigma"][0][0], math.sqrt(R), rel_tol=1e-14)
    assert np.all(out["sigma"][0][1:] < 1e-12)


def test_orthonormal_factors_no_truncation():
    g = np.random.default_rng(2)
    n, R = 12, 8
    U = [np.eye(n)[:, g.permutation(n)[:R]] for _ in range(3)]
    xi = g.standard_normal(R)
    out = oracle.c2t(U, xi, eps=1e-12)
    for l in range(3):
        assert np.allclose(out["sigma"][l], 1.0, atol=1e-15)
    assert out["ranks"] == [R, R, R]
    A = tu.full_from_cp(U, xi)
    assert math.isclose(out["xi_norm"], np.linalg.norm(A), rel_tol=1e-14)   # Cor. 2.4(A)
    assert _rel_err_vs_full(out, A) < 1e-14


def _hadamard_matrix(p):
    H = np.array([[1.0]])
    for _ in range(p):
        H = np.block([[H, H], [H, -H]])
    return H


def test_known_spectrum_end_to_end():
    """Relative sigma^2 = 16,9,4,1,.25,.01,1e-6,1e-10,1e-14 (total 30.26...): eps=1e-2 keeps 6
    (tail .010001 > 3.0e-3 at r=5), 1e-4 keeps 7, 1e-6 keeps 8, 1e-9 keeps 9, 0.5 keeps 2.
    U = Z diag(s) V^T with |V_{nu,k}| = 1/sqrt(R) has unit columns when sum s^2 = R, so the
    normalised side matrix has exactly the chosen singular values."""
    g = np.random.default_rng(4)
    n, p = 24, 6
    R = 2 ** p
    s = np.array([4.0, 3.0, 2.0, 1.0, 0.5, 0.1, 1e-3, 1e-5, 1e-7, 0, 0, 0, 0, 0, 0, 0])
    s = s * math.sqrt(R / np.sum(s ** 2))
    q = s.shape[0]
    V = _hadamard_matrix(p)[:, :q] / math.sqrt(R)
    U = []
    for _ in range(3):
        Zq, _ = np.linalg.qr(g.standard_normal((n, q)))
        U.append(Zq @ np.diag(s) @ V.T)
    xi = g.random(R) + 0.5
    for eps, r_exp in [(1e-2, 6), (1e-4, 7), (1e-6, 8), (1e-9, 9), (0.5, 2)]:
        r_hand = oracle.eps_rank(s, eps)
        assert r_hand == r_exp
        out = oracle.c2t(U, xi, eps=eps)
        assert out["ranks"] == [r_exp] * 3, (eps, out["ranks"])
        for l in range(3):
            nz = s > 0
            assert np.allclose(out["sigma"][l][: int(nz.sum())], s[nz], rtol=1e-12)


# ---------------------------------------------------------------- brute force, bounds

def _bruteforce_case(kind, seed):
    n = 20
    if kind == "gauss":
        cp = workloads.gaussian_sum(n, 60, seed, b=3.0, centre_box=1.5, a_range=(0.5, 8.0))
        return cp.U, cp.xi, True
    cp = workloads.random_cp(n, 50, seed)
    return cp.U, cp.xi, False


@pytest.mark.parametrize("kind,seed,eps", [("gauss", 0, 1e-3), ("gauss", 1, 1e-6), ("random", 2, 0.3),
                                           ("random", 3, 0.05)])
def test_bound_pythagoras_and_core_projection(kind, seed, eps):
    U, xi, monotone = _bruteforce_case(kind, seed)
    out = oracle.c2t(U, xi, eps=eps)
    A = tu.full_from_cp(U, xi)
    Z = out["Z"]
    T = tu.tucker_full(out["beta"], Z)
    err = np.linalg.norm(A - T)
    nA = np.linalg.norm(A)
    # Thm. 2.3: ||A - A0|| <= ||xi|| sum_l (sum_{k>r_l} sigma_{l,k}^2)^{1/2}
    bound = out["xi_norm"] * sum(out["tails"])
    assert err <= bound * (1 + 1e-12) + 1e-13 * nA
    # A0 = A x_l Z0 Z0^T is an orthogonal projection: ||A||^2 = ||beta||^2 + ||A - A0||^2
    assert math.isclose(nA ** 2, np.linalg.norm(out["beta"]) ** 2 + err ** 2, rel_tol=1e-11)
    # the core is the projection of the full tensor onto the Z bases (Prop. 2.2)
    core = A
    for l in range(3):
        core = tu.mode_apply(core, Z[l].T, l)
    assert np.allclose(core, out["beta"], rtol=0, atol=1e-12 * nA)
    # the rank rule held in every mode
    for l in range(3):
        s2 = out["sigma"][l] ** 2
        assert np.sum(s2[out["ranks"][l]:]) <= eps ** 2 * np.sum(s2) * (1 + 1e-12)
    if monotone:
        # Cor. 2.4(B): for monotone sums ||xi|| <= ||A||, so the bound holds with ||A||
        assert out["xi_norm"] <= nA * (1 + 1e-12)
        assert err <= nA * sum(out["tails"]) * (1 + 1e-12) + 1e-13 * nA
    # reported, not asserted: RHOSVD vs the HOSVD of the full tensor at the same ranks
    hc, hZ = tu.hosvd(A, out["ranks"])
    herr = np.linalg.norm(A - tu.tucker_full(hc, hZ))
    assert err <= 50 * herr + 1e-12 * nA


def test_tucker_difference_metric_vs_full():
    g = np.random.default_rng(8)
    n, r = 15, 4
    Za = [np.linalg.qr(g.standard_normal((n, r)))[0] for _ in range(3)]
    Zb = [np.linalg.qr(z + 1e-3 * g.standard_normal((n, r)))[0] for z in Za]
    ba, bb = g.standard_normal((r, r, r)), g.standard_normal((r, r, r))
    full = np.linalg.norm(tu.tucker_full(ba, Za) - tu.tucker_full(bb, Zb)) / np.linalg.norm(tu.tucker_full(bb, Zb))
    assert math.isclose(tu.tucker_rel_diff(ba, Za, bb, Zb), full, rel_tol=1e-10)


# ---------------------------------------------------------------- rank-growth operations

def test_hadamard_of_gaussians_closed_form():
    """exp(-a(x-c1)^2) exp(-b(x-c2)^2) = exp(-ab/(a+b) (c1-c2)^2) exp(-(a+b)(x-m)^2),
    m = (a c1 + b c2)/(a+b)  (Lemma 4.2 uses the same identity)."""
    n = 64
    A = workloads.gaussian_sum(n, 5, 21)
    B = workloads.gaussian_sum(n, 4, 22)
    Uc, xc = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    x = workloads.grid(n, 10.0)
    for j in range(4):
        for i in range(5):
            nu = i + 5 * j
            assert math.isclose(xc[nu], A.xi[i] * B.xi[j], rel_tol=1e-15)
            for l in range(3):
                a, b = A.meta["a"][i], B.meta["a"][j]
                c1, c2 = A.meta["centres"][i, l], B.meta["centres"][j, l]
                m = (a * c1 + b * c2) / (a + b)
                ref = math.exp(-a * b / (a + b) * (c1 - c2) ** 2) * np.exp(-(a + b) * (x - m) ** 2)
                got = Uc[l][:, nu]
                mask = ref > 1e-280
                assert np.allclose(got[mask], ref[mask], rtol=1e-12, atol=0)


def test_cp_hadamard_and_sum_full_tensors():
    A = workloads.random_cp(7, 3, 30)
    B = workloads.random_cp(7, 4, 31)
    Uh, xh = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    Fa, Fb = tu.full_from_cp(A.U, A.xi), tu.full_from_cp(B.U, B.xi)
    assert np.allclose(tu.full_from_cp(Uh, xh), Fa * Fb, rtol=1e-12, atol=1e-12)
    Us, xs = oracle.cp_sum(0.5, A.U, A.xi, -2.0, B.U, B.xi)
    assert np.allclose(tu.full_from_cp(Us, xs), 0.5 * Fa - 2.0 * Fb, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- input generators

def test_sinc_newton_quadrature_converges():
    """sum_k p_k exp(-t_k^2 z^2) -> 1/z (eq. Laplace_Newton); the trapezoid rule in
    u = log t has error ~ exp(-pi^2/(2h)), so halving h must shrink the error a lot."""
    z = np.linspace(0.5, 10.0, 200)

    def err(h, klo, khi):
        t, p = workloads.newton_sinc_nodes(h, klo, khi)
        approx = np.sum(p[:, None] * np.exp(-(t[:, None] ** 2) * z[None, :] ** 2), axis=0)
        return np.max(np.abs(approx * z - 1.0))

    e04 = err(0.4, -60, 30)
    e02 = err(0.2, -120, 60)
    assert e04 < 1e-4
    assert e02 < 1e-8 and e02 < e04 * 1e-3


def test_grid_and_gaussian_generator():
    x = workloads.grid(8, 10.0)
    assert np.allclose(x, -10 + (np.arange(8) + 0.5) * 2.5)
    cp = workloads.gaussian_sum(32, 10, 0)
    assert cp.U[0].flags.f_contiguous and cp.U[0].shape == (32, 10)
    nl = workloads.newton_long_range_sum(n=16, N=3, seed=0)
    assert nl.R == 60 and nl.U[2].shape == (16, 60)


# ---------------------------------------------------------------- edge cases

def test_edge_cases_rank_rule():
    cp = workloads.gaussian_sum(24, 30, 4)
    out = oracle.c2t(cp.U, cp.xi, eps=1.0)
    assert out["ranks"] == [0, 0, 0] and out["beta"].size == 0
    out = oracle.c2t(cp.U, cp.xi, eps=1e-3, ranks=(2, 3, 4))
    assert out["ranks"] == [2, 3, 4]
    out = oracle.c2t(cp.U, cp.xi, eps=1e-3, ranks=(100, 1, 1))
    assert out["ranks"][0] == 24
    U = [u.copy() for u in cp.U]
    for u in U:
        u[:] = 0.0
    out = oracle.c2t(U, cp.xi, eps=1e-6)
    assert out["kept"] == 0 and out["ranks"] == [0, 0, 0]
    with pytest.raises(RuntimeError):
        oracle.c2t(cp.U, cp.xi, eps=1e-12, r_max=3)
