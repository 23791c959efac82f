"""Pins of the C2T-ALS oracle (oracle/als.py) against things other than itself: the unfolding
built from the canonical factors equals the unfolding of the full tensor contracted with the
factors (einsum on the full tensor: pins index order and transposition), a sweep equals HOOI
run on the full tensor's unfoldings with LAPACK SVDs, the captured energy never decreases and
the Tucker error never increases (full tensors), an exact Tucker-rank tensor is reproduced, and
||A||^2 = ||beta||^2 + ||A - A_r||^2 (Pythagoras for an orthogonal projection)."""
import numpy as np

import oracle
import workloads
from oracle import als as oa
from tests import tensor_utils as tu


def _tucker(beta, Z):
    return np.einsum("abc,ia,jb,mc->ijm", beta, *Z)


def test_unfolding_is_the_full_contraction():
    cp = workloads.gaussian_sum(14, 30, 1)
    A = tu.full_from_cp(cp.U, cp.xi)
    tk = oracle.c2t(cp.U, cp.xi, eps=1e-4)
    Z = tk["Z"]
    for l in range(3):
        M = oa.unfolding(cp.U, cp.xi, Z, l)
        m1, m2 = [m for m in range(3) if m != l]
        T = np.moveaxis(A, l, 0)                       # (n_l, n_m1, n_m2)
        F = np.einsum("ijk,ja,kb->iab", T, Z[m1], Z[m2])
        Mf = F.transpose(0, 2, 1).reshape(F.shape[0], -1)   # column a + r_m1 b
        assert np.abs(M - Mf).max() <= 1e-12 * np.abs(Mf).max()


def test_sweep_equals_full_tensor_hooi():
    cp = workloads.gaussian_sum(12, 40, 2)
    A = tu.full_from_cp(cp.U, cp.xi)
    tk = oracle.c2t(cp.U, cp.xi, eps=1e-3)
    res = oa.als(cp.U, cp.xi, tk["Z"], sweeps=2)
    Z = [z.copy() for z in tk["Z"]]
    for _ in range(2):
        for l in range(3):
            m1, m2 = [m for m in range(3) if m != l]
            T = np.moveaxis(A, l, 0)
            F = np.einsum("ijk,ja,kb->iab", T, Z[m1], Z[m2]).reshape(T.shape[0], -1)
            W = np.linalg.svd(F, full_matrices=False)[0]
            Z[l] = W[:, : Z[l].shape[1]]
    for l in range(3):
        P1 = res["Z"][l] @ res["Z"][l].T
        P2 = Z[l] @ Z[l].T
        assert np.abs(P1 - P2).max() <= 1e-9
    beta = np.einsum("ijm,ia,jb,mc->abc", A, *Z)
    assert abs(np.linalg.norm(beta) - np.linalg.norm(res["beta"])) <= 1e-11 * np.linalg.norm(beta)


def test_monotone_and_error_not_increasing():
    for seed, eps in ((3, 1e-2), (4, 1e-3), (5, 1e-5)):
        cp = workloads.gaussian_sum(16, 60, seed)
        A = tu.full_from_cp(cp.U, cp.xi)
        tk = oracle.c2t(cp.U, cp.xi, eps=eps)
        res = oa.als(cp.U, cp.xi, tk["Z"], sweeps=2)
        e = res["energy"]
        assert all(e[i + 1] >= e[i] * (1 - 1e-13) for i in range(len(e) - 1)), e
        err0 = np.linalg.norm(A - _tucker(tk["beta"], tk["Z"]))
        err1 = np.linalg.norm(A - _tucker(res["beta"], res["Z"]))
        assert err1 <= err0 * (1 + 1e-10) + 1e-14 * np.linalg.norm(A)
        # Pythagoras: ||A||^2 = ||beta||^2 + ||A - A_r||^2 (orthonormal Z, projection core)
        assert abs(np.linalg.norm(A) ** 2 - (e[-1] + err1 ** 2)) <= 1e-10 * np.linalg.norm(A) ** 2


def test_exact_tucker_rank_tensor():
    g = np.random.default_rng(7)
    n, r, R = 15, (3, 4, 2), 25
    Zt = [np.linalg.qr(g.standard_normal((n, r[l])))[0] for l in range(3)]
    U = [np.asfortranarray(Zt[l] @ g.standard_normal((r[l], R))) for l in range(3)]
    xi = g.uniform(0.5, 1.5, R)
    A = tu.full_from_cp(U, xi)
    tk = oracle.c2t(U, xi, eps=1e-10)
    assert tk["ranks"] == list(r)
    res = oa.als(U, xi, tk["Z"], sweeps=1)
    assert np.linalg.norm(A - _tucker(res["beta"], res["Z"])) <= 1e-12 * np.linalg.norm(A)
