"""Pins of the T2C / C2C oracle (oracle/t2c.py) against things other than itself: the error
bound of the slice-SVD remark (Sec. 2.4, Remark rem_can_red), exact reconstruction at eps = 0,
a core built with known slice ranks and singular values, the rank bound R <= r3 min(r1, r2),
and C2C against the brute-force full tensor of a small canonical input."""
import numpy as np

import workloads
from oracle import t2c as ot


def _core(shape, seed, decay=0.5):
    g = np.random.default_rng(seed)
    r1, r2, r3 = shape
    A = np.linalg.qr(g.standard_normal((r1, r1)))[0]
    B = np.linalg.qr(g.standard_normal((r2, r2)))[0]
    beta = np.zeros(shape)
    for m in range(r3):
        s = np.exp(-decay * np.arange(min(r1, r2))) * g.uniform(0.5, 2.0) * np.exp(-0.2 * m)
        beta[:, :, m] = (A[:, : len(s)] * s) @ B[:, : len(s)].T + 1e-3 * g.standard_normal((r1, r2)) * s[-1]
    return beta


def test_error_bound_and_rank_bound():
    for shape, seed in [((12, 9, 7), 0), ((20, 20, 20), 1), ((5, 17, 3), 2)]:
        beta = _core(shape, seed)
        for eps in (1e-1, 1e-3, 1e-6):
            res = ot.t2c_core(beta, eps)
            err = np.linalg.norm(beta - ot.beta_from_slices(res, shape))
            assert err <= eps * np.linalg.norm(beta) * (1 + 1e-12), (shape, eps, err)
            assert res["R"] <= shape[2] * min(shape[0], shape[1])
            # p_m is the count of singular values above delta: monotone in eps
        assert ot.t2c_core(beta, 1e-1)["R"] <= ot.t2c_core(beta, 1e-3)["R"] <= ot.t2c_core(beta, 1e-6)["R"]


def test_eps_zero_is_exact():
    beta = np.random.default_rng(3).standard_normal((8, 6, 5))
    res = ot.t2c_core(beta, 0.0)
    assert res["p"] == [6] * 5
    assert np.abs(ot.beta_from_slices(res, beta.shape) - beta).max() <= 1e-13 * np.abs(beta).max()


def test_known_slice_ranks_and_values():
    g = np.random.default_rng(4)
    r1, r2, r3 = 10, 8, 4
    A = np.linalg.qr(g.standard_normal((r1, r1)))[0]
    B = np.linalg.qr(g.standard_normal((r2, r2)))[0]
    q = [1, 3, 0, 8]
    vals = [np.sort(g.uniform(1.0, 3.0, qm))[::-1] for qm in q]
    beta = np.zeros((r1, r2, r3))
    for m in range(r3):
        beta[:, :, m] = (A[:, : q[m]] * vals[m]) @ B[:, : q[m]].T
    res = ot.t2c_core(beta, 1e-8)
    assert res["p"] == q
    for m in range(r3):
        assert np.allclose(res["sigma"][m], vals[m], rtol=1e-13, atol=0)


def test_c2c_against_the_full_tensor():
    cp = workloads.gaussian_sum(16, 600, 5)             # R far above r^2: the reduction pays
    eps_t, eps_c = 1e-6, 1e-4
    res = ot.c2c(cp.U, cp.xi, eps_t, eps_c)
    tk = res["tucker"]
    A = ot.full_from_cp(cp.U, cp.xi)
    A0 = np.einsum("abc,ia,jb,mc->ijm", tk["beta"], *tk["Z"])
    AR = ot.full_from_cp(res["U_can"], res["xi_can"])
    # ||A0 - AR|| = ||beta - beta_R|| (orthonormal Z), at most eps_c ||beta||
    assert abs(np.linalg.norm(A0 - AR) - np.linalg.norm(tk["beta"] - ot.beta_from_slices(res, tk["beta"].shape))) \
        <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(A0 - AR) <= eps_c * np.linalg.norm(tk["beta"]) * (1 + 1e-12)
    assert np.linalg.norm(A - AR) <= np.linalg.norm(A - A0) + eps_c * np.linalg.norm(tk["beta"]) + 1e-12 * np.linalg.norm(A)
    assert res["R"] < cp.xi.shape[0]            # the canonical rank went down


def test_factors_project_back_to_the_slices():
    g = np.random.default_rng(6)
    Z = [np.linalg.qr(g.standard_normal((n, r)))[0] for n, r in ((30, 7), (25, 6), (20, 5))]
    beta = _core((7, 6, 5), 7)
    res = ot.t2c(Z, beta, 1e-4)
    u = Z[0].T @ res["U_can"][0]
    v = Z[1].T @ res["U_can"][1]
    w = Z[2].T @ res["U_can"][2]
    rebuilt = np.einsum("k,ik,jk,mk->ijm", res["xi_can"], u, v, w)
    assert np.abs(rebuilt - ot.beta_from_slices(res, beta.shape)).max() <= 1e-13 * np.abs(beta).max()
