"""GPU parity of the Tucker-to-canonical transform (rhosvd_t2c) and of C2C (rhosvd_c2t followed
by rhosvd_t2c) against the CPU oracle (oracle/t2c.py) on the same seeded inputs.

Tolerances: the slice singular values are FP64 Jacobi (GPU) vs LAPACK SVD (oracle): agreement to
1e-12 of ||beta||.  p_m is equal, except for a singular value within 1e-9 relative of delta.
The reduced core beta_R, rebuilt from the GPU's canonical factors (u = Z1^T U1, ... for
orthonormal Z), matches the oracle's beta_R to 1e-10 of ||beta|| (sums of rank-one terms whose
vectors agree to ~1e-12; signs and rotations within repeated singular values do not matter for
beta_R)."""
import numpy as np
import pytest

import workloads
from oracle import t2c as ot

pytestmark = pytest.mark.gpu


def _dev(P, Z, beta):
    import torch
    Zd = [torch.from_numpy(np.ascontiguousarray(z.T)).cuda().t() for z in Z]
    bd = torch.from_numpy(np.ascontiguousarray(beta.ravel(order="F"))).cuda()
    return Zd, bd


def _gpu_core(res, Z, shape):
    """beta_R from the GPU's canonical factors: u = Z1^T U1, v = Z2^T U2, w = Z3^T U3."""
    R, st = res.rank()
    U = [res.U[l][:, :R].cpu().numpy() for l in range(3)]
    xi = res.xi[:R].cpu().numpy()
    u, v, w = (Z[l].T @ U[l] for l in range(3))
    return np.einsum("k,ik,jk,mk->ijm", xi, u, v, w), R, st


def _check(P, Z, beta, eps):
    Zd, bd = _dev(P, Z, beta)
    ref = ot.t2c_core(beta, eps)
    res = P.rhosvd_t2c(Zd, bd, eps, R_max=beta.shape[2] * min(beta.shape[:2]))
    bR, R, st = _gpu_core(res, Z, beta.shape)
    assert st == 0
    p = res.p.cpu().numpy()[: beta.shape[2]].tolist()
    nb = np.linalg.norm(beta)
    for m in range(beta.shape[2]):
        if p[m] != ref["p"][m]:
            s = np.linalg.svd(beta[:, :, m], compute_uv=False)
            edge = s[min(p[m], ref["p"][m])]
            assert abs(p[m] - ref["p"][m]) == 1 and abs(edge - ref["delta"]) <= 1e-9 * ref["delta"], (m, p[m])
    assert R == sum(p)
    ref_bR = ot.beta_from_slices(ref, beta.shape)
    if p == ref["p"]:
        assert np.linalg.norm(bR - ref_bR) <= 1e-10 * nb
    assert np.linalg.norm(beta - bR) <= eps * nb * (1 + 1e-9)
    return res, ref, p


@pytest.mark.parametrize("shape,eps,seed", [((12, 10, 9), 1e-4, 0), ((33, 40, 17), 1e-6, 1), ((5, 7, 3), 1e-2, 2),
                                            ((64, 64, 50), 1e-5, 3)])
def test_t2c_matches_oracle(rhosvd_cuda, shape, eps, seed):
    Z, beta = workloads.tucker_tensor((80, 70, 60), shape, seed)
    _check(rhosvd_cuda, Z, beta, eps)


def test_t2c_singular_values(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    Z, beta = workloads.tucker_tensor((50, 50, 50), (20, 16, 6), 4)
    res, ref, p = _check(P, Z, beta, 1e-7)
    # each slice's kept u columns reproduce the oracle's singular values: sigma = ||B_m^T u|| (u unit)
    R, _ = res.rank()
    xi = res.xi[:R].cpu().numpy()
    o = 0
    for m in range(beta.shape[2]):
        assert np.allclose(xi[o:o + p[m]], ref["sigma"][m], rtol=0, atol=1e-12 * np.linalg.norm(beta))
        o += p[m]


def test_t2c_eps_zero_and_overflow_and_empty(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    Z, beta = workloads.tucker_tensor((30, 30, 30), (6, 5, 4), 5)
    Zd, bd = _dev(P, Z, beta)
    res = P.rhosvd_t2c(Zd, bd, 0.0, R_max=20)
    bR, R, st = _gpu_core(res, Z, beta.shape)
    assert st == 0 and R == 20 and np.abs(bR - beta).max() <= 1e-13 * np.abs(beta).max()
    res = P.rhosvd_t2c(Zd, bd, 0.0, R_max=7)
    R, st = res.rank()
    assert st == P.RHOSVD_ERR_RANK_OVERFLOW and R == 20
    Ze = [torch.zeros(30, 0, dtype=torch.float64, device="cuda") for _ in range(3)]
    res = P.rhosvd_t2c(Ze, torch.zeros(0, dtype=torch.float64, device="cuda"), 1e-6, R_max=4)
    assert res.rank() == (0, 0)


def test_c2c_against_oracle_and_full_tensor(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    cp = workloads.gaussian_sum(16, 600, 5)
    eps_t, eps_c = 1e-6, 1e-4
    U = [P.to_device_factor(u) for u in cp.U]
    xd = torch.from_numpy(cp.xi).cuda()
    can, tk = P.rhosvd_c2c(U, xd, eps_t, eps_c, R_max=16 * 16 * 16, r_max=16)
    R, st = can.rank()
    assert st == 0
    ref = ot.c2c(cp.U, cp.xi, eps_t, eps_c)
    A = ot.full_from_cp(cp.U, cp.xi)
    Ag = ot.full_from_cp([can.U[l][:, :R].cpu().numpy() for l in range(3)], can.xi[:R].cpu().numpy())
    Ao = ot.full_from_cp(ref["U_can"], ref["xi_can"])
    nb = np.linalg.norm(ref["tucker"]["beta"])
    A0 = np.einsum("abc,ia,jb,mc->ijm", ref["tucker"]["beta"], *ref["tucker"]["Z"])
    bound = np.linalg.norm(A - A0) + eps_c * nb
    assert np.linalg.norm(A - Ag) <= bound * (1 + 1e-6) + 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(A - Ao) <= bound * (1 + 1e-6) + 1e-12 * np.linalg.norm(A)
    assert abs(R - ref["R"]) <= 3                      # p_m may differ at threshold ties
    assert np.linalg.norm(Ag - Ao) <= 2 * eps_c * nb + 1e-10 * np.linalg.norm(A)
    assert R < 600
