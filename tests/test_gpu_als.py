"""GPU parity of the RHOSVD + ALS refinement (rhosvd_c2t_als) against the CPU oracle
(oracle/als.py) and against the full tensor.

Tolerances.  With direct modes (n_l <= r_max + oversample: the basis Q_l is the identity) the
GPU step is the oracle's step up to rounding: both converge to the same HOOI point, so the
refined Tucker tensors agree to the plain-form bar (1e-6 relative) and the captured energies to
1e-9 relative.  With a sketched mode the GPU optimises inside the sketch range, which holds all
but the sketch's missed energy (<= eps^2 of the side matrix): the energies agree to 10 eps^2
relative.  On every input the GPU's captured energy never falls from step to step (1e-12
relative slack for rounding) and the full-tensor error never grows."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import als as oa
from tests import tensor_utils as tu

pytestmark = pytest.mark.gpu


def _dev(P, cp):
    import torch
    return [P.to_device_factor(u) for u in cp.U], torch.from_numpy(np.ascontiguousarray(cp.xi)).cuda()


def _tk(res):
    info = res.info()
    r = [info.r[l] for l in range(3)]
    beta = res.beta[: r[0] * r[1] * r[2]].cpu().numpy().reshape(r, order="F")
    Z = [res.Z[l][:, : r[l]].cpu().numpy() for l in range(3)]
    return info, r, beta, Z


def _monotone(hist):
    for i, (b, a) in enumerate(hist):
        assert a >= b * (1 - 1e-12), (i, b, a)
        if i + 1 < len(hist):
            assert abs(hist[i + 1][0] - a) <= 1e-10 * a, (i, a, hist[i + 1][0])


@pytest.mark.parametrize("n,R,eps,sweeps,seed", [(40, 120, 1e-3, 1, 0), (48, 200, 1e-5, 2, 1), (30, 90, 1e-2, 2, 2)])
def test_als_direct_modes_match_oracle(rhosvd_cuda, n, R, eps, sweeps, seed):
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(n, R, seed)
    U, x = _dev(P, cp)
    res, hist = P.rhosvd_c2t_als(U, x, sweeps=sweeps, eps=eps, r_max=64)
    info, r, beta, Z = _tk(res)
    assert info.status == 0 and all(info.direct[l] for l in range(3))
    o = oa.c2t_als(cp.U, cp.xi, eps, sweeps=sweeps)
    assert r == o["rhosvd"]["ranks"]
    assert tu.tucker_rel_diff(beta, Z, o["beta"], o["Z"]) <= 1e-6
    eo = o["energy"]
    assert len(hist) == 3 * sweeps
    for s, (b, a) in enumerate(hist):
        assert abs(a - eo[s + 1]) <= 1e-9 * eo[s + 1]
    assert abs(hist[0][0] - eo[0]) <= 1e-9 * eo[0]
    _monotone(hist)
    A = tu.full_from_cp(cp.U, cp.xi)
    t0 = o["rhosvd"]
    err0 = np.linalg.norm(A - tu.tucker_full(t0["beta"], t0["Z"]))
    err1 = np.linalg.norm(A - tu.tucker_full(beta, Z))
    assert err1 <= err0 * (1 + 1e-9)


def test_als_sketched_modes(rhosvd_cuda):
    """n = 160 > r_max + oversample: the sketch path; energies within 10 eps^2 of the oracle's."""
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(160, 400, 3)
    eps = 1e-3
    U, x = _dev(P, cp)
    res, hist = P.rhosvd_c2t_als(U, x, sweeps=1, eps=eps, r_max=96, oversample=32)
    info, r, beta, Z = _tk(res)
    assert info.status == 0 and not any(info.direct[l] for l in range(3))
    o = oa.c2t_als(cp.U, cp.xi, eps, sweeps=1)
    if r == o["rhosvd"]["ranks"]:
        for s, (b, a) in enumerate(hist):
            assert abs(a - o["energy"][s + 1]) <= 10 * eps * eps * o["energy"][s + 1]
    _monotone(hist)
    A = tu.full_from_cp(cp.U, cp.xi)
    Ag = tu.tucker_full(beta, Z)
    # Pythagoras for the refined (orthonormal, projection-core) Tucker tensor
    assert abs(np.linalg.norm(A) ** 2 - (np.linalg.norm(beta) ** 2 + np.linalg.norm(A - Ag) ** 2)) \
        <= 1e-9 * np.linalg.norm(A) ** 2
    assert abs(np.linalg.norm(beta) ** 2 - hist[-1][1]) <= 1e-9 * hist[-1][1]


def test_als_zero_sweeps_is_rhosvd(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    cp = workloads.gaussian_sum(64, 150, 4)
    U, x = _dev(P, cp)
    a, h = P.rhosvd_c2t_als(U, x, sweeps=0, eps=1e-5, r_max=64, seed=9)
    b = P.rhosvd_c2t(U, x, eps=1e-5, r_max=64, seed=9)
    assert h == []
    ia, ib = a.info(), b.info()
    r = list(ia.r)
    assert r == list(ib.r)
    assert torch.equal(a.beta[: r[0] * r[1] * r[2]], b.beta[: r[0] * r[1] * r[2]])


def test_als_full_size_hadamard(rhosvd_cuda):
    """The n = 1024, 64 x 64 -> R = 4096 workload at eps = 1e-7 (mixed RHOSVD), one sweep: the
    captured energy never falls, and the refined core's norm equals the last recorded energy up
    to the mixed form's core accuracy (its digit-plane products carry about 2^-40 of sum |a||b|
    per entry; 1e-7 relative on the squared norm)."""
    P = rhosvd_cuda
    import torch
    A, B = workloads.hartree_like_factors(1024, 64, 64, (0, 1))
    Ua, xa = _dev(P, A)
    Ub, xb = _dev(P, B)
    Uc, xc = P.rhosvd_cp_hadamard(Ua, xa, Ub, xb)
    res, hist = P.rhosvd_c2t_als(Uc, xc, sweeps=1, eps=1e-7, r_max=160, oversample=32, seed=12345, precision=1)
    info = res.info()
    assert info.status == 0
    _monotone(hist)
    r = list(info.r)
    beta = res.beta[: r[0] * r[1] * r[2]]
    assert abs(float(torch.sum(beta * beta)) - hist[-1][1]) <= 1e-7 * hist[-1][1]
    assert hist[-1][1] >= hist[0][0]
