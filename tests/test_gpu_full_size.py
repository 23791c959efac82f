"""Full-size parity on the Hadamard workload that bench.py times (two rank-64 Gaussian sums,
n = 1024, product rank R = 4096, eps = 1e-7), in the bench's launch configuration, for both forms.

The oracle's exact RHOSVD at this size takes minutes, so its per-mode singular values, eps-ranks,
tails, kept-term count and ||xi'|| are stored in tests/golden/ by tests/golden/make_full_size.py
(which calls only oracle/).  Z and beta are checked through properties that hold at any size,
on sampled entries computed one by one on the CPU:
  * Z^(l) orthonormal;
  * V^(l)(:, nu) = Z^(l)^T u~_nu for sampled terms nu, with u~_nu the normalised Hadamard column
    formed on the CPU from the two input factors (Prop. 2.2: V = D V_0^T = Z_0^T U);
  * beta(i, j, m) = sum_nu xi'_nu V1(i, nu) V2(j, nu) V3(m, nu) for sampled (i, j, m), from the
    library's own V and xi' (Prop. 2.2), so the Khatri-Rao contraction is checked at full size;
  * the two forms agree on the Tucker tensor.
Tolerances as in test_gpu_parity.py; the mixed core's bound is derived from its digit
rounding relative to the operands' row maxima (see the core check)."""
import json
import math
import os

import numpy as np
import pytest

import workloads
from tests import tensor_utils as tu

pytestmark = pytest.mark.gpu

GOLD_PATH = os.path.join(os.path.dirname(__file__), "golden", "hadamard_n1024_R64x64_eps1e-7.json")
OPTS = dict(eps=1e-7, r_max=160, oversample=32, seed=12345)     # bench.py's options
U64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def gold():
    with open(GOLD_PATH) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def factors():
    return workloads.hartree_like_factors(1024, 64, 64, (0, 1))


_cache = {}


def run_full(P, factors, precision):
    if precision in _cache:
        return _cache[precision]
    import torch
    A, B = factors
    Ua = [P.to_device_factor(u) for u in A.U]
    Ub = [P.to_device_factor(u) for u in B.U]
    xa = torch.from_numpy(A.xi).cuda()
    xb = torch.from_numpy(B.xi).cuda()
    Uc, xc = P.rhosvd_cp_hadamard(Ua, xa, Ub, xb)
    res = P.rhosvd_c2t(Uc, xc, with_V=True, with_xi=True, precision=precision, **OPTS)
    info = res.info()
    r = [info.r[l] for l in range(3)]
    out = dict(info=info, ranks=r,
               beta=res.beta[: r[0] * r[1] * r[2]].cpu().numpy().reshape(r, order="F"),
               Z=[res.Z[l][:, : r[l]].cpu().numpy() for l in range(3)],
               V=[res.V[l][: r[l], :].cpu().numpy() for l in range(3)],
               sigma=res.sigma.cpu().numpy(), xin=res.xi_out.cpu().numpy())
    _cache[precision] = out
    return out


def normalised_column(A, B, l, nu):
    """u~_nu of mode l for the Hadamard term nu = i + 64 j (the product's term order)."""
    i, j = nu % A.U[l].shape[1], nu // A.U[l].shape[1]
    u = A.U[l][:, i] * B.U[l][:, j]
    return u / np.linalg.norm(u)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_ranks_sigma_tails(rhosvd_cuda, factors, gold, precision):
    g = run_full(rhosvd_cuda, factors, precision)
    info = g["info"]
    assert info.status == 0, rhosvd_cuda.rhosvd_strerror(info.status)
    assert info.kept == gold["kept"]
    assert math.isclose(info.xi_norm, gold["xi_norm"], rel_tol=1e-12)
    eps = OPTS["eps"]
    for l in range(3):
        so = np.array(gold["sigma"][l])
        total = gold["total"][l]
        thr = eps * eps * total
        rg, ro = g["ranks"][l], gold["ranks"][l]
        if rg != ro:
            # a difference of one only at a threshold tie (the oracle's tail within 1e-3 of eps^2 total)
            lo = min(rg, ro)
            t1, t0 = np.sum(so[lo + 1:] ** 2), np.sum(so[lo:] ** 2)
            assert abs(rg - ro) == 1 and (abs(t1 - thr) <= 1e-3 * thr or abs(t0 - thr) <= 1e-3 * thr), (l, rg, ro)
        k = info.k[l]
        q = min(len(so), k, rg + 2)
        tol = 6 * U64 * (1024 * k + k * (k + 1)) * so[0] ** 2
        assert np.all(np.abs(g["sigma"][l][:q] ** 2 - so[:q] ** 2) <= tol + 1e-14 * so[:q] ** 2), l
        if rg == ro:
            assert info.tail[l] >= gold["tails"][l] * (1 - 1e-9) - 1e-13 * math.sqrt(total)
        assert info.tail[l] ** 2 <= thr * (1 + 1e-9)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_factors_and_core(rhosvd_cuda, factors, precision):
    g = run_full(rhosvd_cuda, factors, precision)
    A, B = factors
    rng = np.random.default_rng(7)
    for l in range(3):
        Z = g["Z"][l]
        assert np.abs(Z.T @ Z - np.eye(Z.shape[1])).max() <= 1e-12, l
        for nu in rng.choice(4096, size=48, replace=False):
            ref = Z.T @ normalised_column(A, B, l, int(nu))
            assert np.abs(g["V"][l][:, nu] - ref).max() <= 1e-12, (l, nu)
    # core entries from the library's own V and xi'.  Plain: FP64 rounding of the sum.  Mixed:
    # the core's operands a = xi' V1(i, .) and b = V2(j, .) V3(m, .) are cut into 4 base-256
    # digits relative to their row maxima (a row of b uses max|V2(j, .)| max|V3(m, .)|), so each
    # term is off by at most 2^-33 (max|a| |b_nu| + |a_nu| max|b|) from the digit rounding.  The
    # groups s + t = 4, 5 are summed in FP32 over runs of 128 K between readbacks (inexact, the
    # tensor cores truncate); 2^-28 leaves a factor 32 for them and the pair products.
    V1, V2, V3 = g["V"]
    xin = g["xin"]
    r = g["ranks"]
    for _ in range(200):
        i, j, m = (int(rng.integers(r[0])), int(rng.integers(r[1])), int(rng.integers(r[2])))
        a = xin * V1[i]
        bb = V2[j] * V3[m]
        terms = a * bb
        if precision == 0:
            tol = 1e-12 * np.abs(terms).sum()
        else:
            amax = np.abs(a).max()
            bmax = np.abs(V2[j]).max() * np.abs(V3[m]).max()
            tol = 2.0 ** -28 * (amax * np.abs(bb).sum() + bmax * np.abs(a).sum())
        assert abs(g["beta"][i, j, m] - terms.sum()) <= tol, (i, j, m)


def test_full_size_forms_agree(rhosvd_cuda, factors):
    a = run_full(rhosvd_cuda, factors, 0)
    b = run_full(rhosvd_cuda, factors, 1)
    assert a["ranks"] == b["ranks"]
    assert tu.tucker_rel_diff(b["beta"], b["Z"], a["beta"], a["Z"]) < 1e-7


# ---------------------------------------------------------------- range-separated collective potential
# Long-range Newton Gaussians of N = 1000 unit charges (20 a charge): n = 2048, R = 20000, eps = 1e-6.

NEWTON_GOLD = os.path.join(os.path.dirname(__file__), "golden", "newton_n2048_N1000_eps1e-6.json")
NEWTON_OPTS = dict(eps=1e-6, r_max=64, oversample=32, seed=2024)


@pytest.fixture(scope="module")
def newton():
    cp = workloads.newton_long_range_sum(n=2048, N=1000, seed=0)
    with open(NEWTON_GOLD) as f:
        return cp, json.load(f)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_newton(rhosvd_cuda, newton, precision):
    P = rhosvd_cuda
    import torch
    cp, gold = newton
    Ud = [P.to_device_factor(u) for u in cp.U]
    xd = torch.from_numpy(cp.xi).cuda()
    res = P.rhosvd_c2t(Ud, xd, with_V=True, with_xi=True, precision=precision, **NEWTON_OPTS)
    info = res.info()
    assert info.status == 0, P.rhosvd_strerror(info.status)
    assert info.kept == gold["kept"]
    assert math.isclose(info.xi_norm, gold["xi_norm"], rel_tol=1e-12)
    r = [info.r[l] for l in range(3)]
    eps = NEWTON_OPTS["eps"]
    sig = res.sigma.cpu().numpy()
    for l in range(3):
        so = np.array(gold["sigma"][l])
        total = gold["total"][l]
        thr = eps * eps * total
        if r[l] != gold["ranks"][l]:
            lo = min(r[l], gold["ranks"][l])
            t1, t0 = np.sum(so[lo + 1:] ** 2), np.sum(so[lo:] ** 2)
            assert abs(r[l] - gold["ranks"][l]) == 1 and (abs(t1 - thr) <= 1e-3 * thr or abs(t0 - thr) <= 1e-3 * thr)
        else:
            assert info.tail[l] >= gold["tails"][l] * (1 - 1e-9) - 1e-13 * math.sqrt(total)
        k = info.k[l]
        q = min(len(so), k, r[l] + 2)
        tol = 6 * U64 * (2048 * k + k * (k + 1)) * so[0] ** 2
        assert np.all(np.abs(sig[l][:q] ** 2 - so[:q] ** 2) <= tol + 1e-14 * so[:q] ** 2), l
        assert info.tail[l] ** 2 <= thr * (1 + 1e-9)
        Z = res.Z[l][:, : r[l]].cpu().numpy()
        assert np.abs(Z.T @ Z - np.eye(r[l])).max() <= 1e-12
        V = res.V[l][: r[l], :].cpu().numpy()
        for nu in np.random.default_rng(3 + l).choice(cp.U[l].shape[1], size=32, replace=False):
            u = cp.U[l][:, nu] / np.linalg.norm(cp.U[l][:, nu])
            assert np.abs(V[:, nu] - Z.T @ u).max() <= 1e-12, (l, nu)

