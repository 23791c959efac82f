"""GPU parity: the CUDA library (through the C ABI) against the CPU FP64 oracle on the same
seeded inputs.

Tolerances (plain FP64 path), derived from the arithmetic:
  * Tucker tensors: relative Frobenius difference <= 1e-6 (the plain-form bar).
  * ranks: equal; a difference of one is accepted only at a threshold tie, i.e. when the
    oracle's tail at the GPU rank lies within 1e-3 relative of eps^2 * total.
  * singular values: the GPU takes them from the eigenvalues of B B^T with B = Q^T U and Q
    from CholeskyQR, whose orthogonality error is bounded by 6 u (n k + k(k+1)); that bounds
    the relative perturbation of the eigenvalues, so |sigma_g^2 - sigma_o^2| <=
    6 u (n k + k(k+1)) sigma_1^2 (+ 1e-14 sigma_o^2).
  * per-mode truncation errors tau_l (Thm. 2.3): the GPU measures ||U - Z V||_F directly.
    The exact rank-r SVD truncation is optimal, so tau_gpu >= tau_oracle (up to rounding), and
    the GPU's rank satisfies the eps rule by its own measurement: tau_gpu^2 <= eps^2 total.
  * CP Hadamard product and sum: bit-exact (one rounding per entry on both sides).
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests import tensor_utils as tu

pytestmark = pytest.mark.gpu


def to_dev(P, cp_or_U, xi=None):
    import torch
    U = cp_or_U.U if xi is None else cp_or_U
    x = cp_or_U.xi if xi is None else xi
    return [P.to_device_factor(u) for u in U], torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_gpu(P, U, xi, eps, r_max, oversample=32, ranks=(0, 0, 0), seed=1234, precision=0):
    Ud, xd = to_dev(P, U, xi)
    res = P.rhosvd_c2t(Ud, xd, eps=eps, ranks=ranks, r_max=r_max, oversample=oversample, seed=seed,
                       with_V=True, with_xi=True, precision=precision)
    info = res.info()
    r = [info.r[l] for l in range(3)]
    beta = res.beta[: r[0] * r[1] * r[2]].cpu().numpy().reshape((r[0], r[1], r[2]), order="F")
    Z = [res.Z[l][:, : r[l]].cpu().numpy() for l in range(3)]
    sig = res.sigma.cpu().numpy()
    V = [res.V[l][: r[l], :].cpu().numpy() for l in range(3)]
    return dict(info=info, ranks=r, beta=beta, Z=Z, sigma=sig, V=V, xin=res.xi_out.cpu().numpy())


def oracle_tail(sig, r):
    return float(np.sum(sig[r:] ** 2))


def assert_rank_parity(g, o, eps):
    for l in range(3):
        rg, ro = g["ranks"][l], o["ranks"][l]
        if rg == ro:
            continue
        s = o["sigma"][l]
        thr = eps * eps * np.sum(s ** 2)
        assert abs(rg - ro) == 1, (l, rg, ro)
        lo = min(rg, ro)
        # tie: removing sigma_{lo+1} moves the tail across the threshold within 1e-3
        assert abs(oracle_tail(s, lo + 1) - thr) <= 1e-3 * thr or abs(oracle_tail(s, lo) - thr) <= 1e-3 * thr, \
            (l, rg, ro)


U64 = np.finfo(np.float64).eps


def assert_tail_parity(g, o, eps, eps_rule):
    for l in range(3):
        tg, to = g["info"].tail[l], o["tails"][l]
        total = g["info"].total[l]
        assert tg >= to * (1 - 1e-9) - 1e-13 * math.sqrt(total), (l, tg, to)
        if eps_rule:
            assert tg * tg <= eps * eps * total * (1 + 1e-9), (l, tg, eps)


def assert_sigma_parity(g, o, n):
    for l in range(3):
        so = o["sigma"][l]
        k = g["info"].k[l]
        q = min(len(so), k, g["ranks"][l] + 2)
        sg = g["sigma"][l][:q]
        s1 = so[0] if len(so) else 0.0
        tol = 6 * U64 * (n[l] * k + k * (k + 1)) * s1 * s1
        assert np.all(np.abs(sg ** 2 - so[:q] ** 2) <= tol + 1e-14 * so[:q] ** 2), l


def assert_tucker_parity(g, o, tol=1e-6):
    if min(o["ranks"]) == 0:
        assert np.linalg.norm(g["beta"]) == 0.0
        return 0.0
    d = tu.tucker_rel_diff(g["beta"], g["Z"], o["beta"], o["Z"])
    assert d <= tol, d
    for l in range(3):
        Zg = g["Z"][l]
        assert np.allclose(Zg.T @ Zg, np.eye(Zg.shape[1]), atol=1e-10), l
    return d


def oracle_at_ranks(U, xi, o, ranks):
    """The oracle's RHOSVD truncated at other ranks (Def. 2.2 with r_l given): the leading r_l of
    its own singular vectors, V = Z^T U~ and the core by its own loops (Prop. 2.2)."""
    Un, xin, _, _ = oracle.normalize(U, xi)
    Z = [np.asfortranarray(o["Z_full"][l][:, : ranks[l]]) for l in range(3)]
    V = [oracle.project(Z[l], Un[l]) for l in range(3)]
    beta = oracle.core(V, xin) if min(ranks) > 0 else np.zeros(tuple(ranks))
    return dict(o, ranks=list(ranks), Z=Z, V=V, beta=beta,
                tails=[float(np.sqrt(np.sum(o["sigma"][l][ranks[l]:] ** 2))) for l in range(3)])


def check_case(P, U, xi, eps, r_max, oversample=32, ranks=(0, 0, 0), precision=0):
    """GPU vs oracle on one input.  The Tucker tensors are always compared: where a GPU rank is
    one off the oracle's at a threshold tie (assert_rank_parity), against the oracle truncated
    at the GPU's ranks.  Returns (gpu, oracle, Tucker difference)."""
    o = oracle.c2t(U, xi, eps=eps, ranks=ranks)
    g = run_gpu(P, U, xi, eps, r_max, oversample, ranks, precision=precision)
    assert g["info"].status == 0, P.rhosvd_strerror(g["info"].status)
    assert g["info"].kept == o["kept"]
    assert math.isclose(g["info"].xi_norm, o["xi_norm"], rel_tol=1e-13)
    assert np.allclose(g["xin"], o["xin"], rtol=1e-14, atol=0)
    if all(r == 0 for r in ranks):
        assert_rank_parity(g, o, eps)
    assert_sigma_parity(g, o, [u.shape[0] for u in U])
    oc = o if g["ranks"] == o["ranks"] else oracle_at_ranks(U, xi, o, g["ranks"])
    assert_tail_parity(g, oc, eps, all(r == 0 for r in ranks))
    d = assert_tucker_parity(g, oc)
    return g, o, d


# ---------------------------------------------------------------- configurations

def test_gauss_n128_R200_direct(rhosvd_cuda):
    cp = workloads.gaussian_sum(128, 200, 0)
    g, o, d = check_case(rhosvd_cuda, cp.U, cp.xi, 1e-6, r_max=128)
    assert g["info"].direct[0] == 1
    assert g["ranks"] == o["ranks"] and d < 1e-9


def test_gauss_sketch_ragged(rhosvd_cuda):
    """n = 300 > k = 128 forces the range sketch; 300 and 700 are not multiples of the tiles."""
    cp = workloads.gaussian_sum(300, 700, 3)
    g, o, d = check_case(rhosvd_cuda, cp.U, cp.xi, 1e-6, r_max=128, oversample=32)
    assert g["info"].direct[0] == 0
    assert g["info"].resid[0] <= 1e-12 * g["info"].total[0]
    assert d is not None


@pytest.mark.parametrize("precision", [0, 1])
def test_full_width_sketch_grown_by_deflation(rhosvd_cuda, precision):
    """No oversampling: the first sketch keeps all its k = 106 columns, and the deflation sketch
    grows the basis past k.  Every product after the basis (B = Q^T U, B B^T, Z, V, residual)
    must cover the grown width.  Fixed ranks give element-wise parity; with the eps rule the
    rank may exceed the oracle's by one (the basis misses a little more energy than a wider
    sketch), but the measured error must meet the rule."""
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(384, 600, 7)
    g, o, d = check_case(P, cp.U, cp.xi, 1e-6, r_max=106, oversample=0, ranks=(100, 100, 100),
                         precision=precision)
    assert max(g["info"].k[l] for l in range(3)) > 106
    assert d is not None
    o = oracle.c2t(cp.U, cp.xi, eps=1e-6)
    g = run_gpu(P, cp.U, cp.xi, 1e-6, r_max=106, oversample=0, precision=precision)
    info = g["info"]
    assert info.status == 0, P.rhosvd_strerror(info.status)
    for l in range(3):
        assert o["ranks"][l] <= g["ranks"][l] <= o["ranks"][l] + 1, (l, g["ranks"], o["ranks"])
        assert info.tail[l] ** 2 <= 1e-12 * info.total[l] * (1 + 1e-9)


def test_hadamard_then_reduce(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    A = workloads.gaussian_sum(256, 24, 0)
    B = workloads.gaussian_sum(256, 20, 1)
    Ua, xa = to_dev(P, A)
    Ub, xb = to_dev(P, B)
    Uc, xc = P.rhosvd_cp_hadamard(Ua, xa, Ub, xb)
    torch.cuda.synchronize()
    Uo, xo = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    for l in range(3):
        assert np.array_equal(Uc[l].cpu().numpy(), Uo[l])
    assert np.array_equal(xc.cpu().numpy(), xo)
    check_case(P, Uo, xo, 1e-7, r_max=160, oversample=32)


def test_cp_sum_bit_exact(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    A = workloads.gaussian_sum(96, 30, 5)
    B = workloads.random_cp(96, 17, 6)
    Ua, xa = to_dev(P, A)
    Ub, xb = to_dev(P, B)
    Uc, xc = P.rhosvd_cp_sum(0.75, Ua, xa, -1.5, Ub, xb)
    torch.cuda.synchronize()
    Uo, xo = oracle.cp_sum(0.75, A.U, A.xi, -1.5, B.U, B.xi)
    for l in range(3):
        assert np.array_equal(Uc[l].cpu().numpy(), Uo[l])
    assert np.array_equal(xc.cpu().numpy(), xo)


def test_newton_long_range_small(rhosvd_cuda):
    cp = workloads.newton_long_range_sum(n=320, N=40, seed=0)
    check_case(rhosvd_cuda, cp.U, cp.xi, 1e-6, r_max=64, oversample=32)


# ---------------------------------------------------------------- edge cases

def test_rank_one(rhosvd_cuda):
    g0 = np.random.default_rng(11)
    U = [g0.standard_normal((n, 1)) for n in (70, 300, 5)]
    g, o, d = check_case(rhosvd_cuda, U, np.array([2.5]), 1e-12, r_max=8)
    assert g["ranks"] == [1, 1, 1] and d < 1e-14


def test_fewer_terms_than_grid(rhosvd_cuda):
    cp = workloads.gaussian_sum(300, 20, 8)
    g, o, d = check_case(rhosvd_cuda, cp.U, cp.xi, 1e-10, r_max=32, oversample=16)
    assert g["info"].k[0] <= 20


def test_fixed_ranks(rhosvd_cuda):
    cp = workloads.gaussian_sum(200, 300, 9)
    g, o, d = check_case(rhosvd_cuda, cp.U, cp.xi, 1e-6, r_max=64, oversample=96, ranks=(5, 12, 30))
    assert g["ranks"] == [5, 12, 30]


def test_zero_terms_dropped(rhosvd_cuda):
    cp = workloads.gaussian_sum(150, 120, 10)
    U = [u.copy() for u in cp.U]
    U[1][:, 7] = 0.0
    U[2][:, 50] = 0.0
    U[0][:, 90] *= 2.0 ** -1000
    g, o, d = check_case(rhosvd_cuda, U, cp.xi, 1e-6, r_max=150)
    assert g["info"].kept == 118


def test_empty_and_eps_one(rhosvd_cuda):
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(64, 40, 12)
    g = run_gpu(P, cp.U, cp.xi, 1.0, r_max=16)
    assert g["info"].status == 0 and g["ranks"] == [0, 0, 0]
    U0 = [np.zeros((64, 40)) for _ in range(3)]
    g = run_gpu(P, U0, cp.xi, 1e-6, r_max=16)
    assert g["info"].kept == 0 and g["ranks"] == [0, 0, 0]


def test_rank_overflow_reports_needed_rank(rhosvd_cuda):
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(128, 200, 0)
    o = oracle.c2t(cp.U, cp.xi, eps=1e-6)
    g = run_gpu(P, cp.U, cp.xi, 1e-6, r_max=16, oversample=240)
    assert g["info"].status == P.RHOSVD_ERR_RANK_OVERFLOW
    assert [g["info"].r_needed[l] for l in range(3)] == o["ranks"]
    assert g["ranks"] == [16, 16, 16]


def test_nonfinite_input_flagged(rhosvd_cuda):
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(64, 30, 13)
    U = [u.copy() for u in cp.U]
    U[2][3, 4] = np.nan
    g = run_gpu(P, U, cp.xi, 1e-6, r_max=32)
    assert g["info"].status == P.RHOSVD_ERR_NONFINITE


def test_bound_on_full_tensor(rhosvd_cuda):
    """Thm. 2.3 on the GPU result: ||A - A0|| <= ||xi|| sum_l tau_l, with tau_l as measured."""
    cp = workloads.gaussian_sum(24, 70, 15, b=3.0, centre_box=1.5, a_range=(0.5, 8.0))
    g = run_gpu(rhosvd_cuda, cp.U, cp.xi, 1e-4, r_max=24, oversample=0)
    A = tu.full_from_cp(cp.U, cp.xi)
    T = tu.tucker_full(g["beta"], g["Z"])
    err = np.linalg.norm(A - T)
    info = g["info"]
    assert err <= info.xi_norm * sum(info.tail[l] for l in range(3)) * (1 + 1e-9)
    assert math.isclose(np.linalg.norm(A) ** 2, np.linalg.norm(g["beta"]) ** 2 + err ** 2, rel_tol=1e-9)


def test_seed_independence_of_the_result(rhosvd_cuda):
    """The sketch is random; the Tucker tensor is not (up to the parity tolerance)."""
    P = rhosvd_cuda
    cp = workloads.gaussian_sum(400, 500, 14)
    a = run_gpu(P, cp.U, cp.xi, 1e-6, r_max=128, seed=1)
    b = run_gpu(P, cp.U, cp.xi, 1e-6, r_max=128, seed=2)
    assert a["ranks"] == b["ranks"]
    assert tu.tucker_rel_diff(a["beta"], a["Z"], b["beta"], b["Z"]) < 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_workspace_contents_do_not_matter(rhosvd_cuda, precision):
    """The reduction clears what it needs itself: a workspace filled with 0xFF bytes (NaN as
    doubles) gives bit-identical outputs to a zeroed one, and both match the oracle."""
    P = rhosvd_cuda
    import torch
    cp = workloads.gaussian_sum(300, 700, 3)
    Ud, xd = to_dev(P, cp)
    kw = dict(eps=1e-6, r_max=128, oversample=32, seed=77, precision=precision)
    need = P.rhosvd_c2t_workspace_size(P.make_cp(Ud, xd), P.make_opts(**kw))
    outs = []
    for fill in (0x00, 0xFF):
        ws = torch.full((need,), fill, dtype=torch.uint8, device="cuda")
        res = P.rhosvd_c2t(Ud, xd, workspace=ws, **kw)
        info = res.info()
        assert info.status == 0, P.rhosvd_strerror(info.status)
        r = [info.r[l] for l in range(3)]
        outs.append((r, res.beta[: r[0] * r[1] * r[2]].cpu().numpy(),
                     [res.Z[l][:, : r[l]].cpu().numpy() for l in range(3)], res.sigma.cpu().numpy()))
    (ra, ba, Za, sa), (rb, bb, Zb, sb) = outs
    assert ra == rb
    assert np.array_equal(ba, bb) and np.array_equal(sa, sb)
    assert all(np.array_equal(Za[l], Zb[l]) for l in range(3))
    o = oracle.c2t(cp.U, cp.xi, eps=1e-6)
    oc = o if ra == o["ranks"] else oracle_at_ranks(cp.U, cp.xi, o, ra)
    assert tu.tucker_rel_diff(ba.reshape(ra, order="F"), Za, oc["beta"], oc["Z"]) <= 1e-6
