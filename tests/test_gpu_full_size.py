"""Full-size parity on the Hadamard workload that bench.py times (two rank-64 Gaussian sums,
n = 1024, product rank R = 4096, eps = 1e-7) and on the range-separated collective potential
(n = 2048, R = 20000, eps = 1e-6), in the bench's launch configuration, for both forms.

The oracle's exact RHOSVD at these sizes takes from a minute to tens of minutes, so its per-mode
singular values, eps-ranks, tails, kept-term count and ||xi'|| (``<case>.json``) and its leading
left singular vectors Z^(l) (``<case>_Z.npz``, r_l + 4 columns) are stored in tests/golden/ by
tests/golden/make_full_size.py, which calls only oracle/.  From the stored Z the test rebuilds the
oracle's V^(l) = Z^(l)T U~^(l) and core beta with the oracle's own loops (Prop. 2.2) and compares
the Tucker tensors element by element in a common basis (tests/tensor_utils.tucker_rel_diff):
<= 1e-6 relative for both forms (the plain-form bar; the mixed form's products carry FP64-class
digits, its core about 2^-29 of the operands' row scales).  Where a GPU rank is one off at a
threshold tie, the oracle is truncated at the GPU's rank (the stored extra columns).  On top:
  * Z^(l) orthonormal;
  * V^(l)(:, nu) = Z^(l)^T u~_nu for sampled terms nu, with u~_nu the normalised Hadamard column
    formed on the CPU from the two input factors (Prop. 2.2: V = D V_0^T = Z_0^T U);
  * beta(i, j, m) against the sum of xi'_nu V1(i, nu) V2(j, nu) V3(m, nu) over the library's own V
    and xi', for sampled (i, j, m): the Khatri-Rao contraction's arithmetic on its own inputs,
    with the bound derived from its digit scheme (see core_entry_bound);
  * the two forms agree on the Tucker tensor.
Tolerances for ranks, sigma and tails as in test_gpu_parity.py."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads
from tests import tensor_utils as tu

pytestmark = pytest.mark.gpu

GOLD_DIR = os.path.join(os.path.dirname(__file__), "golden")
GOLD_PATH = os.path.join(GOLD_DIR, "hadamard_n1024_R64x64_eps1e-7.json")
OPTS = dict(eps=1e-7, r_max=160, oversample=32, seed=12345)     # bench.py's options
U64 = np.finfo(np.float64).eps
TUCKER_TOL = 1e-6


def load_gold_Z(name):
    z = np.load(os.path.join(GOLD_DIR, f"{name}_Z.npz"))
    return [np.asfortranarray(z[f"Z{l}"]) for l in range(3)]


class OracleTucker:
    """The oracle's Tucker tensor of a full-size case at given ranks, from its stored singular
    vectors: V = Z^T U~ (orc_project) and beta (orc_core) over the oracle's normalisation."""

    def __init__(self, U, xi, Zs):
        self.Un, self.xin, _, _ = oracle.normalize(U, xi)
        self.Zs = Zs
        self._cache = {}

    def at(self, ranks):
        key = tuple(ranks)
        if key not in self._cache:
            assert all(ranks[l] <= self.Zs[l].shape[1] for l in range(3)), (ranks, [z.shape for z in self.Zs])
            Z = [np.asfortranarray(self.Zs[l][:, : ranks[l]]) for l in range(3)]
            V = [oracle.project(Z[l], self.Un[l]) for l in range(3)]
            self._cache[key] = (oracle.core(V, self.xin), Z)
        return self._cache[key]


def assert_ranks_at_tie(rg, ro, so, thr):
    """Equal, or one apart where the oracle's tail is within 1e-3 of the threshold."""
    if rg != ro:
        lo = min(rg, ro)
        t1, t0 = np.sum(so[lo + 1:] ** 2), np.sum(so[lo:] ** 2)
        assert abs(rg - ro) == 1 and (abs(t1 - thr) <= 1e-3 * thr or abs(t0 - thr) <= 1e-3 * thr), (rg, ro)


@pytest.fixture(scope="module")
def gold():
    with open(GOLD_PATH) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def factors():
    return workloads.hartree_like_factors(1024, 64, 64, (0, 1))


@pytest.fixture(scope="module")
def oracle_had(factors):
    A, B = factors
    U, xi = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    return OracleTucker(U, xi, load_gold_Z("hadamard_n1024_R64x64_eps1e-7"))


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


def frexp_scale(x, lo=-126, hi=127, widen=0.0):
    """2^E, an upper bound on the per-row digit scale of the mixed form: E the frexp exponent of
    max|x| (1 + widen) (|x| < 2^E), clamped to [lo, hi] as the slicers clamp it."""
    m = float(np.max(np.abs(x)))
    e = math.frexp(m * (1.0 + widen))[1] if m > 0.0 else lo
    return 2.0 ** min(hi, max(lo, e))


# Bound on one core entry of the mixed form, per term nu and in units of 2^(Ea + Eb) (the two
# operand rows' digit scales): S = 4 balanced base-256 digits per operand, |d1| <= 2^8 and
# |d2|, |d3|, |d4| <= 2^7, the last rounded; every pair s + t <= GMAX = 5 is multiplied, the term
# of pair (s, t) being d_s d'_t 2^(-8 (s + t)).
#   * dropped pairs s + t = 6, 7, 8 (3, 2 and 1 pairs, none with a leading digit): each below
#     2^14 2^(-8 (s + t)):
C_DROP = 3 * 2.0 ** -34 + 2 * 2.0 ** -42 + 2.0 ** -50
#   * rounding: the Khatri-Rao operand's integer is the sum of its FP32 head product and of that
#     product's error, each rounded to the last digit's unit (|x - x^| <= 2^(E - 32)); the other
#     operand is rounded once (2^(E - 33)): 2^-32 + 2^-33 + 2^-65
C_ROUND = 2.0 ** -32 + 2.0 ** -33 + 2.0 ** -65
#   * groups 2 and 3 are accumulated exactly (read back every 256 K, before their FP32 sums can
#     round); groups 4 and 5 share one FP32 accumulator read back at the same cadence.  In that
#     accumulator's units (2^(Ea + Eb - 16)) a term adds at most 1.25 (group 4: 1/2 + 1/4 + 1/2)
#     plus 1.5 2^-8 (group 5), so a 256-term block stays below 256 (1.25 + 1.5 2^-8); it receives
#     7 pairs x 16 K steps of 16 = 112 MMAs, each rounding (the tensor cores truncate) by at most
#     2 2^-23 of (|accumulator| + the sum of its 16 products):
C_ACC = 112 * 2 * 2.0 ** -23 * ((256 + 16) * (1.25 + 1.5 * 2.0 ** -8)) * 2.0 ** -16 / 256
C_CORE = C_DROP + C_ROUND + C_ACC          # about 2^-29.8 per term


def core_entry_bound(precision, a, V2j, V3m, bb):
    """|beta_gpu(i, j, m) - sum_nu a_nu bb_nu| for a = xi' V1(i, .), bb = V2(j, .) V3(m, .)."""
    terms = np.abs(a * bb).sum()
    if precision == 0:
        return 1e-12 * terms                 # FP64 sum of R products: R u sum|terms| < 1e-12 sum|terms|
    R = a.shape[0]
    # the generated Khatri-Rao row is cut with E = e2[j] + e3[m], each taken from the FP32 heads
    # of its factor's row (max |h| (1 + 2^-20), clamped to [-45, 1]); the other operand row with
    # the frexp exponent of its own largest entry
    ev = dict(lo=-45, hi=1, widen=2.0 ** -20 + 2.0 ** -23)
    scale = frexp_scale(a) * frexp_scale(V2j, **ev) * frexp_scale(V3m, **ev)
    return R * C_CORE * scale + 1e-12 * terms


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
        assert_ranks_at_tie(rg, ro, so, thr)
        k = info.k[l]
        q = min(len(so), k, rg + 2)
        tol = 6 * U64 * (1024 * k + k * (k + 1)) * so[0] ** 2
        assert np.all(np.abs(g["sigma"][l][:q] ** 2 - so[:q] ** 2) <= tol + 1e-14 * so[:q] ** 2), l
        # the exact truncation at the GPU's rank is optimal
        assert info.tail[l] >= np.sqrt(np.sum(so[rg:] ** 2)) * (1 - 1e-9) - 1e-13 * math.sqrt(total)
        assert info.tail[l] ** 2 <= thr * (1 + 1e-9)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_tucker_vs_oracle(rhosvd_cuda, factors, oracle_had, precision):
    """||T_gpu - T_oracle||_F / ||T_oracle||_F at the benchmarked size, in a common basis."""
    g = run_full(rhosvd_cuda, factors, precision)
    beta_o, Z_o = oracle_had.at(g["ranks"])
    d = tu.tucker_rel_diff(g["beta"], g["Z"], beta_o, Z_o)
    print(f"hadamard n=1024 R=4096 precision={precision}: ||T_gpu - T_oracle|| / ||T_oracle|| = {d:.3e}")
    assert d <= TUCKER_TOL, d


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
    V1, V2, V3 = g["V"]
    xin = g["xin"]
    r = g["ranks"]
    for _ in range(200):
        i, j, m = (int(rng.integers(r[0])), int(rng.integers(r[1])), int(rng.integers(r[2])))
        a = xin * V1[i]
        bb = V2[j] * V3[m]
        tol = core_entry_bound(precision, a, V2[j], V3[m], bb)
        assert abs(g["beta"][i, j, m] - (a * bb).sum()) <= tol, (i, j, m)


def test_full_size_forms_agree(rhosvd_cuda, factors):
    a = run_full(rhosvd_cuda, factors, 0)
    b = run_full(rhosvd_cuda, factors, 1)
    assert a["ranks"] == b["ranks"]
    assert tu.tucker_rel_diff(b["beta"], b["Z"], a["beta"], a["Z"]) < 1e-7


# ---------------------------------------------------------------- range-separated collective potential
# Long-range Newton Gaussians of N = 1000 unit charges (20 a charge): n = 2048, R = 20000, eps = 1e-6.

NEWTON = "newton_n2048_N1000_eps1e-6"
NEWTON_GOLD = os.path.join(GOLD_DIR, f"{NEWTON}.json")
NEWTON_OPTS = dict(eps=1e-6, r_max=64, oversample=32, seed=2024)


@pytest.fixture(scope="module")
def newton():
    cp = workloads.newton_long_range_sum(n=2048, N=1000, seed=0)
    with open(NEWTON_GOLD) as f:
        return cp, json.load(f), OracleTucker(cp.U, cp.xi, load_gold_Z(NEWTON))


@pytest.mark.parametrize("precision,out_fp32", [(0, False), (1, False), (1, True)])
def test_full_size_newton(rhosvd_cuda, newton, precision, out_fp32):
    """Ranks, sigma, tails, factors and the Tucker tensor against the oracle.  With FP32 outputs
    (Z and beta rounded once to FP32, 2^-24 relative per entry) the Tucker bar is the same."""
    P = rhosvd_cuda
    import torch
    cp, gold, orc = newton
    Ud = [P.to_device_factor(u) for u in cp.U]
    xd = torch.from_numpy(cp.xi).cuda()
    res = P.rhosvd_c2t(Ud, xd, with_V=True, with_xi=True, precision=precision, out_fp32=out_fp32,
                       **NEWTON_OPTS)
    info = res.info()
    assert info.status == 0, P.rhosvd_strerror(info.status)
    assert info.kept == gold["kept"]
    assert math.isclose(info.xi_norm, gold["xi_norm"], rel_tol=1e-12)
    r = [info.r[l] for l in range(3)]
    eps = NEWTON_OPTS["eps"]
    sig = res.sigma.cpu().numpy()
    zt = 1e-6 if out_fp32 else 1e-12
    Zs = []
    for l in range(3):
        so = np.array(gold["sigma"][l])
        total = gold["total"][l]
        thr = eps * eps * total
        assert_ranks_at_tie(r[l], gold["ranks"][l], so, thr)
        assert info.tail[l] >= np.sqrt(np.sum(so[r[l]:] ** 2)) * (1 - 1e-9) - 1e-13 * math.sqrt(total)
        k = info.k[l]
        q = min(len(so), k, r[l] + 2)
        tol = 6 * U64 * (2048 * k + k * (k + 1)) * so[0] ** 2
        assert np.all(np.abs(sig[l][:q] ** 2 - so[:q] ** 2) <= tol + 1e-14 * so[:q] ** 2), l
        assert info.tail[l] ** 2 <= thr * (1 + 1e-9)
        Z = res.Z[l][:, : r[l]].cpu().double().numpy()
        Zs.append(Z)
        assert np.abs(Z.T @ Z - np.eye(r[l])).max() <= zt
        V = res.V[l][: r[l], :].cpu().numpy()
        for nu in np.random.default_rng(3 + l).choice(cp.U[l].shape[1], size=32, replace=False):
            u = cp.U[l][:, nu] / np.linalg.norm(cp.U[l][:, nu])
            assert np.abs(V[:, nu] - Z.T @ u).max() <= zt, (l, nu)
    beta = res.beta[: r[0] * r[1] * r[2]].cpu().double().numpy().reshape(r, order="F")
    beta_o, Z_o = orc.at(r)
    d = tu.tucker_rel_diff(beta, Zs, beta_o, Z_o)
    print(f"newton n=2048 R=20000 precision={precision} fp32={out_fp32}: ||T_gpu - T_oracle|| / ||T_oracle|| = {d:.3e}")
    assert d <= TUCKER_TOL, d
