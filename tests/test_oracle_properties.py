"""Property tests of the oracles on random small inputs (hypothesis): the T2C error bound and
rank bound of Remark rem_can_red, the Horner evaluation with exact reductions against numpy's
polyval, the ALS monotonicity, the energy lemma against the direct pair sum, the RHOSVD error
bound of Thm. 2.3 with the projection identities, and the rank-growth operations (Hadamard
product, linear combination, normalisation) against the full tensors.  Each property is a fact
of the mathematics, independent of the oracle's code."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import workloads  # noqa: E402
from numpy.polynomial import polynomial as npoly  # noqa: E402
from oracle import als as oa  # noqa: E402
from oracle import energy as oe  # noqa: E402
from oracle import horner as oh  # noqa: E402
from oracle import t2c as ot  # noqa: E402

SET = settings(max_examples=15, deadline=None)


@SET
@given(r1=st.integers(1, 9), r2=st.integers(1, 9), r3=st.integers(1, 6), seed=st.integers(0, 10 ** 6),
       leps=st.floats(-12.0, -1.0))
def test_t2c_bounds(r1, r2, r3, seed, leps):
    g = np.random.default_rng(seed)
    beta = g.standard_normal((r1, r2, r3)) * np.exp(-g.uniform(0, 6, (r1, 1, 1)))
    eps = 10.0 ** leps
    res = ot.t2c_core(beta, eps)
    err = np.linalg.norm(beta - ot.beta_from_slices(res, beta.shape))
    assert err <= eps * np.linalg.norm(beta) * (1 + 1e-10) + 1e-14 * np.linalg.norm(beta)
    assert res["R"] <= r3 * min(r1, r2)


@SET
@given(R=st.integers(1, 3), deg=st.integers(0, 3), seed=st.integers(0, 10 ** 6))
def test_horner_exact_reductions(R, deg, seed):
    g = np.random.default_rng(seed)
    cp = workloads.gaussian_sum(8, R, seed % 1000, b=3.0, centre_box=1.5, a_range=(0.3, 2.0))
    coeffs = list(g.uniform(-2.0, 2.0, deg + 1))
    A = ot.full_from_cp(cp.U, cp.xi)
    res = oh.horner(cp.U, cp.xi, coeffs, 0.0, 0.0)
    ref = npoly.polyval(A, coeffs)
    got = ot.full_from_cp(res["U"], res["xi"]) if res["R"] else np.zeros_like(A)
    assert np.abs(got - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1.0)


@SET
@given(R=st.integers(5, 40), seed=st.integers(0, 10 ** 6), leps=st.floats(-6.0, -1.5))
def test_als_never_loses_energy(R, seed, leps):
    cp = workloads.gaussian_sum(10, R, seed % 1000)
    tk = __import__("oracle").c2t(cp.U, cp.xi, eps=10.0 ** leps)
    res = oa.als(cp.U, cp.xi, tk["Z"], sweeps=1)
    e = res["energy"]
    assert all(e[i + 1] >= e[i] * (1 - 1e-12) for i in range(len(e) - 1))


@SET
@given(L1=st.integers(1, 3), L2=st.integers(1, 3), L3=st.integers(1, 2), seed=st.integers(0, 10 ** 6))
def test_energy_lemma_is_the_pair_sum(L1, L2, L3, seed):
    cp = workloads.newton_lattice_long_range(n_cells=48, b=12.0, L=(L1, L2, L3), m=12, seed=seed % 1000)
    M = cp.meta
    E = oe.energy_lemma(cp.U, cp.xi, M["idx"], M["z"], M["p0"])
    Ep = oe.pair_sum(M["coords"], M["z"], oe.long_range_kernel(M["t"], M["p"])) if M["N"] > 1 else 0.0
    assert abs(E - Ep) <= 1e-12 * max(1.0, float(np.abs(M["z"]).sum()) ** 2)


@SET
@given(n=st.integers(3, 10), R=st.integers(1, 24), seed=st.integers(0, 10 ** 6), leps=st.floats(-9.0, -0.5),
       signed=st.booleans())
def test_c2t_bound_and_projection(n, R, seed, leps, signed):
    """Thm. 2.3 on random CP tensors: ||A - A0||_F <= ||xi'|| sum_l tau_l, and A0 is the
    orthogonal projection of A onto the Z bases (Pythagoras; the core is A x_l Z_l^T)."""
    import oracle
    from tests import tensor_utils as tu
    cp = workloads.random_cp(n, R, seed % 100000, signed=signed)
    out = oracle.c2t(cp.U, cp.xi, eps=10.0 ** leps)
    A = tu.full_from_cp(cp.U, cp.xi)
    nA = np.linalg.norm(A)
    T = tu.tucker_full(out["beta"], out["Z"]) if min(out["ranks"]) > 0 else np.zeros_like(A)
    err = np.linalg.norm(A - T)
    assert err <= out["xi_norm"] * sum(out["tails"]) * (1 + 1e-10) + 1e-12 * max(nA, 1.0)
    assert abs(nA ** 2 - np.linalg.norm(out["beta"]) ** 2 - err ** 2) <= 1e-10 * max(nA ** 2, 1.0)
    for l in range(3):
        Z = out["Z"][l]
        assert np.allclose(Z.T @ Z, np.eye(Z.shape[1]), atol=1e-12)


@SET
@given(n=st.integers(2, 8), Ra=st.integers(1, 6), Rb=st.integers(1, 6), seed=st.integers(0, 10 ** 6),
       alpha=st.floats(-3.0, 3.0), beta=st.floats(-3.0, 3.0))
def test_rank_growth_ops_on_full_tensors(n, Ra, Rb, seed, alpha, beta):
    """Hadamard product and linear combination of CP tensors equal the entrywise product and
    the combination of the full tensors; normalisation leaves the full tensor unchanged."""
    import oracle
    from tests import tensor_utils as tu
    a = workloads.random_cp(n, Ra, seed % 100000)
    b = workloads.random_cp(n, Rb, (seed + 1) % 100000)
    A, B = tu.full_from_cp(a.U, a.xi), tu.full_from_cp(b.U, b.xi)
    Uh, xh = oracle.cp_hadamard(a.U, a.xi, b.U, b.xi)
    assert np.allclose(tu.full_from_cp(Uh, xh), A * B, rtol=0, atol=1e-12 * max(np.abs(A * B).max(), 1.0))
    Us, xs = oracle.cp_sum(alpha, a.U, a.xi, beta, b.U, b.xi)
    C = alpha * A + beta * B
    assert np.allclose(tu.full_from_cp(Us, xs), C, rtol=0, atol=1e-12 * max(np.abs(C).max(), 1.0))
    Un, xin, norms, keep = oracle.normalize(a.U, a.xi)
    assert np.allclose(tu.full_from_cp(Un, xin), A, rtol=0, atol=1e-12 * max(np.abs(A).max(), 1.0))
    for l in range(3):
        nz = np.linalg.norm(Un[l], axis=0)
        assert np.allclose(nz[keep.astype(bool)], 1.0, atol=1e-14)
