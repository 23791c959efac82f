"""Host logic of bench.py's CPU legs, on a small Hadamard product: the reference arm's steps
(oracle_pieces) together perform one whole oracle reduction, and the all-cores CPU baseline
(oracle_full_threads) gives the same reduction; both against oracle.c2t on the same input (the
core summed over term slices differs from the one-pass loops only by rounding)."""
import numpy as np
import pytest

import bench
import oracle
import workloads
from tests import tensor_utils as tu

SMALL = dict(bench.WORKLOAD, n=48, Ra=6, Rb=5, seeds=[3, 4])


@pytest.fixture(scope="module")
def reference():
    A, B = workloads.hartree_like_factors(48, 6, 5, [3, 4])
    Uc, xc = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    return oracle.c2t(Uc, xc, eps=SMALL["eps"])


@pytest.mark.parametrize("nsteps", [1, 3, 6, 9])
def test_reference_steps_make_one_whole_reduction(reference, nsteps):
    steps, st = bench.oracle_pieces(nsteps, SMALL)
    assert len(steps) == nsteps
    for f in steps:
        f()
    assert st["r"] == reference["ranks"]
    assert np.abs(st["beta"] - reference["beta"]).max() <= 1e-12 * np.abs(reference["beta"]).max()
    assert tu.tucker_rel_diff(st["beta"], st["Z"], reference["beta"], reference["Z"]) <= 1e-13


def test_threaded_full_reduction_matches(reference):
    res = bench.oracle_full_threads(4, SMALL)
    assert res["ranks"] == reference["ranks"]
    assert tu.tucker_rel_diff(res["beta"], res["Z"], reference["beta"], reference["Z"]) <= 1e-13
    assert res["wall"] > 0 and res["busy"] > 0
    assert bench.tucker_rel_diff_np(res["beta"], res["Z"], reference["beta"], reference["Z"]) <= 1e-13


def test_oracle_threads_matches_single_call():
    cp = workloads.gaussian_sum(40, 90, 2)
    a = oracle.c2t(cp.U, cp.xi, eps=1e-6)
    b = oracle.c2t_threads(cp.U, cp.xi, eps=1e-6)
    assert a["ranks"] == b["ranks"] and a["kept"] == b["kept"]
    assert np.array_equal(a["beta"], b["beta"])
    assert all(np.array_equal(a["sigma"][l], b["sigma"][l]) for l in range(3))
