"""Host logic of bench.py's CPU legs: the three-process timing of the oracle (one mode a spawned
worker) gives the ranks the single-process oracle gives, on a small Hadamard product."""
import numpy as np

import bench
import oracle
import workloads


def test_parallel_modes_match_the_single_process_oracle():
    A, B = workloads.hartree_like_factors(48, 6, 5, [3, 4])
    Uc, xc = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    Un, _, _, _ = oracle.normalize(Uc, xc)
    ranks = [oracle.eps_rank(oracle.side_svd(np.asfortranarray(Un[l]))[0], bench.WORKLOAD["eps"])
             for l in range(3)]
    par = bench.oracle_parallel_modes((Un, 0.0, 0.0))
    assert par["ranks"] == ranks
    assert par["cores"] == 3 and par["kind"] == "oracle" and par["value"] > 0
