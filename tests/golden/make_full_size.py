"""Writes the oracle's results for the full-size workloads: per mode the singular values of the
normalised side matrix (leading NSIG of them), the eps-rank (Thm. 2.3 reading: relative
Frobenius tail), the tail at that rank, the total energy, the number of kept terms and
||xi'||.  The GPU full-size parity tests (tests/test_gpu_full_size.py) compare against these
files.  Calls only oracle/ and the seeded generators of workloads.py.

    python tests/golden/make_full_size.py hadamard_n1024_R64x64_eps1e-7     (about a minute)
    python tests/golden/make_full_size.py newton_n2048_N1000_eps1e-6        (tens of minutes)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle      # noqa: E402
import workloads   # noqa: E402

NSIG = 512
CASES = {
    "hadamard_n1024_R64x64_eps1e-7": dict(kind="hadamard", n=1024, Ra=64, Rb=64, seeds=[0, 1], eps=1e-7),
    "newton_n2048_N1000_eps1e-6": dict(kind="newton", n=2048, N=1000, seed=0, eps=1e-6),
}


def build_cp(c):
    """The canonical input of a case, as the GPU tests build it (Hadamard through the oracle's
    own product, bit-identical to the library's)."""
    if c["kind"] == "hadamard":
        A, B = workloads.hartree_like_factors(c["n"], c["Ra"], c["Rb"], tuple(c["seeds"]))
        return oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
    cp = workloads.newton_long_range_sum(n=c["n"], N=c["N"], seed=c["seed"])
    return cp.U, cp.xi


def main(name):
    c = CASES[name]
    t0 = time.time()
    U, xi = build_cp(c)
    Un, xin, _, keep = oracle.normalize(U, xi)
    out = dict(case=name, params=c, kept=int(keep.sum()), xi_norm=float(np.linalg.norm(xin)),
               ranks=[], tails=[], total=[], sigma=[])
    for l in range(3):
        sig, _ = oracle.side_svd(Un[l])
        r = oracle.eps_rank(sig, c["eps"])
        out["ranks"].append(r)
        out["tails"].append(float(np.sqrt(np.sum(sig[r:] ** 2))))
        out["total"].append(float(np.sum(sig ** 2)))
        out["sigma"].append([float(x) for x in sig[:NSIG]])
        print(f"mode {l}: r = {r}, tail = {out['tails'][-1]:.6e}, {time.time() - t0:.1f} s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1])
