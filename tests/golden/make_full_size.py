"""Writes the oracle's results for the full-size workloads: per mode the singular values of the
normalised side matrix (leading NSIG of them), the eps-rank (Thm. 2.3 reading: relative
Frobenius tail), the tail at that rank, the total energy, the number of kept terms and
||xi'|| (``<case>.json``), and the oracle's leading left singular vectors of eq. SVD_Ul,
ZEXTRA more than the eps-rank (n x (r_l + ZEXTRA), ``<case>_Z.npz``, float64), so that a GPU rank
one off at a threshold tie is compared with the oracle truncated at the GPU's rank.  From the stored Z the GPU tests
rebuild the oracle's V^(l) = Z^(l)T U~^(l) and core beta (Prop. 2.2) with the oracle's own loops
and compare the GPU's Tucker tensor with the oracle's element by element
(tests/test_gpu_full_size.py).  Calls only oracle/ and the seeded generators of workloads.py.

    python tests/golden/make_full_size.py hadamard_n1024_R64x64_eps1e-7     (about a minute)
    python tests/golden/make_full_size.py newton_n2048_N1000_eps1e-6        (tens of minutes)

The three modes' SVDs run in three spawned processes (the oracle's code unchanged, one mode a
process).
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle      # noqa: E402
import workloads   # noqa: E402

NSIG = 512
ZEXTRA = 4
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


def normalised(c):
    U, xi = build_cp(c)
    return oracle.normalize(U, xi)


def mode_svd(args):
    """One mode of the oracle's RHOSVD: the full SVD of the normalised side matrix, its eps-rank
    and the leading r_l left singular vectors."""
    name, l = args
    c = CASES[name]
    t0 = time.time()
    Un, _, _, _ = normalised(c)
    sig, Z = oracle.side_svd(Un[l])
    r = oracle.eps_rank(sig, c["eps"])
    return l, sig, np.ascontiguousarray(Z[:, : r + ZEXTRA]), r, time.time() - t0


def main(name):
    c = CASES[name]
    t0 = time.time()
    Un, xin, _, keep = normalised(c)
    out = dict(case=name, params=c, kept=int(keep.sum()), xi_norm=float(np.linalg.norm(xin)),
               ranks=[0] * 3, tails=[0.0] * 3, total=[0.0] * 3, sigma=[None] * 3)
    Zs = [None] * 3
    with mp.get_context("spawn").Pool(3) as pool:
        for l, sig, Z, r, dt in pool.imap_unordered(mode_svd, [(name, l) for l in range(3)]):
            out["ranks"][l] = r
            out["tails"][l] = float(np.sqrt(np.sum(sig[r:] ** 2)))
            out["total"][l] = float(np.sum(sig ** 2))
            out["sigma"][l] = [float(x) for x in sig[:NSIG]]
            Zs[l] = Z
            print(f"mode {l}: r = {r}, tail = {out['tails'][l]:.6e}, {dt:.1f} s", flush=True)
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, f"{name}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    zpath = os.path.join(here, f"{name}_Z.npz")
    np.savez_compressed(zpath, Z0=Zs[0], Z1=Zs[1], Z2=Zs[2])
    print("wrote", path, zpath, f"{time.time() - t0:.1f} s")


if __name__ == "__main__":
    main(sys.argv[1])
