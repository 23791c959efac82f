"""CPU reference of the canonical-to-Tucker ALS refinement started from the RHOSVD (test
infrastructure only: tests/ and bench.py's CPU legs).  Plain numpy in FP64, written from the
paper's description of one ALS step for d = 3 (Sec. 2.2, after Def. 2.2, eq. can_A_Tuck_als and
Figure figs1:Can_Tuck): with the orthogonal factors of the other two modes fixed, contract the
canonical tensor with them,
    A_2 = xi x_1 (Z1^T U1) x_3 (Z3^T U3),
and take the best rank-r_2 subspace of its r1 r3 x n2 unfolding; likewise for every mode in
turn.  Numpy's SVD serves as that best rank-r SVD.  Nothing here is used by the CUDA library.

The mode-l unfolding of the contraction is, for the other modes m1 < m2,
    M_l = U_l diag(xi) (V_m2 (.) V_m1)^T,   V_m = Z_m^T U_m   (n_l x r_m1 r_m2; Khatri-Rao product),
its r_l leading left singular vectors are the new Z_l, and ||beta||^2 after the update is the sum
of the r_l largest squared singular values of M_l.  For orthonormal factors the Tucker error is
||A||^2 - ||beta||^2, so a sweep never increases it.  Ranks stay those of the RHOSVD start.
"""
import numpy as np

import oracle


def _kr(Va, Vb):
    """Columnwise Kronecker product: column nu = Vb[:, nu] (x) Va[:, nu] (rows j_a + r_a j_b)."""
    ra, R = Va.shape
    rb = Vb.shape[0]
    return (Vb[:, None, :] * Va[None, :, :]).reshape(ra * rb, R)


def unfolding(U, xi, Z, l):
    """M_l = U_l diag(xi) (V_m2 (.) V_m1)^T for the current factors Z (list of three)."""
    m1, m2 = [m for m in range(3) if m != l]
    V1 = Z[m1].T @ U[m1]
    V2 = Z[m2].T @ U[m2]
    return (U[l] * xi) @ _kr(V1, V2).T


def core(U, xi, Z):
    """beta(i, j, m) = sum_nu xi_nu V1(i, nu) V2(j, nu) V3(m, nu), V_l = Z_l^T U_l."""
    V = [Z[l].T @ U[l] for l in range(3)]
    return np.einsum("n,in,jn,mn->ijm", xi, V[0], V[1], V[2])


def als(U, xi, Z0, sweeps=1):
    """ALS sweeps (modes 0, 1, 2 in turn) from the start factors Z0.  Returns dict(Z, beta,
    energy): energy[0] = ||beta||^2 of the start, then one value after every mode update."""
    U = [np.asarray(u, dtype=np.float64) for u in U]
    xi = np.asarray(xi, dtype=np.float64)
    Z = [np.asarray(z, dtype=np.float64).copy() for z in Z0]
    energy = [float(np.sum(core(U, xi, Z) ** 2))]
    for _ in range(sweeps):
        for l in range(3):
            r = Z[l].shape[1]
            if r == 0:
                energy.append(energy[-1])
                continue
            M = unfolding(U, xi, Z, l)
            W, s, _ = np.linalg.svd(M, full_matrices=False)
            Z[l] = np.asfortranarray(W[:, :r])
            energy.append(float(np.sum(s[:r] ** 2)))
    return dict(Z=Z, beta=core(U, xi, Z), energy=energy)


def c2t_als(U, xi, eps, sweeps=1, **kw):
    """RHOSVD (oracle.c2t) for the ranks and the start, then ALS sweeps."""
    tk = oracle.c2t(U, xi, eps=eps, **kw)
    res = als(U, xi, tk["Z"], sweeps)
    res["rhosvd"] = tk
    return res
