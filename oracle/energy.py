"""CPU reference of the interaction energy from the long-range part of a range-separated (RS)
collective potential (test infrastructure only: tests/ and bench.py's CPU legs).  Plain numpy in
FP64, written from the paper's energy lemma (Sec. 4.2, Lemma lem:InterEnergy, eqs.
inter_energy, EnergyFree_Tensor).  Nothing here is used by the CUDA library.

For N charges z_j at grid nodes x_j and the collective long-range potential tensor
P_l = sum_j z_j W_j P_{R_l} (P_{R_l} the long-range part of the reference Newton kernel, W_j its
shift to x_j), given as a canonical tensor (U, xi) of any rank (the generated N R_l terms or a
rank-reduced version):
    p_l(j) = P_l(x_j) = sum_k xi_k U1[i1_j, k] U2[i2_j, k] U3[i3_j, k]   (a sample of the CP tensor)
    E_N = 1/2 <z, p_l> - 1/2 P_{R_l}(0) sum_j z_j^2                     (eq. EnergyFree_Tensor)
in O(R N).  It equals sum_{i<j} z_i z_j P_{R_l}(x_i - x_j) exactly when P_l is the unreduced sum,
and the Coulomb energy sum_{i<j} z_i z_j / |x_i - x_j| (eq. inter_energy) when the short-range
Gaussians have decayed at the smallest distance and the quadrature is accurate there.
"""
import numpy as np


def cp_sample(U, xi, idx):
    """Entries of the canonical tensor at grid index triples idx (N x 3): sum over the terms of
    xi_k times the three factor entries, one term at a time."""
    idx = np.asarray(idx)
    xi = np.asarray(xi, dtype=np.float64)
    out = np.zeros(idx.shape[0])
    for k in range(xi.shape[0]):
        out += xi[k] * U[0][idx[:, 0], k] * U[1][idx[:, 1], k] * U[2][idx[:, 2], k]
    return out


def energy_from_samples(p, z, p0):
    """E_N = 1/2 <z, p> - 1/2 p0 sum z^2 (eq. EnergyFree_Tensor)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * float(np.dot(z, p)) - 0.5 * float(p0) * float(np.dot(z, z))


def energy_lemma(U, xi, idx, z, p0):
    return energy_from_samples(cp_sample(U, xi, idx), z, p0)


def pair_sum(coords, z, kernel):
    """sum_{i<j} z_i z_j kernel(x_i - x_j) by direct O(N^2) summation, row by row."""
    coords = np.asarray(coords, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    E = 0.0
    for i in range(1, coords.shape[0]):
        d = coords[:i] - coords[i]
        E += z[i] * float(np.dot(z[:i], kernel(d)))
    return E


def long_range_kernel(t, p):
    """P_{R_l}(d) = sum_k p_k exp(-t_k^2 |d|^2), the reference kernel's long-range part at the
    continuous offset d (rows of an (M, 3) array)."""
    t = np.asarray(t)
    p = np.asarray(p)

    def f(d):
        r2 = np.sum(d * d, axis=1)
        return np.exp(-np.outer(r2, t * t)) @ p
    return f


def coulomb(d):
    return 1.0 / np.sqrt(np.sum(d * d, axis=1))
