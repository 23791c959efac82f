"""numpy helpers for tests: full tensors, Tucker reconstruction, the Tucker-difference
metric and a reference HOSVD.  Independent of both the oracle and the CUDA library."""
from __future__ import annotations

import numpy as np


def full_from_cp(U, xi):
    """A(i,j,m) = sum_nu xi_nu U1(i,nu) U2(j,nu) U3(m,nu)  (small n only)."""
    return np.einsum("n,in,jn,mn->ijm", np.asarray(xi), U[0], U[1], U[2], optimize=True)


def tucker_full(beta, Z):
    """beta x_1 Z1 x_2 Z2 x_3 Z3 (small n only)."""
    return np.einsum("abc,ia,jb,mc->ijm", beta, Z[0], Z[1], Z[2], optimize=True)


def mode_apply(beta, M, mode):
    """beta x_mode M  (M: new_dim x old_dim)."""
    out = np.tensordot(M, beta, axes=([1], [mode]))
    return np.moveaxis(out, 0, mode)


def tucker_rel_diff(beta_a, Z_a, beta_b, Z_b):
    """||T_a - T_b||_F / ||T_b||_F for Tucker tensors with orthonormal factors, without
    forming n^3: per mode an orthonormal basis P of span[Z_a Z_b], then compare the
    cores expressed in P (the (ra+rb)^3 space)."""
    ca, cb = np.asarray(beta_a), np.asarray(beta_b)
    for l in range(3):
        P, _ = np.linalg.qr(np.hstack([Z_a[l], Z_b[l]]))
        ca = mode_apply(ca, P.T @ Z_a[l], l)
        cb = mode_apply(cb, P.T @ Z_b[l], l)
    den = np.linalg.norm(cb)
    num = np.linalg.norm(ca - cb)
    return num / den if den > 0 else num


def unfold(A, mode):
    return np.moveaxis(A, mode, 0).reshape(A.shape[mode], -1)


def hosvd(A, ranks):
    """Truncated HOSVD of a full tensor via LAPACK SVDs of its unfoldings."""
    Z = []
    for l in range(3):
        u, s, _ = np.linalg.svd(unfold(A, l), full_matrices=False)
        Z.append(u[:, : ranks[l]])
    core = A
    for l in range(3):
        core = mode_apply(core, Z[l].T, l)
    return core, Z
