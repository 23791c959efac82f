"""CPU reference of the Tucker-to-canonical transform (T2C) and of the canonical-to-canonical
reduction C2C = C2T followed by T2C (test infrastructure only: tests/ and bench.py's CPU legs).
Plain numpy in FP64, written from the paper's remark on reducing the canonical rank of a
Tucker core (Sec. 2.4, Remark rem_can_red, eqs. T2C_slice, T2C_SVD, beta_R); numpy's SVD
serves as the slice SVD.  Nothing here is used by the CUDA library.

The remark, for a core beta of size r1 x r2 x r3 (slices along the third mode):
  beta = sum_m B_m (x) z_m, B_m = beta(:, :, m), z_m the m-th unit vector (eq. T2C_slice);
  each B_m is cut to its singular values above a threshold delta (p_m of them, eq. T2C_SVD);
  beta_R = sum_m B_{p_m} (x) z_m (eq. beta_R), canonical rank R = sum_m p_m <= r3 min(r1, r2),
  and ||beta - beta_R|| <= sum_m ||B_m - B_{p_m}||.
Reading of the threshold (the remark states eps / r^{3/2} for an r x r x r core with an absolute
eps): delta = eps ||beta||_F / (r3 sqrt(min(r1, r2))), so that every slice drops at most
min(r1, r2) values below delta and the remark's bound becomes ||beta - beta_R|| <= eps ||beta||.
A singular value at or below the slice's FP64 resolution min(r1, r2) u ||B_m||_F counts as zero
(also for eps = 0): it is rounding, not a direction of the slice.
The canonical factors of the whole tensor A = beta x_1 Z1 x_2 Z2 x_3 Z3 are
  xi_(m,k) = sigma_k(B_m),  u1 = Z1 u_k,  u2 = Z2 v_k,  u3 = Z3(:, m).
"""
import numpy as np

import oracle


def threshold(beta, eps):
    """delta = eps ||beta||_F / (r3 sqrt(min(r1, r2)))."""
    r1, r2, r3 = beta.shape
    if min(r1, r2, r3) == 0:
        return 0.0
    return float(eps) * float(np.linalg.norm(beta)) / (r3 * np.sqrt(min(r1, r2)))


def t2c_core(beta, eps):
    """Slice SVDs of the core.  Returns dict(delta, p (list), sigma, U, V (lists per slice, the
    kept p_m columns), R)."""
    beta = np.asarray(beta, dtype=np.float64)
    r1, r2, r3 = beta.shape
    delta = threshold(beta, eps)
    out = dict(delta=delta, p=[], sigma=[], U=[], V=[])
    for m in range(r3):
        Bm = beta[:, :, m]
        U, s, Vt = np.linalg.svd(Bm, full_matrices=False)
        floor = min(r1, r2) * np.finfo(np.float64).eps * float(np.linalg.norm(Bm))
        p = int(np.sum(s > max(delta, floor)))
        out["p"].append(p)
        out["sigma"].append(s[:p].copy())
        out["U"].append(U[:, :p].copy())
        out["V"].append(Vt[:p].T.copy())
    out["R"] = int(sum(out["p"]))
    return out


def beta_from_slices(res, shape):
    """beta_R = sum_m (sum_k sigma_k u_k v_k^T) (x) z_m."""
    r1, r2, r3 = shape
    b = np.zeros(shape)
    for m in range(r3):
        if res["p"][m]:
            b[:, :, m] = (res["U"][m] * res["sigma"][m]) @ res["V"][m].T
    return b


def t2c(Z, beta, eps):
    """Canonical factors (U1, U2, U3 each n_l x R, column-major) and weights xi of the Tucker
    tensor (Z, beta), plus the slice data of t2c_core."""
    res = t2c_core(beta, eps)
    R = res["R"]
    cols1, cols2, cols3, xi = [], [], [], []
    for m in range(beta.shape[2]):
        for k in range(res["p"][m]):
            cols1.append(Z[0] @ res["U"][m][:, k])
            cols2.append(Z[1] @ res["V"][m][:, k])
            cols3.append(Z[2][:, m].copy())
            xi.append(res["sigma"][m][k])
    shp = [z.shape[0] for z in Z]
    U = [np.asfortranarray(np.stack(c, axis=1)) if R else np.zeros((shp[l], 0)) for l, c in enumerate((cols1, cols2, cols3))]
    res.update(U_can=U, xi_can=np.array(xi))
    return res


def c2c(U, xi, eps_tucker, eps_t2c, **kw):
    """The canonical-to-canonical reduction: RHOSVD (oracle.c2t) then T2C of its Tucker tensor."""
    tk = oracle.c2t(U, xi, eps=eps_tucker, **kw)
    res = t2c(tk["Z"], tk["beta"], eps_t2c)
    res["tucker"] = tk
    return res


def full_from_cp(U, xi):
    """The full n1 x n2 x n3 tensor of a canonical representation (small n only)."""
    return np.einsum("k,ik,jk,mk->ijm", np.asarray(xi), U[0], U[1], U[2])
