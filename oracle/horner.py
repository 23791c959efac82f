"""CPU reference of the polynomial of a canonical tensor evaluated by the Horner scheme with a
rank reduction after every product (test infrastructure only: tests/ and bench.py's CPU legs).
Plain numpy in FP64, written from the paper's section on Green's kernels (Sec. 5, the
tensor-valued polynomial P(A) and its Horner form), with the products of Sec. 3 (eq. rho_ten)
and the canonical-to-canonical reduction of Sec. 2.4 (oracle.t2c.c2c).  Nothing here is used by
the CUDA library.

For a canonical tensor A and coefficients a_0..a_n (Hadamard products, I the all-ones tensor):
    P(A) = a_0 I + a_1 A + ... + a_n A^n = a_0 + A (a_1 + A (a_2 + ... + A (a_{n-1} + a_n A)...)).
Reading of "n applications of RHOSVD": start from Y_n = a_n I (rank one) and for k = n-1..0
    Y_k = C2C( A (.) Y_{k+1} + a_k I ),
one Hadamard product and one reduction per degree, the constant joined as a rank-one term
(omitted when a_k = 0).  Trailing zero coefficients are dropped first (the degree is that of the
last nonzero a_k); the zero polynomial has rank 0.  If the exact Y_k are Y*_k, the error
obeys Y_k - Y*_k = A (.) (Y_{k+1} - Y*_{k+1}) + E_k, E_k the reduction error of step k, so
    ||Y_0 - P(A)||_F <= sum_k max|A|^k ||E_k||_F.
"""
import numpy as np

import oracle
from oracle import t2c as ot


def _ones_term(n, a):
    return [np.ones((n[l], 1), order="F") for l in range(3)], np.array([float(a)])


def degree(coeffs):
    """Index of the last nonzero coefficient, -1 for the zero polynomial."""
    c = np.asarray(coeffs, dtype=np.float64)
    nz = np.nonzero(c)[0]
    return int(nz[-1]) if nz.size else -1


def horner(U, xi, coeffs, eps_tucker, eps_t2c, r_max=None, keep_steps=False):
    """P(A) as a canonical tensor.  Returns dict(U, xi, R, steps) where steps[j] (j = 0 for the
    first reduction, k = n-1) holds R_in (rank entering the reduction), ranks (Tucker r_l) and R
    (canonical rank after T2C); with keep_steps the step's input factors and result too."""
    U = [np.asfortranarray(u, dtype=np.float64) for u in U]
    xi = np.asarray(xi, dtype=np.float64)
    c = np.asarray(coeffs, dtype=np.float64)
    n = [u.shape[0] for u in U]
    deg = degree(c)
    if deg < 0:
        return dict(U=[np.zeros((n[l], 0)) for l in range(3)], xi=np.zeros(0), R=0, steps=[])
    YU, Yx = _ones_term(n, c[deg])
    steps = []
    for k in range(deg - 1, -1, -1):
        PU, Px = oracle.cp_hadamard(U, xi, YU, Yx)               # A (.) Y_{k+1}
        if c[k] != 0.0:
            OU, Ox = _ones_term(n, 1.0)
            PU, Px = oracle.cp_sum(1.0, PU, Px, c[k], OU, Ox)    # + a_k I
        kw = {} if r_max is None else dict(r_max=r_max)
        res = ot.c2c(PU, Px, eps_tucker, eps_t2c, **kw)
        YU, Yx = res["U_can"], res["xi_can"]
        st = dict(k=k, R_in=int(Px.shape[0]), ranks=list(res["tucker"]["ranks"]), R=int(res["R"]))
        if keep_steps:
            st.update(U_in=PU, xi_in=Px, U=YU, xi=Yx)
        steps.append(st)
    return dict(U=YU, xi=Yx, R=int(Yx.shape[0]), steps=steps)


def power_direct(U, xi, m, eps_tucker, eps_t2c, r_max=None):
    """A^m by m-1 exact Hadamard products (rank R^m) and one C2C reduction (the paper's
    P^(3) = P (.) P (.) P example, Sec. 5)."""
    PU, Px = [np.asfortranarray(u, dtype=np.float64) for u in U], np.asarray(xi, dtype=np.float64)
    for _ in range(m - 1):
        PU, Px = oracle.cp_hadamard(PU, Px, U, xi)
    kw = {} if r_max is None else dict(r_max=r_max)
    res = ot.c2c(PU, Px, eps_tucker, eps_t2c, **kw)
    res["R_in"] = int(Px.shape[0])
    return res
