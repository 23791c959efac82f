"""Seeded synthetic canonical (CP) tensors for RHOSVD.

This module only *generates inputs*: factor matrices U^(l) (n_l x R, column-major,
FP64) and weights xi (length R) of a d=3 canonical tensor
A = sum_k xi_k u1_k (x) u2_k (x) u3_k (paper Sec. 2.1, eq. can_A3).  It holds none
of the RHOSVD arithmetic; both the CPU oracle (``oracle/``) and the CUDA library
consume what it returns.

Grid (paper Sec. 3 collocation at the interval midpoints, Sec. 4.1 mesh h=2b/n):
cell centres x_i = -b + (i - 1/2) h, h = 2b/n, i = 1..n.  Factor columns are the
Gaussians sampled at those points (collocation).

Random numbers come from numpy's PCG64 generator seeded with the stated seed;
every draw below is listed in the order it is made, so a workload is fully fixed
by (recipe, seed).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class CP:
    """A d=3 canonical tensor: U[l] is (n_l, R) Fortran-ordered float64, xi is (R,)."""

    U: list
    xi: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return [u.shape[0] for u in self.U]

    @property
    def R(self):
        return int(self.xi.shape[0])


def grid(n: int, b: float) -> np.ndarray:
    """Cell-centre grid on [-b, b] with h = 2b/n."""
    h = 2.0 * b / n
    return -b + (np.arange(n, dtype=np.float64) + 0.5) * h


def gaussian_columns(x: np.ndarray, centres: np.ndarray, expo: np.ndarray) -> np.ndarray:
    """Column k = exp(-expo_k (x - centre_k)^2) sampled on x; (n, R) Fortran order."""
    d = x[:, None] - centres[None, :]
    return np.asfortranarray(np.exp(-expo[None, :] * d * d))


def gaussian_sum(n: int, R: int, seed: int, b: float = 10.0, centre_box: float = 5.0,
                 a_range=(0.5, 20.0), c_range=(0.1, 1.0)) -> CP:
    """Sum of R isotropic Gaussians c_k exp(-a_k |x - x_k|^2) on an n^3 grid.

    Draw order with PCG64(seed): centres (R,3) uniform in [-centre_box, centre_box],
    then log a_k uniform in [log a_lo, log a_hi], then c_k uniform in c_range.
    The 3D Gaussian separates: u_k^(l)(i) = exp(-a_k (x_i - x_{k,l})^2), xi_k = c_k.
    """
    g = np.random.default_rng(seed)
    centres = g.uniform(-centre_box, centre_box, size=(R, 3))
    a = np.exp(g.uniform(math.log(a_range[0]), math.log(a_range[1]), size=R))
    c = g.uniform(c_range[0], c_range[1], size=R)
    x = grid(n, b)
    U = [gaussian_columns(x, centres[:, l].copy(), a) for l in range(3)]
    return CP(U=U, xi=c.astype(np.float64),
              meta=dict(kind="gaussian_sum", n=n, R=R, seed=seed, b=b,
                        centres=centres, a=a))


def gaussian_sum_params(n: int, R: int, seed: int, b: float = 10.0, centre_box: float = 5.0,
                        a_range=(0.5, 20.0), c_range=(0.1, 1.0)):
    """The random parameters of gaussian_sum(n, R, seed) in the same draw order, without the
    factor columns: (grid x, centres (R,3), exponents a (R,), weights c (R,)).  The columns
    are u_k^(l)(i) = exp(-a_k (x_i - centres[k, l])^2); large batches evaluate them on the
    device."""
    g = np.random.default_rng(seed)
    centres = g.uniform(-centre_box, centre_box, size=(R, 3))
    a = np.exp(g.uniform(math.log(a_range[0]), math.log(a_range[1]), size=R))
    c = g.uniform(c_range[0], c_range[1], size=R)
    return grid(n, b), centres, a, c


def newton_sinc_nodes(h: float = 0.4, k_lo: int = -19, k_hi: int = 0):
    """Quadrature nodes/weights for 1/z = (2/sqrt(pi)) int_0^inf exp(-z^2 t^2) dt.

    With t = e^u the integrand becomes (2/sqrt(pi)) e^u exp(-z^2 e^{2u}); the step-h
    trapezoid (sinc) rule gives t_k = e^{k h}, p_k = (2/sqrt(pi)) h e^{k h}
    (paper Sec. 4.1, eqs. laplace, sinc_Newt, Laplace_Newton).  The long-range part
    keeps t_k <= 1, i.e. k <= 0 (eq. RS_repres).
    """
    k = np.arange(k_lo, k_hi + 1, dtype=np.float64)
    t = np.exp(k * h)
    p = (2.0 / math.sqrt(math.pi)) * h * np.exp(k * h)
    return t, p


def newton_long_range_sum(n: int = 2048, N: int = 1000, seed: int = 0, b: float = 10.0,
                          centre_box: float = 8.0, h: float = 0.4, k_lo: int = -19,
                          k_hi: int = 0) -> CP:
    """Collective long-range Newton potential of N unit charges.

    Each centre x_j carries the long-range Gaussians of the sinc-quadrature Newton
    kernel: p_k exp(-t_k^2 |x - x_j|^2), k = k_lo..k_hi (t_k <= 1).  R = N (k_hi-k_lo+1).
    Draw order with PCG64(seed): centres (N,3) uniform in [-centre_box, centre_box].
    Term index nu = j * M + (k - k_lo), M = k_hi - k_lo + 1.
    """
    g = np.random.default_rng(seed)
    centres = g.uniform(-centre_box, centre_box, size=(N, 3))
    t, p = newton_sinc_nodes(h, k_lo, k_hi)
    M = t.shape[0]
    x = grid(n, b)
    expo = np.tile(t * t, N)
    U = []
    for l in range(3):
        cen = np.repeat(centres[:, l], M)
        U.append(gaussian_columns(x, cen, expo))
    xi = np.tile(p, N).astype(np.float64)
    return CP(U=U, xi=xi, meta=dict(kind="newton_long_range", n=n, N=N, seed=seed, b=b,
                                    h=h, k_lo=k_lo, k_hi=k_hi, centres=centres))


def batched_gaussian_sums(count: int = 512, seed0: int = 0, n_choices=(128, 256, 512, 1024),
                          R_range=(100, 8000)):
    """Shapes and seeds of the batched workload: member i uses seed seed0+i.

    Draw order with PCG64(seed0 + 10**6): n_i uniform over n_choices, then
    R_i = round(exp(uniform(log R_lo, log R_hi))).  Returns a list of (n, R, seed).
    """
    g = np.random.default_rng(seed0 + 10**6)
    ns = g.choice(np.asarray(n_choices), size=count)
    Rs = np.rint(np.exp(g.uniform(math.log(R_range[0]), math.log(R_range[1]), size=count)))
    return [(int(ns[i]), int(Rs[i]), seed0 + i) for i in range(count)]


def learned_instances(count: int, first_seed: int, n: int = 1024, R_range=(2000, 8000)):
    """Shapes and seeds of the learned-proposal workload: instance i uses seed first_seed + i
    and R_i = round(exp(uniform(log R_lo, log R_hi))) drawn with PCG64([first_seed + i, 1]) (a
    stream apart from the instance's own Gaussian parameters).  Training uses first_seed = 10**6,
    held-out evaluation the seeds after the largest training set (10**6 + 20000 on).
    Returns a list of (n, R, seed)."""
    out = []
    for i in range(count):
        s = first_seed + i
        g = np.random.default_rng([s, 1])
        R = int(np.rint(np.exp(g.uniform(math.log(R_range[0]), math.log(R_range[1])))))
        out.append((int(n), R, s))
    return out


def tucker_tensor(n, r, seed, decay=0.15):
    """A seeded Tucker tensor (Z, beta) for the Tucker-to-canonical transform: Z_l (n_l x r_l)
    with orthonormal columns (QR of Gaussian matrices), and a core whose mode-3 slice m is
    A_m diag(s_m) B_m^T + noise, A_m, B_m random orthonormal, s_m(k) = exp(-decay k - 0.05 m)
    scaled by a uniform [0.5, 2] factor; noise 1e-3 of the smallest s_m.  Draw order with
    PCG64(seed): Z_1, Z_2, Z_3, then per slice A_m, B_m, the factor, the noise.
    Returns (Z list of column-major float64 arrays, beta (r1, r2, r3) array)."""
    g = np.random.default_rng(seed)
    Z = [np.asfortranarray(np.linalg.qr(g.standard_normal((n[l], r[l])))[0]) for l in range(3)]
    r1, r2, r3 = r
    q = min(r1, r2)
    beta = np.zeros((r1, r2, r3))
    for m in range(r3):
        A = np.linalg.qr(g.standard_normal((r1, q)))[0]
        B = np.linalg.qr(g.standard_normal((r2, q)))[0]
        s = np.exp(-decay * np.arange(q) - 0.05 * m) * g.uniform(0.5, 2.0)
        beta[:, :, m] = (A * s) @ B.T + 1e-3 * s[-1] * g.standard_normal((r1, r2))
    return Z, np.asfortranarray(beta)


def newton_kernel(n: int = 257, b: float = 10.0, M: int = 9, h: float = 0.7,
                  long_range: bool = False) -> CP:
    """The discretised Newton kernel 1/|x| as the R = 2M+1 term canonical tensor P_R of the
    sinc quadrature (Sec. 4.1, eqs. laplace, sinc_Newt, Laplace_Newton, galten_int,
    sinc_general): t_k = e^{k h}, p_k = (2/sqrt(pi)) h e^{k h}, k = -M..M, and the factor
    columns b_i(t_k) = cell average of exp(-t_k^2 x^2) over cell i of the n-cell grid on [-b, b]
    (piecewise-constant basis; with n odd the middle cell is centred on the singularity):
        b_i(t) = sqrt(pi) / (2 t h_x) [erf(t (x_i + h_x/2)) - erf(t (x_i - h_x/2))].
    All three modes share one factor matrix; the weights are xi_k = p_k.  long_range keeps the
    terms with t_k <= 1 (k <= 0, eq. RS_repres): R_l = M + 1.  No random draws."""
    from scipy.special import erf
    x = grid(n, b)
    hx = 2.0 * b / n
    k = np.arange(-M, (0 if long_range else M) + 1, dtype=np.float64)
    t = np.exp(k * h)
    p = (2.0 / math.sqrt(math.pi)) * h * t
    lo = (x - hx / 2)[:, None] * t[None, :]
    hi = (x + hx / 2)[:, None] * t[None, :]
    B = np.asfortranarray(math.sqrt(math.pi) / (2.0 * hx * t[None, :]) * (erf(hi) - erf(lo)))
    return CP(U=[B, B.copy(order="F"), B.copy(order="F")], xi=p.astype(np.float64),
              meta=dict(kind="newton_kernel", n=n, b=b, M=M, h=h, long_range=long_range))


def point_grid(n_cells: int, b: float) -> np.ndarray:
    """Collocation grid including the origin (Sec. 4.1, for continuous radial functions the mode
    size becomes n+1): x_i = -b + i 2b/n_cells, i = 0..n_cells."""
    return -b + np.arange(n_cells + 1, dtype=np.float64) * (2.0 * b / n_cells)


def lattice(n_cells: int, L, m: int):
    """Nodes of an L1 x L2 x L3 lattice centred on the origin with spacing m grid steps, on the
    grid of point_grid(n_cells, .) (m even or L odd keeps every node on a grid point).  Returns
    the (N, 3) grid indices, node j = j1 + L1 (j2 + L2 j3)."""
    c = n_cells // 2
    ax = [c + np.round((np.arange(L[l]) - (L[l] - 1) / 2.0) * m).astype(np.int64) for l in range(3)]
    I = np.stack(np.meshgrid(ax[0], ax[1], ax[2], indexing="ij"), axis=-1)
    I = I.transpose(2, 1, 0, 3).reshape(-1, 3)           # j1 fastest
    if I.min() < 0 or I.max() > n_cells:
        raise ValueError("lattice leaves the grid")
    return np.ascontiguousarray(I)


def slater_sinc_nodes(lam: float = 0.5, h: float = 1.56, k_lo: int = -2, k_hi: int = 2):
    """Gaussian exponents tau_k and weights p_k of the sinc rule for the Slater function
    exp(-lam |x|) = exp(-2 sqrt(alpha rho)), rho = |x|^2, alpha = lam^2 / 4, from its Laplace
    transform with weight sqrt(alpha/pi) tau^{-3/2} exp(-alpha/tau) (Sec. 4.3, eq.
    Slater_Laplace_tr, Lemma lem:sincSlater): tau = e^u, step h,
        tau_k = e^{k h},  p_k = h sqrt(alpha/pi) tau_k^{-1/2} exp(-alpha/tau_k).
    exp(-lam |x|) ~ sum_k p_k exp(-tau_k |x|^2).  Long range: tau_k <= 1 (k <= 0).  Defaults:
    R = 5 terms, R_l = 3 (k = -2..0), h from minimising the maximum error over |x| in [1, 20]
    at lam = 0.5 (about 4e-3)."""
    al = lam * lam / 4.0
    k = np.arange(k_lo, k_hi + 1, dtype=np.float64)
    tau = np.exp(k * h)
    p = h * math.sqrt(al / math.pi) * tau ** -0.5 * np.exp(-al / tau)
    return tau, p


def slater_amplitude(x, y, z, c1: float = 6.0, c2: float = 0.1):
    """F(x,y,z) = c1 cos(x + 2y + 4z) exp(-c2 sqrt(x^2 + 2y^2 + 4z^2)) (Sec. 4.4, eq. func2)."""
    return c1 * np.cos(x + 2 * y + 4 * z) * np.exp(-c2 * np.sqrt(x * x + 2 * y * y + 4 * z * z))


def multi_slater_long_range(n_cells: int = 384, b: float = 10.0, L=(4, 4, 4), m: int = 20, lam: float = 0.5,
                            h: float = 1.56, amplitudes: str = "random", seed: int = 0) -> CP:
    """Long-range part G_{N,l} = sum_j c_j W_j G_l of a sum of Slater functions placed on the nodes
    of an L1 x L2 x L3 lattice (Sec. 4.4, eq. Slater_interp_multi; Tables Tab:random_ranks and
    Tab:func_ranks): every node contributes the R_l long-range Gaussians of slater_sinc_nodes
    centred on it (collocation on point_grid(n_cells, b), nodes on grid points, so the shifted
    reference vectors are the Gaussians sampled at the grid).  Amplitudes c_j: "random" draws
    U[-5, 5] with PCG64(seed) in node order; "func" evaluates slater_amplitude at the node.
    Term index nu = j R_l + k.  R = N R_l."""
    x = point_grid(n_cells, b)
    idx = lattice(n_cells, L, m)
    N = idx.shape[0]
    tau, p = slater_sinc_nodes(lam, h)
    keep = tau <= 1.0
    tau, p = tau[keep], p[keep]
    Rl = tau.shape[0]
    if amplitudes == "random":
        c = np.random.default_rng(seed).uniform(-5.0, 5.0, size=N)
    elif amplitudes == "func":
        c = slater_amplitude(x[idx[:, 0]], x[idx[:, 1]], x[idx[:, 2]])
    else:
        raise ValueError(amplitudes)
    expo = np.tile(tau, N)
    U = [gaussian_columns(x, np.repeat(x[idx[:, l]], Rl), expo) for l in range(3)]
    xi = (np.repeat(c, Rl) * np.tile(p, N)).astype(np.float64)
    return CP(U=U, xi=xi, meta=dict(kind="multi_slater_long_range", n_cells=n_cells, b=b, L=tuple(L), m=m,
                                    lam=lam, h=h, amplitudes=amplitudes, seed=seed, N=N, R_l=Rl, idx=idx, c=c))


def newton_lattice_long_range(n_cells: int = 384, b: float = 24.0, L=(16, 16, 16), m: int = 24, h: float = 0.4,
                              k_lo: int = -19, seed: int = 0) -> CP:
    """Collective long-range Newton potential P_l = sum_j z_j W_j P_{R_l} of N = L1 L2 L3 charges on
    the nodes of a lattice (Sec. 4.2, eq. RS_repres; Lemma lem:InterEnergy): the long-range sinc
    Gaussians t_k <= 1 of newton_sinc_nodes(h, k_lo, 0) centred on every node, collocation on
    point_grid(n_cells, b).  Charges z_j ~ U[-1, 1] from PCG64(seed) in node order.  Term
    nu = j R_l + k, weight z_j p_k.  meta: idx (N x 3 grid indices), z, coords (N x 3), p0 =
    P_{R_l}(0) = sum_k p_k (the single reference kernel's long-range part at its centre)."""
    x = point_grid(n_cells, b)
    idx = lattice(n_cells, L, m)
    N = idx.shape[0]
    t, p = newton_sinc_nodes(h, k_lo, 0)
    Rl = t.shape[0]
    z = np.random.default_rng(seed).uniform(-1.0, 1.0, size=N)
    expo = np.tile(t * t, N)
    U = [gaussian_columns(x, np.repeat(x[idx[:, l]], Rl), expo) for l in range(3)]
    xi = (np.repeat(z, Rl) * np.tile(p, N)).astype(np.float64)
    coords = np.stack([x[idx[:, l]] for l in range(3)], axis=1)
    return CP(U=U, xi=xi, meta=dict(kind="newton_lattice_long_range", n_cells=n_cells, b=b, L=tuple(L), m=m, h=h,
                                    k_lo=k_lo, seed=seed, N=N, R_l=Rl, idx=idx, z=z, coords=coords,
                                    p0=float(p.sum()), t=t, p=p))


# Named workloads (sizes, distributions and thresholds).
CONFIGS = {
    "gauss_n128_R200": dict(n=128, R=200, seed=0, eps=1e-6),
    "hadamard_n1024_R64x64": dict(n=1024, Ra=64, Rb=64, seeds=(0, 1), eps=1e-7),
    "newton_lr_n2048_N1000": dict(n=2048, N=1000, seed=0, eps=1e-6),
    "learned_n1024_R2000_8000": dict(n=1024, R_range=(2000, 8000), train_seed=10**6, n_train=20000,
                                     eval_seed=10**6 + 20000, n_eval=2000, eps=1e-6, nprop=32),
    # long-range multi-Slater lattice sums (Tables Tab:random_ranks, Tab:func_ranks), C2C thresholds
    "slater_lattice_random_n384": dict(n_cells=384, b=10.0, m=20, lam=0.5, h=1.56, amplitudes="random", seed=0,
                                       lattices=[(4, 4, 4), (6, 6, 6), (8, 8, 8), (16, 16, 8), (16, 16, 16)],
                                       eps_tucker=1e-3, eps_t2c=1e-5),
    "slater_lattice_func_n232": dict(n_cells=232, b=10.0, m=12, lam=0.5, h=1.56, amplitudes="func", seed=0,
                                     lattices=[(4, 4, 4), (6, 6, 6), (8, 8, 8), (16, 16, 8), (16, 16, 16)],
                                     eps_tucker=1e-3, eps_t2c=1e-5),
    # interaction energy of 16^3 charges from the reduced long-range potential (Lemma lem:InterEnergy)
    "newton_lattice_energy_N4096": dict(n_cells=384, b=24.0, L=(16, 16, 16), m=24, h=0.4, k_lo=-40, seed=0,
                                        eps_tucker=1e-6, eps_t2c=1e-8),
}


def hartree_like_factors(n: int = 1024, Ra: int = 64, Rb: int = 64, seeds=(0, 1)):
    """The two rank-64 Gaussian sums whose Hadamard product is the rank-4096 input."""
    return gaussian_sum(n, Ra, seeds[0]), gaussian_sum(n, Rb, seeds[1])


def random_cp(n, R, seed, signed=True, dist="normal") -> CP:
    """Unstructured random CP tensor (tests): factors N(0,1) or U[0,1), weights N(0,1)."""
    g = np.random.default_rng(seed)
    ns = [n] * 3 if np.isscalar(n) else list(n)
    U = []
    for l in range(3):
        if dist == "normal":
            U.append(np.asfortranarray(g.standard_normal((ns[l], R))))
        else:
            U.append(np.asfortranarray(g.random((ns[l], R))))
    xi = g.standard_normal(R) if signed else g.random(R) + 0.1
    return CP(U=U, xi=xi.astype(np.float64), meta=dict(kind="random", seed=seed))


def gaussian_sum_device(n: int, R: int, seed: int, device="cuda", **kw):
    """gaussian_sum(n, R, seed) with the factor columns evaluated on the device (torch):
    returns (U list of column-major float64 CUDA tensors, xi, params) where params holds the
    centres (R x 3), log-exponents and weights as CUDA float64 tensors (the inputs of the
    learned proposal's features).  Same parameter draws as gaussian_sum."""
    import torch
    x, centres, a, c = gaussian_sum_params(n, R, seed, **kw)
    xt = torch.from_numpy(x).to(device)
    at = torch.from_numpy(a).to(device)
    U = []
    for l in range(3):
        d = xt[:, None] - torch.from_numpy(centres[:, l].copy()).to(device)[None, :]
        U.append(torch.exp(-at[None, :] * d * d).t().contiguous().t())
    params = dict(centres=torch.from_numpy(np.ascontiguousarray(centres)).to(device),
                  loga=torch.from_numpy(np.log(a)).to(device), c=torch.from_numpy(c).to(device))
    return U, torch.from_numpy(c).to(device), params
