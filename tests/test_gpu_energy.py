"""GPU parity of the node sampling of a canonical tensor (rhosvd_cp_sample) and of the interaction
energy from the long-range part of the collective Newton potential (rhosvd_rs_energy,
Lemma lem:InterEnergy) against the CPU oracle (oracle/energy.py).

Tolerances.  A sample is a sum of R products of four FP64 numbers, summed in another order on
each side: |p_gpu - p_orc| <= 4 R u sum_k |xi_k u1 u2 u3| (bound on a reordered sum).  The energy
adds N such samples: |E_gpu - E_orc| <= 1/2 sum_j |z_j| (that bound) + 4 N u (1/2 sum |z_j p_j| +
1/2 p0 sum z_j^2).  The energy of the C2C-reduced potential differs from the unreduced one by at
most 1/2 sum |z_j| max |P - P_red| <= 1/2 sum |z_j| (||xi'|| (sum_l tau_l^2)^(1/2) + eps_t2c
||beta||) (Thm. 2.3 with the measured tau_l, and the T2C bound)."""
import numpy as np
import pytest

import workloads
from oracle import energy as oe

pytestmark = pytest.mark.gpu
U_RND = 2.0 ** -53


def _dev(P, cp):
    import torch
    return [P.to_device_factor(u) for u in cp.U], torch.from_numpy(np.ascontiguousarray(cp.xi)).cuda()


def _abs_terms(U, xi, idx):
    return oe.cp_sample([np.abs(u) for u in U], np.abs(xi), idx)


def test_sample_matches_oracle(rhosvd_cuda):
    P = rhosvd_cuda
    cp = workloads.random_cp((50, 41, 33), 37, 3)
    g = np.random.default_rng(8)
    idx = np.stack([g.integers(0, n, 300) for n in (50, 41, 33)], axis=1)
    idx[0] = (0, 0, 0)
    idx[1] = (49, 40, 32)
    U, x = _dev(P, cp)
    got = P.rhosvd_cp_sample(U, x, idx).cpu().numpy()
    ref = oe.cp_sample(cp.U, cp.xi, idx)
    bound = 4 * cp.R * U_RND * _abs_terms(cp.U, cp.xi, idx)
    assert np.all(np.abs(got - ref) <= bound)
    bad = np.array([[0, 0, 33], [-1, 0, 0], [10, 10, 10]])
    out = P.rhosvd_cp_sample(U, x, bad).cpu().numpy()
    assert np.isnan(out[0]) and np.isnan(out[1]) and out[2] == pytest.approx(oe.cp_sample(cp.U, cp.xi, bad[2:])[0])


def test_energy_matches_oracle_and_pair_sum(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    cp = workloads.newton_lattice_long_range(n_cells=96, b=12.0, L=(4, 3, 3), m=24, seed=2)
    M = cp.meta
    U, x = _dev(P, cp)
    z = torch.from_numpy(M["z"]).cuda()
    E, p = P.rhosvd_rs_energy(U, x, M["idx"], z, M["p0"])
    Eg = float(E.item())
    pr = oe.cp_sample(cp.U, cp.xi, M["idx"])
    Eo = oe.energy_from_samples(pr, M["z"], M["p0"])
    sb = 4 * cp.R * U_RND * _abs_terms(cp.U, cp.xi, M["idx"])
    assert np.all(np.abs(p.cpu().numpy() - pr) <= sb)
    N = M["N"]
    eb = 0.5 * float(np.abs(M["z"]) @ sb) + 4 * N * U_RND * (0.5 * float(np.abs(M["z"] * pr).sum())
                                                             + 0.5 * M["p0"] * float(M["z"] @ M["z"]))
    assert abs(Eg - Eo) <= eb
    Ep = oe.pair_sum(M["coords"], M["z"], oe.long_range_kernel(M["t"], M["p"]))
    assert abs(Eg - Ep) <= eb + 1e-12 * abs(Ep)


def test_energy_empty_and_single_charge(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    cp = workloads.newton_lattice_long_range(n_cells=48, b=12.0, L=(1, 1, 1), m=24, seed=1)
    M = cp.meta
    U, x = _dev(P, cp)
    E, _ = P.rhosvd_rs_energy(U, x, M["idx"], torch.from_numpy(M["z"]).cuda(), M["p0"])
    # one charge: its own long-range potential at its centre is exactly the self term
    assert abs(float(E.item())) <= 8 * U_RND * M["p0"] * M["z"][0] ** 2
    E0, _ = P.rhosvd_rs_energy(U, x, np.zeros((0, 3), dtype=np.int64), torch.zeros(0, dtype=torch.float64).cuda(), 1.0)
    assert float(E0.item()) == 0.0


def test_energy_of_reduced_lattice_potential(rhosvd_cuda):
    """N = 16^3 = 4096 charges, R_l = 41 long-range Gaussians each (R = 167936 terms), n = 385:
    the C2C-reduced potential's energy against the unreduced one (both on the GPU, and the oracle's
    unreduced samples) within the reduction bound, and against the Coulomb sum within the kernel's
    own error."""
    P = rhosvd_cuda
    import torch
    C = dict(workloads.CONFIGS["newton_lattice_energy_N4096"])
    eps_t, eps_c = C.pop("eps_tucker"), C.pop("eps_t2c")
    cp = workloads.newton_lattice_long_range(**C)
    M = cp.meta
    U, x = _dev(P, cp)
    z = torch.from_numpy(M["z"]).cuda()
    E_full, p_full = P.rhosvd_rs_energy(U, x, M["idx"], z, M["p0"])
    can, tk = P.rhosvd_c2c(U, x, eps_t, eps_c, R_max=160 * 160, r_max=160)
    R, st = can.rank()
    info = tk.info()
    assert st == 0 and info.status == 0 and R < cp.R
    E_red, _ = P.rhosvd_rs_energy([can.U[l][:, :R] for l in range(3)], can.xi[:R], M["idx"], z, M["p0"])
    r = [info.r[l] for l in range(3)]
    beta = tk.beta[: r[0] * r[1] * r[2]]
    dP = info.xi_norm * float(np.sqrt(sum(t * t for t in info.tail))) + eps_c * float(torch.linalg.norm(beta))
    sz = float(np.abs(M["z"]).sum())
    assert abs(float(E_red.item()) - float(E_full.item())) <= 0.5 * sz * dP
    pr = oe.cp_sample(cp.U, cp.xi, M["idx"])
    sb = 4 * cp.R * U_RND * _abs_terms(cp.U, cp.xi, M["idx"])
    assert np.all(np.abs(p_full.cpu().numpy() - pr) <= sb)
    Ec = oe.pair_sum(M["coords"], M["z"], oe.coulomb)
    K = oe.long_range_kernel(M["t"], M["p"])
    kb = oe.pair_sum(M["coords"], np.abs(M["z"]), lambda d: np.abs(K(d) - oe.coulomb(d)))
    assert abs(float(E_full.item()) - Ec) <= kb * (1 + 1e-9) + 1e-10 * abs(Ec)
