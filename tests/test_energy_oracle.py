"""Pins of the RS interaction-energy oracle (oracle/energy.py) and of the lattice workloads:
the lemma's energy from the unreduced collective long-range potential equals the direct pair sum
of the long-range kernel (an algebraic identity: only the self terms are removed), and the
Coulomb energy of eq. inter_energy when the short-range Gaussians have decayed at the lattice
spacing; the sinc rules against their closed forms; and the energy from a C2C-reduced potential
within the bound given by the reduction's error."""
import math

import numpy as np

import workloads
from oracle import energy as oe
from oracle import t2c as ot


def test_lemma_equals_long_range_pair_sum():
    cp = workloads.newton_lattice_long_range(n_cells=96, b=12.0, L=(3, 3, 2), m=24, seed=3)
    M = cp.meta
    E = oe.energy_lemma(cp.U, cp.xi, M["idx"], M["z"], M["p0"])
    Ep = oe.pair_sum(M["coords"], M["z"], oe.long_range_kernel(M["t"], M["p"]))
    assert abs(E - Ep) <= 1e-12 * sum(abs(M["z"])) ** 2


def test_lemma_matches_coulomb_up_to_the_kernel_error():
    # |E_lemma - E_Coulomb| <= sum_{i<j} |z_i z_j| |P_{R_l}(r_ij) - 1/r_ij| (triangle inequality);
    # a wrong self-term correction would miss by 1/2 p0 sum z^2, far above the bound
    for k_lo, seed in ((-19, 4), (-40, 6)):
        cp = workloads.newton_lattice_long_range(n_cells=96, b=12.0, L=(4, 3, 3), m=24, k_lo=k_lo, seed=seed)
        M = cp.meta
        E = oe.energy_lemma(cp.U, cp.xi, M["idx"], M["z"], M["p0"])
        Ec = oe.pair_sum(M["coords"], M["z"], oe.coulomb)
        K = oe.long_range_kernel(M["t"], M["p"])
        bound = oe.pair_sum(M["coords"], np.abs(M["z"]), lambda d: np.abs(K(d) - oe.coulomb(d)))
        assert abs(E - Ec) <= bound * (1 + 1e-9) + 1e-12 * abs(Ec)
        assert 0.5 * M["p0"] * float(np.dot(M["z"], M["z"])) > 100 * bound


def test_sinc_rules_against_closed_forms():
    # 1/r: the step-0.4 trapezoid rule is good to ~1e-5 relative (its discretisation error), and
    # truncated at t_min = e^{-16} it misses about (2/sqrt(pi)) t_min of the integral
    t, p = workloads.newton_sinc_nodes(0.4, -40, 19)
    r = np.linspace(1.0, 30.0, 200)
    approx = np.exp(-np.outer(r * r, t * t)) @ p
    assert np.max(np.abs(approx * r - 1.0)) <= 2e-5
    assert abs(approx[-1] - 1.0 / r[-1]) <= 2e-5 / r[-1] + 1.2 * (2 / math.sqrt(math.pi)) * math.exp(-16.0)
    tau, q = workloads.slater_sinc_nodes(0.5, 1.56, -2, 2)
    approx = np.exp(-np.outer(r[r <= 20] ** 2, tau)) @ q
    assert np.max(np.abs(approx - np.exp(-0.5 * r[r <= 20]))) <= 5e-3
    # long-range Slater terms: tau <= 1, three of them (R_l = 3, R = 5)
    assert int(np.sum(tau <= 1.0)) == 3


def test_slater_lattice_structure():
    cp = workloads.multi_slater_long_range(n_cells=64, b=10.0, L=(2, 3, 2), m=10, amplitudes="random", seed=1)
    M = cp.meta
    assert cp.R == M["N"] * 3 and M["N"] == 12
    # the sum of the node Gaussians at a grid point equals the closed form of the long-range part
    x = workloads.point_grid(64, 10.0)
    tau, q = workloads.slater_sinc_nodes(0.5, 1.56)
    keep = tau <= 1.0
    g = (7, 30, 41)
    ref = 0.0
    for j in range(M["N"]):
        d2 = sum((x[g[l]] - x[M["idx"][j, l]]) ** 2 for l in range(3))
        ref += M["c"][j] * float(np.dot(q[keep], np.exp(-tau[keep] * d2)))
    val = float(oe.cp_sample(cp.U, cp.xi, np.array([g]))[0])
    assert abs(val - ref) <= 1e-13 * (np.abs(M["c"]).sum())
    F = workloads.slater_amplitude(np.array([0.0]), np.array([0.0]), np.array([0.0]))
    assert F[0] == 6.0


def test_energy_of_reduced_potential_within_bound():
    cp = workloads.newton_lattice_long_range(n_cells=40, b=12.0, L=(3, 3, 2), m=12, seed=5)
    M = cp.meta
    res = ot.c2c(cp.U, cp.xi, 1e-6, 1e-8)
    E0 = oe.energy_lemma(cp.U, cp.xi, M["idx"], M["z"], M["p0"])
    E1 = oe.energy_lemma(res["U_can"], res["xi_can"], M["idx"], M["z"], M["p0"])
    dP = np.linalg.norm(ot.full_from_cp(cp.U, cp.xi) - ot.full_from_cp(res["U_can"], res["xi_can"]))
    # |E1 - E0| = 1/2 |<z, dp>| <= 1/2 sum|z| max|dP| <= 1/2 sum|z| ||dP||_F
    assert abs(E1 - E0) <= 0.5 * np.abs(M["z"]).sum() * dP * (1 + 1e-9) + 1e-14 * abs(E0)
    assert res["R"] < cp.R
