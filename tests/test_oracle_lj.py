"""Pins of the oracle's thermalized Lennard-Jones pair terms (App. C.1: the
12-6 pair potential averaged over the third-degree rule; no density, no
embedding).  CPU only.

sigma -> 0 reproduces the static 12-6 lattice energy written out in numpy
with occupancies; the three gradients match central differences of F; on a
perfect lattice the forces vanish and mu is uniform; the average converges
to the exact Gaussian expectation at fourth order in sigma.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_01235_gb300 import workloads as W

from test_oracle_pins import check_fd, np_min_image_d


def np_lj(pot, r):
    """4 eps [(s / r)^12 - (s / r)^6] times the quintic switch, in numpy."""
    t = np.clip((r - pot.r_switch) / (pot.r_cut - pot.r_switch), 0.0, 1.0)
    Sw = 1 - 10 * t**3 + 15 * t**4 - 6 * t**5
    eps, s = pot.lj_eps[0, 0], pot.lj_sigma[0, 0]
    x6 = (s / r) ** 6
    return 4.0 * eps * (x6 * x6 - x6) * Sw


def lj_lattice(seed=3, amp_q=0.05, amp_s=0.02, vac_min=0.05):
    s = W.config_vacancy_lattice(cells=4, pot=W.potential_lj())
    s = W.perturb(s, amp_q, amp_s, seed=seed)
    return W.random_fractions(s, vac_min=vac_min, seed=seed + 1)


def test_sigma_to_zero_reproduces_static_lj():
    s = lj_lattice()
    s.sigma[:] = 1e-7
    fe = O.free_energy(s, mode=1)
    assert fe["status"] == O.OK
    d = np_min_image_d(s.q, s.L)
    r = np.sqrt(np.sum(d * d, axis=2))
    np.fill_diagonal(r, 1e9)
    E = 0.5 * np.sum(np.outer(s.x[0], s.x[0]) * np_lj(s.pot, r))
    np.testing.assert_allclose(fe["F4"][0], E, rtol=1e-12)


def test_lj_gradients_match_central_differences():
    s = lj_lattice()
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    assert st == O.OK
    check_fd(s, (off, idx), [0, 17, 101, s.n - 1])


def test_lj_perfect_lattice_zero_force_uniform_mu():
    s = W.config_vacancy_lattice(cells=4, pot=W.potential_lj(), x0=0.9)
    s.x[:] = 0.9
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    assert fe["status"] == O.OK
    assert np.abs(fe["gq"]).max() < 1e-13
    np.testing.assert_allclose(fe["mu_ex"], fe["mu_ex"][0, 0], rtol=1e-13)
    # with no density the excess chemical potential is the pair sum alone:
    # mu_ex = sum_j x_j <phi>_ij, i.e. 2 E_V / (n x^2) * x
    np.testing.assert_allclose(fe["mu_ex"][0, 0], 2.0 * fe["F4"][0] / (s.n * 0.9), rtol=1e-12)


def exact_gaussian_lj(pot, dbar, s2, n=48):
    """Gaussian expectation of the pair term over a separation of variance s2
    per axis, by a Gauss-Hermite product rule of n points per axis."""
    x, w = np.polynomial.hermite.hermgauss(n)
    w = w / np.sqrt(np.pi)
    off = np.sqrt(2.0 * s2) * x
    X, Y, Z = np.meshgrid(dbar[0] + off, dbar[1] + off, dbar[2] + off, indexing="ij")
    Wt = w[:, None, None] * w[None, :, None] * w[None, None, :]
    return float(np.sum(Wt * np_lj(pot, np.sqrt(X * X + Y * Y + Z * Z))))


def test_lj_average_converges_to_gaussian_at_fourth_order():
    """The rule is exact to degree 3, so <phi>_rule - <phi>_Gauss ~ sigma^4:
    doubling sigma multiplies the difference by ~16."""
    pot = W.potential_lj()
    dbar = np.array([2.3, 0.9, -0.6])
    errs = []
    for sg in (0.02, 0.04):
        rule = O.pair_average(pot, 0, 0, 0, dbar, sg, sg)
        exact = exact_gaussian_lj(pot, dbar, 2 * sg * sg)
        errs.append(abs(rule - exact) / abs(exact))
    assert errs[1] < 1e-3
    ratio = errs[1] / errs[0]
    assert 10.0 < ratio < 24.0, (errs, ratio)
