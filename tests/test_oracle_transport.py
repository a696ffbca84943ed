"""Pins of the oracle's transport variants (Sec. 3, Eq. Transport and Eq.
MassTransport): host exchange and the ballistic term.  CPU only.

Host exchange: species exchange with a host species instead of the vacancy.
Pinned by conservation of every species, reduction to the vacancy law when
the host plays the vacancy's part, and the detailed-balance fixed point
x_k / x_host ~ exp(-2 beta (mu_k - mu_host)) of the symmetric exponents.
Ballistic term: tau x'' + x' = R.  Pinned by the tau -> 0 limit (Euler
step) and, with the potential off (R linear: a graph Laplacian on the FCC
bonds), by convergence to the closed-form solution of one Fourier mode,
tau e'' + e' + D lambda e = 0 with lambda from the FCC neighbour vectors.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_01235_gb300 import workloads as W

KB = 8.617333262e-5


def lattice_bonds(s):
    rb = 0.5 * (s.a / np.sqrt(2.0) + s.a)
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    return O.bonds(s, rb, off, idx)


def alloy_no_vacancy(seed=1, cells=4):
    s = W.config_binary_alloy(cells=cells, seed=seed)
    s.x[0] = 1.0 - s.x[1]          # x_A + x_B = 1: no vacancies
    return s


def test_host_exchange_conserves_every_species_and_site_totals():
    s = W.config_binary_alloy(cells=4)          # x_v = 1e-3
    bonds = lattice_bonds(s)
    rng = np.random.default_rng(2)
    mu = rng.normal(scale=0.05, size=s.x.shape)
    dt = s.dt_default() * 0.1
    st, x1, _ = O.transport_step(s, mu, bonds, dt, host=0)
    assert st == O.OK
    assert np.abs(x1 - s.x).max() > 1e-6                                   # mass moved
    np.testing.assert_allclose(x1.sum(axis=1), s.x.sum(axis=1), rtol=1e-13)  # each species
    np.testing.assert_allclose(x1.sum(axis=0), s.x.sum(axis=0), rtol=0, atol=1e-15)  # x_v per site


def test_host_exchange_reduces_to_the_vacancy_law():
    """With no vacancies and the host (A) in the vacancy's place, the B
    fractions follow the vacancy law of a one-species system x = x_B; a
    uniform host potential shifts nothing."""
    s2 = alloy_no_vacancy()
    bonds = lattice_bonds(s2)
    rng = np.random.default_rng(3)
    muB = rng.normal(scale=0.05, size=s2.n)
    dt = s2.dt_default() * 0.1
    s1 = s2.copy()
    s1.x = s2.x[1:2].copy()
    st, x1v = O.diffuse_step(s1, muB[None, :], bonds, dt)
    assert st == O.OK
    for c in (0.0, 0.37):
        mu2 = np.stack([np.full(s2.n, c), muB])
        st, x2, _ = O.transport_step(s2, mu2, bonds, dt, host=0)
        assert st == O.OK
        np.testing.assert_allclose(x2[1], x1v[0], rtol=0, atol=1e-14)
        np.testing.assert_allclose(x2[0], 1.0 - x2[1], rtol=0, atol=1e-14)


def test_host_exchange_detailed_balance_fixed_point():
    s = alloy_no_vacancy(seed=4)
    s.T[:] = 700.0
    bonds = lattice_bonds(s)
    rng = np.random.default_rng(5)
    muA = rng.normal(scale=0.05, size=s.n)
    muB = rng.normal(scale=0.05, size=s.n)
    beta = 1.0 / (KB * 700.0)
    ratio = 0.1 * np.exp(-2.0 * beta * (muB - muA))       # x_B / x_A at the fixed point
    s.x = np.stack([1.0 / (1.0 + ratio), ratio / (1.0 + ratio)])
    dt = s.dt_default()
    st, x1, _ = O.transport_step(s, np.stack([muA, muB]), bonds, dt, host=0)
    assert st == O.OK
    np.testing.assert_allclose(x1, s.x, rtol=0, atol=1e-14)
    # the same fractions with the host potential's sign flipped are not balanced
    st, x2, _ = O.transport_step(s, np.stack([-muA, muB]), bonds, dt, host=0)
    assert np.abs(x2 - s.x).max() > 1e-6


def test_ballistic_tau_to_zero_is_the_euler_step():
    s = W.random_fractions(W.config_vacancy_lattice(cells=4), vac_min=0.05, seed=6)
    bonds = lattice_bonds(s)
    rng = np.random.default_rng(7)
    mu = rng.normal(scale=0.02, size=s.x.shape)
    dt = s.dt_default() * 0.05
    st, xe = O.diffuse_step(s, mu, bonds, dt)
    v0 = rng.normal(scale=1.0, size=s.x.shape) * 0.0
    st, xb, vb = O.transport_step(s, mu, bonds, dt, tau=1e-30 * dt, v=v0)
    assert st == O.OK
    np.testing.assert_allclose(xb, xe, rtol=0, atol=1e-15)
    st, x0, v1 = O.transport_step(s, mu, bonds, dt, tau=0.0, v=v0)
    np.testing.assert_allclose(x0, xe, rtol=0, atol=0)


@pytest.mark.parametrize("tau_lambda", [0.1, 2.0])     # overdamped and oscillating modes
def test_ballistic_converges_to_the_closed_form_mode(tau_lambda):
    cells, a = 4, 3.6
    s = W.config_vacancy_lattice(cells=cells, a=a)
    s.T[:] = 800.0
    L = cells * a
    k = 2.0 * np.pi / L
    x0, eps0 = 0.5, 0.01
    s.x = (x0 + eps0 * np.cos(k * s.q[0]))[None, :]
    bonds = lattice_bonds(s)
    D = s.nu0 * np.exp(-s.Qm / (KB * 800.0))
    lam = 8.0 * (1.0 - np.cos(k * a / 2.0))              # 8 of the 12 FCC neighbours have x offsets +-a/2
    tau = tau_lambda / (D * lam)
    t_end = 3.0 / (D * lam)
    mu = np.zeros_like(s.x)
    r = np.roots([tau, 1.0, D * lam]).astype(complex)
    A = -eps0 * r[1] / (r[0] - r[1])
    B = eps0 * r[0] / (r[0] - r[1])
    exact = (A * np.exp(r[0] * t_end) + B * np.exp(r[1] * t_end)).real
    errs = []
    for K in (100, 200, 400):
        x = s.x.copy()
        v = np.zeros_like(x)
        for _ in range(K):
            st, x, v = O.transport_step(s, mu, bonds, t_end / K, tau=tau, v=v, x=x)
            assert st == O.OK
        amp = 2.0 * np.mean((x[0] - x0) * np.cos(k * s.q[0]))
        errs.append(abs(amp - exact))
    assert abs(exact) < eps0 and abs(exact - eps0) > 1e-3 * eps0       # the mode decayed
    assert errs[2] < 2e-3 * eps0
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4   # first order in dt


def test_transport_step_rejects_bad_arguments():
    s = W.config_vacancy_lattice(cells=4)
    bonds = lattice_bonds(s)
    mu = np.zeros_like(s.x)
    st, _, _ = O.transport_step(s, mu, bonds, 1e-12, host=1)        # host >= S
    assert st == O.ERR_ARG
    st, _, _ = O.transport_step(s, mu, bonds, 1e-12, tau=1.0)       # tau > 0 needs v
    assert st == O.ERR_ARG
