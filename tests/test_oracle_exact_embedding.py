"""Pins of the oracle's exact embedding average (App. B.2: App. A's
third-degree rule applied to F_k(rho_i) over site i and its neighbours
inside r_cut, which the paper replaces by the Taylor form Eq. F_taylor_mxe).

Each test checks the oracle against something other than itself: the
static EAM energy in numpy (sigma -> 0), App. A's pair rule (a rule of two
sites is the pair rule, whose nodes are pinned separately), the Gaussian
expectation by a tensor Gauss-Hermite rule (the third-degree rule's error
falls as sigma^4), central differences of the free energy, and the symmetry
of a perfect lattice.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1910_01235_gb300 import workloads as W
from test_oracle_pins import np_pair_fn, small_lattice, small_slab, static_eam_energy


def cluster(points, pot=None, x=None, sigma=0.1, L=24.0):
    """A few sites in a large periodic box (no interaction across images)."""
    pot = pot or W.potential_single()
    s = W.config_vacancy_lattice(cells=3, pot=pot)
    n = len(points)
    s.L = np.array([L, L, L])
    s.q = (np.asarray(points, float) + L / 2).T.copy()
    s.sigma = np.full(n, sigma)
    s.T = np.full(n, 800.0)
    s.sublattice = np.zeros(n, np.uint8)
    s.x = np.asarray(x, float) if x is not None else np.ones((pot.n_species, n))
    return s


def np_embedding(pot, k, rho):
    return -pot.E[k] * np.sqrt(rho)


# ---------------------------------------------------------------- static limit
@pytest.mark.parametrize("which", ["single", "binary", "slab"])
def test_sigma_to_zero_reproduces_static_eam(which):
    if which == "slab":
        s = small_slab()
    else:
        s = small_lattice(pot=W.potential_binary() if which == "binary" else None)
    s.sigma[:] = 1e-7
    fe = O.free_energy_exact(s)
    assert fe["status"] == O.OK
    np.testing.assert_allclose(fe["F4"][0], static_eam_energy(s), rtol=1e-12)


# ---------------------------------------------------------------- rule of two sites
@pytest.mark.parametrize("binary", [False, True])
def test_two_site_rule_is_the_pair_rule(binary):
    """N = 2 sites: N_q = 6, M = 12 nodes moving one site by sqrt(6) sigma --
    App. A's pair rule, so <F(rho_i)> = (1/12) sum over the pair nodes of
    F(sum_l x_jl f_kl(r_node))."""
    pot = W.potential_binary() if binary else W.potential_single()
    x = np.array([[0.7, 0.4], [0.25, 0.5]]) if binary else None
    s = cluster([[0, 0, 0], [1.9, 1.2, -0.7]], pot=pot, x=x)
    s.sigma[:] = [0.09, 0.14]
    fe = O.free_energy_exact(s)
    assert fe["status"] == O.OK
    d = s.q[:, 1] - s.q[:, 0]
    disp, _, _, _ = O.quad_nodes(d, s.sigma[0], s.sigma[1])
    r = np.sqrt(np.sum(disp * disp, axis=1))
    for k in range(s.S):
        for i, j in ((0, 1), (1, 0)):
            rho = sum(s.x[l, j] * np_pair_fn(pot, 1, k, l, r) for l in range(s.S))
            ref = np.mean(np_embedding(pot, k, rho))
            np.testing.assert_allclose(fe["emb"][k, i], ref, rtol=1e-13)


# ---------------------------------------------------------------- third degree
def gauss_hermite_expectation(fn, means, sigma, npts=4):
    """E[fn(q)] for independent Gaussians q_s ~ N(means_s, sigma_s^2 I) by the
    tensor-product Gauss-Hermite rule (exact for degree 2 npts - 1 per axis)."""
    t, w = np.polynomial.hermite.hermgauss(npts)
    w = w / np.sqrt(np.pi)
    nsite = len(means)
    dims = 3 * nsite
    grid = np.array(list(itertools.product(range(npts), repeat=dims)))
    wt = np.prod(w[grid], axis=1)
    coords = np.sqrt(2.0) * t[grid]                          # standard normal nodes
    q = [means[s][None, :] + sigma[s] * coords[:, 3 * s:3 * s + 3] for s in range(nsite)]
    return np.sum(wt * fn(q))


def test_embedding_error_falls_as_sigma_to_the_fourth():
    """The rule integrates every polynomial of degree <= 3 in the 3N
    coordinates exactly (App. A), so its error against the Gaussian
    expectation of F(rho_0) falls as sigma^4: a wrong node distance or
    weight leaves an error of order sigma^2 or 1."""
    pot = W.potential_single()
    pts = np.array([[0.0, 0.0, 0.0], [2.5, 0.3, 0.1], [0.2, 2.4, -0.4]])

    def F_rho0(q):
        rho = sum(np_pair_fn(pot, 1, 0, 0, np.sqrt(np.sum((q[j] - q[0]) ** 2, axis=1))) for j in (1, 2))
        return np_embedding(pot, 0, rho)

    errs = []
    for sg in (0.08, 0.04):
        s = cluster(pts, sigma=sg)
        fe = O.free_energy_exact(s)
        assert fe["status"] == O.OK
        ref = gauss_hermite_expectation(F_rho0, list(pts), [sg] * 3)
        errs.append(abs(fe["emb"][0, 0] - ref))
    ratio = errs[0] / errs[1]
    assert errs[1] > 0.0
    assert 10.0 < ratio < 24.0, (errs, ratio)   # error ~ sigma^4


# ---------------------------------------------------------------- gradients by FD
def energy(s, nb, **kw):
    fe = O.free_energy_exact(s, nb, **kw)
    assert fe["status"] == O.OK
    return fe["F4"]


def check_fd_exact(s, nb, sites, h=1e-5, rtol=1e-7, atol=3e-8):
    fe = O.free_energy_exact(s, nb)
    assert fe["status"] == O.OK
    for i in sites:
        for c in range(3):
            qp, qm = s.q.copy(), s.q.copy()
            qp[c, i] += h
            qm[c, i] -= h
            fd = (energy(s, nb, q=qp)[3] - energy(s, nb, q=qm)[3]) / (2 * h)
            assert abs(fd - fe["gq"][c, i]) <= atol + rtol * abs(fe["gq"][c, i]), ("q", i, c, fd, fe["gq"][c, i])
        sp, sm = s.sigma.copy(), s.sigma.copy()
        sp[i] += h
        sm[i] -= h
        fd = (energy(s, nb, sigma=sp)[3] - energy(s, nb, sigma=sm)[3]) / (2 * h)
        assert abs(fd - fe["gs"][i]) <= atol + rtol * abs(fe["gs"][i]), ("sigma", i, fd, fe["gs"][i])
        for k in range(s.S):
            hx = 1e-6
            if s.x[k, i] < 2 * hx or 1 - s.x[:, i].sum() < 2 * hx:
                continue
            xp, xm = s.x.copy(), s.x.copy()
            xp[k, i] += hx
            xm[k, i] -= hx
            Fp, Fm = energy(s, nb, x=xp), energy(s, nb, x=xm)
            fd = (Fp[3] - Fm[3]) / (2 * hx)
            assert abs(fd - fe["mu"][k, i]) <= 1e-6 + 1e-7 * abs(fe["mu"][k, i]), ("mu", i, k, fd, fe["mu"][k, i])
            fd_ex = (Fp[0] - Fm[0]) / (2 * hx)
            assert abs(fd_ex - fe["mu_ex"][k, i]) <= 1e-6 + 1e-7 * abs(fe["mu_ex"][k, i])


def margin_to_cutoff(s, nb, sites):
    """Smallest distance of a mean pair distance of these sites from r_cut
    (the rule's membership changes there, and with it the free energy)."""
    off, idx = nb
    m = np.inf
    for i in sites:
        for j in idx[off[i]:off[i + 1]]:
            d = s.q[:, j] - s.q[:, i]
            d -= s.L * np.rint(d / s.L)
            m = min(m, abs(np.linalg.norm(d) - s.pot.r_cut))
    return m


@pytest.mark.parametrize("which", ["single", "binary", "slab"])
def test_exact_gradients_match_central_differences(which):
    if which == "slab":
        # octahedral sites are 1.8 A from their hosts and have ~80 sites in
        # their rule: at sigma = 0.1 A the nodes (sigma sqrt(3 N) ~ 1.5 A) come
        # closer than 0.5 A, so the slab runs at sigma ~ 0.03 A
        s = small_slab()
        s.sigma *= 0.3
        sites = [0, 5, s.n // 2 + 3, s.n - 1]
    else:
        s = small_lattice(pot=W.potential_binary() if which == "binary" else None)
        sites = [0, 17, 101, s.n - 1]
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    assert st == O.OK
    assert margin_to_cutoff(s, (off, idx), sites) > 1e-3
    check_fd_exact(s, (off, idx), sites)


# ---------------------------------------------------------------- symmetry
def test_perfect_lattice_zero_force_uniform_mu():
    s = W.config_vacancy_lattice(x0=0.99)
    s.x[:] = 0.99
    fe = O.free_energy_exact(s)
    assert fe["status"] == O.OK
    assert np.abs(fe["gq"]).max() < 1e-12
    # ~11,000 node terms per site: uniform to rounding
    np.testing.assert_allclose(fe["mu_ex"], fe["mu_ex"][0, 0], rtol=1e-12)
    np.testing.assert_allclose(fe["gs"], fe["gs"][0], rtol=1e-12)
    # the two averages differ: the exact rule moves each site by sigma sqrt(3 N)
    ft = O.free_energy(s)
    assert abs(fe["F4"][0] - ft["F4"][0]) > 1e-3 * s.n * 1e-3


def test_translation_invariance():
    s = small_lattice(pot=W.potential_binary())
    fe = O.free_energy_exact(s)
    t = s.copy()
    t.q = s.q + np.array([[0.37], [-1.21], [2.9]])
    t.q -= t.L[:, None] * np.floor(t.q / t.L[:, None])
    ft = O.free_energy_exact(t)
    assert fe["status"] == ft["status"] == O.OK
    np.testing.assert_allclose(ft["F4"], fe["F4"], rtol=1e-12)
    np.testing.assert_allclose(ft["gq"], fe["gq"], rtol=0, atol=1e-11)
