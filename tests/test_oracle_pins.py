"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
printed constants of the quadrature rule (App. A), exact Gaussian moments,
the exact Gaussian expectation, the static EAM energy written out
independently, central finite differences of the free energy, the symmetry
of a perfect lattice, translation invariance, a brute-force neighbour search
in numpy, the closed form of the linear (potential-free) master equation on
the FCC lattice, and the stationarity of a FIRE fixed point.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1910_01235_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def small_lattice(cells=4, pot=None, seed=7, amp_q=0.05, amp_s=0.02, S=None):
    s = W.config_vacancy_lattice(cells=cells, pot=pot)
    if pot is not None and pot.n_species != 1:
        s.x = np.zeros((pot.n_species, s.n))
    s = W.perturb(s, amp_q, amp_s, seed=seed)
    s = W.random_fractions(s, vac_min=0.05, seed=seed + 1)
    return s


def small_slab(nx=4, ny=4, nz=2, seed=11):
    s = W.config_interstitial_slab(nx, ny, nz, top=100.0, xmax=0.3, seed=seed)
    return W.perturb(s, 0.03, 0.01, seed=seed + 1)


def np_pair_fn(pot, kind, k, l, r):
    """The potential tables of the configuration, evaluated in numpy."""
    t = np.clip((r - pot.r_switch) / (pot.r_cut - pot.r_switch), 0.0, 1.0)
    Sw = 1 - 10 * t**3 + 15 * t**4 - 6 * t**5
    if kind == 0:
        if pot.cross_geomean and k != l:
            return np.sqrt(np_pair_fn(pot, 0, k, k, r) * np_pair_fn(pot, 0, l, l, r))
        A, p, r0 = pot.phi_A[k, l], pot.phi_p[k, l], pot.phi_r0[k, l]
    else:
        A, p, r0 = pot.f_xi[k, l], pot.f_q[k, l], pot.f_r0[k, l]
    return A * np.exp(-p * (r / r0 - 1.0)) * Sw


def np_min_image_d(q, L):
    d = q.T[None, :, :] - q.T[:, None, :]          # d[i, j] = q_j - q_i
    d = d - L * np.rint(d * (1.0 / L))
    return d


# ---------------------------------------------------------------- App. A
def test_rule_constants_match_printed_values():
    g = json.load(open(os.path.join(GOLDEN, "app_a_rule.json")))
    Nq = g["sites_per_pair"] * g["N_q_per_site"]
    M = g["M_over_N_q"] * Nq
    sigma = 0.137
    disp, which, axis, dsig = O.quad_nodes(np.zeros(3), sigma, sigma)
    assert disp.shape[0] == M == g["overhead_vs_plain_force_evaluation"]
    # each node moves one site by r*sqrt(2)*sigma along one axis, r^2 = N_q/2
    r = np.sqrt(g["r2_over_N_q"] * Nq)
    np.testing.assert_allclose(np.abs(disp).max(axis=1), r * np.sqrt(2.0) * sigma, rtol=1e-15)
    # equal weights W_k = pi^(N_q/2)/(2 N_q): normalised weight 1/M
    assert g["weight_times_2Nq_over_pi_pow_Nq_half"] == 1.0
    assert sorted(zip(which.tolist(), axis.tolist())) == sorted(
        [(s, a) for s in (0, 1) for a in range(3) for _ in (0, 1)])


def gaussian_moment(dbar, s2, powers):
    """E[prod_a d_a^{p_a}] for d ~ N(dbar, s2 I), degree <= 3 (exact)."""
    out = 1.0
    for a, pa in enumerate(powers):
        m = dbar[a]
        out *= {0: 1.0, 1: m, 2: m * m + s2, 3: m**3 + 3 * m * s2}[pa]
    return out


@pytest.mark.parametrize("si,sj", [(0.1, 0.1), (0.05, 0.17), (0.2, 0.0)])
def test_nodes_integrate_degree3_exactly(si, sj):
    dbar = np.array([2.1, -0.7, 0.4])
    disp, which, axis, dsig = O.quad_nodes(dbar, si, sj)
    s2 = si * si + sj * sj
    for powers in itertools.product(range(4), repeat=3):
        if sum(powers) > 3:
            continue
        rule = np.mean(np.prod(disp ** np.array(powers), axis=1))
        np.testing.assert_allclose(rule, gaussian_moment(dbar, s2, powers), rtol=1e-13, atol=1e-13)
    # degree 4 is NOT exact (third-degree rule): E[(d_x - m_x)^2 (d_y - m_y)^2] = s2^2
    rule4 = np.mean((disp[:, 0] - dbar[0]) ** 2 * (disp[:, 1] - dbar[1]) ** 2)
    assert abs(rule4 - s2**2) > 0.5 * s2**2


def test_node_sigma_derivative_by_fd():
    dbar = np.array([1.9, 0.3, -1.1])
    h = 1e-6
    for site in (0, 1):
        a = [0.11, 0.07]
        b = list(a)
        b[site] += h
        c = list(a)
        c[site] -= h
        d0, which, axis, dsig = O.quad_nodes(dbar, *a)
        dp = O.quad_nodes(dbar, *b)[0]
        dm = O.quad_nodes(dbar, *c)[0]
        fd = (dp - dm) / (2 * h)
        for p in range(12):
            expect = np.zeros(3)
            if which[p] == site:
                expect[axis[p]] = dsig[p]
            np.testing.assert_allclose(fd[p], expect, atol=1e-8)


def exact_gaussian_average(pot, kind, k, l, dbar, s2, n=48):
    x, w = np.polynomial.hermite.hermgauss(n)
    w = w / np.sqrt(np.pi)
    off = np.sqrt(2.0 * s2) * x
    X, Y, Z = np.meshgrid(dbar[0] + off, dbar[1] + off, dbar[2] + off, indexing="ij")
    Wt = w[:, None, None] * w[None, :, None] * w[None, None, :]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    return float(np.sum(Wt * np_pair_fn(pot, kind, k, l, r)))


@pytest.mark.parametrize("kind", [0, 1])
def test_pair_average_converges_to_gaussian_at_fourth_order(kind):
    pot = W.potential_single()
    dbar = np.array([2.2, 0.9, -0.6])
    errs = []
    for sg in (0.02, 0.04):
        rule = O.pair_average(pot, kind, 0, 0, dbar, sg, sg)
        exact = exact_gaussian_average(pot, kind, 0, 0, dbar, 2 * sg * sg)
        errs.append(abs(rule - exact) / abs(exact))
    assert errs[1] < 1e-4
    ratio = errs[1] / errs[0]
    assert 10.0 < ratio < 24.0, (errs, ratio)   # error ~ sigma^4


# ---------------------------------------------------------------- static limit
def static_eam_energy(sys):
    """Textbook EAM with occupancies (Eqs. EAM-Substitutional and
    EAM-density-substitutional with n replaced by x), written out in numpy."""
    pot = sys.pot
    d = np_min_image_d(sys.q, sys.L)
    r = np.sqrt(np.sum(d * d, axis=2))
    np.fill_diagonal(r, 1e9)
    S = sys.S
    E = 0.0
    for k in range(S):
        rho = np.zeros(sys.n)
        for l in range(S):
            E += 0.5 * np.sum(np.outer(sys.x[k], sys.x[l]) * np_pair_fn(pot, 0, k, l, r))
            rho += np_pair_fn(pot, 1, k, l, r) @ sys.x[l]
        E += np.sum(sys.x[k] * (-pot.E[k] * np.sqrt(rho)))
    return E


@pytest.mark.parametrize("which", ["single", "binary", "slab"])
def test_sigma_to_zero_reproduces_static_eam(which):
    if which == "slab":
        s = small_slab()
    else:
        s = small_lattice(pot=W.potential_binary() if which == "binary" else None)
    s.sigma[:] = 1e-7
    fe = O.free_energy(s, mode=1)
    assert fe["status"] == O.OK
    np.testing.assert_allclose(fe["F4"][0], static_eam_energy(s), rtol=1e-12)


def test_perfect_lattice_reference_values():
    """Perfect FCC a = 3.6 A, x = 1 (values recomputed independently with
    numpy, outside the oracle): E_V/site -1.198691 eV at sigma -> 0
    and -1.230738 eV at sigma = 0.1 A, dE_V/dsigma_i = -0.69263 eV/A."""
    s = W.config_vacancy_lattice(x0=1.0)
    s.x[:] = 1.0
    s.sigma[:] = 1e-7
    assert abs(O.free_energy(s, mode=1)["F4"][0] / s.n - (-1.198691)) < 1e-6
    s.sigma[:] = 0.1
    fe = O.free_energy(s)
    assert abs(fe["F4"][0] / s.n - (-1.230738)) < 1e-6
    dEV = fe["gs"] + 3 * O.KB * s.T / s.sigma
    np.testing.assert_allclose(dEV, -0.69263, atol=1e-5)


# ---------------------------------------------------------------- gradients by FD
def fd_energy(s, **kw):
    fe = O.free_energy(s, mode=1, **kw)
    assert fe["status"] == O.OK
    return fe["F4"][3]


def check_fd(s, nb, sites, h=1e-5, rtol=1e-7, atol=3e-8, species=True):
    fe = O.free_energy(s, nb)
    assert fe["status"] == O.OK
    for i in sites:
        for c in range(3):
            qp, qm = s.q.copy(), s.q.copy()
            qp[c, i] += h
            qm[c, i] -= h
            fd = (fd_energy(s, nb=nb, q=qp) - fd_energy(s, nb=nb, q=qm)) / (2 * h)
            assert abs(fd - fe["gq"][c, i]) <= atol + rtol * abs(fe["gq"][c, i]), ("q", i, c, fd, fe["gq"][c, i])
        sp, sm = s.sigma.copy(), s.sigma.copy()
        sp[i] += h
        sm[i] -= h
        fd = (fd_energy(s, nb=nb, sigma=sp) - fd_energy(s, nb=nb, sigma=sm)) / (2 * h)
        assert abs(fd - fe["gs"][i]) <= atol + rtol * abs(fe["gs"][i]), ("sigma", i, fd, fe["gs"][i])
        if not species:
            continue
        for k in range(s.S):
            hx = 1e-6
            if s.x[k, i] < 2 * hx or 1 - s.x[:, i].sum() < 2 * hx:
                continue
            xp, xm = s.x.copy(), s.x.copy()
            xp[k, i] += hx
            xm[k, i] -= hx
            fd = (fd_energy(s, nb=nb, x=xp) - fd_energy(s, nb=nb, x=xm)) / (2 * hx)
            assert abs(fd - fe["mu"][k, i]) <= 1e-6 + 1e-7 * abs(fe["mu"][k, i]), ("mu", i, k, fd, fe["mu"][k, i])
            # the excess part alone: derivative of E_V
            ep = O.free_energy(s, nb, mode=1, x=xp)["F4"][0]
            em = O.free_energy(s, nb, mode=1, x=xm)["F4"][0]
            fd_ex = (ep - em) / (2 * hx)
            assert abs(fd_ex - fe["mu_ex"][k, i]) <= 1e-6 + 1e-7 * abs(fe["mu_ex"][k, i])


@pytest.mark.parametrize("which", ["single", "binary", "slab"])
def test_gradients_match_central_differences(which):
    if which == "slab":
        s = small_slab()
        sites = [0, 5, s.n // 2 + 3, s.n - 1]
    else:
        s = small_lattice(pot=W.potential_binary() if which == "binary" else None)
        sites = [0, 17, 101, s.n - 1]
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    assert st == O.OK
    check_fd(s, (off, idx), sites)


# ---------------------------------------------------------------- symmetry
def test_perfect_lattice_zero_force_uniform_mu_zero_flux():
    s = W.config_vacancy_lattice(x0=0.99)
    s.x[:] = 0.99
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    assert fe["status"] == O.OK
    assert np.abs(fe["gq"]).max() < 1e-12
    np.testing.assert_allclose(fe["mu_ex"], fe["mu_ex"][0, 0], rtol=1e-13)
    np.testing.assert_allclose(fe["gs"], fe["gs"][0], rtol=1e-13)
    boff, bidx = O.bonds(s, 3.0, off, idx)
    assert np.all(np.diff(boff) == 12)
    st, x1 = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), s.dt_default())
    assert st == O.OK
    assert np.abs(x1 - s.x).max() < 1e-15


def test_translation_invariance():
    s = small_lattice(pot=W.potential_binary())
    t = s.copy()
    t.q = t.q + np.array([0.123, -0.456, 0.789])[:, None]
    t.q = t.q - np.floor(t.q / t.L[:, None]) * t.L[:, None]
    rl = O.r_list_for(s)
    _, o1, i1 = O.neighbors(s.q, s.L, rl)
    _, o2, i2 = O.neighbors(t.q, t.L, rl)
    np.testing.assert_array_equal(o1, o2)
    np.testing.assert_array_equal(i1, i2)
    a = O.free_energy(s, (o1, i1))
    b = O.free_energy(t, (o2, i2))
    np.testing.assert_allclose(a["F4"], b["F4"], rtol=1e-12)
    np.testing.assert_allclose(a["gq"], b["gq"], atol=1e-10)
    np.testing.assert_allclose(a["mu_ex"], b["mu_ex"], rtol=1e-11)


# ---------------------------------------------------------------- neighbours
def np_neighbors(q, L, r_list):
    """Brute force in numpy with the same rounding rule, no FMA."""
    d = np_min_image_d(q, L)
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    n = q.shape[1]
    mask = r2 < r_list * r_list
    mask[np.arange(n), np.arange(n)] = False
    off = np.concatenate([[0], np.cumsum(mask.sum(axis=1))]).astype(np.int32)
    idx = np.nonzero(mask)[1].astype(np.int32)
    return off, idx


@pytest.mark.parametrize("case", ["c1", "perturbed", "tight_box", "slab"])
def test_neighbors_brute_force_binned_numpy_agree(case):
    if case == "c1":
        s = W.config_vacancy_lattice()
        rl = O.r_list_for(s)
    elif case == "perturbed":
        s = W.perturb(W.config_vacancy_lattice(), 0.3, 0.05)
        rl = O.r_list_for(s)
    elif case == "tight_box":
        s = W.perturb(W.config_vacancy_lattice(cells=4), 0.2, 0.0)
        rl = s.L[0] / 2.0 - 1e-9     # L = 2 r_list + tiny
    else:
        s = small_slab()
        rl = O.r_list_for(s)
    st, o1, i1 = O.neighbors(s.q, s.L, rl, binned=False)
    assert st == O.OK
    st, o2, i2 = O.neighbors(s.q, s.L, rl, binned=True)
    assert st == O.OK
    o3, i3 = np_neighbors(s.q, s.L, rl)
    np.testing.assert_array_equal(o1, o3)
    np.testing.assert_array_equal(i1, i3)
    np.testing.assert_array_equal(o2, o3)
    np.testing.assert_array_equal(i2, i3)
    for i in (0, s.n // 3, s.n - 1):
        np.testing.assert_array_equal(O.neighbor_row(s.q, s.L, rl, i), i3[o3[i]:o3[i + 1]])


def test_box_too_small():
    s = W.config_vacancy_lattice(cells=4)
    st, _, _ = O.neighbors(s.q, s.L, s.L[0] / 2 + 1e-9)
    assert st == O.ERR_BOX_TOO_SMALL


def test_fcc_coordination():
    s = W.config_vacancy_lattice()
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    assert np.all(np.diff(off) == 54)          # 12 + 6 + 24 + 12 shells within 5.445 A
    slab = W.config_interstitial_slab(6, 6, 6, gap_z=0.0)
    st, off, idx = O.neighbors(slab.q, slab.L, O.r_list_for(slab))
    boff, bidx = O.bonds(slab, 3.0, off, idx)
    nb = np.diff(boff)
    assert np.all(nb[: slab.n // 2] == 0)      # host sublattice immobile
    assert np.all(nb[slab.n // 2:] == 12)      # octahedral sites form an FCC lattice


# ---------------------------------------------------------------- master equation
def test_mass_conservation_and_antisymmetry():
    s = small_lattice(pot=W.potential_binary(), amp_q=0.1)
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    boff, bidx = O.bonds(s, 3.0, off, idx)
    st, x1 = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), s.dt_default() * 0.1)
    assert st == O.OK
    assert np.abs(x1 - s.x).max() > 1e-6          # something moved
    eps = np.finfo(float).eps
    for k in range(s.S):
        assert abs(x1[k].sum() - s.x[k].sum()) <= 4 * s.n * eps


def test_x_range_rejects_and_keeps_x():
    s = small_lattice(amp_q=0.0)
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    boff, bidx = O.bonds(s, 3.0, off, idx)
    st, x1 = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), s.dt_default() * 1e4)
    assert st == O.ERR_X_RANGE
    np.testing.assert_array_equal(x1, s.x)


def fcc_laplacian_eigs_fourier(cells, a):
    """Eigenvalues of the 12-neighbour graph Laplacian of a periodic FCC
    lattice: lambda(k) = sum_delta (cos k.delta - 1), k = 2 pi m / (cells a).
    m over {0..2 cells-1}^3 lists every Bloch character exactly twice."""
    deltas = [np.array(v) * a / 2 for v in itertools.product((-1, 0, 1), repeat=3)
              if sorted(map(abs, v)) == [0, 1, 1]]
    ms = np.array(list(itertools.product(range(2 * cells), repeat=3)), dtype=float)
    k = 2 * np.pi * ms / (cells * a)
    lam = sum(np.cos(k @ d) - 1.0 for d in deltas)
    return np.sort(lam)[::2]


def test_linear_fick_closed_form():
    """Pair and embedding prefactors zero: every excess chemical potential is
    0, J_{i->j} - J_{j->i} = D (x_i - x_j), and K Euler steps are the matrix
    power (I + dt D L)^K of the FCC nearest-neighbour Laplacian."""
    s = W.config_vacancy_lattice(pot=W.potential_off(), x0=0.9)
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    assert fe["status"] == O.OK
    assert np.all(fe["mu_ex"] == 0.0)
    boff, bidx = O.bonds(s, 3.0, off, idx)
    dt = s.dt_default()
    x = s.x.copy()
    K = 25
    for _ in range(K):
        st, x = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), dt, x=x)
        assert st == O.OK
    # independent closed form
    d = np_min_image_d(s.q, s.L)
    r = np.sqrt(np.sum(d * d, axis=2))
    A = ((r > 0.1) & (r < 3.0)).astype(float)
    Lap = A - np.diag(A.sum(axis=1))
    lam, V = np.linalg.eigh(Lap)
    np.testing.assert_allclose(lam, fcc_laplacian_eigs_fourier(5, s.a), atol=1e-10)
    D = s.nu0 * np.exp(-s.Qm / (W.KB_EV_PER_K * s.T[0]))
    xK = V @ ((1.0 + dt * D * lam) ** K * (V.T @ s.x[0]))
    np.testing.assert_allclose(x[0], xK, atol=1e-13)


# ---------------------------------------------------------------- FIRE
def test_fire_converges_to_stationary_point_variant_s():
    s = W.config_vacancy_lattice(cells=4, pot=W.potential_variant_s(), x0=1.0)
    s.x[:] = 1.0
    s = W.perturb(s, 0.05, 0.03)
    F_start = O.free_energy(s, mode=1)["F4"][3]
    st, it, fm, q, sg = O.relax(s, 1e-6, 3000)
    assert st == O.OK, (st, it, fm)
    assert fm <= 1e-6
    t = s.copy()
    t.q, t.sigma = q, sg
    F_end = O.free_energy(t, mode=1)["F4"][3]
    assert F_end < F_start
    # stationarity by central differences of F (independent of the analytic gradient)
    h = 1e-5
    for i in (0, 77, t.n - 1):
        for c in range(3):
            qp, qm = t.q.copy(), t.q.copy()
            qp[c, i] += h
            qm[c, i] -= h
            g = (fd_energy(t, q=qp) - fd_energy(t, q=qm)) / (2 * h)
            assert abs(g) < 1e-5
        sp, sm = t.sigma.copy(), t.sigma.copy()
        sp[i] += h
        sm[i] -= h
        assert abs((fd_energy(t, sigma=sp) - fd_energy(t, sigma=sm)) / (2 * h)) < 1e-5
    # on the perfect lattice the fixed point has uniform sigma: the minimum of
    # F over one common sigma (1-D, by bisection on its FD slope)
    def slope(sv):
        u = t.copy()
        u.q = W.fcc_positions(4, 4, 4, s.a)
        u.sigma[:] = sv + h
        fp = fd_energy(u)
        u.sigma[:] = sv - h
        return (fp - fd_energy(u)) / (2 * h)
    lo, hi = 0.05, 0.4
    assert slope(lo) < 0 < slope(hi)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if slope(mid) < 0 else (lo, mid)
    np.testing.assert_allclose(sg, 0.5 * (lo + hi), atol=1e-6)


def test_literal_potential_has_no_sigma_minimum():
    """With p = 3 < q = 5 the thermal force never changes sign: dF/dsigma < 0
    for every uniform sigma, so FIRE cannot converge: sigma runs away until
    the neighbour range r_cut + sqrt6 sigma + skin outgrows half the box."""
    s = W.config_vacancy_lattice(x0=1.0)
    s.x[:] = 1.0
    for sv in (0.05, 0.1, 0.2, 0.4):
        s.sigma[:] = sv
        fe = O.free_energy(s)
        assert np.all(fe["gs"] < 0)
    s.sigma[:] = 0.1
    st, it, fm, q, sg = O.relax(s, 1e-6, 15)
    assert st == O.ERR_NO_CONVERGE and it == 15
    assert np.all(sg > 0.3)
    st, it, fm, q, sg = O.relax(s, 1e-6, 60)
    assert st == O.ERR_BOX_TOO_SMALL
    np.testing.assert_array_equal(sg, s.sigma)      # input state restored


def test_fire_restores_state_on_geometry_error():
    s = W.config_vacancy_lattice(cells=4, x0=1.0)
    s.x[:] = 1.0
    s.q[:, 1] = s.q[:, 0] + 0.3        # two sites 0.3 A apart
    st, it, fm, q, sg = O.relax(s, 1e-6, 5)
    assert st == O.ERR_GEOMETRY
    np.testing.assert_array_equal(q, s.q)
    np.testing.assert_array_equal(sg, s.sigma)


# ---------------------------------------------------------------- workloads
def test_cu_vacancy_shape_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "cu_vacancy_shape.json")))
    s = W.config_cu_vacancy()
    assert s.n == g["sites"]
    assert s.a == g["a0_angstrom"]
    c_vac = float(np.sum(1.0 - s.x.sum(axis=0))) / s.n
    assert abs(c_vac - g["c_vac"]) / g["c_vac"] < g["c_vac_rel_tol"]
    assert (s.nu0, s.Qm) == (g["nu0_per_s"], g["Qm_eV"])


# ---------------------------------------------------------------- reservoirs
def test_reservoir_steady_state_detailed_balance():
    """Sec. 4 reservoir fixes.  Potential off (mu_ex = 0 in the bulk); one
    layer holds x_r (setatomicfraction) and mu_r (setchemicalpotential).  The
    steady state of the rate law has every bulk site at detailed balance with
    the layer: x_b / (1 - x_b) = x_r / (1 - x_r) exp(2 beta (mu_r - 0))."""
    s = W.config_vacancy_lattice(cells=4, pot=W.potential_off(), x0=0.3)
    s.x[:] = 0.3
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    assert np.all(fe["mu_ex"] == 0.0)
    boff, bidx = O.bonds(s, 3.0, off, idx)
    layer = s.q[2] < 0.5 * s.a * 0.5
    x_r, mu_r = 0.5, 0.01
    fix_x = (layer, np.full((1, s.n), x_r))
    fix_mu = (layer, np.full((1, s.n), mu_r))
    dt = 20 * s.dt_default()
    x = s.x.copy()
    for _ in range(4000):
        st, x = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), dt, x=x, fix_x=fix_x, fix_mu=fix_mu)
        assert st == O.OK
    beta = 1.0 / (O.KB * s.T[0])
    r = x_r / (1 - x_r) * np.exp(2 * beta * mu_r)
    np.testing.assert_allclose(x[0, layer], x_r, rtol=0, atol=0)
    np.testing.assert_allclose(x[0, ~layer], r / (1 + r), rtol=0, atol=1e-9)


# ---------------------------------------------------------------- FIRE trajectory
def test_fire_trajectory_worked_by_hand():
    """The relaxation's FIRE update (Bitzek et al., PRL 97, 170201 (2006)) in
    the order fixed for both implementations -- power check (from the second
    iteration), kick v += dt f, mixing v <- (1 - a) v + a |v| f/|f|, drift
    y += dt v -- on F = 1/2 (q_x^2 + 30 q_y^2 + 4 q_z^2) from (1, 1, 1), with
    dt0 = 0.3, dt_max = 0.5, f_inc = 1.1, f_dec = 0.5, a0 = 0.2, f_a = 0.99,
    n_min = 0.  The stiff y axis overshoots, so iterations 1 and 3 reset
    (P <= 0: v = 0, dt halved, a = a0) and iterations 2 and 4 grow dt.  Each
    iteration is written out below; a swapped kick/mixing/check order, a
    wrong reset or a wrong mixing norm changes the positions at once."""
    fp = O.FireParams(dt0=0.3, dt_max=0.5, f_inc=1.1, f_dec=0.5, alpha0=0.2, f_alpha=0.99, n_min=0)
    k = np.array([1.0, 30.0, 4.0])
    traj = O.fire_quadratic(k[:, None], np.ones((3, 1)), 5, fp)[:, :, 0]
    nrm = np.linalg.norm

    def mixed(v, f, a):
        return (1.0 - a) * v + a * nrm(v) / nrm(f) * f

    # iteration 0 (no power check): v and f are parallel, mixing keeps v
    y0 = np.array([1.0, 1.0, 1.0])
    f = -k * y0                                   # (-1, -30, -4)
    v = mixed(0.0 + 0.3 * f, f, 0.2)              # (-0.3, -9, -1.2)
    y1 = y0 + 0.3 * v
    np.testing.assert_allclose(y1, [0.91, -1.7, 0.64], rtol=1e-15)
    # iteration 1: P = f.v = 0.273 - 459 + 3.072 < 0 -> v = 0, dt = 0.15, a = 0.2
    f = -k * y1
    assert f @ v < 0
    v = mixed(0.15 * f, f, 0.2)
    y2 = y1 + 0.15 * v
    np.testing.assert_allclose(y2, [0.889525, -0.5525, 0.5824], rtol=1e-14)
    # iteration 2: P > 0 and n_pos = 1 > n_min -> dt = 0.165, a = 0.198
    f = -k * y2
    assert f @ v > 0
    v = mixed(v + 0.165 * f, f, 0.198)
    y3 = y2 + 0.165 * v
    # iteration 3: the y axis overshoots again, P < 0 -> v = 0, dt = 0.0825, a = 0.2
    f = -k * y3
    assert f @ v < 0
    v = mixed(0.0825 * f, f, 0.2)
    y4 = y3 + 0.0825 * v
    # iteration 4: P > 0 -> dt = 0.09075, a = 0.198
    f = -k * y4
    assert f @ v > 0
    v = mixed(v + 0.09075 * f, f, 0.198)
    y5 = y4 + 0.09075 * v
    np.testing.assert_allclose(traj, np.array([y0, y1, y2, y3, y4, y5]), rtol=1e-13, atol=1e-15)
