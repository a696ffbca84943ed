"""The seeded synthetic inputs follow their stated recipe (sizes, value
distributions, site numbering, sublattices, determinism).  CPU only; no
arithmetic of the method is involved."""
import numpy as np
import pytest

from paper_1910_01235_gb300 import workloads as W


def test_fcc_numbering_cells_lexicographic_z_fastest_then_basis():
    q = W.fcc_positions(3, 4, 5, 2.0)
    assert q.shape == (3, 4 * 3 * 4 * 5)
    for (ix, iy, iz, b) in [(0, 0, 0, 0), (0, 0, 1, 0), (0, 1, 0, 3), (2, 3, 4, 2), (1, 2, 3, 1)]:
        i = W.site_index(3, 4, 5, ix, iy, iz, b)
        np.testing.assert_allclose(q[:, i], (np.array([ix, iy, iz]) + W.FCC_BASIS[b]) * 2.0)


def test_vacancy_lattice_recipe():
    s = W.config_vacancy_lattice()
    assert s.n == 500 and s.S == 1
    np.testing.assert_allclose(s.L, 5 * 3.6)
    assert np.all(s.T == 800.0) and np.all(s.sigma == 0.1)
    zero = np.flatnonzero(s.x[0] == 0.0)
    assert zero.tolist() == [W.site_index(5, 5, 5, 2, 2, 2, 0)]
    assert np.all(np.delete(s.x[0], zero) == 0.99)
    assert (s.nu0, s.Qm) == (1e13, 0.69)


def test_binary_alloy_recipe_and_determinism():
    s = W.config_binary_alloy()
    assert s.n == 256_000 and s.S == 2
    np.testing.assert_allclose(s.L, 40 * 3.6)
    xa, xb = s.x
    assert xa.min() >= 0.85 and xa.max() < 0.95
    np.testing.assert_allclose(xa + xb, 0.999, rtol=0, atol=1e-15)
    # uniform: mean and spread of U(0.85, 0.95)
    assert abs(xa.mean() - 0.90) < 1e-3 and abs(xa.std() - 0.1 / np.sqrt(12.0)) < 1e-3
    assert np.all(s.T == 1000.0) and np.all(s.sigma == 0.1)
    t = W.config_binary_alloy()
    assert np.array_equal(s.x, t.x) and np.array_equal(s.q, t.q)
    u = W.config_binary_alloy(seed=W.SEED + 7)
    assert not np.array_equal(s.x, u.x)


def test_surface_alloy_has_the_vacuum_gap():
    s = W.config_surface_alloy()
    assert s.n == 108_000
    np.testing.assert_allclose(s.L, [30 * 3.6, 30 * 3.6, 30 * 3.6 + 20.0])
    assert s.q[2].max() < 30 * 3.6


def test_interstitial_slab_recipe():
    s = W.config_interstitial_slab()
    nh = no = 4 * 100 * 100 * 50
    assert s.n == nh + no == 4_000_000 and s.S == 2
    np.testing.assert_allclose(s.L, [360.0, 360.0, 50 * 3.6 + 20.0])
    assert np.all(s.sublattice[:nh] == 0) and np.all(s.sublattice[nh:] == 1)
    assert s.mobile_mask == 0b10
    assert np.all(s.x[0, :nh] == 1.0) and np.all(s.x[0, nh:] == 0.0)
    assert np.all(s.x[1, :nh] == 0.0)
    sol = s.x[1, nh:]
    z = s.q[2, nh:]
    zmax = 49 * 3.6 + 0.5 * 3.6
    assert np.all(sol[z < zmax - 10.0] == 0.0)
    top = z >= zmax - 10.0
    assert sol[top].max() < 0.05 and sol[top].mean() > 0.02
    # every octahedral site inside the periodic box
    assert np.all(s.q[:, nh:] >= 0.0) and np.all(s.q[:, nh:] < s.L[:, None])
    assert (s.nu0, s.Qm, float(s.T[0])) == (8.1e12, 0.294, 600.0)


def test_cu_vacancy_shape():
    s = W.config_cu_vacancy()
    assert s.n == 864_000
    assert np.count_nonzero(s.x[0] == 0.0) == 1 and s.x[0, W.site_index(60, 60, 60, 30, 30, 30, 0)] == 0.0
    np.testing.assert_allclose(s.L, 60 * 3.615)


def test_ensemble_recipe():
    systems = W.config_ensemble()
    assert len(systems) == 512
    assert sum(s.n for s in systems) == 2_850_284
    for s in systems:
        c = round(s.L[0] / 3.6)
        assert 4 <= c <= 16 and s.n == 4 * c ** 3
        assert 300.0 <= s.T[0] < 1200.0 and np.all(s.T == s.T[0])
        xv = 1.0 - s.x[0]
        assert xv.min() >= 0.0 and xv.max() < 2e-2
