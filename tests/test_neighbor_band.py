"""CPU check of the FP32 prefilter of the cell-staged neighbour kernels.

On grids of >= 3 cells per axis the kernels decide |d| < r_list from FP32
positions within each site's cell, shifted into the home cell's frame by the
stencil offset times the FP32 cell width; inside an error band around r_list^2
they defer to the FP64 minimum-image rule (Algorithm 1's neighbour list).  The
claim that makes the lists exact is: wherever the FP32 test decides, it agrees
with the FP64 rule.  Here numpy float32 arithmetic follows the kernels'
operation order (cell assignment, staging, the difference and the fused dot
product, the band comparisons), the band follows the bound the host computes
before each build, and pairs are placed from 1e-7 to 1e-2 relative of the
cutoff, across the band's edge, where a too-narrow band would show.
"""
import numpy as np
import pytest

U = 2.0 ** -24


def band_bound(qmax, Lmax, r_list):
    """The list builder's band on |d|^2 (per-component delta, both forms)."""
    delta = max(2.0 * (6.0 * U * qmax + U * Lmax + U * r_list), 8.0 * U * Lmax / 3.0)
    b = 2.0 * (2.0 * np.sqrt(3.0) * r_list * delta + 3.0 * delta * delta + 4.0 * U * r_list * r_list)
    return np.float32(b * (1.0 + 1e-6))


def cell_assign(q, L, nc):
    """Unwrapped cell index and FP32 position within the cell, per axis."""
    h = L / nc
    u = q * (1.0 / L)
    w = np.floor(u)
    c = ((u - w) * nc).astype(np.int64)
    c = np.clip(c, 0, nc - 1)
    ac = w.astype(np.int64) * nc + c
    rel = (q - ac.astype(np.float64) * h).astype(np.float32)
    return ac, c, rel


def fma32(a, b, c):
    # the product of two floats is exact in FP64; one rounding to float32
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def fp32_r2(qi, qj, L, nc):
    """FP32 |d|^2 as the kernels form it, and whether j lies in i's 27-cell
    stencil (only those pairs are staged; others get r2 = inf here)."""
    h = L / nc
    h_f = np.float32(h)
    _, ci, ri = cell_assign(qi, L, nc)
    _, cj, rj = cell_assign(qj, L, nc)
    o = (cj - ci) % nc
    o = np.where(o == nc - 1, -1, o)
    staged = np.all(np.abs(o) <= 1, axis=-1)
    o = np.where(np.abs(o) <= 1, o, 0)
    shift = o.astype(np.float32) * h_f
    cq = (rj + shift).astype(np.float32)
    d = (cq - ri).astype(np.float32)
    r2 = (d[..., 0] * d[..., 0]).astype(np.float32)
    r2 = fma32(d[..., 1], d[..., 1], r2)
    r2 = fma32(d[..., 2], d[..., 2], r2)
    return np.where(staged, r2, np.float32(np.inf)), staged


def fp64_r2(qi, qj, L):
    da = qj - qi
    k = np.rint(da * (1.0 / L))
    d = da - L * k
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


@pytest.mark.parametrize("L,r_list,outside", [
    (144.0, 5.5, False),     # 256,000-site alloy box, 26 cells per axis
    (360.0, 6.1, False),     # 4M-site slab scale
    (18.0, 5.6, True),       # 3 cells per axis, positions up to a box outside
])
def test_fp32_decisions_outside_the_band_match_fp64(L, r_list, outside):
    rng = np.random.default_rng(1910)
    nc = int(np.floor(L / (r_list * (1.0 + 1e-9))))
    assert nc >= 3
    m = 200_000
    qi = rng.uniform(0.0, L, (m, 3))
    if outside:
        qi += L * rng.integers(-1, 2, (m, 3))
    v = rng.normal(size=(m, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # |r / r_list - 1| log-uniform in [1e-7, 1e-2], either sign: across the
    # band's edge (~1e-4 relative at these sizes) and well inside it
    eps = np.exp(rng.uniform(np.log(1e-7), np.log(1e-2), m)) * rng.choice([-1.0, 1.0], m)
    r = r_list * (1.0 + eps)
    qj = qi + r[:, None] * v
    qj += L * rng.integers(-1, 2, (m, 3))     # another image of the same site
    qmax = max(np.abs(qi).max(), np.abs(qj).max())
    band = band_bound(qmax, L, r_list)
    rl2 = r_list * r_list
    cut = np.float32(rl2)
    lo, hi = np.float32(cut - band), np.float32(cut + band)
    r2f, staged = fp32_r2(qi, qj, L, nc)
    exact_in = fp64_r2(qi, qj, L) < rl2
    assert not np.any(exact_in & ~staged)   # the stencil holds every list pair
    says_in, says_out = r2f < lo, r2f > hi
    assert not np.any(says_in & ~exact_in)
    assert not np.any(says_out & exact_in)
    # both outcomes occur on each side of the band, and the band stays narrow
    undecided = ~(says_in | says_out)
    assert says_in.any() and says_out.any() and undecided.any()
    assert np.abs(eps[undecided]).max() < 1e-3


def test_band_covers_the_home_frame_error_bound():
    """8 u h per component is inside the band's delta for any grid of >= 3
    cells (h <= L / 3), whatever the positions' magnitude."""
    for L in (10.0, 144.0, 360.0, 1000.0):
        for nc in (3, 7, 26):
            h = L / nc
            delta = max(2.0 * (6.0 * U * 0.0 + U * L + U * h), 8.0 * U * L / 3.0)
            assert 8.0 * U * h <= delta


@pytest.mark.parametrize("L,r_list,outside", [(144.0, 5.5, False), (360.0, 6.1, False), (18.0, 5.6, True)])
def test_home_frame_error_within_its_own_bound(L, r_list, outside):
    """The home-frame form's |d|^2 error stays below the bound built from
    8 u h per component (without the band's factor 2), and that bound is not
    vacuous: the largest error seen is a sizeable fraction of it."""
    rng = np.random.default_rng(7)
    nc = int(np.floor(L / (r_list * (1.0 + 1e-9))))
    h = L / nc
    m = 400_000
    qi = rng.uniform(0.0, L, (m, 3))
    if outside:
        qi += L * rng.integers(-1, 2, (m, 3))
    v = rng.normal(size=(m, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    eps = rng.uniform(-1e-3, 1e-3, m)
    qj = qi + (r_list * (1.0 + eps))[:, None] * v + L * rng.integers(-1, 2, (m, 3))
    r2f, staged = fp32_r2(qi, qj, L, nc)
    err = np.abs(r2f[staged].astype(np.float64) - fp64_r2(qi, qj, L)[staged]).max()
    d = 8.0 * U * h
    bound = 2.0 * np.sqrt(3.0) * r_list * d + 3.0 * d * d + 4.0 * U * r_list * r_list
    assert err <= bound
    assert err >= 0.05 * bound
