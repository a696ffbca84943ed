"""Seeded synthetic inputs for the MXE hot path.

This module builds lattices, molar fractions, temperatures and potential
parameter tables.  It holds none of the method's arithmetic (no quadrature,
no energies, no rates): both the CUDA path and the CPU oracle consume its
plain arrays, so the same seeded input reaches both sides.

Shapes follow the paper's workloads: an FCC lattice of conventional cubic
cells with a four-site basis (Sec. 5.1 vacancy diffusion in Cu; Sec. 5.4
octahedral interstitial sublattice for H in Pd), periodic boxes, vacuum gaps
modelled as a periodic box longer than the slab.

Site order: conventional cells in lexicographic (ix, iy, iz) order with iz
fastest, then the basis index; for two-sublattice systems all host sites come
first, then all octahedral sites in the same cell order.

Random draws use numpy's PCG64 with a fixed seed and a fixed draw order.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

SEED = 1910012350
KB_EV_PER_K = 8.617333262e-5   # Boltzmann constant, eV/K (CODATA 2018)

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
OCTA_BASIS = np.array([[0.5, 0.0, 0.0], [0.0, 0.5, 0.0], [0.0, 0.0, 0.5], [0.5, 0.5, 0.5]])

MAXS = 4


@dataclasses.dataclass
class Potential:
    """Analytic Finnis-Sinclair-type EAM tables for S species (App. B.2).

    phi_kl(r) = A_kl exp(-p_kl (r / r0_kl - 1)) S(r)     pair term
    f_kl(r)   = xi_kl exp(-q_kl (r / r0f_kl - 1)) S(r)   density at a k-site from an l-neighbour
    F_k(rho)  = -E_k sqrt(rho)                             embedding
    S(r)      quintic switch from r_switch to r_cut.
    cross_geomean: off-diagonal pair terms are sqrt(phi_kk phi_ll) pointwise
    (the tables' off-diagonal phi entries are then ignored).
    """
    n_species: int
    phi_A: np.ndarray
    phi_p: np.ndarray
    phi_r0: np.ndarray
    f_xi: np.ndarray
    f_q: np.ndarray
    f_r0: np.ndarray
    E: np.ndarray
    r_switch: float = 4.5
    r_cut: float = 5.0
    cross_geomean: bool = False
    # thermalized Lennard-Jones pair terms in place of phi (App. C.1):
    # 4 eps_kl [(s_kl / r)^12 - (s_kl / r)^6] S(r); E_k = 0 removes the embedding
    lj: bool = False
    lj_eps: Optional[np.ndarray] = None
    lj_sigma: Optional[np.ndarray] = None


def _tables(S):
    z = lambda: np.zeros((S, S))
    return z(), z(), np.ones((S, S)), z(), z(), np.ones((S, S))


def potential_single(A=0.3, p=3.0, r0=2.55, xi=1.0, q=5.0, r0f=2.55, E=1.0,
                     r_switch=4.5, r_cut=5.0) -> Potential:
    """One species: the analytic EAM of the 500-site and 864,000-site lattices."""
    pA, pp, pr0, fx, fq, fr0 = _tables(1)
    pA[0, 0], pp[0, 0], pr0[0, 0] = A, p, r0
    fx[0, 0], fq[0, 0], fr0[0, 0] = xi, q, r0f
    return Potential(1, pA, pp, pr0, fx, fq, fr0, np.array([E]), r_switch, r_cut, False)


def potential_variant_s(**kw) -> Potential:
    """The single-species potential with the exponents swapped (p=5, q=3).

    With the literal exponents (p=3 < q=5) the lattice has no free-energy
    minimum in sigma; swapping them gives a stable lattice whose relaxation
    converges.  Used where a test needs a converged relaxation.
    """
    return potential_single(p=5.0, q=3.0, **kw)


def potential_binary() -> Potential:
    """Two species A, B: B has prefactors x1.1 and length scale 2.65 A; the
    cross pair is the pointwise geometric mean; the density from an
    l-neighbour is that neighbour's own f_ll."""
    S = 2
    pA, pp, pr0, fx, fq, fr0 = _tables(S)
    pA[0, 0], pp[0, 0], pr0[0, 0] = 0.3, 3.0, 2.55
    pA[1, 1], pp[1, 1], pr0[1, 1] = 0.33, 3.0, 2.65
    for k in range(S):
        fx[k, 0], fq[k, 0], fr0[k, 0] = 1.0, 5.0, 2.55
        fx[k, 1], fq[k, 1], fr0[k, 1] = 1.1, 5.0, 2.65
    return Potential(S, pA, pp, pr0, fx, fq, fr0, np.array([1.0, 1.1]), 4.5, 5.0, True)


def potential_binary_variant_s() -> Potential:
    """The binary tables with the exponents swapped (p = 5, q = 3) for both
    species: a stable alloy whose relaxation converges."""
    P = potential_binary()
    P.phi_p[:] = np.where(P.phi_p != 0, 5.0, 0.0)
    P.f_q[:] = np.where(P.f_q != 0, 3.0, 0.0)
    return P


def potential_lj(eps=0.1, sigma_lj=2.3) -> Potential:
    """One species with a 12-6 Lennard-Jones pair term (minimum at
    2^(1/6) sigma_lj = 2.58 A, near the nearest-neighbour distance 2.55 A of
    the a = 3.6 A lattice), no density and no embedding; same switch."""
    S = 1
    pA, pp, pr0, fx, fq, fr0 = _tables(S)
    return Potential(S, pA, pp, pr0, fx, fq, fr0, np.array([0.0]), 4.5, 5.0, False, True,
                     np.full((1, 1), eps), np.full((1, 1), sigma_lj))


# The eight parameters differentiated in the surface-alloy workload: for each
# element e in (A, B): pair prefactor A_e, pair exponent p_e, density exponent
# q_e and length scale r0_e (shared by the element's pair and density terms).
THETA_NAMES = ("A_A", "p_A", "q_A", "r0_A", "A_B", "p_B", "q_B", "r0_B")


def theta_of(pot: Potential) -> np.ndarray:
    return np.array([pot.phi_A[0, 0], pot.phi_p[0, 0], pot.f_q[0, 0], pot.phi_r0[0, 0],
                     pot.phi_A[1, 1], pot.phi_p[1, 1], pot.f_q[0, 1], pot.phi_r0[1, 1]])


def binary_from_theta(theta, base: Potential = None) -> Potential:
    """The binary tables with element e's (A_e, p_e, q_e, r0_e) replaced;
    the density from an e-neighbour uses q_e and r0_e at every site."""
    P = dataclasses.replace(base if base is not None else potential_binary())
    P.phi_A, P.phi_p, P.phi_r0 = P.phi_A.copy(), P.phi_p.copy(), P.phi_r0.copy()
    P.f_q, P.f_r0 = P.f_q.copy(), P.f_r0.copy()
    for e in range(2):
        A, p, q, r0 = (float(v) for v in theta[4 * e:4 * e + 4])
        P.phi_A[e, e], P.phi_p[e, e], P.phi_r0[e, e] = A, p, r0
        P.f_q[:, e], P.f_r0[:, e] = q, r0
    return P


def potential_host_solute() -> Potential:
    """Species 0 = host, 1 = interstitial solute.  Host-host as the single
    species potential; host-solute pair and density with prefactor 0.5 and
    length scale 2.0 A; no solute-solute interaction."""
    S = 2
    pA, pp, pr0, fx, fq, fr0 = _tables(S)
    pA[0, 0], pp[0, 0], pr0[0, 0] = 0.3, 3.0, 2.55
    fx[0, 0], fq[0, 0], fr0[0, 0] = 1.0, 5.0, 2.55
    for (k, l) in ((0, 1), (1, 0)):
        pA[k, l], pp[k, l], pr0[k, l] = 0.5, 3.0, 2.0
        fx[k, l], fq[k, l], fr0[k, l] = 0.5, 5.0, 2.0
    return Potential(S, pA, pp, pr0, fx, fq, fr0, np.array([1.0, 1.0]), 4.5, 5.0, False)


def potential_off(S=1) -> Potential:
    """Pair and embedding prefactors zero, densities kept positive: every
    excess chemical potential is exactly zero, so the rate law reduces to
    linear Fick exchange."""
    pA, pp, pr0, fx, fq, fr0 = _tables(S)
    pp[:], pr0[:] = 3.0, 2.55
    fx[:], fq[:], fr0[:] = 1.0, 5.0, 2.55
    return Potential(S, pA, pp, pr0, fx, fq, fr0, np.zeros(S), 4.5, 5.0, False)


@dataclasses.dataclass
class System:
    """State of one periodic system (all arrays float64 / uint8, SoA)."""
    name: str
    L: np.ndarray               # [3] box lengths (A), periodic on all axes
    q: np.ndarray               # [3, n] mean positions (A)
    sigma: np.ndarray           # [n] per-component standard deviation (A)
    x: np.ndarray               # [S, n] molar fractions; vacancy = 1 - sum_k
    T: np.ndarray               # [n] temperature (K)
    sublattice: np.ndarray      # [n] uint8
    mobile_mask: int            # bit s set: sublattice s carries mass flux
    pot: Potential
    a: float                    # lattice parameter (A)
    nu0: float                  # attempt frequency (1/s)
    Qm: float                   # migration energy (eV)
    notes: str = ""

    @property
    def n(self) -> int:
        return self.q.shape[1]

    @property
    def S(self) -> int:
        return self.x.shape[0]

    def copy(self) -> "System":
        return dataclasses.replace(self, q=self.q.copy(), sigma=self.sigma.copy(),
                                   x=self.x.copy(), T=self.T.copy(),
                                   sublattice=self.sublattice.copy())

    def dt_default(self) -> float:
        """Euler step 0.02 / (12 nu0 exp(-Qm / kB T)) at the hottest site."""
        Tm = float(self.T.max())
        return 0.02 / (12.0 * self.nu0 * np.exp(-self.Qm / (KB_EV_PER_K * Tm)))


def fcc_positions(nx, ny, nz, a, basis=FCC_BASIS) -> np.ndarray:
    """[3, 4 nx ny nz] positions, cells lexicographic with iz fastest, then basis."""
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + basis[None, :, :]) * a
    return np.ascontiguousarray(pos.reshape(-1, 3).T)


def site_index(nx, ny, nz, ix, iy, iz, b) -> int:
    return ((ix * ny + iy) * nz + iz) * 4 + b


def config_vacancy_lattice(cells=5, a=3.6, T=800.0, sigma0=0.1, x0=0.99, pot=None,
                           vacancy_cell=(2, 2, 2)) -> System:
    """Single species with vacancies: x = x0 everywhere except one site at 0.
    Default: 5x5x5 cells (500 sites), a = 3.6 A, T = 800 K, sigma = 0.1 A."""
    q = fcc_positions(cells, cells, cells, a)
    n = q.shape[1]
    x = np.full((1, n), x0)
    x[0, site_index(cells, cells, cells, *vacancy_cell, 0)] = 0.0
    return System(f"vacancy_{cells}c", np.full(3, cells * a), q, np.full(n, sigma0), x,
                  np.full(n, T), np.zeros(n, np.uint8), 1,
                  pot if pot is not None else potential_single(), a, 1e13, 0.69)


def config_binary_alloy(cells=40, a=3.6, T=1000.0, sigma0=0.1, seed=SEED, gap_z=0.0) -> System:
    """Two species plus vacancy on every site: x_A ~ U(0.85, 0.95),
    x_B = 0.999 - x_A, vacancy 1e-3.  Default 40^3 cells (256,000 sites)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    q = fcc_positions(cells, cells, cells, a)
    n = q.shape[1]
    xa = rng.uniform(0.85, 0.95, n)
    x = np.stack([xa, 0.999 - xa])
    L = np.array([cells * a, cells * a, cells * a + gap_z])
    return System(f"binary_{cells}c", L, q, np.full(n, sigma0), x, np.full(n, T),
                  np.zeros(n, np.uint8), 1, potential_binary(), a, 1e13, 0.69)


def config_surface_alloy(cells=30, a=3.6, T=1000.0, seed=SEED) -> System:
    """Binary alloy slab with a 20 A vacuum gap along z (30^3 cells, 108,000 sites)."""
    s = config_binary_alloy(cells, a, T, seed=seed, gap_z=20.0)
    s.name = f"surface_{cells}c"
    return s


def config_interstitial_slab(nx=100, ny=100, nz=50, a=3.6, T=600.0, sigma0=0.1,
                             seed=SEED, gap_z=20.0, top=10.0, xmax=0.05) -> System:
    """Host FCC sublattice (0, immobile, x_host = 1) plus octahedral sublattice
    (1, mobile) holding one solute with x ~ U(0, xmax) in the top `top` A of
    the slab and 0 elsewhere.  Default 100x100x50 cells: 2 M + 2 M sites."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    qh = fcc_positions(nx, ny, nz, a)
    qo = fcc_positions(nx, ny, nz, a, OCTA_BASIS)
    L = np.array([nx * a, ny * a, nz * a + gap_z])
    # octahedral sites at the periodic seam (coordinate = n a) are wrapped
    qo = qo - np.floor(qo / L[:, None]) * L[:, None] * (qo >= L[:, None])
    nh, no = qh.shape[1], qo.shape[1]
    q = np.ascontiguousarray(np.concatenate([qh, qo], axis=1))
    x = np.zeros((2, nh + no))
    x[0, :nh] = 1.0
    draw = rng.uniform(0.0, xmax, no)
    zmax = (nz - 1) * a + 0.5 * a
    draw[qo[2] < zmax - top] = 0.0
    x[1, nh:] = draw
    sub = np.concatenate([np.zeros(nh, np.uint8), np.ones(no, np.uint8)])
    return System(f"slab_{nx}x{ny}x{nz}", L, q, np.full(nh + no, sigma0), x,
                  np.full(nh + no, T), sub, 0b10, potential_host_solute(), a, 8.1e12, 0.294)


def config_cu_vacancy(cells=60, a=3.615, T=300.0) -> System:
    """The paper's scaling case shape: 60^3 cells (864,000 sites), one vacancy
    at the centre, x = 1 elsewhere (Sec. 5.1, Sec. 6)."""
    s = config_vacancy_lattice(cells, a, T, x0=1.0, vacancy_cell=(cells // 2,) * 3)
    s.name = f"cu_vacancy_{cells}c"
    return s


def perturb(sys: System, amp_q=0.05, amp_sigma=0.02, seed=SEED + 1) -> System:
    """Random displacement of mean positions and widths (uniform), for tests."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    s = sys.copy()
    s.q = s.q + rng.uniform(-amp_q, amp_q, s.q.shape)
    s.sigma = s.sigma + rng.uniform(-amp_sigma, amp_sigma, s.sigma.shape)
    return s


def random_fractions(sys: System, lo=0.0, hi=1.0, vac_min=0.0, seed=SEED + 2) -> System:
    """Random molar fractions with sum_k x_k <= 1 - vac_min on mobile sites."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    s = sys.copy()
    raw = rng.uniform(lo, hi, (s.S + 1, s.n))
    raw /= raw.sum(axis=0, keepdims=True)
    s.x = np.ascontiguousarray(raw[: s.S] * (1.0 - vac_min))
    return s


def config_ensemble(n_systems=512, cmin=4, cmax=16, a=3.6, sigma0=0.1, seed=SEED, pot=None) -> List[System]:
    """Independent periodic single-species lattices: cells per side ~ U{cmin..cmax},
    T ~ U(300, 1200) K, vacancy fraction c_v ~ U(1e-4, 1e-2) per system; per
    site x_v = c_v * 2 u, u ~ U(0, 1), so the fluxes are non-trivial.
    Draw order: all cell counts, all T, all c_v, then each system's u."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    cells = rng.integers(cmin, cmax + 1, n_systems)
    Ts = rng.uniform(300.0, 1200.0, n_systems)
    cvs = rng.uniform(1e-4, 1e-2, n_systems)
    out = []
    for s_ in range(n_systems):
        c = int(cells[s_])
        q = fcc_positions(c, c, c, a)
        n = q.shape[1]
        xv = cvs[s_] * 2.0 * rng.uniform(0.0, 1.0, n)
        out.append(System(f"ensemble_{s_}_{c}c", np.full(3, c * a), q, np.full(n, sigma0), (1.0 - xv)[None, :].copy(),
                          np.full(n, Ts[s_]), np.zeros(n, np.uint8), 1,
                          pot if pot is not None else potential_single(), a, 1e13, 0.69))
    return out


CONFIGS = {
    "vacancy_500": lambda: config_vacancy_lattice(),
    "binary_256k": lambda: config_binary_alloy(),
    "surface_108k": lambda: config_surface_alloy(),
    "slab_4M": lambda: config_interstitial_slab(),
    "cu_vacancy_864k": lambda: config_cu_vacancy(),
}
