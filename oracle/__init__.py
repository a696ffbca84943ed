"""Plain FP64 CPU oracle of the MXE hot path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product path (the CUDA library and
its binding) never imports, links or runs anything here, and this package
shares no code with it: the only common input is the seeded arrays built by
`paper_1910_01235_gb300.workloads`, which hold none of the method's
arithmetic.

The arithmetic lives in `mxe_oracle.c` (plain loops, FP64, no FMA
contraction); this module compiles it with gcc and marshals numpy arrays.
Each wrapper names the passage of the paper its C function follows.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mxe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXS = 4
KB = 8.617333262e-5

OK, ERR_ARG, ERR_BOX_TOO_SMALL, ERR_NBR_OVERFLOW = 0, 1, 4, 5
ERR_GEOMETRY, ERR_NONFINITE, ERR_X_RANGE, ERR_NO_CONVERGE = 6, 7, 8, 9


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (OpenMP over sites if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB)
    return _LIB


class _Pot(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("cross_geomean", C.c_int32)] + [
        (nm, (C.c_double * MAXS) * MAXS) for nm in ("phi_A", "phi_p", "phi_r0", "f_xi", "f_q", "f_r0")
    ] + [("E", C.c_double * MAXS), ("r_switch", C.c_double), ("r_cut", C.c_double),
         ("lj", C.c_int32), ("pad", C.c_int32), ("lj_eps", (C.c_double * MAXS) * MAXS),
         ("lj_sigma", (C.c_double * MAXS) * MAXS)]


class _Sys(C.Structure):
    _fields_ = [("n", C.c_int64), ("S", C.c_int32), ("pad", C.c_int32), ("L", C.c_double * 3),
                ("q", C.c_void_p), ("sigma", C.c_void_p), ("x", C.c_void_p), ("T", C.c_void_p)]


class _Fire(C.Structure):
    _fields_ = [("dt0", C.c_double), ("dt_max", C.c_double), ("f_inc", C.c_double),
                ("f_dec", C.c_double), ("alpha0", C.c_double), ("f_alpha", C.c_double),
                ("sigma_max", C.c_double), ("n_min", C.c_int32), ("pad", C.c_int32)]


@dataclasses.dataclass
class FireParams:
    """FIRE constants (Bitzek et al. 2006 defaults; dt in the units of
    sqrt(A^2 / (eV/A)) with unit masses)."""
    dt0: float = 0.02
    dt_max: float = 0.1
    f_inc: float = 1.1
    f_dec: float = 0.5
    alpha0: float = 0.1
    f_alpha: float = 0.99
    n_min: int = 5
    sigma_max: float = 0.0    # <= 0: no upper bound on sigma


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            p = C.c_void_p
            L.orc_neighbors.argtypes = [C.c_int64, p, p, C.c_double, p, p, C.c_int64, p]
            L.orc_neighbors_binned.argtypes = L.orc_neighbors.argtypes
            L.orc_neighbor_row.argtypes = [C.c_int64, p, p, C.c_double, C.c_int64, p, C.c_int64, p]
            L.orc_bonds.argtypes = [C.c_int64, p, p, C.c_double, p, C.c_uint32, p, p, p, p, C.c_int64, p]
            L.orc_quad_nodes.argtypes = [p, C.c_double, C.c_double, p, p, p, p]
            L.orc_quad_nodes.restype = None
            L.orc_pair_average_value.argtypes = [p, C.c_int, C.c_int, C.c_int, p, C.c_double, C.c_double]
            L.orc_pair_average_value.restype = C.c_double
            L.orc_free_energy.argtypes = [p, p, p, p, C.c_int] + [p] * 10
            L.orc_free_energy_exact.argtypes = [p, p, p, p] + [p] * 6
            L.orc_diffuse_step.argtypes = [C.c_int64, C.c_int, p, p, p, p, p, C.c_double, C.c_double, C.c_double]
            L.orc_diffuse_step_res.argtypes = [C.c_int64, C.c_int, p, p, p, p, p, C.c_double, C.c_double,
                                               C.c_double, p, p, p, p]
            L.orc_relax.argtypes = [p, p, p, p, C.c_double, C.c_double, C.c_int, p, p, p, C.c_int]
            L.orc_transport_step.argtypes = [C.c_int64, C.c_int, p, p, p, p, p, C.c_double, C.c_double,
                                             C.c_double, C.c_int, C.c_double, p]
            L.orc_fire_quadratic.argtypes = [C.c_int64, p, p, C.c_int, p, p]
            L.orc_fire_quadratic.restype = None
            L.orc_num_threads.argtypes = []
            _lib = L
        return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def make_potential(pot) -> _Pot:
    P = _Pot()
    S = pot.n_species
    P.n_species = S
    P.cross_geomean = 1 if pot.cross_geomean else 0
    for nm in ("phi_A", "phi_p", "phi_r0", "f_xi", "f_q", "f_r0"):
        tab = getattr(pot, nm)
        dst = getattr(P, nm)
        for k in range(MAXS):
            for l in range(MAXS):
                dst[k][l] = float(tab[k, l]) if (k < S and l < S) else (1.0 if nm.endswith("r0") else 0.0)
    for k in range(S):
        P.E[k] = float(pot.E[k])
    P.r_switch = float(pot.r_switch)
    P.r_cut = float(pot.r_cut)
    if getattr(pot, "lj", False):
        P.lj = 1
        for k in range(S):
            for l in range(S):
                P.lj_eps[k][l] = float(pot.lj_eps[k, l])
                P.lj_sigma[k][l] = float(pot.lj_sigma[k, l])
    return P


class _SysRef:
    """Keeps numpy buffers alive for the ctypes struct."""

    def __init__(self, sys, q=None, sigma=None, x=None):
        self.q = _f64(sys.q if q is None else q)
        self.sigma = _f64(sys.sigma if sigma is None else sigma)
        self.x = _f64(sys.x if x is None else x)
        self.T = _f64(sys.T)
        s = _Sys()
        s.n = sys.n
        s.S = self.x.shape[0]
        for a in range(3):
            s.L[a] = float(sys.L[a])
        s.q, s.sigma, s.x, s.T = _ptr(self.q), _ptr(self.sigma), _ptr(self.x), _ptr(self.T)
        self.s = s


def neighbors(q, L, r_list, binned=None):
    """Neighbour CSR (offsets [n+1] int32, idx int32), rows sorted by j.
    Brute force for n <= 4000 unless `binned` is given."""
    q = _f64(q)
    n = q.shape[1]
    L = _f64(L)
    if binned is None:
        binned = n > 4000
    fn = lib().orc_neighbors_binned if binned else lib().orc_neighbors
    off = np.zeros(n + 1, np.int32)
    cap = 80 * n + 64
    while True:
        idx = np.zeros(cap, np.int32)
        cnt = C.c_int64(0)
        st = fn(n, _ptr(q), _ptr(L), float(r_list), _ptr(off), _ptr(idx), cap, C.byref(cnt))
        if st == ERR_NBR_OVERFLOW:
            cap = cnt.value + 64
            continue
        if st != OK:
            return st, None, None
        return OK, off, idx[: cnt.value].copy()


def neighbor_row(q, L, r_list, i):
    q = _f64(q)
    L = _f64(L)
    row = np.zeros(4096, np.int32)
    cnt = C.c_int64(0)
    st = lib().orc_neighbor_row(q.shape[1], _ptr(q), _ptr(L), float(r_list), int(i), _ptr(row), 4096, C.byref(cnt))
    assert st == OK
    return row[: cnt.value].copy()


def bonds(sys, r_bond, nb_off, nb_idx):
    """Nearest-neighbour bond CSR on mobile sublattices (Sec. 3)."""
    q = _f64(sys.q)
    L = _f64(sys.L)
    sub = np.ascontiguousarray(sys.sublattice, dtype=np.uint8)
    off = np.zeros(sys.n + 1, np.int32)
    cap = int(nb_idx.shape[0]) + 64
    idx = np.zeros(cap, np.int32)
    cnt = C.c_int64(0)
    st = lib().orc_bonds(sys.n, _ptr(q), _ptr(L), float(r_bond), _ptr(sub), int(sys.mobile_mask),
                         _ptr(nb_off), _ptr(nb_idx), _ptr(off), _ptr(idx), cap, C.byref(cnt))
    assert st == OK, st
    return off, idx[: cnt.value].copy()


def quad_nodes(dbar, s_first, s_second):
    """App. A nodes for one pair: (disp [12,3], which [12], axis [12], dsig [12])."""
    d = _f64(dbar)
    disp = np.zeros((12, 3))
    which = np.zeros(12, np.int32)
    axis = np.zeros(12, np.int32)
    dsig = np.zeros(12)
    lib().orc_quad_nodes(_ptr(d), float(s_first), float(s_second), _ptr(disp), _ptr(which), _ptr(axis), _ptr(dsig))
    return disp, which, axis, dsig


def pair_average(pot, kind, k, l, dbar, s_first, s_second):
    """<phi_kl> (kind 0) or <f_kl> (kind 1) over the 12 nodes (App. A, B)."""
    P = make_potential(pot)
    d = _f64(dbar)
    return lib().orc_pair_average_value(C.byref(P), int(kind), int(k), int(l), _ptr(d),
                                        float(s_first), float(s_second))


def r_list_for(sys, skin=0.2):
    return sys.pot.r_cut + np.sqrt(6.0) * float(np.max(sys.sigma)) + skin


def free_energy(sys, nb=None, mode=0, q=None, sigma=None, x=None, r_list=None):
    """Free energy and gradients (App. B.2, Sec. 2.1).  Returns a dict with
    status, F4 = (E_V, F_vib, F_mix, F), gq [3,n], gs [n], mu_ex [S,n],
    mu [S,n] and the per-site rho_bar, rho_avg, a, b, e [S,n]."""
    ref = _SysRef(sys, q, sigma, x)
    n, S = sys.n, ref.x.shape[0]
    if nb is None:
        rl = r_list if r_list is not None else sys.pot.r_cut + np.sqrt(6.0) * float(ref.sigma.max()) + 0.2
        st, off, idx = neighbors(ref.q, sys.L, rl)
        assert st == OK, st
    else:
        off, idx = nb
    P = make_potential(sys.pot)
    out = dict(F4=np.zeros(4), gq=np.zeros((3, n)), gs=np.zeros(n), mu_ex=np.zeros((S, n)),
               mu=np.zeros((S, n)), rho_bar=np.zeros((S, n)), rho_avg=np.zeros((S, n)),
               a=np.zeros((S, n)), b=np.zeros((S, n)), e=np.zeros((S, n)))
    st = lib().orc_free_energy(C.byref(ref.s), C.byref(P), _ptr(off), _ptr(idx), int(mode),
                               *[_ptr(out[k]) for k in ("F4", "gq", "gs", "mu_ex", "mu", "rho_bar",
                                                        "rho_avg", "a", "b", "e")])
    out["status"] = int(st)
    return out


def free_energy_exact(sys, nb=None, q=None, sigma=None, x=None, r_list=None):
    """Free energy and gradients with the exact phase average of the
    embedding term (App. B.2: App. A's third-degree rule over a site and its
    neighbours inside r_cut, in place of the Taylor form Eq. F_taylor_mxe).
    Returns a dict with status, F4, gq, gs, mu_ex, mu and emb [S, n] =
    <F_k(rho_i^k)>."""
    ref = _SysRef(sys, q, sigma, x)
    n, S = sys.n, ref.x.shape[0]
    if nb is None:
        rl = r_list if r_list is not None else sys.pot.r_cut + np.sqrt(6.0) * float(ref.sigma.max()) + 0.2
        st, off, idx = neighbors(ref.q, sys.L, rl)
        assert st == OK, st
    else:
        off, idx = nb
    P = make_potential(sys.pot)
    out = dict(F4=np.zeros(4), gq=np.zeros((3, n)), gs=np.zeros(n), mu_ex=np.zeros((S, n)),
               mu=np.zeros((S, n)), emb=np.zeros((S, n)))
    st = lib().orc_free_energy_exact(C.byref(ref.s), C.byref(P), _ptr(off), _ptr(idx),
                                     *[_ptr(out[k]) for k in ("F4", "gq", "gs", "mu_ex", "mu", "emb")])
    out["status"] = int(st)
    return out


def diffuse_step(sys, mu_ex, bond_csr, dt, x=None, nu0=None, Qm=None, fix_x=None, fix_mu=None):
    """One forward-Euler step of Eq. MassTransport (reading described in the
    C source).  fix_x / fix_mu: optional (mask [n] bool, values [S, n])
    reservoirs (Sec. 4: setatomicfraction, setchemicalpotential).
    Returns (status, x_new)."""
    xx = _f64(sys.x if x is None else x).copy()
    T = _f64(sys.T)
    mu = _f64(mu_ex)
    off, idx = bond_csr
    fxm = fxv = fmm = fmv = None
    if fix_x is not None:
        fxm = np.ascontiguousarray(fix_x[0], dtype=np.uint8)
        fxv = _f64(fix_x[1])
    if fix_mu is not None:
        fmm = np.ascontiguousarray(fix_mu[0], dtype=np.uint8)
        fmv = _f64(fix_mu[1])
    st = lib().orc_diffuse_step_res(sys.n, xx.shape[0], _ptr(xx), _ptr(T), _ptr(mu), _ptr(off), _ptr(idx),
                                    float(dt), float(sys.nu0 if nu0 is None else nu0),
                                    float(sys.Qm if Qm is None else Qm), _ptr(fxm), _ptr(fxv), _ptr(fmm), _ptr(fmv))
    return int(st), xx


def transport_step(sys, mu_ex, bond_csr, dt, host=-1, tau=0.0, v=None, x=None, nu0=None, Qm=None):
    """One step of the transport variants (host exchange, ballistic term;
    definitions in the C source).  v: [S, n] rates for tau > 0 (in-out copy).
    Returns (status, x_new, v_new)."""
    xx = _f64(sys.x if x is None else x).copy()
    vv = None if v is None else _f64(v).copy()
    T = _f64(sys.T)
    mu = _f64(mu_ex)
    off, idx = bond_csr
    st = lib().orc_transport_step(sys.n, xx.shape[0], _ptr(xx), _ptr(T), _ptr(mu), _ptr(off), _ptr(idx),
                                  float(dt), float(sys.nu0 if nu0 is None else nu0),
                                  float(sys.Qm if Qm is None else Qm), int(host), float(tau), _ptr(vv))
    return int(st), xx, vv


def relax(sys, ftol, max_iter, fire: FireParams | None = None, skin=0.2, q=None, sigma=None, x=None, exact=False):
    """FIRE relaxation of (q, sigma) at fixed x (exact: the exact embedding
    average of free_energy_exact in place of the Taylor form).  Returns
    (status, iters, fmax, q_new, sigma_new)."""
    fire = fire or FireParams()
    ref = _SysRef(sys, q, sigma, x)
    qq = ref.q.copy()
    ss = ref.sigma.copy()
    P = make_potential(sys.pot)
    fp = _Fire(fire.dt0, fire.dt_max, fire.f_inc, fire.f_dec, fire.alpha0, fire.f_alpha, fire.sigma_max,
               fire.n_min, 0)
    it = C.c_int(0)
    fm = C.c_double(0.0)
    rl = sys.pot.r_cut + skin
    st = lib().orc_relax(C.byref(ref.s), _ptr(qq), _ptr(ss), C.byref(P), float(rl), float(ftol),
                         int(max_iter), C.byref(fp), C.byref(it), C.byref(fm), 1 if exact else 0)
    return int(st), int(it.value), float(fm.value), qq, ss


def fire_quadratic(kq, q0, iters, fire: FireParams | None = None):
    """The relaxation's FIRE update on F = 1/2 sum kq q^2 (q [3, n]): the
    trajectory [iters + 1, 3, n], the start first."""
    fire = fire or FireParams()
    q = _f64(q0).copy()
    n = q.shape[1]
    k = _f64(kq)
    traj = np.zeros((iters + 1,) + q.shape)
    fp = _Fire(fire.dt0, fire.dt_max, fire.f_inc, fire.f_dec, fire.alpha0, fire.f_alpha, fire.sigma_max,
               fire.n_min, 0)
    lib().orc_fire_quadratic(n, _ptr(k), _ptr(q), int(iters), C.byref(fp), _ptr(traj))
    return traj


def staggered(sys, n_steps, dt, ftol, max_iter, r_bond, fire=None, initial_relax=True, skin=0.2):
    """Staggered scheme (Sec. 4): relax, then per step: excess chemical
    potentials -> one Euler step of x -> relax at fixed x.  Returns
    (status, system copy at the end, list of per-step FIRE iteration counts)."""
    s = sys.copy()
    iters = []
    if initial_relax:
        st, it, fm, s.q, s.sigma = relax(s, ftol, max_iter, fire, skin)
        if st not in (OK, ERR_NO_CONVERGE):
            return st, s, iters
        iters.append(it)
    for _ in range(n_steps):
        st, off, idx = neighbors(s.q, s.L, r_list_for(s, skin))
        if st != OK:
            return st, s, iters
        fe = free_energy(s, (off, idx))
        if fe["status"] != OK:
            return fe["status"], s, iters
        boff, bidx = bonds(s, r_bond, off, idx)
        st, s.x = diffuse_step(s, fe["mu_ex"], (boff, bidx), dt)
        if st != OK:
            return st, s, iters
        st, it, fm, s.q, s.sigma = relax(s, ftol, max_iter, fire, skin)
        iters.append(it)
        if st not in (OK, ERR_NO_CONVERGE):
            return st, s, iters
    return OK, s, iters
