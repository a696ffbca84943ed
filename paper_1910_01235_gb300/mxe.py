"""Thin Python binding of the MXE C ABI (include/mxe.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library `libmxe.so`; PyTorch supplies device memory and the stream.  The
low-level functions carry the C names and return the C status code (plus the
C out-parameters); `MxeSystem` wraps one context with device-resident state
and raises `MxeError` on failure.  There is no CPU fallback: if the library
cannot be built or loaded, importing the functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

MAXS = 4
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_BOX_TOO_SMALL, ERR_NBR_OVERFLOW = 0, 1, 2, 3, 4, 5
ERR_GEOMETRY, ERR_NONFINITE, ERR_X_RANGE, ERR_NO_CONVERGE, ERR_STATE = 6, 7, 8, 9, 10
FP64, FP32_MIXED, FP32_FF = 0, 1, 2
PRECISIONS = {"fp64": FP64, "mixed": FP32_MIXED, "ff": FP32_FF}


class MxeError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        super().__init__(f"{where}: {mxe_status_string(status)} (status {status})")


class mxe_box(C.Structure):
    _fields_ = [("L", C.c_double * 3)]


class mxe_potential(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("cross_geomean", C.c_int32)] + [
        (nm, (C.c_double * MAXS) * MAXS) for nm in ("phi_A", "phi_p", "phi_r0", "f_xi", "f_q", "f_r0")
    ] + [("E", C.c_double * MAXS), ("r_switch", C.c_double), ("r_cut", C.c_double),
         ("lj", C.c_int32), ("pad", C.c_int32), ("lj_eps", (C.c_double * MAXS) * MAXS),
         ("lj_sigma", (C.c_double * MAXS) * MAXS)]


class mxe_state(C.Structure):
    _fields_ = [("n", C.c_int64), ("q", C.c_void_p), ("sigma", C.c_void_p), ("x", C.c_void_p),
                ("T", C.c_void_p), ("sublattice", C.c_void_p), ("mobile_mask", C.c_uint32),
                ("pad", C.c_uint32)]


class mxe_transport(C.Structure):
    _fields_ = [("host_species", C.c_int32), ("pad", C.c_int32), ("tau_r", C.c_double)]


class mxe_grad_info(C.Structure):
    _fields_ = [("relax_iters_total", C.c_int32), ("recomputed_steps", C.c_int32),
                ("cg_iters_total", C.c_int32), ("cg_iters_max", C.c_int32), ("cg_resid_max", C.c_double)]


class mxe_fire_params(C.Structure):
    _fields_ = [("dt0", C.c_double), ("dt_max", C.c_double), ("f_inc", C.c_double),
                ("f_dec", C.c_double), ("alpha0", C.c_double), ("f_alpha", C.c_double),
                ("sigma_max", C.c_double), ("n_min", C.c_int32), ("check_every", C.c_int32)]


EXPORTS = ["mxe_status_string", "mxe_create", "mxe_create_batch", "mxe_destroy", "mxe_build_neighbors",
           "mxe_export_neighbors", "mxe_export_bonds", "mxe_free_energy_grad", "mxe_free_energy_grad_async",
           "mxe_sync_status", "mxe_relax", "mxe_relax_info", "mxe_diffuse_step", "mxe_diffuse_step_async",
           "mxe_diffuse_step_noalloc", "mxe_timing_enable", "mxe_timing_read", "mxe_set_reservoirs",
           "mxe_set_dt_scale", "mxe_run_staggered", "mxe_autotune", "mxe_set_pass_shape",
           "mxe_potential_terms", "mxe_tangent", "mxe_flux_vjp", "mxe_unrolled_grad", "mxe_transport_step",
           "mxe_set_embedding", "mxe_element_param_grad", "mxe_unrolled_grad_multi", "mxe_set_pair_block",
           "mxe_get_pass_shape", "mxe_run_stats", "mxe_pair_form",
           "mxe_potential_pair_form"]
EMBED_TAYLOR, EMBED_EXACT = 0, 1
TIMING_NAME_LEN = 48
NOALLOC_SCRATCH_DOUBLES = 1 << 19


def noalloc_max_sites(S: int) -> int:
    return NOALLOC_SCRATCH_DOUBLES // (3 + 3 * S)

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libmxe.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            p, i64, d = C.c_void_p, C.c_int64, C.c_double
            L.mxe_status_string.restype = C.c_char_p
            L.mxe_status_string.argtypes = [C.c_int]
            L.mxe_create.argtypes = [C.POINTER(C.c_void_p), p, p, i64, C.c_int, p]
            L.mxe_create_batch.argtypes = [C.POINTER(C.c_void_p), C.c_int32, p, p, p, i64, C.c_int, p]
            L.mxe_set_dt_scale.argtypes = [p, p]
            L.mxe_relax_info.argtypes = [p, C.c_int32, p, p, p]
            L.mxe_run_staggered.argtypes = [p, p, C.c_int32, d, d, d, d, C.c_int32, p, C.POINTER(C.c_int32)]
            L.mxe_autotune.argtypes = [p, p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
            L.mxe_set_pass_shape.argtypes = [p, C.c_int32, C.c_int32]
            L.mxe_set_embedding.argtypes = [p, C.c_int32]
            L.mxe_set_pair_block.argtypes = [p, C.c_int32]
            L.mxe_get_pass_shape.argtypes = [p, p, p, p]
            L.mxe_pair_form.argtypes = [p, p, p]
            L.mxe_potential_pair_form.argtypes = [p, p, p, p, p]
            L.mxe_run_stats.argtypes = [p, p, p]
            L.mxe_element_param_grad.argtypes = [p, p, p]
            L.mxe_unrolled_grad_multi.argtypes = [p, p, C.c_int32, d, d, d, d, C.c_int32, p, C.c_int32, C.c_int32,
                                                  p, d, C.c_int32, p, p, p]
            i32p = C.POINTER(C.c_int32)
            L.mxe_potential_terms.argtypes = [p, i32p, i32p, p, p, p]
            L.mxe_tangent.argtypes = [p, p] + [p] * 10
            L.mxe_flux_vjp.argtypes = [p, p, p, d, d, d, p, p, p]
            L.mxe_transport_step.argtypes = [p, p, p, p, p, d, d, d]
            L.mxe_unrolled_grad.argtypes = [p, p, C.c_int32, d, d, d, d, C.c_int32, p, C.c_int32, p, d, C.c_int32,
                                            p, p, p]
            L.mxe_destroy.argtypes = [p]
            L.mxe_build_neighbors.argtypes = [p, p, d, d, C.POINTER(i64), C.POINTER(d)]
            L.mxe_export_neighbors.argtypes = [p, p, p]
            L.mxe_export_bonds.argtypes = [p, p, p, C.POINTER(i64)]
            L.mxe_free_energy_grad.argtypes = [p, p, p, p, p, p, p]
            L.mxe_free_energy_grad_async.argtypes = [p, p, p, p, p, p, p]
            L.mxe_sync_status.argtypes = [p]
            L.mxe_relax.argtypes = [p, p, d, C.c_int32, p, C.POINTER(C.c_int32), C.POINTER(d)]
            L.mxe_diffuse_step.argtypes = [p, p, p, d, d, d]
            L.mxe_diffuse_step_async.argtypes = [p, p, p, d, d, d]
            L.mxe_diffuse_step_noalloc.argtypes = [i64, C.c_int32, p, p, p, p, p, d, d, d, p]
            L.mxe_timing_enable.argtypes = [p, C.c_int32]
            L.mxe_set_reservoirs.argtypes = [p, p, p, p, p]
            L.mxe_timing_read.argtypes = [p, C.c_int32, p, p, p, C.POINTER(C.c_int32)]
            for nm in EXPORTS:
                if nm != "mxe_status_string":
                    getattr(L, nm).restype = C.c_int
            _lib = L
        return _lib


# ------------------------------------------------------------------ C names
def mxe_status_string(status) -> str:
    return lib().mxe_status_string(int(status)).decode()


def mxe_create(box: mxe_box, pot: mxe_potential, n: int, precision: int, stream: int):
    ctx = C.c_void_p()
    st = lib().mxe_create(C.byref(ctx), C.byref(box), C.byref(pot), int(n), int(precision), C.c_void_p(stream))
    return st, ctx


def mxe_create_batch(boxes, offsets, pot: mxe_potential, precision: int, stream: int):
    """boxes: sequence of 3-vectors; offsets: n_systems + 1 site offsets."""
    m = len(boxes)
    barr = (mxe_box * max(m, 1))()
    for b, L in enumerate(boxes):
        barr[b] = mxe_box((C.c_double * 3)(*[float(v) for v in L]))
    off = (C.c_int64 * (m + 1))(*[int(v) for v in offsets])
    ctx = C.c_void_p()
    st = lib().mxe_create_batch(C.byref(ctx), m, barr, off, C.byref(pot), int(offsets[-1]), int(precision),
                                C.c_void_p(stream))
    return st, ctx


def mxe_destroy(ctx):
    return lib().mxe_destroy(ctx)


def mxe_set_dt_scale(ctx, scale=None):
    if scale is None:
        return lib().mxe_set_dt_scale(ctx, None)
    arr = (C.c_double * len(scale))(*[float(v) for v in scale])
    return lib().mxe_set_dt_scale(ctx, arr)


def mxe_relax_info(ctx, m):
    it = (C.c_int32 * m)()
    fm = (C.c_double * m)()
    cv = (C.c_int32 * m)()
    st = lib().mxe_relax_info(ctx, m, it, fm, cv)
    return st, np.array(it[:], np.int32), np.array(fm[:]), np.array(cv[:], bool)


def mxe_run_staggered(ctx, state, n_steps, dt, nu0, Qm, ftol, max_iter, fire: mxe_fire_params | None = None):
    done = C.c_int32(0)
    st = lib().mxe_run_staggered(ctx, C.byref(state), int(n_steps), float(dt), float(nu0), float(Qm), float(ftol),
                                 int(max_iter), C.byref(fire) if fire is not None else None, C.byref(done))
    return st, done.value


def mxe_autotune(ctx, state):
    lanes, threads = C.c_int32(0), C.c_int32(0)
    st = lib().mxe_autotune(ctx, C.byref(state), C.byref(lanes), C.byref(threads))
    return st, lanes.value, threads.value


def mxe_set_pass_shape(ctx, lanes, threads):
    return lib().mxe_set_pass_shape(ctx, int(lanes), int(threads))


def mxe_set_embedding(ctx, mode):
    return lib().mxe_set_embedding(ctx, int(mode))


def mxe_potential_terms(ctx):
    """(n_phi, n_f, terms [T, 3] = (A, kappa, lambda), phi_of [4, 4], f_of [4, 4])."""
    nphi, nf = C.c_int32(0), C.c_int32(0)
    terms = (C.c_double * (3 * (MAXS * (MAXS + 1) // 2 + MAXS * MAXS)))()
    phi_of = (C.c_int32 * (MAXS * MAXS))()
    f_of = (C.c_int32 * (MAXS * MAXS))()
    st = lib().mxe_potential_terms(ctx, C.byref(nphi), C.byref(nf), terms, phi_of, f_of)
    T = nphi.value + nf.value
    return (st, nphi.value, nf.value, np.array(terms[:3 * T]).reshape(T, 3),
            np.array(phi_of[:]).reshape(MAXS, MAXS), np.array(f_of[:]).reshape(MAXS, MAXS))


def mxe_tangent(ctx, state, dq, dsigma, dx, gq, gs, mu, gq_t, gs_t, mu_t, dterm):
    """All arguments after the state are device pointers (0 = none)."""
    return lib().mxe_tangent(ctx, C.byref(state), *[C.c_void_p(v or 0) for v in
                                                    (dq, dsigma, dx, gq, gs, mu, gq_t, gs_t, mu_t, dterm)])


def mxe_transport_step(ctx, state, host, tau, mu_ex_ptr, v_ptr, dt, nu0, Qm):
    opt = mxe_transport(int(host), 0, float(tau))
    return lib().mxe_transport_step(ctx, C.byref(state), C.byref(opt), C.c_void_p(mu_ex_ptr or 0),
                                    C.c_void_p(v_ptr or 0), float(dt), float(nu0), float(Qm))


def mxe_flux_vjp(ctx, state, mu_ex, dt, nu0, Qm, xbar_next, xbar, mubar):
    return lib().mxe_flux_vjp(ctx, C.byref(state), C.c_void_p(mu_ex), float(dt), float(nu0), float(Qm),
                              C.c_void_p(xbar_next), C.c_void_p(xbar), C.c_void_p(mubar))


def mxe_unrolled_grad(ctx, state, n_steps, dt, nu0, Qm, ftol, max_iter, fire, every, w_ptr, cg_tol, cg_max,
                      n_terms, dx0_ptr=0):
    dterm = (C.c_double * max(2 * n_terms, 1))()
    info = mxe_grad_info()
    st = lib().mxe_unrolled_grad(ctx, C.byref(state), int(n_steps), float(dt), float(nu0), float(Qm), float(ftol),
                                 int(max_iter), C.byref(fire) if fire is not None else None, int(every),
                                 C.c_void_p(w_ptr), float(cg_tol), int(cg_max), dterm, C.c_void_p(dx0_ptr or 0),
                                 C.byref(info))
    return st, np.array(dterm[:2 * n_terms]), {nm: getattr(info, nm) for nm, _ in mxe_grad_info._fields_}


def mxe_unrolled_grad_multi(ctx, state, n_steps, dt, nu0, Qm, ftol, max_iter, fire, every, n_obj, w_ptr, cg_tol,
                            cg_max, n_terms, dx0_ptr=0):
    dterm = (C.c_double * max(2 * n_terms * n_obj, 1))()
    info = mxe_grad_info()
    st = lib().mxe_unrolled_grad_multi(ctx, C.byref(state), int(n_steps), float(dt), float(nu0), float(Qm),
                                       float(ftol), int(max_iter), C.byref(fire) if fire is not None else None,
                                       int(every), int(n_obj), C.c_void_p(w_ptr), float(cg_tol), int(cg_max), dterm,
                                       C.c_void_p(dx0_ptr or 0), C.byref(info))
    return (st, np.array(dterm[:2 * n_terms * n_obj]).reshape(n_obj, 2 * n_terms),
            {nm: getattr(info, nm) for nm, _ in mxe_grad_info._fields_})


def mxe_build_neighbors(ctx, state: mxe_state, skin: float, r_bond: float):
    npairs = C.c_int64(0)
    rl = C.c_double(0.0)
    st = lib().mxe_build_neighbors(ctx, C.byref(state), float(skin), float(r_bond), C.byref(npairs), C.byref(rl))
    return st, npairs.value, rl.value


def mxe_export_neighbors(ctx, offsets_ptr: int, idx_ptr: int):
    return lib().mxe_export_neighbors(ctx, C.c_void_p(offsets_ptr), C.c_void_p(idx_ptr))


def mxe_export_bonds(ctx, offsets_ptr: int, idx_ptr: int):
    nb = C.c_int64(0)
    st = lib().mxe_export_bonds(ctx, C.c_void_p(offsets_ptr), C.c_void_p(idx_ptr), C.byref(nb))
    return st, nb.value


def mxe_free_energy_grad(ctx, state, F4, gq, gs, mu_ex, mu, asynchronous=False):
    fn = lib().mxe_free_energy_grad_async if asynchronous else lib().mxe_free_energy_grad
    return fn(ctx, C.byref(state), *[C.c_void_p(p) for p in (F4, gq, gs, mu_ex, mu)])


def mxe_sync_status(ctx):
    return lib().mxe_sync_status(ctx)


def mxe_relax(ctx, state, ftol, max_iter, fire: mxe_fire_params | None = None):
    it = C.c_int32(0)
    fm = C.c_double(0.0)
    st = lib().mxe_relax(ctx, C.byref(state), float(ftol), int(max_iter),
                         C.byref(fire) if fire is not None else None, C.byref(it), C.byref(fm))
    return st, it.value, fm.value


def mxe_diffuse_step(ctx, state, mu_ex_ptr, dt, nu0, Qm, asynchronous=False):
    fn = lib().mxe_diffuse_step_async if asynchronous else lib().mxe_diffuse_step
    return fn(ctx, C.byref(state), C.c_void_p(mu_ex_ptr or 0), float(dt), float(nu0), float(Qm))


def mxe_set_reservoirs(ctx, fix_x_mask_ptr=0, fix_x_value_ptr=0, fix_mu_mask_ptr=0, fix_mu_value_ptr=0):
    return lib().mxe_set_reservoirs(ctx, *[C.c_void_p(p) for p in (fix_x_mask_ptr, fix_x_value_ptr,
                                                                   fix_mu_mask_ptr, fix_mu_value_ptr)])


def mxe_timing_enable(ctx, enable: bool):
    return lib().mxe_timing_enable(ctx, 1 if enable else 0)


def mxe_timing_read(ctx, max_entries=64):
    """Returns (status, {class: (launches, total_ms)}) and clears the record."""
    names = C.create_string_buffer(max_entries * TIMING_NAME_LEN)
    counts = (C.c_int64 * max_entries)()
    total = (C.c_double * max_entries)()
    k = C.c_int32(0)
    st = lib().mxe_timing_read(ctx, max_entries, names, counts, total, C.byref(k))
    out = {}
    for e in range(k.value):
        nm = names.raw[e * TIMING_NAME_LEN:(e + 1) * TIMING_NAME_LEN].split(b"\0", 1)[0].decode()
        out[nm] = (int(counts[e]), float(total[e]))
    return st, out


def mxe_diffuse_step_noalloc(n, S, x_ptr, T_ptr, mu_ex_ptr, bond_off_ptr, bond_idx_ptr, dt, nu0, Qm, stream):
    """Euler step with no device allocation (see include/mxe.h)."""
    return lib().mxe_diffuse_step_noalloc(int(n), int(S), C.c_void_p(x_ptr), C.c_void_p(T_ptr),
                                          C.c_void_p(mu_ex_ptr), C.c_void_p(bond_off_ptr),
                                          C.c_void_p(bond_idx_ptr), float(dt), float(nu0), float(Qm),
                                          C.c_void_p(stream))


def potential_pair_form(pot):
    """(table pattern, power form, m [2], n [2]) of a potential, decided on the
    host as a context would (include/mxe.h, mxe_potential_pair_form)."""
    P = make_potential(pot)
    v = (C.c_int32 * 6)()
    st = lib().mxe_potential_pair_form(C.byref(P), C.byref(v, 0), C.byref(v, 4), C.byref(v, 8), C.byref(v, 16))
    if st != OK:
        raise MxeError(st, "mxe_potential_pair_form")
    return v[0], v[1], (v[2], v[3]), (v[4], v[5])


# ------------------------------------------------------------------ helpers
def make_potential(pot) -> mxe_potential:
    P = mxe_potential()
    S = pot.n_species
    P.n_species = S
    P.cross_geomean = 1 if pot.cross_geomean else 0
    for nm in ("phi_A", "phi_p", "phi_r0", "f_xi", "f_q", "f_r0"):
        tab, dst = getattr(pot, nm), getattr(P, nm)
        for k in range(MAXS):
            for l in range(MAXS):
                dst[k][l] = float(tab[k, l]) if (k < S and l < S) else (1.0 if nm.endswith("r0") else 0.0)
    for k in range(S):
        P.E[k] = float(pot.E[k])
    P.r_switch, P.r_cut = float(pot.r_switch), float(pot.r_cut)
    if getattr(pot, "lj", False):
        P.lj = 1
        for k in range(S):
            for l in range(S):
                P.lj_eps[k][l] = float(pot.lj_eps[k, l])
                P.lj_sigma[k][l] = float(pot.lj_sigma[k, l])
    return P


def make_fire(dt0=0.02, dt_max=0.1, f_inc=1.1, f_dec=0.5, alpha0=0.1, f_alpha=0.99, n_min=5, check_every=16,
              sigma_max=0.0):
    return mxe_fire_params(dt0, dt_max, f_inc, f_dec, alpha0, f_alpha, sigma_max, n_min, check_every)


def _ptr(t):
    return 0 if t is None else int(t.data_ptr())


class MxeSystem:
    """One context plus device-resident state (torch tensors on `device`)."""

    def __init__(self, sys, precision="fp64", device="cuda:0", stream=None, skin=0.2, r_bond=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.sys = sys
        self.n, self.S = sys.n, sys.S
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        dev = self.device
        self.q = torch.as_tensor(np.ascontiguousarray(sys.q), dtype=torch.float64, device=dev).contiguous()
        self.sigma = torch.as_tensor(np.ascontiguousarray(sys.sigma), dtype=torch.float64, device=dev).contiguous()
        self.x = torch.as_tensor(np.ascontiguousarray(sys.x), dtype=torch.float64, device=dev).contiguous()
        self.T = torch.as_tensor(np.ascontiguousarray(sys.T), dtype=torch.float64, device=dev).contiguous()
        self.sub = torch.as_tensor(np.ascontiguousarray(sys.sublattice), dtype=torch.uint8, device=dev).contiguous()
        self.F4 = torch.zeros(4, dtype=torch.float64, device=dev)
        self.gq = torch.zeros((3, self.n), dtype=torch.float64, device=dev)
        self.gs = torch.zeros(self.n, dtype=torch.float64, device=dev)
        self.mu_ex = torch.zeros((self.S, self.n), dtype=torch.float64, device=dev)
        self.mu = torch.zeros((self.S, self.n), dtype=torch.float64, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.pot = make_potential(sys.pot)
        with torch.cuda.device(dev):
            self._create()
        self.skin = skin
        # bonds: nearest neighbours of the FCC sublattice (a/sqrt2), cut halfway to the second shell (a)
        self.r_bond = r_bond if r_bond is not None else 0.5 * (sys.a / np.sqrt(2.0) + sys.a)
        self.state = mxe_state()
        self._refresh_state()

    def _create(self):
        self.box = mxe_box((C.c_double * 3)(*[float(v) for v in self.sys.L]))
        st, self.ctx = mxe_create(self.box, self.pot, self.n, self.precision, self.stream.cuda_stream)
        if st != OK:
            raise MxeError(st, "mxe_create")

    def _refresh_state(self):
        s = self.state
        s.n = self.n
        s.q, s.sigma, s.x, s.T = _ptr(self.q), _ptr(self.sigma), _ptr(self.x), _ptr(self.T)
        s.sublattice = _ptr(self.sub)
        s.mobile_mask = int(self.sys.mobile_mask)

    def close(self):
        if getattr(self, "ctx", None):
            mxe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where, allow=()):
        if st != OK and st not in allow:
            raise MxeError(st, where)
        return st

    def build_neighbors(self):
        st, npairs, rl = mxe_build_neighbors(self.ctx, self.state, self.skin, self.r_bond)
        self._check(st, "mxe_build_neighbors")
        self.n_pairs, self.r_list = npairs, rl
        return npairs, rl

    def export_neighbors(self):
        t = self.torch
        off = t.zeros(self.n + 1, dtype=t.int32, device=self.device)
        idx = t.zeros(max(self.n_pairs, 1), dtype=t.int32, device=self.device)
        self._check(mxe_export_neighbors(self.ctx, _ptr(off), _ptr(idx)), "mxe_export_neighbors")
        return off, idx[: self.n_pairs]

    def export_bonds(self):
        t = self.torch
        off = t.zeros(self.n + 1, dtype=t.int32, device=self.device)
        st, nb = mxe_export_bonds(self.ctx, _ptr(off), 0)
        self._check(st, "mxe_export_bonds")
        idx = t.zeros(max(nb, 1), dtype=t.int32, device=self.device)
        st, nb = mxe_export_bonds(self.ctx, _ptr(off), _ptr(idx))
        self._check(st, "mxe_export_bonds")
        return off, idx[:nb]

    def free_energy_grad(self, with_mu=True, asynchronous=False):
        st = mxe_free_energy_grad(self.ctx, self.state, _ptr(self.F4), _ptr(self.gq), _ptr(self.gs),
                                  _ptr(self.mu_ex), _ptr(self.mu) if with_mu else 0, asynchronous)
        return self._check(st, "mxe_free_energy_grad")

    def sync_status(self, allow=()):
        return self._check(mxe_sync_status(self.ctx), "mxe_sync_status", allow)

    def relax(self, ftol, max_iter, fire=None, allow=(ERR_NO_CONVERGE,)):
        st, it, fm = mxe_relax(self.ctx, self.state, ftol, max_iter, fire)
        self._check(st, "mxe_relax", allow)
        return st, it, fm

    def diffuse_step(self, dt, mu_ex=None, nu0=None, Qm=None, asynchronous=False, allow=()):
        st = mxe_diffuse_step(self.ctx, self.state, _ptr(mu_ex), dt,
                              self.sys.nu0 if nu0 is None else nu0, self.sys.Qm if Qm is None else Qm,
                              asynchronous)
        return self._check(st, "mxe_diffuse_step", allow)

    def transport_step(self, dt, host=-1, tau=0.0, v=None, mu_ex=None, nu0=None, Qm=None, allow=()):
        """One step of the transport variants (mxe_transport_step): exchange
        with a host species and/or the ballistic term; v: [S, n] rates."""
        st = mxe_transport_step(self.ctx, self.state, host, tau, _ptr(mu_ex), _ptr(v), dt,
                                self.sys.nu0 if nu0 is None else nu0, self.sys.Qm if Qm is None else Qm)
        return self._check(st, "mxe_transport_step", allow)

    def set_reservoirs(self, fix_x=None, fix_mu=None):
        """fix_x / fix_mu: (mask [n] bool, values [S, n]) numpy arrays or None
        (Sec. 4: setatomicfraction / setchemicalpotential)."""
        t = self.torch
        self._res = []
        ptrs = []
        for grp in (fix_x, fix_mu):
            if grp is None:
                ptrs += [0, 0]
                continue
            m = t.as_tensor(np.ascontiguousarray(grp[0], dtype=np.uint8), device=self.device).contiguous()
            v = t.as_tensor(np.ascontiguousarray(grp[1], dtype=np.float64), device=self.device).contiguous()
            self._res += [m, v]
            ptrs += [_ptr(m), _ptr(v)]
        self._check(mxe_set_reservoirs(self.ctx, *ptrs), "mxe_set_reservoirs")

    def relax_info(self):
        """Per-system (iterations, fmax, converged) of the last relaxation."""
        st, it, fm, cv = mxe_relax_info(self.ctx, getattr(self, "n_systems", 1))
        self._check(st, "mxe_relax_info")
        return it, fm, cv

    def run_staggered(self, n_steps, dt, ftol, max_iter, fire=None, nu0=None, Qm=None, allow=()):
        """n_steps staggered steps replayed from one captured CUDA graph."""
        st, done = mxe_run_staggered(self.ctx, self.state, n_steps, dt, self.sys.nu0 if nu0 is None else nu0,
                                     self.sys.Qm if Qm is None else Qm, ftol, max_iter, fire)
        self._check(st, "mxe_run_staggered", allow)
        return st, done

    def run_stats(self):
        """(graph launches, kernels per step) of the last run_staggered."""
        v = (C.c_int32 * 2)()
        self._check(lib().mxe_run_stats(self.ctx, C.byref(v, 0), C.byref(v, 4)), "mxe_run_stats")
        return tuple(v)

    def autotune(self):
        st, lanes, threads = mxe_autotune(self.ctx, self.state)
        self._check(st, "mxe_autotune")
        return lanes, threads

    def set_pass_shape(self, lanes, threads, pair_threads=None):
        self._check(mxe_set_pass_shape(self.ctx, lanes, threads), "mxe_set_pass_shape")
        if pair_threads is not None:
            self._check(lib().mxe_set_pair_block(self.ctx, int(pair_threads)), "mxe_set_pair_block")

    def pass_shape(self):
        """(lanes per site, threads per block, pairs per block of the pair kernels)."""
        v = (C.c_int32 * 3)()
        self._check(lib().mxe_get_pass_shape(self.ctx, C.byref(v, 0), C.byref(v, 4), C.byref(v, 8)),
                    "mxe_get_pass_shape")
        return tuple(v)

    def pair_form(self):
        """(table pattern, power form) of the pair kernels (see include/mxe.h)."""
        v = (C.c_int32 * 2)()
        self._check(lib().mxe_pair_form(self.ctx, C.byref(v, 0), C.byref(v, 4)), "mxe_pair_form")
        return tuple(v)

    def set_embedding(self, mode):
        """"taylor" (Eq. F_taylor_mxe, default) or "exact" (App. A's rule over
        each site and its neighbours inside r_cut)."""
        m = {"taylor": EMBED_TAYLOR, "exact": EMBED_EXACT}[mode] if isinstance(mode, str) else int(mode)
        self._check(mxe_set_embedding(self.ctx, m), "mxe_set_embedding")

    # ---------------------------------------------------------- second order
    def potential_terms(self):
        st, nphi, nf, terms, phi_of, f_of = mxe_potential_terms(self.ctx)
        self._check(st, "mxe_potential_terms")
        return nphi, nf, terms, phi_of, f_of

    def tangent(self, dq=None, dsigma=None, dx=None):
        """Values and directional derivatives of (dF/dq, dF/dsigma, mu_ex) and
        of the term sensitivities along (dq, dsigma, dx) (device tensors or None)."""
        t = self.torch
        nphi, nf, _, _, _ = self.potential_terms()
        T = nphi + nf
        z = lambda *shape: t.zeros(shape, dtype=t.float64, device=self.device)
        out = dict(gq=z(3, self.n), gs=z(self.n), mu_ex=z(self.S, self.n), gq_t=z(3, self.n), gs_t=z(self.n),
                   mu_ex_t=z(self.S, self.n), dterm=z(4 * T))
        st = mxe_tangent(self.ctx, self.state, _ptr(dq), _ptr(dsigma), _ptr(dx), _ptr(out["gq"]), _ptr(out["gs"]),
                         _ptr(out["mu_ex"]), _ptr(out["gq_t"]), _ptr(out["gs_t"]), _ptr(out["mu_ex_t"]),
                         _ptr(out["dterm"]))
        self._check(st, "mxe_tangent")
        return out

    def flux_vjp(self, mu_ex, dt, xbar_next, nu0=None, Qm=None):
        t = self.torch
        xbar = t.zeros_like(xbar_next)
        mubar = t.zeros_like(xbar_next)
        st = mxe_flux_vjp(self.ctx, self.state, _ptr(mu_ex), dt, self.sys.nu0 if nu0 is None else nu0,
                          self.sys.Qm if Qm is None else Qm, _ptr(xbar_next), _ptr(xbar), _ptr(mubar))
        self._check(st, "mxe_flux_vjp")
        return xbar, mubar

    def unrolled_grad(self, n_steps, dt, w, ftol=1e-10, max_iter=50000, every=5, cg_tol=1e-10, cg_max=5000,
                      fire=None, nu0=None, Qm=None):
        """dL/d(term parameters) and dL/dx_0 for L = sum w x after n_steps
        staggered steps (mxe_unrolled_grad).  Returns (dterm [2 T], dx0, info)."""
        nphi, nf, _, _, _ = self.potential_terms()
        w = self.torch.as_tensor(w, dtype=self.torch.float64, device=self.device).contiguous()
        dx0 = self.torch.zeros_like(w)
        st, dterm, info = mxe_unrolled_grad(self.ctx, self.state, n_steps, dt, self.sys.nu0 if nu0 is None else nu0,
                                            self.sys.Qm if Qm is None else Qm, ftol, max_iter, fire, every,
                                            _ptr(w), cg_tol, cg_max, nphi + nf, _ptr(dx0))
        self._check(st, "mxe_unrolled_grad")
        return dterm, dx0, info

    def unrolled_grad_multi(self, n_steps, dt, w, ftol=1e-10, max_iter=50000, every=5, cg_tol=1e-10, cg_max=5000,
                            fire=None, nu0=None, Qm=None):
        """As unrolled_grad for the objectives w [n_obj, S, n] at once
        (mxe_unrolled_grad_multi).  Returns (dterm [n_obj, 2 T], dx0, info)."""
        nphi, nf, _, _, _ = self.potential_terms()
        w = self.torch.as_tensor(w, dtype=self.torch.float64, device=self.device).contiguous()
        dx0 = self.torch.zeros_like(w)
        st, dterm, info = mxe_unrolled_grad_multi(self.ctx, self.state, n_steps, dt,
                                                  self.sys.nu0 if nu0 is None else nu0,
                                                  self.sys.Qm if Qm is None else Qm, ftol, max_iter, fire, every,
                                                  w.shape[0], _ptr(w), cg_tol, cg_max, nphi + nf, _ptr(dx0))
        self._check(st, "mxe_unrolled_grad_multi")
        return dterm, dx0, info

    def staggered_step(self, dt, ftol, max_iter, fire=None):
        """One step of the staggered scheme (Sec. 4): excess chemical potentials,
        one Euler step of x, then relaxation of (q, sigma) at fixed x."""
        self.free_energy_grad(with_mu=False)
        self.diffuse_step(dt, mu_ex=self.mu_ex)
        return self.relax(ftol, max_iter, fire)


def element_param_grad(pot, dterm):
    """dL/d(A_e, p_e, q_e, r0_e) for each element e ([S, 4]) from the term
    sensitivities dterm = [dL/dc (T), dL/dlambda (T)] (mxe_element_param_grad:
    the closed-form chain rule, computed by the library)."""
    P = make_potential(pot)
    d = np.ascontiguousarray(dterm, dtype=np.float64)
    out = np.zeros((pot.n_species, 4))
    st = lib().mxe_element_param_grad(C.byref(P), d.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p))
    if st != OK:
        raise MxeError(st, "mxe_element_param_grad")
    return out


def concatenate(systems):
    """One System holding `systems` site block after site block, plus the
    site offsets (argument marshalling for a batched context).  The systems
    must share the potential, the mobile sublattice mask, the lattice
    parameter and nu0, Qm."""
    first = systems[0]
    for t in systems[1:]:
        if (t.S != first.S or t.mobile_mask != first.mobile_mask or t.a != first.a or t.nu0 != first.nu0
                or t.Qm != first.Qm):
            raise ValueError("systems of one batch must share S, mobile_mask, a, nu0 and Qm")
    offsets = np.zeros(len(systems) + 1, np.int64)
    offsets[1:] = np.cumsum([t.n for t in systems])
    merged = first.copy()
    merged.name = f"batch_{len(systems)}"
    merged.q = np.concatenate([t.q for t in systems], axis=1)
    merged.sigma = np.concatenate([t.sigma for t in systems])
    merged.x = np.concatenate([t.x for t in systems], axis=1)
    merged.T = np.concatenate([t.T for t in systems])
    merged.sublattice = np.concatenate([t.sublattice for t in systems])
    return merged, offsets


class MxeBatch(MxeSystem):
    """A batched context: many independent systems in one set of device
    arrays (sites concatenated; see mxe_create_batch).  F4 is [n_systems, 4];
    `part(t, b)` slices a per-site tensor to system b."""

    def __init__(self, systems, precision="fp64", device="cuda:0", stream=None, skin=0.2, r_bond=None):
        self.systems = list(systems)
        self.n_systems = len(self.systems)
        merged, self.offsets = concatenate(self.systems)
        super().__init__(merged, precision, device, stream, skin, r_bond)
        self.F4 = self.torch.zeros((self.n_systems, 4), dtype=self.torch.float64, device=self.device)

    def _create(self):
        boxes = [t.L for t in self.systems]
        st, self.ctx = mxe_create_batch(boxes, self.offsets, self.pot, self.precision, self.stream.cuda_stream)
        if st != OK:
            raise MxeError(st, "mxe_create_batch")

    def part(self, t, b):
        return t[..., int(self.offsets[b]):int(self.offsets[b + 1])]

    def set_dt_scale(self, scale=None):
        self._check(mxe_set_dt_scale(self.ctx, scale), "mxe_set_dt_scale")


def _autograd_function():
    import torch

    class MxeFreeEnergy(torch.autograd.Function):
        """F(q, sigma, x) as a differentiable scalar.  forward runs the CUDA
        free-energy pass (neighbour sets rebuilt for the given state); backward
        returns grad_out times (dF/dq, dF/dsigma, dF/dx) from that same pass,
        with the vacancy fraction dependent (dF/dx = mu)."""

        @staticmethod
        def forward(ctx, q, sigma, x, system):
            system.q.copy_(q.detach())
            system.sigma.copy_(sigma.detach())
            system.x.copy_(x.detach())
            system.build_neighbors()
            system.free_energy_grad(with_mu=True)
            ctx.save_for_backward(system.gq.clone(), system.gs.clone(), system.mu.clone())
            return system.F4[3].clone()

        @staticmethod
        def backward(ctx, grad_out):
            gq, gs, mu = ctx.saved_tensors
            return grad_out * gq, grad_out * gs, grad_out * mu, None

    return MxeFreeEnergy


_MxeFreeEnergy = None


def free_energy(q, sigma, x, system):
    """Differentiable free energy of `system` (an MxeSystem) at (q, sigma, x)."""
    global _MxeFreeEnergy
    if _MxeFreeEnergy is None:
        _MxeFreeEnergy = _autograd_function()
    return _MxeFreeEnergy.apply(q, sigma, x, system)
