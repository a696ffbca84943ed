"""Thermalized Lennard-Jones pair terms (App. C.1) through the C ABI against
the oracle: free energy and gradients (FP64 tolerances: 1e-10 relative on
energies, 1e-9 absolute on gradients), a fixed-length relaxation, and the
Euler step; contexts other than FP64 are refused."""
import numpy as np
import pytest

import oracle as O
from paper_1910_01235_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_01235_gb300 import mxe as M  # noqa: E402


def lj_lattice(seed=3):
    s = W.config_vacancy_lattice(cells=5, pot=W.potential_lj())
    s = W.perturb(s, 0.05, 0.02, seed=seed)
    return W.random_fractions(s, vac_min=0.05, seed=seed + 1)


def test_lj_free_energy_fp64_parity():
    s = lj_lattice()
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    g.free_energy_grad()
    st, off, idx = O.neighbors(s.q, s.L, g.r_list)
    fe = O.free_energy(s, (off, idx))
    assert fe["status"] == O.OK
    np.testing.assert_allclose(g.F4.cpu().numpy(), fe["F4"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(g.gq.cpu().numpy(), fe["gq"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(g.gs.cpu().numpy(), fe["gs"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(g.mu_ex.cpu().numpy(), fe["mu_ex"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(g.mu.cpu().numpy(), fe["mu"], rtol=1e-12, atol=1e-9)
    g.close()


def test_lj_relax_and_euler_step_parity():
    s = lj_lattice(seed=5)
    K = 8
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    st, it, fm = g.relax(0.0, K)
    assert it == K
    sto, ito, fmo, qo, so = O.relax(s, 0.0, K)
    assert ito == K
    np.testing.assert_allclose(g.q.cpu().numpy(), qo, rtol=0, atol=1e-9)
    np.testing.assert_allclose(g.sigma.cpu().numpy(), so, rtol=0, atol=1e-9)
    r = s.copy()
    r.q, r.sigma = qo, so
    g.build_neighbors()
    g.free_energy_grad()
    st, off, idx = O.neighbors(r.q, r.L, g.r_list)
    fe = O.free_energy(r, (off, idx))
    boff, bidx = O.bonds(r, g.r_bond, off, idx)
    dt = r.dt_default() * 1e-3
    st, xo = O.diffuse_step(r, fe["mu_ex"], (boff, bidx), dt)
    assert st == O.OK
    g.diffuse_step(dt, mu_ex=g.mu_ex)
    np.testing.assert_allclose(g.x.cpu().numpy(), xo, rtol=0, atol=1e-12)
    assert np.abs(xo - r.x).max() > 1e-9
    g.close()


def test_lj_only_in_fp64_contexts():
    s = lj_lattice()
    for prec in ("mixed", "ff"):
        with pytest.raises(M.MxeError) as e:
            M.MxeSystem(s, prec)
        assert e.value.status == M.ERR_ARG
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    st = M.mxe_tangent(g.ctx, g.state, 0, 0, 0, M._ptr(g.gq), 0, 0, 0, 0, 0, 0)
    assert st == M.ERR_ARG
    g.close()
