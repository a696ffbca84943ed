"""Exact embedding average (App. B.2: App. A's rule over each site and its
neighbours inside r_cut) on the GPU against the oracle, element by element.

Tolerances as for the Taylor form: FP64 energies 1e-10 relative, gradients
and chemical potentials 1e-9 eV/A (eV) absolute; in the FP32 modes the
chemical potentials and energies come from FP64 passes (same bounds), the
forces from FP32 pair passes (1e-4 relative to max(max |g|, 1 eV/A)).
Relaxations of K FIRE iterations: 1e-9 A in FP64, 1e-4 A in FP32 modes.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_01235_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_01235_gb300 import mxe as M  # noqa: E402


def single(seed=3):
    s = W.perturb(W.config_vacancy_lattice(cells=5), 0.08, 0.03, seed=seed)
    return W.random_fractions(s, vac_min=0.02, seed=seed + 1)


def binary(seed=5):
    s = W.perturb(W.config_binary_alloy(cells=6), 0.08, 0.03, seed=seed)
    return W.random_fractions(s, vac_min=0.01, seed=seed + 1)


def slab(seed=9):
    # sigma ~ 0.03 A: with ~80 sites in an octahedral site's rule the nodes
    # move a site by sigma sqrt(3 N) (0.5 A here)
    s = W.config_interstitial_slab(5, 5, 3, top=100.0, xmax=0.4, seed=seed)
    s = W.perturb(s, 0.04, 0.01, seed=seed + 1)
    s.sigma *= 0.3
    return s


CASES = {"single": single, "binary": binary, "slab": slab}


def gpu_exact(s, prec):
    g = M.MxeSystem(s, prec)
    g.set_embedding("exact")
    g.build_neighbors()
    g.free_energy_grad()
    torch.cuda.synchronize()
    out = dict(F4=g.F4.cpu().numpy(), gq=g.gq.cpu().numpy(), gs=g.gs.cpu().numpy(),
               mu_ex=g.mu_ex.cpu().numpy(), mu=g.mu.cpu().numpy())
    return g, out


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
@pytest.mark.parametrize("case", list(CASES))
def test_exact_embedding_free_energy_parity(case, prec):
    s = CASES[case]()
    g, out = gpu_exact(s, prec)
    st, off, idx = O.neighbors(s.q, s.L, g.r_list)
    assert st == O.OK
    fe = O.free_energy_exact(s, (off, idx))
    assert fe["status"] == O.OK
    np.testing.assert_allclose(out["F4"], fe["F4"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(out["mu_ex"], fe["mu_ex"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(out["mu"], fe["mu"], rtol=1e-12, atol=1e-9)
    if prec == "fp64":
        np.testing.assert_allclose(out["gq"], fe["gq"], rtol=0, atol=1e-9)
        np.testing.assert_allclose(out["gs"], fe["gs"], rtol=0, atol=1e-9)
    else:
        scale = max(np.abs(fe["gq"]).max(), np.abs(fe["gs"]).max(), 1.0)
        assert np.abs(out["gq"] - fe["gq"]).max() <= 1e-4 * scale
        assert np.abs(out["gs"] - fe["gs"]).max() <= 1e-4 * scale
    # the Taylor form differs (the exact path really ran)
    ft = O.free_energy(s, (off, idx))
    assert abs(ft["F4"][0] - fe["F4"][0]) > 1e-6 * abs(fe["F4"][0])
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "ff"])
def test_exact_embedding_relaxation_parity(prec):
    """K FIRE iterations with the exact average (FP32 modes: FP32 node
    arithmetic for the forces) against the oracle's FIRE on the same form."""
    s = W.perturb(W.config_vacancy_lattice(cells=4, x0=0.97), 0.05, 0.02)
    K = 8
    g = M.MxeSystem(s, prec)
    g.set_embedding("exact")
    g.build_neighbors()
    st, it, fm = g.relax(0.0, K)
    assert st == M.ERR_NO_CONVERGE and it == K
    sto, ito, fmo, qo, so = O.relax(s, 0.0, K, exact=True)
    assert sto == O.ERR_NO_CONVERGE and ito == K
    tol = 1e-9 if prec == "fp64" else 1e-4
    np.testing.assert_allclose(g.q.cpu().numpy(), qo, rtol=0, atol=tol)
    np.testing.assert_allclose(g.sigma.cpu().numpy(), so, rtol=0, atol=tol)
    assert abs(fm - fmo) <= (1e-8 if prec == "fp64" else 1e-4 * max(fmo, 1.0))
    # back to the Taylor form: the same context evaluates it again
    g.set_embedding("taylor")
    t = s.copy()
    t.q, t.sigma = g.q.cpu().numpy(), g.sigma.cpu().numpy()
    g.build_neighbors()
    g.free_energy_grad()
    ft = O.free_energy(t, r_list=g.r_list)
    np.testing.assert_allclose(g.F4.cpu().numpy(), ft["F4"], rtol=1e-10, atol=1e-10)
    g.close()


def test_exact_embedding_rejected_by_derivative_calls():
    s = single()
    g = M.MxeSystem(s, "fp64")
    g.set_embedding("exact")
    g.build_neighbors()
    with pytest.raises(M.MxeError):
        g.tangent()
    assert M.mxe_set_embedding(g.ctx, 7) == M.ERR_ARG
    g.close()
