"""The free energy as a torch.autograd.Function: backward against central
differences of the CUDA forward (FP64, h = 1e-6) and against the oracle's
gradients, on a binary alloy slab with a 20 A vacuum gap (free surfaces)."""
import numpy as np
import pytest

import oracle as O
from paper_1910_01235_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_01235_gb300 import mxe as M  # noqa: E402


def surface_alloy():
    s = W.config_surface_alloy(cells=4)
    s = W.perturb(s, 0.05, 0.02, seed=41)
    return W.random_fractions(s, vac_min=0.02, seed=42)


def test_backward_matches_central_differences_and_oracle():
    s = surface_alloy()
    g = M.MxeSystem(s, "fp64")
    dev = g.device
    q = torch.tensor(s.q, device=dev, requires_grad=True)
    sg = torch.tensor(s.sigma, device=dev, requires_grad=True)
    x = torch.tensor(s.x, device=dev, requires_grad=True)
    F = M.free_energy(q, sg, x, g)
    F.backward()
    gq, gs, gx = q.grad.cpu().numpy(), sg.grad.cpu().numpy(), x.grad.cpu().numpy()

    def F_at(qq, ss, xx):
        with torch.no_grad():
            return M.free_energy(qq, ss, xx, g).item()

    h = 1e-6
    rng = np.random.default_rng(5)
    for i in rng.choice(s.n, 6, replace=False):
        for c in range(3):
            qp, qm = q.detach().clone(), q.detach().clone()
            qp[c, i] += h
            qm[c, i] -= h
            fd = (F_at(qp, sg.detach(), x.detach()) - F_at(qm, sg.detach(), x.detach())) / (2 * h)
            assert abs(fd - gq[c, i]) <= 2e-7 + 1e-7 * abs(gq[c, i])
        sp, sm = sg.detach().clone(), sg.detach().clone()
        sp[i] += h
        sm[i] -= h
        fd = (F_at(q.detach(), sp, x.detach()) - F_at(q.detach(), sm, x.detach())) / (2 * h)
        assert abs(fd - gs[i]) <= 2e-7 + 1e-7 * abs(gs[i])
        for k in range(s.S):
            xp, xm = x.detach().clone(), x.detach().clone()
            xp[k, i] += h
            xm[k, i] -= h
            fd = (F_at(q.detach(), sg.detach(), xp) - F_at(q.detach(), sg.detach(), xm)) / (2 * h)
            assert abs(fd - gx[k, i]) <= 2e-6 + 1e-7 * abs(gx[k, i])
    st, off, idx = O.neighbors(s.q, s.L, g.r_list)
    fe = O.free_energy(s, (off, idx))
    np.testing.assert_allclose(gq, fe["gq"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gs, fe["gs"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gx, fe["mu"], rtol=1e-12, atol=1e-9)
    g.close()


def test_grad_out_scales_and_fp32_modes():
    s = surface_alloy()
    for prec in ("mixed", "ff"):
        g = M.MxeSystem(s, prec)
        q = torch.tensor(s.q, device=g.device, requires_grad=True)
        sg = torch.tensor(s.sigma, device=g.device, requires_grad=True)
        x = torch.tensor(s.x, device=g.device, requires_grad=True)
        F = M.free_energy(q, sg, x, g)
        (3.0 * F).backward()
        st, off, idx = O.neighbors(s.q, s.L, g.r_list)
        fe = O.free_energy(s, (off, idx))
        scale = max(np.abs(fe["gq"]).max(), 1.0)
        assert np.abs(q.grad.cpu().numpy() - 3.0 * fe["gq"]).max() <= 3e-4 * scale
        np.testing.assert_allclose(x.grad.cpu().numpy(), 3.0 * fe["mu"], rtol=1e-11, atol=3e-9)
        g.close()
