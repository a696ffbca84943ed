"""The free energy as a torch.autograd.Function: backward against central
differences of the oracle's free energy (FP64, h = 1e-6) and against the
oracle's gradients, on binary alloy slabs with a 20 A vacuum gap (free
surfaces), including the full 108,000-site workload."""
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


def oracle_F(s, r_list):
    st, off, idx = O.neighbors(s.q, s.L, r_list, binned=s.n > 20000)
    assert st == O.OK
    fe = O.free_energy(s, (off, idx))
    assert fe["status"] == O.OK
    return fe


def check_backward(s, n_sites, seed, h=1e-6, tol=2e-7, hx=None, tolx=None, full_oracle=True):
    """backward of the CUDA free energy at (q, sigma, x) against central
    differences (step h, FP64) of the oracle's F at sampled components, and
    element by element against the oracle's analytic gradients.  tol: the
    error budget of the difference quotient (truncation ~h^2 plus the
    rounding of F, ~1e-16 |F| / h); hx, tolx: the same for x, whose third
    derivative kB T / x_v^2 (mixing entropy) is large at small x_v."""
    hx = h if hx is None else hx
    tolx = 10 * tol if tolx is None else tolx
    g = M.MxeSystem(s, "fp64")
    dev = g.device
    q = torch.tensor(s.q, device=dev, requires_grad=True)
    sg = torch.tensor(s.sigma, device=dev, requires_grad=True)
    x = torch.tensor(s.x, device=dev, requires_grad=True)
    F = M.free_energy(q, sg, x, g)
    F.backward()
    gq, gs, gx = q.grad.cpu().numpy(), sg.grad.cpu().numpy(), x.grad.cpu().numpy()
    rl = g.r_list
    fe = oracle_F(s, rl)
    assert abs(F.item() - fe["F4"][3]) <= 1e-10 * abs(fe["F4"][3])

    def fd(field, idx):
        step = hx if field == "x" else h
        vals = []
        for sgn in (1, -1):
            t = s.copy()
            arr = getattr(t, field)
            arr[idx] += sgn * step
            vals.append(oracle_F(t, rl)["F4"][3])
        return (vals[0] - vals[1]) / (2 * step)

    rng = np.random.default_rng(seed)
    for i in rng.choice(s.n, n_sites, replace=False):
        for c in range(3):
            assert abs(fd("q", (c, i)) - gq[c, i]) <= tol + 1e-7 * abs(gq[c, i])
        assert abs(fd("sigma", i) - gs[i]) <= tol + 1e-7 * abs(gs[i])
        for k in range(s.S):
            assert abs(fd("x", (k, i)) - gx[k, i]) <= tolx + 1e-7 * abs(gx[k, i])
    if full_oracle:
        np.testing.assert_allclose(gq, fe["gq"], rtol=0, atol=1e-9)
        np.testing.assert_allclose(gs, fe["gs"], rtol=0, atol=1e-9)
        np.testing.assert_allclose(gx, fe["mu"], rtol=1e-12, atol=1e-9)
    g.close()


def test_backward_matches_oracle_differences_and_gradients():
    check_backward(surface_alloy(), 6, 5)


def test_backward_full_size_surface_alloy_108k():
    """The 108,000-site surface alloy (30^3 cells, 20 A gap): every gradient
    element against the oracle's, and the oracle's differences at two
    sampled sites.  |F| ~ 3.5e5 eV here, so a step of 1e-6 would leave
    ~2e-5 of rounding in the quotient; h = 1e-4 keeps truncation (~1e-8)
    and rounding (~2e-7) both below the 1e-6 budget for q and sigma.  For x
    (x_v = 1e-3, third derivative ~9e4) h = 1e-5: truncation ~1.4e-6,
    rounding ~3.5e-6, budget 1e-5."""
    s = W.perturb(W.config_surface_alloy(), 0.03, 0.01, seed=43)
    check_backward(s, 2, 6, h=1e-4, tol=1e-6, hx=1e-5, tolx=1e-5)


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
