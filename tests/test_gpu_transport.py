"""Transport variants (host exchange, ballistic term of Eq. Transport)
through the C ABI against the oracle, element by element (FP64 step: 1e-12
absolute in x and 1e-12 relative in the rates, as the Euler-step parity
tests)."""
import numpy as np
import pytest

import oracle as O
from paper_1910_01235_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_01235_gb300 import mxe as M  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def setup(s, prec="fp64"):
    g = M.MxeSystem(s, prec)
    g.build_neighbors()
    g.free_energy_grad()
    boff, bidx = (t.cpu().numpy() for t in g.export_bonds())
    return g, g.mu_ex.cpu().numpy(), (boff, bidx)


def cases():
    alloy = W.perturb(W.config_binary_alloy(cells=5), 0.04, 0.02, seed=61)       # x_v = 1e-3
    novac = W.perturb(W.config_binary_alloy(cells=4, seed=62), 0.04, 0.02, seed=63)
    novac.x[0] = 1.0 - novac.x[1]                                                # no vacancies
    single = W.random_fractions(W.perturb(W.config_vacancy_lattice(), 0.04, 0.02, seed=64), vac_min=0.05, seed=65)
    return {"alloy": alloy, "novac": novac, "single": single}


@pytest.mark.parametrize("case,host", [("alloy", 0), ("alloy", 1), ("novac", 0), ("single", -1), ("alloy", -1)])
def test_host_exchange_step_parity(case, host):
    s = cases()[case]
    g, mu, bonds = setup(s)
    dt = s.dt_default() * 0.05
    st, xo, _ = O.transport_step(s, mu, bonds, dt, host=host)
    assert st == O.OK
    g.transport_step(dt, host=host, mu_ex=g.mu_ex)
    np.testing.assert_allclose(g.x.cpu().numpy(), xo, rtol=0, atol=1e-12)
    assert np.abs(xo - s.x).max() > 1e-8
    if host >= 0:   # every species conserved, site totals unchanged
        x1 = g.x.cpu().numpy()
        np.testing.assert_allclose(x1.sum(axis=1), s.x.sum(axis=1), rtol=1e-12)
        np.testing.assert_allclose(x1.sum(axis=0), s.x.sum(axis=0), rtol=0, atol=1e-14)
    g.close()


def test_vacancy_variant_equals_the_euler_step():
    s = cases()["alloy"]
    g, mu, bonds = setup(s)
    dt = s.dt_default() * 0.05
    x0 = g.x.clone()
    g.diffuse_step(dt, mu_ex=g.mu_ex)
    ref = g.x.clone()
    g.x.copy_(x0)
    g.transport_step(dt, host=-1, tau=0.0, mu_ex=g.mu_ex)
    assert (g.x - ref).abs().max().item() <= 1e-14
    g.close()


@pytest.mark.parametrize("host,tau_scale", [(-1, 0.3), (0, 3.0)])
def test_ballistic_steps_parity(host, tau_scale):
    """Several steps carrying the rates v, against the oracle's steps."""
    s = cases()["alloy"]
    g, mu, bonds = setup(s)
    dt = s.dt_default() * 0.05
    tau = tau_scale * dt
    v = torch.zeros_like(g.x)
    xo, vo = s.x.copy(), np.zeros_like(s.x)
    for _ in range(4):
        g.transport_step(dt, host=host, tau=tau, v=v, mu_ex=g.mu_ex)
        st, xo, vo = O.transport_step(s, mu, bonds, dt, host=host, tau=tau, v=vo, x=xo)
        assert st == O.OK
    np.testing.assert_allclose(g.x.cpu().numpy(), xo, rtol=0, atol=1e-12)
    scale = np.abs(vo).max()
    np.testing.assert_allclose(v.cpu().numpy(), vo, rtol=0, atol=1e-12 * scale)
    assert np.abs(xo - s.x).max() > 1e-8
    g.close()


def test_range_error_keeps_x_and_rates():
    s = cases()["single"]
    g, mu, bonds = setup(s)
    v = dev(np.full(s.x.shape, 3.0))
    x0, v0 = g.x.clone(), v.clone()
    st = g.transport_step(s.dt_default() * 1e6, tau=1e-9, v=v, mu_ex=g.mu_ex, allow=(M.ERR_X_RANGE,))
    assert st == M.ERR_X_RANGE
    assert torch.equal(g.x, x0) and torch.equal(v, v0)
    g.close()


def test_transport_step_arguments():
    s = cases()["alloy"]
    g, mu, bonds = setup(s)
    assert M.mxe_transport_step(g.ctx, g.state, 2, 0.0, 0, 0, 1e-12, s.nu0, s.Qm) == M.ERR_ARG   # host >= S
    assert M.mxe_transport_step(g.ctx, g.state, -1, 1.0, 0, 0, 1e-12, s.nu0, s.Qm) == M.ERR_ARG  # tau needs v
    assert M.mxe_transport_step(g.ctx, g.state, -1, -1.0, 0, 0, 1e-12, s.nu0, s.Qm) == M.ERR_ARG
    # mu computed when not given: same result as with the pass's own mu
    x0 = g.x.clone()
    g.transport_step(s.dt_default() * 0.05, host=0)
    a = g.x.clone()
    g.x.copy_(x0)
    g.transport_step(s.dt_default() * 0.05, host=0, mu_ex=g.mu_ex)
    assert torch.equal(a, g.x)
    g.close()
