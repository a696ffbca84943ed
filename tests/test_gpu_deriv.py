"""Second-order passes, the Euler-step VJP and the gradient of unrolled
staggered steps, through the C ABI, against central differences of the oracle.

Every expected value is a difference quotient of oracle results (the plain
definition of a derivative); the CUDA side computes the same derivatives
analytically (forward-mode dual numbers, a hand-written VJP, conjugate
gradients on the relaxation Hessian).  Tolerances are set by the truncation
error of the differences (step h ~1e-5 relative: error ~h^2 ~1e-10 relative
plus rounding ~1e-16/h): 1e-6 of the largest component unless stated.
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


_RELAXED = {}


def alloy(seed=3, relaxed=False):
    """256-site binary alloy (x_A ~ U(0.85, 0.95), x_B = 0.999 - x_A), exponent-
    swapped tables so that the relaxation has a minimum, perturbed."""
    s = W.perturb(W.config_binary_alloy(cells=4), 0.05, 0.02, seed=seed)
    s.pot = W.potential_binary_variant_s()
    if relaxed:
        if seed not in _RELAXED:
            st, it, fm, q, sg = O.relax(s, 1e-10, 50000)
            assert st == O.OK
            _RELAXED[seed] = (q, sg)
        s.q, s.sigma = (a.copy() for a in _RELAXED[seed])
    return s


def oracle_grads(s, r_list):
    st, off, idx = O.neighbors(s.q, s.L, r_list)
    assert st == O.OK
    fe = O.free_energy(s, (off, idx))
    assert fe["status"] == O.OK
    return fe


def ctx_for(s):
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    return g


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def direction(s, seed=7):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1, 1, (3, s.n)), rng.uniform(-1, 1, s.n) * 0.1, rng.uniform(-1, 1, (s.S, s.n)) * 0.01)


def close(a, b, rel=1e-6):
    scale = max(np.abs(b).max(), 1e-30)
    err = np.abs(np.asarray(a) - np.asarray(b)).max()
    assert err <= rel * scale, (err, scale)


def test_tangent_pass_values_equal_the_gradient_pass():
    s = alloy()
    g = ctx_for(s)
    out = g.tangent()
    fe = oracle_grads(s, g.r_list)
    np.testing.assert_allclose(out["gq"].cpu().numpy(), fe["gq"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(out["gs"].cpu().numpy(), fe["gs"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(out["mu_ex"].cpu().numpy(), fe["mu_ex"], rtol=0, atol=1e-9)
    nphi, nf, _, _, _ = g.potential_terms()
    T = nphi + nf
    assert float(out["gq_t"].abs().max()) == 0.0 and float(out["dterm"][2 * T:].abs().max()) == 0.0
    g.close()


def test_parameter_gradient_against_oracle_differences():
    """dE_V/dtheta for the eight (A, p, q, r0) of both elements: per-term
    sensitivities from the CUDA pass, chain rule on the host, against central
    differences of the oracle's E_V."""
    s = alloy()
    g = ctx_for(s)
    nphi, nf, terms, phi_of, f_of = g.potential_terms()
    T = nphi + nf
    dterm = g.tangent()["dterm"].cpu().numpy()
    theta = W.theta_of(s.pot)
    base = s.pot
    grad = M.element_param_grad(base, dterm[:2 * T]).reshape(-1)
    fd = np.zeros_like(theta)
    for m in range(theta.size):
        h = 1e-5 * abs(theta[m])
        vals = []
        for sgn in (1, -1):
            t = s.copy()
            th = theta.copy()
            th[m] += sgn * h
            t.pot = W.binary_from_theta(th, base)
            vals.append(oracle_grads(t, g.r_list)["F4"][0])
        fd[m] = (vals[0] - vals[1]) / (2 * h)
    print("dE_V/dtheta", dict(zip(W.THETA_NAMES, grad)))
    np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
    g.close()


def test_hessian_vector_products_against_oracle_differences():
    s = alloy()
    g = ctx_for(s)
    dq, dsg, dx = direction(s)
    out = g.tangent(dev(dq), dev(dsg), dev(dx))
    h = 1e-5
    res = []
    for sgn in (1, -1):
        t = s.copy()
        t.q = s.q + sgn * h * dq
        t.sigma = s.sigma + sgn * h * dsg
        t.x = s.x + sgn * h * dx
        res.append(oracle_grads(t, g.r_list))
    for key, got in (("gq", "gq_t"), ("gs", "gs_t"), ("mu_ex", "mu_ex_t")):
        fd = (res[0][key] - res[1][key]) / (2 * h)
        close(out[got].cpu().numpy(), fd)
    g.close()


def test_mixed_parameter_state_derivatives_against_oracle_differences():
    """The tangent of the term sensitivities along v is d/dtheta of
    (grad E_V . v): compare through the chain rule with differences over
    theta of the oracle's gradients dotted with v."""
    s = alloy()
    g = ctx_for(s)
    nphi, nf, terms, phi_of, f_of = g.potential_terms()
    T = nphi + nf
    dq, dsg, dx = direction(s, seed=11)
    out = g.tangent(dev(dq), dev(dsg), dev(dx))
    dt_term = out["dterm"].cpu().numpy()[2 * T:]
    theta = W.theta_of(s.pot)
    base = s.pot
    got = M.element_param_grad(base, dt_term).reshape(-1)
    fd = np.zeros_like(theta)
    for m in range(theta.size):
        h = 1e-5 * abs(theta[m])
        vals = []
        for sgn in (1, -1):
            t = s.copy()
            th = theta.copy()
            th[m] += sgn * h
            t.pot = W.binary_from_theta(th, base)
            fe = oracle_grads(t, g.r_list)
            vals.append((fe["gq"] * dq).sum() + (fe["gs"] * dsg).sum() + (fe["mu_ex"] * dx).sum())
        fd[m] = (vals[0] - vals[1]) / (2 * h)
    np.testing.assert_allclose(got, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    g.close()


def euler_dt(s, r_bond, target=1e-4):
    fe = oracle_grads(s, O.r_list_for(s))
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    boff, bidx = O.bonds(s, r_bond, off, idx)
    trial = s.dt_default() * 1e-9
    st, x1 = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), trial)
    return trial * target / np.abs(x1 - s.x).max(), (boff, bidx), fe


def test_euler_step_vjp_against_oracle_differences():
    s = alloy()
    g = ctx_for(s)
    dt, bonds, fe = euler_dt(s, g.r_bond, target=1e-4)
    mu = fe["mu_ex"]
    rng = np.random.default_rng(13)
    w = rng.uniform(-1, 1, s.x.shape)
    vx = rng.uniform(-1, 1, s.x.shape) * 1e-3
    vm = rng.uniform(-1, 1, mu.shape) * 1e-2
    xbar, mubar = g.flux_vjp(dev(mu), dt, dev(w))
    got = (xbar.cpu().numpy() * vx).sum() + (mubar.cpu().numpy() * vm).sum()
    h = 1e-4
    vals = []
    for sgn in (1, -1):
        t = s.copy()
        t.x = s.x + sgn * h * vx
        st, x1 = O.diffuse_step(t, mu + sgn * h * vm, bonds, dt)
        assert st == O.OK
        vals.append((w * x1).sum())
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(got - fd) <= 1e-7 * max(abs(fd), 1e-12) + 1e-12, (got, fd)
    g.close()


# ---------------------------------------------------------------- unrolled steps
N_STEPS = 2


def unrolled_case():
    s = alloy(relaxed=True)
    rb = 0.5 * (s.a / np.sqrt(2.0) + s.a)
    dt, _, _ = euler_dt(s, rb, target=1e-4)
    rng = np.random.default_rng(17)
    w = np.zeros_like(s.x)
    w[1] = rng.uniform(-1, 1, s.n)          # a weighting of the B fractions
    return s, rb, dt, w


def oracle_L(s, pot, dt, w, rb, x0=None):
    t = s.copy()
    t.pot = pot
    if x0 is not None:
        t.x = x0
    st, so, iters = O.staggered(t, N_STEPS, dt, 1e-10, 50000, rb, initial_relax=True)
    assert st == O.OK
    return float((w * so.x).sum()), so


def test_unrolled_gradient_against_oracle_differences():
    """dL/dtheta (two of the eight parameters) and dL/dx_0 along a direction,
    for L = w . x after two staggered steps with converged relaxations,
    against central differences of the oracle's staggered run."""
    s, rb, dt, w = unrolled_case()
    g = ctx_for(s)
    nphi, nf, terms, phi_of, f_of = g.potential_terms()
    dterm, dx0, info = g.unrolled_grad(N_STEPS, dt, w, ftol=1e-10, every=1)
    print("info", info)
    L0, so = oracle_L(s, s.pot, dt, w, rb)
    np.testing.assert_allclose(g.x.cpu().numpy(), so.x, rtol=0, atol=1e-10)   # forward run
    theta = W.theta_of(s.pot)
    base = s.pot
    grad = M.element_param_grad(base, dterm).reshape(-1)
    for m in (W.THETA_NAMES.index("q_B"), W.THETA_NAMES.index("r0_A")):
        h = 3e-4 * abs(theta[m])
        vals = []
        for sgn in (1, -1):
            th = theta.copy()
            th[m] += sgn * h
            vals.append(oracle_L(s, W.binary_from_theta(th, base), dt, w, rb)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        print(W.THETA_NAMES[m], grad[m], fd)
        assert abs(grad[m] - fd) <= 1e-4 * abs(fd) + 1e-12, (W.THETA_NAMES[m], grad[m], fd)
    rng = np.random.default_rng(19)
    v = np.zeros_like(s.x)
    v[1] = rng.uniform(-1, 1, s.n) * 1e-4
    v[0] = -v[1]                          # exchange A for B, vacancy unchanged
    h = 1.0
    vals = [oracle_L(s, s.pot, dt, w, rb, x0=s.x + sgn * h * v)[0] for sgn in (1, -1)]
    fd = (vals[0] - vals[1]) / (2 * h)
    got = float((dx0.cpu().numpy() * v).sum())
    print("dL/dx0 . v", got, fd)
    assert abs(got - fd) <= 1e-4 * abs(fd) + 1e-12
    g.close()


def test_unrolled_gradient_checkpoint_interval_does_not_matter():
    s, rb, dt, w = unrolled_case()
    res = []
    for every in (1, 2, 5):
        g = ctx_for(s)
        dterm, dx0, info = g.unrolled_grad(4, dt, w, ftol=1e-10, every=every)
        res.append((dterm, dx0.cpu().numpy(), info))
        g.close()
    assert res[0][2]["recomputed_steps"] == 0 and res[1][2]["recomputed_steps"] > 0
    for dterm, dx0, info in res[1:]:
        np.testing.assert_allclose(dterm, res[0][0], rtol=1e-7, atol=1e-9 * np.abs(res[0][0]).max())
        np.testing.assert_allclose(dx0, res[0][1], rtol=0, atol=1e-7 * np.abs(res[0][1]).max())


def test_unrolled_gradient_rejects_fp32_contexts_and_reservoirs():
    s, rb, dt, w = unrolled_case()
    g = M.MxeSystem(s, "mixed")
    g.build_neighbors()
    st, dterm, info = M.mxe_unrolled_grad(g.ctx, g.state, 1, dt, s.nu0, s.Qm, 1e-10, 100, None, 1,
                                          M._ptr(dev(w)), 1e-10, 100, 5)
    assert st == M.ERR_ARG
    g.close()


def z_profile_weights(s, nbins):
    """Mean x_B of the sites in each of nbins slabs along z (the B-fraction
    z-profile): w[b] = indicator(bin b) / (sites in bin b) on species B."""
    z = s.q[2] % s.L[2]
    b = np.minimum((z / s.L[2] * nbins).astype(int), nbins - 1)
    w = np.zeros((nbins,) + s.x.shape)
    for k in range(nbins):
        m = b == k
        w[k, 1, m] = 1.0 / m.sum()
    return w


def test_z_profile_jacobian_shares_one_forward_sweep():
    """The whole B-fraction z-profile (4 bins) x 8 parameters from one call:
    every row equals the single-objective gradient of that bin, and two
    entries match central differences of the oracle's staggered run."""
    s, rb, dt, _ = unrolled_case()
    W4 = z_profile_weights(s, 4)
    g = ctx_for(s)
    dterm, dx0, info = g.unrolled_grad_multi(N_STEPS, dt, W4, ftol=1e-10, every=1)
    g.close()
    assert dterm.shape[0] == 4
    jac = np.array([M.element_param_grad(s.pot, dterm[b]).reshape(-1) for b in range(4)])
    for b in (0, 3):
        g = ctx_for(s)
        d1, x1, _ = g.unrolled_grad(N_STEPS, dt, W4[b], ftol=1e-10, every=1)
        g.close()
        np.testing.assert_allclose(dterm[b], d1, rtol=1e-9, atol=1e-12 * np.abs(d1).max())
        np.testing.assert_allclose(dx0[b].cpu().numpy(), x1.cpu().numpy(), rtol=0,
                                   atol=1e-9 * np.abs(x1.cpu().numpy()).max())
    theta = W.theta_of(s.pot)
    m = W.THETA_NAMES.index("p_B")
    h = 3e-4 * abs(theta[m])
    for b in (1, 2):
        vals = []
        for sgn in (1, -1):
            th = theta.copy()
            th[m] += sgn * h
            vals.append(oracle_L(s, W.binary_from_theta(th, s.pot), dt, W4[b], rb)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        print("bin", b, jac[b, m], fd)
        assert abs(jac[b, m] - fd) <= 1e-4 * abs(fd) + 1e-12
