"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances:
  FP64 path: energies 1e-10 relative; dF/dq, dF/dsigma, mu 1e-9 eV/A (eV)
  absolute; x 1e-10 absolute after a run; neighbour and bond CSR bit-exact.
  FP32-compute paths: energies 1e-5 relative; gradients 1e-4 relative to
  max(max|g_oracle|, 1 eV/A); mu 1e-4 relative to max(max|mu_oracle|, 1 eV);
  x 1e-7 absolute after a run.
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

PRECS = ["fp64", "mixed", "ff"]


# ---------------------------------------------------------------- cases
def perturbed_single(cells=5, seed=3):
    s = W.perturb(W.config_vacancy_lattice(cells=cells), 0.08, 0.03, seed=seed)
    return W.random_fractions(s, vac_min=0.02, seed=seed + 1)


def perturbed_binary(cells=6, seed=5):
    s = W.perturb(W.config_binary_alloy(cells=cells), 0.08, 0.03, seed=seed)
    return W.random_fractions(s, vac_min=0.01, seed=seed + 1)


def small_slab(seed=9):
    s = W.config_interstitial_slab(5, 5, 3, top=100.0, xmax=0.4, seed=seed)
    return W.perturb(s, 0.04, 0.01, seed=seed + 1)


def ragged(seed=13):
    """A lattice with 37 sites removed at random: no regular row lengths."""
    s = perturbed_single(seed=seed)
    rng = np.random.default_rng(seed)
    keep = np.sort(rng.choice(s.n, s.n - 37, replace=False))
    t = s.copy()
    t.q, t.sigma, t.x, t.T = t.q[:, keep].copy(), t.sigma[keep].copy(), t.x[:, keep].copy(), t.T[keep].copy()
    t.sublattice = t.sublattice[keep].copy()
    return t


CASES = {
    "c1": lambda: W.config_vacancy_lattice(),
    "single": perturbed_single,
    "binary": perturbed_binary,
    "slab": small_slab,
    "ragged": ragged,
}


def stable_dt(s, r_bond, target=1e-3):
    """An Euler step for which the largest |x' - x| of the oracle is `target`
    (the explicit step is only stable for small enough dt, Sec. 4)."""
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    boff, bidx = O.bonds(s, r_bond, off, idx)
    trial = s.dt_default() * 1e-9
    st, x1 = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), trial)
    assert st == O.OK
    return trial * target / np.abs(x1 - s.x).max()


def r_bond_of(s):
    return 0.5 * (s.a / np.sqrt(2.0) + s.a)


def gpu_eval(sys, prec, **kw):
    g = M.MxeSystem(sys, prec, **kw)
    g.build_neighbors()
    g.free_energy_grad()
    torch.cuda.synchronize()
    out = dict(F4=g.F4.cpu().numpy(), gq=g.gq.cpu().numpy(), gs=g.gs.cpu().numpy(),
               mu_ex=g.mu_ex.cpu().numpy(), mu=g.mu.cpu().numpy(), r_list=g.r_list)
    return g, out


def oracle_eval(sys, r_list):
    st, off, idx = O.neighbors(sys.q, sys.L, r_list)
    assert st == O.OK
    fe = O.free_energy(sys, (off, idx))
    assert fe["status"] == O.OK
    return fe


def check_fp64(gpu, ora):
    np.testing.assert_allclose(gpu["F4"], ora["F4"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(gpu["gq"], ora["gq"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gpu["gs"], ora["gs"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gpu["mu_ex"], ora["mu_ex"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gpu["mu"], ora["mu"], rtol=1e-12, atol=1e-9)


def check_mixed(gpu, ora):
    """FP32 node arithmetic for the forces; with mu requested, mu and the
    energies come from the FP64 (mixed) or float-float (ff) passes."""
    gscale = max(np.abs(ora["gq"]).max(), np.abs(ora["gs"]).max(), 1.0)
    assert np.abs(gpu["gq"] - ora["gq"]).max() <= 1e-4 * gscale
    assert np.abs(gpu["gs"] - ora["gs"]).max() <= 1e-4 * gscale
    np.testing.assert_allclose(gpu["F4"], ora["F4"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(gpu["mu_ex"], ora["mu_ex"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gpu["mu"], ora["mu"], rtol=1e-12, atol=1e-9)


def check_forces_only(g, ora):
    """Forces-only call of an FP32 mode: energies from the FP32 pass (1e-5)."""
    st = M.mxe_free_energy_grad(g.ctx, g.state, M._ptr(g.F4), M._ptr(g.gq), M._ptr(g.gs), 0, 0)
    assert st == M.OK
    np.testing.assert_allclose(g.F4.cpu().numpy(), ora["F4"], rtol=1e-5)
    gscale = max(np.abs(ora["gq"]).max(), np.abs(ora["gs"]).max(), 1.0)
    assert np.abs(g.gq.cpu().numpy() - ora["gq"]).max() <= 1e-4 * gscale


# ---------------------------------------------------------------- neighbours
@pytest.mark.parametrize("case", ["c1", "single", "binary", "slab", "ragged", "tight"])
def test_neighbors_and_bonds_bit_exact(case):
    if case == "tight":
        s = W.perturb(W.config_vacancy_lattice(cells=4), 0.2, 0.0)
        skin = s.L[0] / 2 - 1e-9 - (s.pot.r_cut + np.sqrt(6.0) * s.sigma.max())
        g = M.MxeSystem(s, "fp64", skin=skin)
    else:
        s = CASES[case]()
        g = M.MxeSystem(s, "fp64")
    npairs, rl = g.build_neighbors()
    off, idx = g.export_neighbors()
    st, o_off, o_idx = O.neighbors(s.q, s.L, rl)
    assert st == O.OK
    np.testing.assert_array_equal(off.cpu().numpy(), o_off)
    np.testing.assert_array_equal(idx.cpu().numpy(), o_idx)
    boff, bidx = g.export_bonds()
    ob_off, ob_idx = O.bonds(s, g.r_bond, o_off, o_idx)
    np.testing.assert_array_equal(boff.cpu().numpy(), ob_off)
    np.testing.assert_array_equal(bidx.cpu().numpy(), ob_idx)
    g.close()


@pytest.mark.parametrize("case", ["single", "slab", "tight"])
def test_neighbor_builders_agree(case, monkeypatch):
    """The cell-staged builder and the warp-per-site fallback give the same CSR."""
    if case == "tight":
        s = W.perturb(W.config_vacancy_lattice(cells=4), 0.2, 0.0)
    else:
        s = CASES[case]()
    lists = []
    for per_site in (False, True):
        if per_site:
            monkeypatch.setenv("MXE_NEIGHBOR_PER_SITE", "1")
        g = M.MxeSystem(s, "fp64")
        g.build_neighbors()
        lists.append([t.cpu().numpy() for t in (*g.export_neighbors(), *g.export_bonds())])
        g.close()
    for a, b in zip(*lists):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("which", ["binary_256k", "slab_4M"])
def test_neighbors_full_size_sampled_rows(which):
    s = W.CONFIGS[which]()
    g = M.MxeSystem(s, "mixed")
    npairs, rl = g.build_neighbors()
    off, idx = g.export_neighbors()
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    assert off[-1] == npairs
    rng = np.random.default_rng(0)
    rows = np.concatenate([[0, s.n - 1], rng.choice(s.n, 30, replace=False)])
    for i in rows:
        np.testing.assert_array_equal(idx[off[i]:off[i + 1]], O.neighbor_row(s.q, s.L, rl, i))
    # every row is sorted and free of self-pairs
    lens = np.diff(off)
    starts = off[:-1]
    for i in rows:
        r = idx[off[i]:off[i + 1]]
        assert np.all(np.diff(r) > 0) and i not in r
    assert lens.max() <= 200 and starts[0] == 0
    g.close()


# ---------------------------------------------------------------- free energy
@pytest.mark.parametrize("case", list(CASES))
def test_free_energy_fp64_parity(case):
    s = CASES[case]()
    g, out = gpu_eval(s, "fp64")
    check_fp64(out, oracle_eval(s, out["r_list"]))
    g.close()


@pytest.mark.parametrize("prec", ["mixed", "ff"])
@pytest.mark.parametrize("case", list(CASES))
def test_free_energy_fp32_parity(prec, case):
    s = CASES[case]()
    g, out = gpu_eval(s, prec)
    ora = oracle_eval(s, out["r_list"])
    check_mixed(out, ora)
    check_forces_only(g, ora)
    g.close()


@pytest.mark.parametrize("nl", ["4", "16"])
def test_team_width_does_not_change_results(nl, monkeypatch):
    s = perturbed_binary()
    _, ref = gpu_eval(s, "fp64")
    monkeypatch.setenv("MXE_LANES_PER_SITE", nl)
    g, out = gpu_eval(s, "fp64")
    check_fp64(out, dict(ref))
    g.close()


def test_free_energy_full_size_binary_256k():
    """The 256,000-site binary alloy at the launch shape the benchmark times,
    every site compared (oracle on all host cores)."""
    s = W.perturb(W.config_binary_alloy(), 0.05, 0.02)
    ora = None
    for prec in PRECS:
        g, out = gpu_eval(s, prec)
        if ora is None:
            ora = oracle_eval(s, out["r_list"])
        (check_fp64 if prec == "fp64" else check_mixed)(out, ora)
        g.close()


# ---------------------------------------------------------------- diffusion
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["c1", "binary", "slab"])
def test_diffuse_step_parity_and_mass(prec, case):
    s = CASES[case]()
    if case == "binary":
        s = W.perturb(W.config_binary_alloy(cells=6), 0.03, 0.01)
    g, out = gpu_eval(s, prec)
    dt = stable_dt(s, g.r_bond)
    x0 = g.x.clone()
    g.diffuse_step(dt, mu_ex=g.mu_ex)
    x1 = g.x.cpu().numpy()
    st, off, idx = O.neighbors(s.q, s.L, out["r_list"])
    fe = O.free_energy(s, (off, idx))
    boff, bidx = O.bonds(s, g.r_bond, off, idx)
    st, xo = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), dt)
    assert st == O.OK
    assert np.abs(xo - s.x).max() > 1e-4       # the step moved mass
    # every precision mode evaluates mu and the step in FP64
    np.testing.assert_allclose(x1, xo, rtol=0, atol=1e-12)
    eps = np.finfo(float).eps
    for k in range(s.S):
        assert abs(x1[k].sum() - x0[k].sum().item()) <= 4 * s.n * eps
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "ff"])
def test_diffuse_with_reservoirs_parity(prec):
    """Reservoir groups (Sec. 4): held x after the step, held mu in every rate."""
    s = perturbed_single()
    rng = np.random.default_rng(31)
    mx = rng.random(s.n) < 0.1
    mm = (rng.random(s.n) < 0.1) & ~mx
    fix_x = (mx, np.clip(s.x + 0.05, 0.0, 0.97))
    fix_mu = (mm, np.full((1, s.n), -2.3))
    g, out = gpu_eval(s, prec)
    g.set_reservoirs(fix_x=fix_x, fix_mu=fix_mu)
    dt = stable_dt(s, g.r_bond, target=1e-4)
    g.diffuse_step(dt, mu_ex=g.mu_ex)
    st, off, idx = O.neighbors(s.q, s.L, out["r_list"])
    fe = O.free_energy(s, (off, idx))
    boff, bidx = O.bonds(s, g.r_bond, off, idx)
    st, xo = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), dt, fix_x=fix_x, fix_mu=fix_mu)
    assert st == O.OK
    x1 = g.x.cpu().numpy()
    np.testing.assert_array_equal(x1[:, mx], fix_x[1][:, mx])
    np.testing.assert_allclose(x1, xo, rtol=0, atol=1e-12)
    # without the groups the step differs
    g.set_reservoirs()
    g.x.copy_(torch.as_tensor(s.x))
    g.diffuse_step(dt, mu_ex=g.mu_ex)
    assert np.abs(g.x.cpu().numpy() - x1).max() > 1e-6
    g.close()


def test_diffuse_x_range_rejected_and_x_kept():
    s = perturbed_single()
    g, out = gpu_eval(s, "fp64")
    x0 = g.x.clone()
    dt = stable_dt(s, g.r_bond)
    st = g.diffuse_step(dt * 1e4, mu_ex=g.mu_ex, allow=(M.ERR_X_RANGE,))
    assert st == M.ERR_X_RANGE
    assert torch.equal(g.x, x0)
    # the context stays usable
    g.diffuse_step(dt, mu_ex=g.mu_ex)
    g.close()


def test_diffuse_without_mu_recomputes_it():
    s = perturbed_single()
    g, _ = gpu_eval(s, "fp64")
    dt = stable_dt(s, g.r_bond)
    ref = g.x.clone()
    g.diffuse_step(dt, mu_ex=g.mu_ex)
    a = g.x.clone()
    g.x.copy_(ref)
    g.diffuse_step(dt, mu_ex=None)
    assert torch.equal(g.x, a)
    g.close()


# ---------------------------------------------------------------- relaxation
@pytest.mark.parametrize("pot", ["variant_s", "literal"])
def test_relax_fixed_iterations_fp64_parity(pot):
    p = W.potential_variant_s() if pot == "variant_s" else W.potential_single()
    s = W.perturb(W.config_vacancy_lattice(cells=4, pot=p, x0=0.97), 0.05, 0.02)
    K = 12
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    st, it, fm = g.relax(0.0, K)
    assert st == M.ERR_NO_CONVERGE and it == K
    sto, ito, fmo, qo, so = O.relax(s, 0.0, K)
    assert sto == O.ERR_NO_CONVERGE and ito == K
    np.testing.assert_allclose(g.q.cpu().numpy(), qo, rtol=0, atol=1e-9)
    np.testing.assert_allclose(g.sigma.cpu().numpy(), so, rtol=0, atol=1e-9)
    assert abs(fm - fmo) <= 1e-8
    g.close()


@pytest.mark.parametrize("pot", ["literal", "variant_s"])
def test_relax_fixed_iterations_fp64_binary_parity(pot):
    """FP64 FIRE on the binary alloy: with the literal tables the half-list
    force pass takes the power form (rates 3/r0 and 5/r0: two exponentials
    per node, the terms as products), with the swapped exponents the general
    form; both against the oracle's trajectory at 1e-9 A."""
    s = W.perturb(W.config_binary_alloy(cells=4), 0.05, 0.02, seed=13)
    s = W.random_fractions(s, vac_min=0.01, seed=14)
    if pot == "variant_s":
        s.pot = W.potential_binary_variant_s()
    K = 12
    g = M.MxeSystem(s, "fp64")
    assert g.pair_form() == (1, 1)
    g.build_neighbors()
    st, it, fm = g.relax(0.0, K)
    assert st == M.ERR_NO_CONVERGE and it == K
    sto, ito, fmo, qo, so = O.relax(s, 0.0, K)
    assert sto == O.ERR_NO_CONVERGE and ito == K
    np.testing.assert_allclose(g.q.cpu().numpy(), qo, rtol=0, atol=1e-9)
    np.testing.assert_allclose(g.sigma.cpu().numpy(), so, rtol=0, atol=1e-9)
    assert abs(fm - fmo) <= 1e-8
    g.close()


@pytest.mark.parametrize("prec", PRECS)
def test_relax_converges_variant_s(prec):
    s = W.perturb(W.config_vacancy_lattice(pot=W.potential_variant_s(), x0=1.0), 0.05, 0.03)
    s.x[:] = 1.0
    g = M.MxeSystem(s, prec)
    g.build_neighbors()
    ftol = 1e-6 if prec == "fp64" else 2e-4
    st, it, fm = g.relax(ftol, 4000)
    assert st == M.OK and fm <= ftol
    sto, ito, fmo, qo, so = O.relax(s, ftol, 4000)
    assert sto == O.OK
    tol = 1e-7 if prec == "fp64" else 2e-4
    np.testing.assert_allclose(g.q.cpu().numpy(), qo, rtol=0, atol=tol)
    np.testing.assert_allclose(g.sigma.cpu().numpy(), so, rtol=0, atol=tol)
    if prec == "fp64":
        assert abs(it - ito) <= 2
    g.close()


def test_relax_rebuilds_neighbor_list_on_skin_violation():
    """The literal potential grows sigma quickly: the list must be rebuilt
    during the relaxation, and the result still matches the oracle (which
    rebuilds every iteration)."""
    s = W.config_vacancy_lattice()
    g = M.MxeSystem(s, "fp64", skin=0.05)
    g.build_neighbors()
    rl0 = g.r_list
    st, it, fm = g.relax(0.0, 14)
    sto, ito, fmo, qo, so = O.relax(s, 0.0, 14)
    np.testing.assert_allclose(g.sigma.cpu().numpy(), so, rtol=0, atol=1e-9)
    np.testing.assert_allclose(g.q.cpu().numpy(), qo, rtol=0, atol=1e-9)
    g.build_neighbors()
    assert g.r_list > rl0 + 0.05
    g.close()


# ---------------------------------------------------------------- staggered run
def dip_lattice():
    """500-site lattice (variant S) with x = 0.99 and one site at 0.5."""
    s = W.config_vacancy_lattice(pot=W.potential_variant_s())
    s.x[s.x == 0.0] = 0.5
    return s


def relaxed_dt(s, ftol, K, target, fire=None):
    r = s.copy()
    _, _, _, r.q, r.sigma = O.relax(s, ftol, K, fire)
    return stable_dt(r, r_bond_of(s), target=target)


@pytest.mark.parametrize("prec,ftol,K", [("fp64", 0.0, 15), ("fp64", 1e-5, 2000)])
def test_staggered_run_x_parity(prec, ftol, K):
    """Staggered scheme (Sec. 4): relax, then per step mu -> Euler step ->
    relax.  Fixed iteration counts compare FIRE trajectories; converged
    relaxations compare fixed points."""
    s = dip_lattice()
    steps = 5
    dt = relaxed_dt(s, ftol, K, 1e-3)
    g = M.MxeSystem(s, prec)
    g.build_neighbors()
    g.relax(ftol, K)
    for _ in range(steps):
        g.build_neighbors()
        g.staggered_step(dt, ftol, K)
    st, so, iters = O.staggered(s, steps, dt, ftol, K, g.r_bond)
    assert st == O.OK
    assert np.abs(so.x - s.x).max() > 1e-3          # mass moved
    np.testing.assert_allclose(g.x.cpu().numpy(), so.x, rtol=0, atol=1e-10)
    np.testing.assert_allclose(g.q.cpu().numpy(), so.q, rtol=0, atol=1e-8)
    g.close()


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_staggered_run_fp32_forces_x_within_1e7(prec):
    """FP32-compute paths on a stable binary alloy (x_v = 1e-3 as in the
    256,000-site workload): FIRE trajectories of fixed length with FP32
    forces, mu and the Euler step in FP64; x after the run within 1e-7."""
    s = W.perturb(W.config_binary_alloy(cells=5), 0.05, 0.02)
    s.pot = W.potential_binary_variant_s()
    steps, K = 5, 60
    dt = relaxed_dt(s, 0.0, K, 2e-4)
    g = M.MxeSystem(s, prec)
    g.build_neighbors()
    g.relax(0.0, K)
    for _ in range(steps):
        g.build_neighbors()
        g.staggered_step(dt, 0.0, K)
    st, so, iters = O.staggered(s, steps, dt, 0.0, K, g.r_bond)
    assert st == O.OK
    assert np.abs(so.x - s.x).max() > 1e-4
    dx = np.abs(g.x.cpu().numpy() - so.x).max()
    dq = np.abs(g.q.cpu().numpy() - so.q).max()
    print(f"{prec}: max |x - x_oracle| = {dx:.3e}, max |q - q_oracle| = {dq:.3e} A")
    assert dx <= 1e-7
    assert dq <= 1e-4
    g.close()


def test_sigma_box_keeps_empty_site_bounded():
    """A site with zero occupied fraction has nothing but -3 kB T ln sigma: with
    sigma_max its width stops at the bound (velocity zeroed) and the
    relaxation of the rest converges; GPU and oracle agree."""
    s = W.config_vacancy_lattice(pot=W.potential_variant_s())
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    fire = M.make_fire(sigma_max=0.5)
    st, it, fm = g.relax(1e-6, 3000, fire)
    assert st == M.OK
    sto, ito, fmo, qo, so = O.relax(s, 1e-6, 3000, O.FireParams(sigma_max=0.5))
    assert sto == O.OK
    sg = g.sigma.cpu().numpy()
    assert sg[s.x[0] == 0.0].max() == 0.5
    np.testing.assert_allclose(sg, so, rtol=0, atol=1e-7)
    np.testing.assert_allclose(g.q.cpu().numpy(), qo, rtol=0, atol=1e-7)
    g.close()


# ---------------------------------------------------------------- errors / edges
def test_status_geometry_and_state_restored():
    s = W.config_vacancy_lattice(cells=4)
    s.q[:, 1] = s.q[:, 0] + 0.3
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    st = M.mxe_free_energy_grad(g.ctx, g.state, M._ptr(g.F4), 0, 0, 0, 0)
    assert st == M.ERR_GEOMETRY
    q0 = g.q.clone()
    st, it, fm = g.relax(1e-6, 5, allow=(M.ERR_GEOMETRY,))
    assert st == M.ERR_GEOMETRY
    assert torch.equal(g.q, q0)
    g.close()


def test_status_nonfinite_on_zero_sigma():
    s = W.config_vacancy_lattice(cells=4)
    s.sigma[7] = 0.0
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    assert M.mxe_free_energy_grad(g.ctx, g.state, M._ptr(g.F4), 0, 0, 0, 0) == M.ERR_NONFINITE
    g.close()


def test_status_box_too_small_and_call_order():
    s = W.config_vacancy_lattice(cells=4)
    g = M.MxeSystem(s, "fp64", skin=3.0)
    assert M.mxe_free_energy_grad(g.ctx, g.state, M._ptr(g.F4), 0, 0, 0, 0) == M.ERR_STATE
    st, _, _ = M.mxe_build_neighbors(g.ctx, g.state, 3.0, 3.0)
    assert st == M.ERR_BOX_TOO_SMALL
    g.close()


def test_create_rejects_unsupported_species_count():
    pot = M.make_potential(W.potential_single())
    pot.n_species = 3
    box = M.mxe_box((M.C.c_double * 3)(18.0, 18.0, 18.0))
    st, ctx = M.mxe_create(box, pot, 10, M.FP64, 0)
    assert st == M.ERR_ARG and not ctx.value


@pytest.mark.parametrize("prec", PRECS)
def test_empty_system(prec):
    s = W.config_vacancy_lattice(cells=5)
    e = s.copy()
    e.q, e.sigma, e.x, e.T, e.sublattice = (np.zeros((3, 0)), np.zeros(0), np.zeros((1, 0)), np.zeros(0),
                                            np.zeros(0, np.uint8))
    g = M.MxeSystem(e, prec)
    npairs, _ = g.build_neighbors()
    assert npairs == 0
    g.free_energy_grad()
    assert np.all(g.F4.cpu().numpy() == 0.0)
    g.diffuse_step(1e-12, mu_ex=g.mu_ex)
    g.diffuse_step(1e-12, mu_ex=None)
    st, it, fm = g.relax(1e-6, 10)
    assert st == M.OK and it == 0
    g.close()


@pytest.mark.parametrize("case", ["single", "binary", "slab"])
def test_second_build_without_count_pass_is_bit_exact(case):
    """A context that has built once fills its next lists at a fixed stride
    (previous longest row plus a margin) without a count pass; rows that
    grow past the stride fall back to count + fill.  Both must give the
    oracle's sets bit for bit."""
    s = CASES[case]()
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    rng = np.random.default_rng(29)
    for grow in (0.0, 0.6):   # the second state: same widths, then much wider (longer rows)
        t = s.copy()
        t.q = s.q + rng.uniform(-0.05, 0.05, s.q.shape)
        t.sigma = s.sigma + grow
        g.q.copy_(torch.as_tensor(t.q, device=g.device))
        g.sigma.copy_(torch.as_tensor(t.sigma, device=g.device))
        g.build_neighbors()
        off, idx = (a.cpu().numpy() for a in g.export_neighbors())
        st, oo, oi = O.neighbors(t.q, t.L, g.r_list)
        assert st == O.OK
        np.testing.assert_array_equal(off, oo)
        np.testing.assert_array_equal(idx, oi)
        boff, bidx = (a.cpu().numpy() for a in g.export_bonds())
        bo, bi = O.bonds(t, g.r_bond, oo, oi)
        np.testing.assert_array_equal(boff, bo)
        np.testing.assert_array_equal(bidx, bi)
    g.close()
