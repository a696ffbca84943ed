"""Batched ensembles, the graph-captured staggered loop and the autotuner,
through the C ABI, against the oracle run on each system alone.

A batch is a set of independent instances of the problem (Sec. 4), so every
per-system result must equal what the oracle gives for that system by itself:
neighbour and bond sets bit-exact (indices shifted by the system's first
site), energies and gradients at the FP64 tolerances of the single-system
tests (1e-10 relative, 1e-9 absolute), relaxations and staggered runs at the
tolerances of the single-system relaxation tests.
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


def r_bond_of(s):
    return 0.5 * (s.a / np.sqrt(2.0) + s.a)


def empty_like(s):
    e = s.copy()
    e.name = "empty"
    e.q = np.zeros((3, 0))
    e.sigma = np.zeros(0)
    e.x = np.zeros((s.S, 0))
    e.T = np.zeros(0)
    e.sublattice = np.zeros(0, np.uint8)
    return e


def ensemble(n=5, seed=31, pot=None, with_empty=True):
    """Uneven single-species systems (4 or 5 cells per side, T and vacancy
    fraction per system as in the ensemble workload), perturbed so that
    forces and fluxes are non-trivial, plus an empty system in the middle."""
    systems = W.config_ensemble(n_systems=n, cmin=4, cmax=5, seed=seed, pot=pot)
    out = []
    for k, s in enumerate(systems):
        out.append(W.perturb(s, 0.05, 0.02, seed=seed + 7 * k))
    if with_empty:
        out.insert(2, empty_like(out[0]))
    return out


def binary_pair(seed=41):
    a = W.perturb(W.config_binary_alloy(cells=4), 0.05, 0.02, seed=seed)
    b = W.perturb(W.config_binary_alloy(cells=5), 0.06, 0.02, seed=seed + 1)
    return [W.random_fractions(a, vac_min=0.01, seed=seed + 2), W.random_fractions(b, vac_min=0.01, seed=seed + 3)]


def oracle_fe(s, r_list):
    st, off, idx = O.neighbors(s.q, s.L, r_list)
    assert st == O.OK
    fe = O.free_energy(s, (off, idx))
    assert fe["status"] == O.OK
    return fe, off, idx


# ---------------------------------------------------------------- lists and energies
@pytest.mark.parametrize("case", ["single", "binary"])
def test_batch_lists_bit_exact_per_system(case):
    systems = ensemble() if case == "single" else binary_pair()
    g = M.MxeBatch(systems, "fp64")
    g.build_neighbors()
    off, idx = (t.cpu().numpy() for t in g.export_neighbors())
    boff, bidx = (t.cpu().numpy() for t in g.export_bonds())
    for b, s in enumerate(systems):
        o0, o1 = int(g.offsets[b]), int(g.offsets[b + 1])
        rows = off[o0:o1 + 1] - off[o0]
        ent = idx[off[o0]:off[o1]]
        if s.n == 0:
            assert off[o1] == off[o0] and boff[o1] == boff[o0]
            continue
        assert ent.min() >= o0 and ent.max() < o1          # no pair crosses systems
        st, ro, ri = O.neighbors(s.q, s.L, g.r_list)
        assert st == O.OK
        np.testing.assert_array_equal(rows, ro)
        np.testing.assert_array_equal(ent - o0, ri)
        bro, bri = O.bonds(s, g.r_bond, ro, ri)
        np.testing.assert_array_equal(boff[o0:o1 + 1] - boff[o0], bro)
        np.testing.assert_array_equal(bidx[boff[o0]:boff[o1]] - o0, bri)
    g.close()


@pytest.mark.parametrize("case", ["single", "binary"])
def test_batch_free_energy_fp64_per_system(case):
    systems = ensemble() if case == "single" else binary_pair()
    g = M.MxeBatch(systems, "fp64")
    g.build_neighbors()
    g.free_energy_grad()
    F4 = g.F4.cpu().numpy()
    for b, s in enumerate(systems):
        if s.n == 0:
            assert np.all(F4[b] == 0.0)
            continue
        fe, _, _ = oracle_fe(s, g.r_list)
        np.testing.assert_allclose(F4[b], fe["F4"], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(g.part(g.gq, b).cpu().numpy(), fe["gq"], rtol=0, atol=1e-9)
        np.testing.assert_allclose(g.part(g.gs, b).cpu().numpy(), fe["gs"], rtol=0, atol=1e-9)
        np.testing.assert_allclose(g.part(g.mu_ex, b).cpu().numpy(), fe["mu_ex"], rtol=0, atol=1e-9)
        np.testing.assert_allclose(g.part(g.mu, b).cpu().numpy(), fe["mu"], rtol=1e-12, atol=1e-9)
    g.close()


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_batch_free_energy_fp32_per_system(prec):
    """FP32-compute tolerances: energies 1e-5 relative, gradients 1e-4 of
    max(max|g|, 1), mu 1e-4 of max(max|mu|, 1)."""
    systems = binary_pair()
    g = M.MxeBatch(systems, prec)
    g.build_neighbors()
    g.free_energy_grad()
    F4 = g.F4.cpu().numpy()
    for b, s in enumerate(systems):
        fe, _, _ = oracle_fe(s, g.r_list)
        np.testing.assert_allclose(F4[b], fe["F4"], rtol=1e-5)
        for key, t in (("gq", g.gq), ("gs", g.gs)):
            ref = fe[key]
            np.testing.assert_allclose(g.part(t, b).cpu().numpy(), ref, rtol=0,
                                       atol=1e-4 * max(np.abs(ref).max(), 1.0))
        ref = fe["mu_ex"]
        np.testing.assert_allclose(g.part(g.mu_ex, b).cpu().numpy(), ref, rtol=0,
                                   atol=1e-4 * max(np.abs(ref).max(), 1.0))
    g.close()


def test_batch_of_one_matches_single_context():
    s = ensemble(with_empty=False)[0]
    a = M.MxeSystem(s, "fp64")
    a.build_neighbors()
    a.free_energy_grad()
    b = M.MxeBatch([s], "fp64")
    b.build_neighbors()
    b.free_energy_grad()
    np.testing.assert_allclose(b.F4.cpu().numpy()[0], a.F4.cpu().numpy(), rtol=1e-13, atol=1e-12)
    assert torch.equal(a.gq, b.gq) and torch.equal(a.gs, b.gs) and torch.equal(a.mu_ex, b.mu_ex)
    a.close()
    b.close()


def test_batch_box_too_small_names_the_system():
    systems = ensemble(n=3, with_empty=False)
    tiny = W.perturb(W.config_vacancy_lattice(cells=2, vacancy_cell=(1, 1, 1)), 0.01, 0.0)   # L = 7.2 A < 2 r_list
    g = M.MxeBatch(systems + [tiny], "fp64")
    st, _, _ = M.mxe_build_neighbors(g.ctx, g.state, g.skin, g.r_bond)
    assert st == M.ERR_BOX_TOO_SMALL
    g.close()


# ---------------------------------------------------------------- relaxation
def test_batch_relax_fixed_iterations_per_system():
    systems = ensemble(pot=W.potential_variant_s())
    K = 10
    g = M.MxeBatch(systems, "fp64")
    g.build_neighbors()
    st, it, fm = g.relax(0.0, K)
    assert st == M.ERR_NO_CONVERGE and it == K
    iters, fmax, conv = g.relax_info()
    for b, s in enumerate(systems):
        if s.n == 0:
            assert conv[b] and iters[b] == 0
            continue
        sto, ito, fmo, qo, so = O.relax(s, 0.0, K)
        assert sto == O.ERR_NO_CONVERGE and ito == K and iters[b] == K
        np.testing.assert_allclose(g.part(g.q, b).cpu().numpy(), qo, rtol=0, atol=1e-9)
        np.testing.assert_allclose(g.part(g.sigma, b).cpu().numpy(), so, rtol=0, atol=1e-9)
        assert abs(fmax[b] - fmo) <= 1e-8
    g.close()


def test_batch_relax_systems_converge_independently():
    """Variant S relaxes to a minimum; systems perturbed by different amounts
    need different iteration counts, and each stops on its own."""
    base = W.config_vacancy_lattice(pot=W.potential_variant_s(), x0=1.0)
    systems = []
    for k, amp in enumerate((0.01, 0.05, 0.03)):
        s = W.perturb(base, amp, 0.02, seed=50 + k)
        s.x[:] = 1.0
        systems.append(s)
    ftol = 1e-6
    g = M.MxeBatch(systems, "fp64")
    g.build_neighbors()
    st, it, fm = g.relax(ftol, 4000)
    assert st == M.OK and fm <= ftol
    iters, fmax, conv = g.relax_info()
    assert conv.all()
    seen = []
    for b, s in enumerate(systems):
        sto, ito, fmo, qo, so = O.relax(s, ftol, 4000)
        assert sto == O.OK
        assert abs(int(iters[b]) - ito) <= 2
        seen.append(ito)
        np.testing.assert_allclose(g.part(g.q, b).cpu().numpy(), qo, rtol=0, atol=1e-7)
        np.testing.assert_allclose(g.part(g.sigma, b).cpu().numpy(), so, rtol=0, atol=1e-7)
    assert len(set(seen)) > 1                  # the systems really stopped at different iterations
    assert it == max(iters)
    g.close()


# ---------------------------------------------------------------- Euler step
def test_batch_diffuse_step_per_system_dt():
    systems = ensemble()
    g = M.MxeBatch(systems, "fp64")
    g.build_neighbors()
    g.free_energy_grad()
    live = [s for s in systems if s.n]
    dt = min(s.dt_default() for s in live) * 1e-3
    scale = [1.0 + 0.5 * b for b in range(len(systems))]
    g.set_dt_scale(scale)
    x0 = g.x.clone()
    g.diffuse_step(dt, mu_ex=g.mu_ex)
    moved = 0.0
    for b, s in enumerate(systems):
        if s.n == 0:
            continue
        fe, off, idx = oracle_fe(s, g.r_list)
        boff, bidx = O.bonds(s, g.r_bond, off, idx)
        st, xo = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), dt * scale[b])
        assert st == O.OK
        np.testing.assert_allclose(g.part(g.x, b).cpu().numpy(), xo, rtol=0, atol=1e-12)
        # mass of each system is conserved on its own
        assert abs(g.part(g.x, b).sum().item() - g.part(x0, b).sum().item()) <= 1e-10
        moved = max(moved, np.abs(xo - s.x).max())
    assert moved > 1e-9
    g.set_dt_scale(None)
    g.close()


def test_set_dt_scale_rejects_single_context_and_bad_values():
    s = ensemble(with_empty=False)[0]
    a = M.MxeSystem(s, "fp64")
    assert M.mxe_set_dt_scale(a.ctx, [1.0]) == M.ERR_ARG
    a.close()
    g = M.MxeBatch(ensemble(n=2, with_empty=False), "fp64")
    assert M.mxe_set_dt_scale(g.ctx, [1.0, -1.0]) == M.ERR_ARG
    assert M.mxe_set_dt_scale(g.ctx, [1.0, float("nan")]) == M.ERR_ARG
    g.close()


# ---------------------------------------------------------------- graph-captured staggered loop
def dip_lattice():
    s = W.config_vacancy_lattice(pot=W.potential_variant_s())
    s.x[s.x == 0.0] = 0.5
    return s


def relaxed(s, ftol, K, fire=None):
    r = s.copy()
    _, _, _, r.q, r.sigma = O.relax(s, ftol, K, fire)
    return r


def stable_dt(s, r_bond, target):
    st, off, idx = O.neighbors(s.q, s.L, O.r_list_for(s))
    fe = O.free_energy(s, (off, idx))
    boff, bidx = O.bonds(s, r_bond, off, idx)
    trial = s.dt_default() * 1e-9
    st, x1 = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), trial)
    assert st == O.OK
    return trial * target / np.abs(x1 - s.x).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_graph_run_matches_step_by_step_calls(prec):
    """The captured loop runs the same kernels as mu -> mxe_diffuse_step ->
    mxe_relax issued call by call."""
    s = relaxed(dip_lattice(), 0.0, 12)
    K, steps = 12, 4
    dt = stable_dt(s, r_bond_of(s), 1e-3)
    a = M.MxeSystem(s, prec)
    a.build_neighbors()
    for _ in range(steps):
        a.staggered_step(dt, 0.0, K)
    b = M.MxeSystem(s, prec)
    b.build_neighbors()
    st, done = b.run_staggered(steps, dt, 0.0, K)
    assert st == M.OK and done == steps
    # every step of the run from one graph launch (a device-side loop); per
    # FIRE iteration at least the four force passes, the reduction and the update
    launches, kernels = b.run_stats()
    assert launches == 1 and kernels >= 6 * (K + 1)
    dx = (a.x - b.x).abs().max().item()
    dq = (a.q - b.q).abs().max().item()
    ds = (a.sigma - b.sigma).abs().max().item()
    print(f"{prec}: graph vs calls: |dx| {dx:.3e} |dq| {dq:.3e} |dsigma| {ds:.3e}")
    assert dx <= 1e-13 and dq <= 1e-11 and ds <= 1e-11
    assert (b.x - torch.as_tensor(s.x, device=b.device)).abs().max().item() > 1e-4   # mass moved
    a.close()
    b.close()


@pytest.mark.parametrize("skin", [0.2, 0.01])
def test_graph_run_fp64_oracle_parity(skin):
    """Staggered run against the oracle (which rebuilds its lists at every
    evaluation).  skin = 0.01 A makes the captured loop stop itself for
    rebuilds inside the relaxation, which the host then finishes."""
    s = relaxed(dip_lattice(), 0.0, 15)
    K, steps = 15, 5
    dt = stable_dt(s, r_bond_of(s), 1e-3)
    g = M.MxeSystem(s, "fp64", skin=skin)
    g.build_neighbors()
    st, done = g.run_staggered(steps, dt, 0.0, K)
    assert st == M.OK and done == steps
    launches, _ = g.run_stats()
    if skin == 0.2:
        assert launches == 1
    else:
        assert launches > 1       # the loop stopped for rebuilds and was launched again
    sto, so, iters = O.staggered(s, steps, dt, 0.0, K, g.r_bond, initial_relax=False)
    assert sto == O.OK
    assert np.abs(so.x - s.x).max() > 1e-3
    np.testing.assert_allclose(g.x.cpu().numpy(), so.x, rtol=0, atol=1e-10)
    np.testing.assert_allclose(g.q.cpu().numpy(), so.q, rtol=0, atol=1e-8)
    np.testing.assert_allclose(g.sigma.cpu().numpy(), so.sigma, rtol=0, atol=1e-8)
    g.close()


def test_graph_run_batch_per_system_oracle_parity():
    """Batched staggered run with per-system Euler steps: every system
    follows its own oracle run."""
    systems = []
    for k in range(3):
        s = dip_lattice()
        s.T[:] = 700.0 + 150.0 * k
        systems.append(relaxed(W.perturb(s, 0.01, 0.0, seed=60 + k), 0.0, 10))
    K, steps = 10, 4
    dts = [stable_dt(s, r_bond_of(s), 1e-3) for s in systems]
    dt = min(dts)
    scale = [d / dt for d in dts]
    g = M.MxeBatch(systems, "fp64")
    g.build_neighbors()
    g.set_dt_scale(scale)
    st, done = g.run_staggered(steps, dt, 0.0, K)
    assert st == M.OK and done == steps
    for b, s in enumerate(systems):
        sto, so, iters = O.staggered(s, steps, dt * scale[b], 0.0, K, g.r_bond, initial_relax=False)
        assert sto == O.OK
        np.testing.assert_allclose(g.part(g.x, b).cpu().numpy(), so.x, rtol=0, atol=1e-10)
        np.testing.assert_allclose(g.part(g.q, b).cpu().numpy(), so.q, rtol=0, atol=1e-8)
    g.close()


def test_graph_run_x_range_stops_and_keeps_x():
    s = relaxed(dip_lattice(), 0.0, 5)
    g = M.MxeSystem(s, "fp64")
    g.build_neighbors()
    x0 = g.x.clone()
    st, done = g.run_staggered(3, s.dt_default() * 1e6, 0.0, 5, allow=(M.ERR_X_RANGE,))
    assert st == M.ERR_X_RANGE and done == 0
    assert torch.equal(g.x, x0)
    assert g.sync_status() == M.OK        # the error was reported once
    g.close()


def test_graph_run_zero_steps_and_call_order():
    s = dip_lattice()
    g = M.MxeSystem(s, "fp64")
    st, done = M.mxe_run_staggered(g.ctx, g.state, 2, 1e-12, s.nu0, s.Qm, 0.0, 3)
    assert st == M.ERR_STATE
    g.build_neighbors()
    st, done = M.mxe_run_staggered(g.ctx, g.state, 0, 1e-12, s.nu0, s.Qm, 0.0, 3)
    assert st == M.OK and done == 0
    st, done = M.mxe_run_staggered(g.ctx, g.state, 2, -1.0, s.nu0, s.Qm, 0.0, 3)
    assert st == M.ERR_ARG
    g.close()


# ---------------------------------------------------------------- autotuner
def test_autotune_picks_a_valid_shape_and_keeps_results():
    systems = ensemble(with_empty=False)
    g = M.MxeBatch(systems, "mixed")
    g.build_neighbors()
    g.free_energy_grad()
    ref = (g.gq.clone(), g.mu_ex.clone())
    lanes, threads = g.autotune()
    assert lanes in (4, 8, 16) and threads in (128, 256)
    g.free_energy_grad()
    scale = max(ref[0].abs().max().item(), 1.0)
    assert (g.gq - ref[0]).abs().max().item() <= 1e-6 * scale
    assert (g.mu_ex - ref[1]).abs().max().item() <= 1e-10
    assert g.pass_shape()[2] in (64, 128, 256)     # pairs per block of the pair kernels
    for lanes, threads, pairs in ((4, 128, 64), (16, 256, 256)):
        g.set_pass_shape(lanes, threads, pairs)
        assert g.pass_shape() == (lanes, threads, pairs)
        g.free_energy_grad()
        assert (g.gq - ref[0]).abs().max().item() <= 1e-6 * scale
        assert (g.mu_ex - ref[1]).abs().max().item() <= 1e-10
    assert M.mxe_set_pass_shape(g.ctx, 5, 256) == M.ERR_ARG
    assert M.mxe_set_pass_shape(g.ctx, 8, 96) == M.ERR_ARG
    assert M.lib().mxe_set_pair_block(g.ctx, 96) == M.ERR_ARG
    g.close()
