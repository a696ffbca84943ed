"""The benchmarked step against the oracle, and relaxations whose neighbour
lists are rebuilt many times inside one call.

The step is the one bench.py times on the 256,000-site binary alloy (FCC 40^3
cells, App. B.2 alloy tables): autotuned pass shape, neighbour build, free
energy with the excess chemical potentials, one Euler step of Eq.
MassTransport, then 10 FIRE iterations (Sec. 4, Algorithm 1) in which the
lists are rebuilt once the skin criterion fails.  In the float-float context
the forces of every evaluation after the first relaxation come from the
half-list FP32 pair kernels (each unordered pair once, App. A nodes) and
their per-site gathers; the halted-pass logic re-evaluates a pass that
started on lists found stale.

Tolerances (FP32-compute modes): forces and width derivatives 1e-4 relative
to max(max |g_oracle|, 1 eV/A); energies 1e-10 relative when the chemical
potentials are requested (they come from the accurate passes); x 1e-7
absolute; positions and widths after K FIRE iterations 1e-4 A (a force error
e moves y by at most K^2 dt_max^2 e).
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

K_BENCH = 10


def builds_in(timing):
    """List builds in a timing record: one fill launch per build."""
    return timing.get("build_fill", (0, 0.0))[0]


def force_scale(fe):
    return max(np.abs(fe["gq"]).max(), np.abs(fe["gs"]).max(), 1.0)


def oracle_step(s, r_list, r_bond, dt, K):
    """Oracle form of the step: free energy at the input state, Euler step,
    then K FIRE iterations at the new composition (lists rebuilt for every
    evaluation)."""
    st, off, idx = O.neighbors(s.q, s.L, r_list)
    assert st == O.OK
    fe = O.free_energy(s, (off, idx))
    assert fe["status"] == O.OK
    boff, bidx = O.bonds(s, r_bond, off, idx)
    st, xo = O.diffuse_step(s, fe["mu_ex"], (boff, bidx), dt)
    assert st == O.OK
    r = s.copy()
    r.x = xo
    sto, ito, fmo, qo, so = O.relax(r, 0.0, K)
    assert sto == O.ERR_NO_CONVERGE and ito == K
    return fe, xo, qo, so, fmo


@pytest.mark.parametrize("prec", ["ff", "mixed"])
def test_bench_step_256k_against_oracle(prec):
    """bench.py's timed step, float-float and FP64-sum contexts, full size,
    with at least one list rebuild inside the relaxation; then the forces at
    the GPU's final state (half-list kernels on lists built mid-relaxation)
    against the oracle's at that same state."""
    s = W.config_binary_alloy()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        g = M.MxeSystem(s, prec, device=dev, stream=stream)
    g.build_neighbors()
    g.autotune()
    fire = M.make_fire(check_every=K_BENCH + 1)
    dt = s.dt_default()
    M.mxe_timing_enable(g.ctx, True)
    npairs, r_list = g.build_neighbors()
    g.free_energy_grad(with_mu=False, asynchronous=True)
    g.diffuse_step(dt, mu_ex=g.mu_ex, asynchronous=True)
    st, it, fm = g.relax(0.0, K_BENCH, fire)
    _, timing = M.mxe_timing_read(g.ctx)
    M.mxe_timing_enable(g.ctx, False)
    assert it == K_BENCH
    # the step's first forces come from the half-list pair kernel (the
    # autotuner made the relaxation records), and the relaxation rebuilt
    assert timing.get("pair32_force", (0, 0.0))[0] >= K_BENCH + 2
    assert builds_in(timing) >= 2, timing
    F4 = g.F4.cpu().numpy()
    gq0, gs0 = g.gq.cpu().numpy(), g.gs.cpu().numpy()
    x1, q1, s1 = g.x.cpu().numpy(), g.q.cpu().numpy(), g.sigma.cpu().numpy()

    fe, xo, qo, so, fmo = oracle_step(s, r_list, g.r_bond, dt, K_BENCH)
    gscale = force_scale(fe)
    np.testing.assert_allclose(F4, fe["F4"], rtol=1e-10, atol=1e-10)
    eq = np.abs(gq0 - fe["gq"]).max()
    es = np.abs(gs0 - fe["gs"]).max()
    ex = np.abs(x1 - xo).max()
    dq = np.abs(q1 - qo).max()
    ds = np.abs(s1 - so).max()
    print(f"256k {prec} step: |dF/dq| err {eq:.2e}, |dF/dsigma| err {es:.2e} (scale {gscale:.2f}), "
          f"x {ex:.2e}, q {dq:.2e} A, sigma {ds:.2e} A, fmax {fm:.6f} vs {fmo:.6f}")
    assert eq <= 1e-4 * gscale and es <= 1e-4 * gscale
    assert np.abs(xo - s.x).max() > 1e-6          # the Euler step moved mass (x_v = 1e-3)
    assert ex <= 1e-7
    assert dq <= 1e-4 and ds <= 1e-4
    assert abs(fm - fmo) <= 1e-4 * max(fmo, 1.0)

    # forces at the GPU's own final state, on the lists of the last rebuild
    g.free_energy_grad(with_mu=False)
    t = s.copy()
    t.q, t.sigma, t.x = q1, s1, x1
    st, off, idx = O.neighbors(t.q, t.L, O.r_list_for(t))
    assert st == O.OK
    fe2 = O.free_energy(t, (off, idx))
    assert fe2["status"] == O.OK
    sc2 = force_scale(fe2)
    assert np.abs(g.gq.cpu().numpy() - fe2["gq"]).max() <= 1e-4 * sc2
    assert np.abs(g.gs.cpu().numpy() - fe2["gs"]).max() <= 1e-4 * sc2
    np.testing.assert_allclose(g.F4.cpu().numpy(), fe2["F4"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(g.mu_ex.cpu().numpy(), fe2["mu_ex"], rtol=0, atol=1e-9)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
@pytest.mark.parametrize("pot", ["literal", "variant_s"])
def test_relax_many_rebuilds(prec, pot):
    """A skin of 0.01 A makes nearly every FIRE iteration rebuild the lists
    and the pair index (and resize the relaxation records), so most passes
    start on lists found stale and are evaluated again after the rebuild.
    The trajectory of K iterations must still be the oracle's: 1e-9 A in
    FP64, 1e-4 A with FP32 node arithmetic."""
    p = W.potential_single() if pot == "literal" else W.potential_variant_s()
    s = W.perturb(W.config_vacancy_lattice(pot=p, x0=0.97), 0.05, 0.02)
    K = 14
    g = M.MxeSystem(s, prec, skin=0.01)
    g.build_neighbors()
    # a first relaxation makes the relaxation records; restart from s
    g.relax(0.0, 1)
    g.q.copy_(torch.as_tensor(s.q))
    g.sigma.copy_(torch.as_tensor(s.sigma))
    g.build_neighbors()
    M.mxe_timing_enable(g.ctx, True)
    st, it, fm = g.relax(0.0, K)
    _, timing = M.mxe_timing_read(g.ctx)
    M.mxe_timing_enable(g.ctx, False)
    assert st == M.ERR_NO_CONVERGE and it == K
    assert builds_in(timing) >= 4, timing
    pair_force = "pair64_force" if prec == "fp64" else "pair32_force"
    assert timing.get(pair_force, (0, 0.0))[0] >= K + 1, timing
    sto, ito, fmo, qo, so = O.relax(s, 0.0, K)
    assert sto == O.ERR_NO_CONVERGE and ito == K
    dq = np.abs(g.q.cpu().numpy() - qo).max()
    ds = np.abs(g.sigma.cpu().numpy() - so).max()
    print(f"{prec}/{pot}: {builds_in(timing)} builds, q {dq:.2e} A, sigma {ds:.2e} A")
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert dq <= tol and ds <= tol
    assert abs(fm - fmo) <= (1e-8 if prec == "fp64" else 1e-4 * max(fmo, 1.0))
    g.close()


def test_binary_alloy_tables_take_the_specialised_pattern():
    """The benchmark's alloy has two like pair terms, one cross term and a
    density that depends on the neighbour's species only: the pair kernels
    specialised for that table pattern (phi_of = {{0, 1}, {1, 2}}, f_of[k][l]
    = l) must see exactly these tables; the slab's host-solute tables must
    not match it."""
    g = M.MxeSystem(W.config_binary_alloy(cells=5), "ff")
    nphi, nf, terms, phi_of, f_of = g.potential_terms()
    assert (nphi, nf) == (3, 2)
    np.testing.assert_array_equal(phi_of[:2, :2], [[0, 1], [1, 2]])
    np.testing.assert_array_equal(f_of[:2, :2], [[nphi + 0, nphi + 1], [nphi + 0, nphi + 1]])
    g.close()
    g = M.MxeSystem(W.config_interstitial_slab(4, 4, 2, top=100.0, xmax=0.3), "ff")
    nphi, nf, terms, phi_of, f_of = g.potential_terms()
    assert phi_of[1, 1] == -1
    g.close()


def _binary_with(p_a=None, q_b=None, cells=5, seed=21):
    s = W.perturb(W.config_binary_alloy(cells=cells), 0.06, 0.02, seed=seed)
    s = W.random_fractions(s, vac_min=0.01, seed=seed + 1)
    if p_a is not None:
        s.pot.phi_p[0, 0] = p_a
    if q_b is not None:
        s.pot.f_q[:, 1] = q_b
    return s


def test_power_form_taken_where_the_rates_allow_it():
    """The alloy's pair and density rates are 3/r0 and 5/r0 per species
    (integer powers 6 and 10 of exp(-r / (2 r0)), cross term powers 3 and 3):
    the accurate pass takes the power form; a pair exponent of 3.1 (a ratio
    31/50) or a density exponent of 4.9 for B leaves the general form, and so
    does any potential outside the binary table pattern."""
    for s, want in ((W.config_binary_alloy(cells=4), (1, 1)),
                    (_binary_with(), (1, 1)),
                    (_binary_with(p_a=3.1), (1, 0)),
                    (_binary_with(q_b=4.9), (1, 0))):
        g = M.MxeSystem(s, "ff")
        assert g.pair_form() == want
        g.close()
    s = W.config_binary_alloy(cells=4)
    s.pot = W.potential_binary_variant_s()
    g = M.MxeSystem(s, "fp64")
    assert g.pair_form() == (1, 1)   # rates 5/r0 and 3/r0: powers 10 and 6
    g.close()
    g = M.MxeSystem(W.config_vacancy_lattice(cells=4), "ff")
    assert g.pair_form()[1] == 0
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
@pytest.mark.parametrize("form", ["power", "general"])
def test_accurate_pass_parity_in_both_forms(prec, form):
    """Energies and chemical potentials (the accurate pass) against the oracle
    with the power form taken and not taken (same tolerances as the other
    parity tests: energies 1e-10 relative, mu^ex 1e-9 eV)."""
    s = _binary_with() if form == "power" else _binary_with(p_a=3.1)
    g = M.MxeSystem(s, prec)
    assert g.pair_form()[1] == (1 if form == "power" else 0)
    g.build_neighbors()
    g.free_energy_grad()
    torch.cuda.synchronize()
    fe = O.free_energy(s, r_list=g.r_list)
    assert fe["status"] == O.OK
    np.testing.assert_allclose(g.F4.cpu().numpy(), fe["F4"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(g.mu_ex.cpu().numpy(), fe["mu_ex"], rtol=0, atol=1e-9)
    g.close()
