"""Host decision of the pair kernels' forms (no GPU): the species-table
pattern and the power form of the accurate pass (each species' pair and
density terms as integer powers of one exponential exp(-beta_s r), App. B.2
tables).  The power form must be taken exactly when the rates allow it."""
import numpy as np
import pytest

from paper_1910_01235_gb300 import workloads as W

M = pytest.importorskip("paper_1910_01235_gb300.mxe")


def _lib_or_skip():
    try:
        M.lib()
    except Exception as e:  # the library is built by __graft_entry__.build()
        pytest.skip(f"libmxe not built: {e}")


def _binary(p_a=None, q_b=None, geo=True):
    pot = W.potential_binary()
    if p_a is not None:
        pot.phi_p[0, 0] = p_a
    if q_b is not None:
        pot.f_q[:, 1] = q_b
    pot.cross_geomean = geo
    return pot


def test_binary_alloy_takes_the_power_form():
    _lib_or_skip()
    # rates 3/r0 and 5/r0 per species: c_s = exp(-r / (2 r0_s)), powers 6 and 10
    assert M.potential_pair_form(W.potential_binary()) == (1, 1, (6, 6), (10, 10))
    # swapped exponents (p = 5, q = 3): powers 10 and 6
    assert M.potential_pair_form(W.potential_binary_variant_s()) == (1, 1, (10, 10), (6, 6))


@pytest.mark.parametrize("kw", [{"p_a": 3.1}, {"q_b": 4.9}, {"p_a": 2.0 + 1e-9}])
def test_rates_without_small_integer_ratios_keep_the_general_form(kw):
    _lib_or_skip()
    tab, power, m, n = M.potential_pair_form(_binary(**kw))
    assert tab == 1 and power == 0 and m == (0, 0) and n == (0, 0)


def test_other_patterns_keep_the_general_form():
    _lib_or_skip()
    assert M.potential_pair_form(_binary(geo=False))[1] == 0          # cross term not a geometric mean
    assert M.potential_pair_form(W.potential_single())[:2] == (0, 0)  # one species
    assert M.potential_pair_form(W.potential_lj())[1] == 0


def test_power_form_identity_for_the_alloy_tables():
    """exp(c - lambda r) = exp(c) exp(-beta r)^m with lambda = m beta: the
    alloy's pair and density terms and the geometric-mean cross term, on a
    grid of distances, to rounding."""
    pot = W.potential_binary()
    r = np.linspace(1.5, 6.0, 200)
    c = [np.exp(-r / (2.0 * pot.phi_r0[s, s])) for s in range(2)]
    for s in range(2):
        phi = pot.phi_A[s, s] * np.exp(-pot.phi_p[s, s] * (r / pot.phi_r0[s, s] - 1.0))
        np.testing.assert_allclose(pot.phi_A[s, s] * np.exp(pot.phi_p[s, s]) * c[s] ** 6, phi, rtol=1e-13)
        f = pot.f_xi[0, s] * np.exp(-pot.f_q[0, s] * (r / pot.f_r0[0, s] - 1.0))
        np.testing.assert_allclose(pot.f_xi[0, s] * np.exp(pot.f_q[0, s]) * c[s] ** 10, f, rtol=1e-13)
    phi0 = pot.phi_A[0, 0] * np.exp(-pot.phi_p[0, 0] * (r / pot.phi_r0[0, 0] - 1.0))
    phi1 = pot.phi_A[1, 1] * np.exp(-pot.phi_p[1, 1] * (r / pot.phi_r0[1, 1] - 1.0))
    cross = np.sqrt(pot.phi_A[0, 0] * pot.phi_A[1, 1]) * np.exp(0.5 * (pot.phi_p[0, 0] + pot.phi_p[1, 1]))
    np.testing.assert_allclose(cross * c[0] ** 3 * c[1] ** 3, np.sqrt(phi0 * phi1), rtol=1e-13)
