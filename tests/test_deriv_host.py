"""Host side of the parameter derivatives (no GPU): the map from the eight
alloy parameters to the radial terms' (c = ln A + exponent, lambda =
exponent / length) and the chain rule through it, against the closed-form
Jacobian of that map."""
import numpy as np

from paper_1910_01235_gb300 import mxe as M
from paper_1910_01235_gb300 import workloads as W

# the binary tables' term layout: pair terms AA, AB (geometric mean), BB, then
# the density terms of an A-neighbour and of a B-neighbour
PHI_OF = -np.ones((4, 4), int)
F_OF = -np.ones((4, 4), int)
PHI_OF[0, 0], PHI_OF[0, 1], PHI_OF[1, 0], PHI_OF[1, 1] = 0, 1, 1, 2
F_OF[0, 0] = F_OF[1, 0] = 3
F_OF[0, 1] = F_OF[1, 1] = 4


def test_theta_round_trip():
    P = W.potential_binary_variant_s()
    th = W.theta_of(P)
    Q = W.binary_from_theta(th, P)
    for nm in ("phi_A", "phi_p", "phi_r0", "f_xi", "f_q", "f_r0"):
        assert np.array_equal(getattr(P, nm), getattr(Q, nm))
    assert list(W.THETA_NAMES) == ["A_A", "p_A", "q_A", "r0_A", "A_B", "p_B", "q_B", "r0_B"]


def test_term_parameters_closed_form():
    P = W.potential_binary()
    c, lam = M.term_parameters(P, PHI_OF, F_OF, 3, 2)
    AA, pA, rA, AB, pB, rB = 0.3, 3.0, 2.55, 0.33, 3.0, 2.65
    np.testing.assert_allclose(c[0], np.log(AA) + pA)
    np.testing.assert_allclose(lam[0], pA / rA)
    np.testing.assert_allclose(c[1], 0.5 * (np.log(AA) + pA + np.log(AB) + pB))
    np.testing.assert_allclose(lam[1], 0.5 * (pA / rA + pB / rB))
    np.testing.assert_allclose(c[2], np.log(AB) + pB)
    np.testing.assert_allclose(c[3], np.log(1.0) + 5.0)
    np.testing.assert_allclose(lam[4], 5.0 / 2.65)


def test_chain_rule_matches_the_analytic_jacobian():
    P = W.potential_binary_variant_s()
    th = W.theta_of(P)
    rng = np.random.default_rng(1)
    dterm = rng.normal(size=10)
    got = M.chain_to_parameters(dterm, lambda t: W.binary_from_theta(t, P), th, PHI_OF, F_OF, 3, 2)
    dc, dl = dterm[:5], dterm[5:]
    A_A, p_A, q_A, r_A, A_B, p_B, q_B, r_B = th
    exp = np.array([
        (dc[0] + 0.5 * dc[1]) / A_A,
        dc[0] + dl[0] / r_A + 0.5 * (dc[1] + dl[1] / r_A),
        dc[3] + dl[3] / r_A,
        -p_A / r_A ** 2 * (dl[0] + 0.5 * dl[1]) - q_A / r_A ** 2 * dl[3],
        (dc[2] + 0.5 * dc[1]) / A_B,
        dc[2] + dl[2] / r_B + 0.5 * (dc[1] + dl[1] / r_B),
        dc[4] + dl[4] / r_B,
        -p_B / r_B ** 2 * (dl[2] + 0.5 * dl[1]) - q_B / r_B ** 2 * dl[4],
    ])
    np.testing.assert_allclose(got, exp, rtol=1e-8)
