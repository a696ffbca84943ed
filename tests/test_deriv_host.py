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


def term_parameters(pot):
    """(c, lambda) of the binary tables' five radial terms (layout above):
    c = ln A + exponent, lambda = exponent / length scale; the cross pair
    averages the two like pairs (its pointwise geometric mean)."""
    A, p, r0 = pot.phi_A, pot.phi_p, pot.phi_r0
    c = np.array([np.log(A[0, 0]) + p[0, 0],
                  0.5 * (np.log(A[0, 0]) + p[0, 0] + np.log(A[1, 1]) + p[1, 1]),
                  np.log(A[1, 1]) + p[1, 1],
                  np.log(pot.f_xi[0, 0]) + pot.f_q[0, 0],
                  np.log(pot.f_xi[0, 1]) + pot.f_q[0, 1]])
    lam = np.array([p[0, 0] / r0[0, 0], 0.5 * (p[0, 0] / r0[0, 0] + p[1, 1] / r0[1, 1]), p[1, 1] / r0[1, 1],
                    pot.f_q[0, 0] / pot.f_r0[0, 0], pot.f_q[0, 1] / pot.f_r0[0, 1]])
    return c, lam


def fd_chain(dterm, P, rel_step=1e-6):
    """dL/dtheta by central differences of theta -> (c, lambda)."""
    th = W.theta_of(P)
    out = np.zeros(th.size)
    for m in range(th.size):
        h = rel_step * max(abs(th[m]), 1.0)
        tp, tm = th.copy(), th.copy()
        tp[m] += h
        tm[m] -= h
        cp, lp = term_parameters(W.binary_from_theta(tp, P))
        cm, lm = term_parameters(W.binary_from_theta(tm, P))
        out[m] = dterm[:5] @ ((cp - cm) / (2 * h)) + dterm[5:] @ ((lp - lm) / (2 * h))
    return out


def test_term_parameters_closed_form():
    P = W.potential_binary()
    c, lam = term_parameters(P)
    AA, pA, rA, AB, pB, rB = 0.3, 3.0, 2.55, 0.33, 3.0, 2.65
    np.testing.assert_allclose(c[0], np.log(AA) + pA)
    np.testing.assert_allclose(lam[0], pA / rA)
    np.testing.assert_allclose(c[1], 0.5 * (np.log(AA) + pA + np.log(AB) + pB))
    np.testing.assert_allclose(lam[1], 0.5 * (pA / rA + pB / rB))
    np.testing.assert_allclose(c[2], np.log(AB) + pB)
    np.testing.assert_allclose(c[3], np.log(1.0) + 5.0)
    np.testing.assert_allclose(lam[4], 5.0 / 2.65)


def test_library_chain_rule_matches_differences_and_closed_form():
    """mxe_element_param_grad (host arithmetic of the library) against central
    differences of the map and the hand-written Jacobian of it."""
    P = W.potential_binary_variant_s()
    th = W.theta_of(P)
    rng = np.random.default_rng(1)
    dterm = rng.normal(size=10)
    got = M.element_param_grad(P, dterm).reshape(-1)
    np.testing.assert_allclose(got, fd_chain(dterm, P), rtol=1e-8, atol=1e-9)
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
    np.testing.assert_allclose(got, exp, rtol=1e-13)


def test_library_chain_rule_single_species_and_rejections():
    P = W.potential_variant_s()
    dterm = np.array([0.7, -1.3, 0.25, 2.0])      # dc(phi), dc(f), dl(phi), dl(f)
    got = M.element_param_grad(P, dterm).reshape(-1)
    A, p, q, r0 = 0.3, 5.0, 3.0, 2.55
    np.testing.assert_allclose(got, [0.7 / A, 0.7 + 0.25 / r0, -1.3 + 2.0 / r0,
                                     -p / r0 ** 2 * 0.25 - q / r0 ** 2 * 2.0], rtol=1e-14)
    # density length scale not the pair's: no element structure
    Q = W.potential_variant_s()
    Q.f_r0 = Q.f_r0 + 0.1
    try:
        M.element_param_grad(Q, dterm)
        raise AssertionError("expected MxeError")
    except M.MxeError as e:
        assert e.status == M.ERR_ARG
