"""Pins of the oracle's 1D SBP operators (Appendix; Eqs. (2)-(6))."""
import numpy as np
import pytest

import oracle
from tests import appendix

SIZES = [4, 5, 6, 8, 20, 100]


@pytest.mark.parametrize("n", SIZES)
def test_operators_match_printed_appendix(n):
    """The oracle's D+, D-, P+, P- equal the matrices printed in the Appendix."""
    assert np.array_equal(oracle.dplus(n), appendix.d_plus_printed(n))
    assert np.array_equal(oracle.dminus(n), appendix.d_minus_printed(n))
    assert np.array_equal(oracle.pplus(n), appendix.p_plus(n))
    assert np.array_equal(oracle.pminus(n), appendix.p_minus(n))


@pytest.mark.parametrize("n", SIZES)
def test_d_equals_p_inverse_q(n):
    """Eq. (3): D = P^-1 Q, with Q taken from the printed Q matrices."""
    Qp = np.diag(oracle.pplus(n)) @ oracle.dplus(n)
    Qm = np.diag(oracle.pminus(n)) @ oracle.dminus(n)
    assert np.array_equal(Qp, appendix.q_plus(n))
    assert np.array_equal(Qm, appendix.q_minus(n))


@pytest.mark.parametrize("n", SIZES)
def test_sbp_identity_exact(n):
    """Eq. (QB): Q+ + Q-^T = B exactly (all entries are dyadic)."""
    Qp = np.diag(oracle.pplus(n)) @ oracle.dplus(n)
    Qm = np.diag(oracle.pminus(n)) @ oracle.dminus(n)
    assert np.array_equal(Qp + Qm.T, appendix.boundary_b(n))


@pytest.mark.parametrize("n", SIZES)
def test_accuracy_on_monomials(n):
    """Eq. (2): D+ x-^k = k x+^{k-1} and D- x+^k = k x-^{k-1}, k = 0, 1."""
    xp = np.arange(n + 1, dtype=float)
    xm = np.concatenate([[0.0], np.arange(n) + 0.5, [float(n)]])
    Dp, Dm = oracle.dplus(n), oracle.dminus(n)
    np.testing.assert_allclose(Dp @ np.ones(n + 2), 0.0, atol=1e-14)
    np.testing.assert_allclose(Dm @ np.ones(n + 1), 0.0, atol=1e-14)
    np.testing.assert_allclose(Dp @ xm, np.ones(n + 1), rtol=0, atol=1e-13)
    np.testing.assert_allclose(Dm @ xp, np.ones(n + 2), rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", SIZES)
def test_boundary_form(n):
    """Eq. (6): x+^T B x- = x_n x_n - x_0 x_0 for grid functions sampled at the ends."""
    rng = np.random.default_rng(n)
    u, v = rng.standard_normal(n + 1), rng.standard_normal(n + 2)
    Qp = np.diag(oracle.pplus(n)) @ oracle.dplus(n)
    Qm = np.diag(oracle.pminus(n)) @ oracle.dminus(n)
    lhs = u @ Qp @ v + v @ Qm @ u
    assert lhs == pytest.approx(u[n] * v[n + 1] - u[0] * v[0], abs=1e-12)


@pytest.mark.parametrize("n", SIZES)
def test_norms_are_quadratures(n):
    """P+ and P- are positive and integrate 1 and x exactly over [0, n]."""
    pp, pm = oracle.pplus(n), oracle.pminus(n)
    assert (pp > 0).all() and (pm > 0).all()
    xp = np.arange(n + 1, dtype=float)
    xm = np.concatenate([[0.0], np.arange(n) + 0.5, [float(n)]])
    assert pp.sum() == pytest.approx(n) and pm.sum() == pytest.approx(n)
    assert pp @ xp == pytest.approx(n * n / 2) and pm @ xm == pytest.approx(n * n / 2)


def test_closed_operator_spectrum_below_yee():
    """D+ closed by the PEC-type SAT (-P-^-1 Q+^T) composed with D+: its largest
    eigenvalue stays below the Yee value 4/h^2 (Sec. VI-A: same CFL as FDTD)."""
    n = 100
    Dp = oracle.dplus(n)
    Pm = np.diag(oracle.pminus(n))
    Qp = np.diag(oracle.pplus(n)) @ Dp
    Hop = -np.linalg.solve(Pm, Qp.T)          # D- closed by the PEC SAT
    lam = np.linalg.eigvals(-(Dp @ Hop))
    assert np.max(lam.real) < 4.0
    assert np.max(np.abs(lam.imag)) < 1e-8
