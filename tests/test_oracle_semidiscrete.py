"""Pins of the oracle's semi-discrete operator (Eqs. (7)-(23), (EPBC1-6)) on tiny grids."""
import math

import numpy as np
import pytest

import oracle
from oracle import PEC, PMC, ABSORBING
from tests import oracle_helpers as oh

GRIDS = [((4, 5, 6), (0.3, 0.2, 0.25)), ((6, 4, 5), (1.0, 1.0, 1.0))]
FACE_SETS = [
    (PEC,) * 6,
    (PMC,) * 6,
    (PEC, PMC, PMC, PEC, PEC, PMC),
    (PMC, PEC, PEC, PMC, PMC, PEC),
]


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("n,h", GRIDS)
@pytest.mark.parametrize("faces", FACE_SETS)
def test_operator_equals_kronecker_closed_form(n, h, faces):
    """With PEC/PMC SATs the oracle's operator equals the Kronecker construction of
    Eqs. (ED_1)-(ED_3) from the printed Q, P with Q- - B^T (PEC, H side) and Q+ - B
    (PMC, E side) at the penalised ends."""
    blk = oracle.Block(n, h, 1e-12, faces)
    M = oh.dense_operator([blk])
    K = oh.kronecker_operator(blk, faces)
    assert _rel(M, K) < 1e-13


@pytest.mark.parametrize("n,h", GRIDS)
@pytest.mark.parametrize("faces", FACE_SETS)
def test_energy_neutral_pec_pmc(n, h, faces):
    """Eqs. (17)/(18) and (22)/(23): dE/dt = 0, i.e. W M + M^T W = 0 in the energy norm."""
    blk = oracle.Block(n, h, 1e-12, faces)
    M = oh.dense_operator([blk])
    W = np.diag(oh.energy_matrix([blk]))
    S = W @ M + M.T @ W
    assert np.max(np.abs(S)) <= 1e-12 * np.max(np.abs(W @ M))


def test_energy_neutral_dielectric():
    """Uniform eps_r = 4: the same identity in the eps-weighted norm."""
    n, h = (4, 5, 6), (0.3, 0.2, 0.25)
    eps = np.full((n[2], n[1], n[0]), 4.0)
    blk = oracle.Block(n, h, 1e-12, (PEC, PMC) * 3, eps_r=eps)
    M = oh.dense_operator([blk])
    W = np.diag(oh.energy_matrix([blk], eps_r=4.0))
    S = W @ M + M.T @ W
    assert np.max(np.abs(S)) <= 1e-12 * np.max(np.abs(W @ M))


def test_sat_sign_flip_breaks_neutrality():
    """Sanity of the pin: the negated PEC penalty (sigma -> -sigma) is not energy-neutral.
    Built by subtracting twice the SAT part (PEC minus no-penalty closed form)."""
    n, h = (4, 5, 6), (0.3, 0.2, 0.25)
    blk = oracle.Block(n, h, 1e-12, (PEC,) * 6)
    M = oh.dense_operator([blk])
    K_free = oh.kronecker_operator(blk, (-1,) * 6)       # no penalties at all
    M_flip = M - 2.0 * (M - K_free)
    W = np.diag(oh.energy_matrix([blk]))
    S = W @ M_flip + M_flip.T @ W
    assert np.max(np.abs(S)) > 1e-3 * np.max(np.abs(W @ M))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_interface_energy_neutral(axis):
    """Interface SAT (zero-phase periodic SAT with +-1/2, Eqs. (EPBC1-6), (EPBCP)) between two
    blocks: the coupled operator is skew in the joint energy norm."""
    nA = [4, 5, 4]
    nB = [4, 5, 4]
    nB[axis] = 5
    h = (0.3, 0.2, 0.25)
    hB = list(h)
    hB[axis] = 0.4
    fa = [PEC, PMC, PEC, PMC, PMC, PEC]
    fb = list(fa)
    A = oracle.Block(nA, h, 1e-12, fa)
    B = oracle.Block(nB, hB, 1e-12, fb)
    oracle.connect(A, 2 * axis + 1, B, 2 * axis)
    M = oh.dense_operator([A, B])
    W = np.diag(oh.energy_matrix([A, B]))
    S = W @ M + M.T @ W
    assert np.max(np.abs(S)) <= 1e-12 * np.max(np.abs(W @ M))


def test_periodic_self_interface_energy_neutral():
    """A block joined to itself across z (periodic with zero phase) stays energy-neutral."""
    A = oracle.Block((4, 5, 6), (0.3, 0.2, 0.25), 1e-12, (PEC, PEC, PMC, PMC, PEC, PEC))
    oracle.connect(A, 5, A, 4)
    M = oh.dense_operator([A])
    W = np.diag(oh.energy_matrix([A]))
    S = W @ M + M.T @ W
    assert np.max(np.abs(S)) <= 1e-12 * np.max(np.abs(W @ M))


@pytest.mark.parametrize("faces", [(ABSORBING,) * 6, (PEC, ABSORBING, PMC, ABSORBING, ABSORBING, PEC)])
def test_absorbing_dissipative(faces):
    """Absorbing SAT: W M + M^T W is negative semidefinite (energy can only leave)."""
    blk = oracle.Block((4, 5, 6), (0.3, 0.2, 0.25), 1e-12, faces)
    M = oh.dense_operator([blk])
    W = np.diag(oh.energy_matrix([blk]))
    S = W @ M + M.T @ W
    Dm = np.diag(1.0 / np.sqrt(np.diag(W)))
    lam = np.linalg.eigvalsh(Dm @ S @ Dm)
    scale = np.max(np.abs(lam))
    assert lam.max() <= 1e-12 * scale
    assert lam.min() < -1e-3 * scale            # and it does dissipate


def test_spectral_radius_within_cfl():
    """Sec. VI-A: the SBP-SAT time-step limit equals FDTD's.  The operator's largest |eigenvalue|
    times dt_CFL = 1/(c sqrt(sum 1/h^2)) stays below 2 (leapfrog bound).
    With W the diagonal energy norm of Eq. (16), S = W^{1/2} M W^{-1/2} has the spectrum of M.
    S is skew-symmetric to rounding (so the spectrum is purely imaginary), and its largest
    |eigenvalue| is then its 2-norm: the square root of the top eigenvalue of S^T S (sparse)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    n, h = (8, 8, 8), (1.0, 1.0, 1.0)
    blk = oracle.Block(n, h, 1e-12, (PEC,) * 6)
    M = oh.dense_operator([blk])
    r = np.sqrt(oh.energy_matrix([blk]))
    S = (r[:, None] * M) / r[None, :]
    assert np.max(np.abs(S + S.T)) < 1e-12 * np.max(np.abs(S))      # purely imaginary spectrum
    Ss = sp.csr_matrix(S)
    StS = sla.LinearOperator(S.shape, matvec=lambda v: Ss.T @ (Ss @ v), dtype=float)
    rho = math.sqrt(sla.eigsh(StS, k=1, which="LA", tol=1e-10, return_eigenvectors=False)[0])
    dt = oracle.dt_cfl(1.0, *h)
    assert rho * dt < 2.0
