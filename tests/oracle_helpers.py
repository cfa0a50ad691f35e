"""Dense-matrix views of the oracle for the semi-discrete pins (tiny grids only)."""
import numpy as np

import oracle
from tests import appendix

EPS0, MU0 = oracle.EPS0, oracle.MU0


def sizes(blk):
    return [int(np.prod(blk.shape(c))) for c in range(6)]


def dense_operator(blocks):
    """Matrix M of the semi-discrete system dU/dt = M U (oracle.rhs), columns by unit vectors.
    U stacks, block by block, the six components flattened x fastest."""
    layout = []
    off = 0
    for b in blocks:
        for c in range(6):
            m = int(np.prod(b.shape(c)))
            layout.append((b, c, off, m))
            off += m
    N = off
    M = np.zeros((N, N))
    zero = {(id(b), c): np.zeros(b.shape(c)) for b, c, _, _ in layout}
    for b, c, _, _ in layout:
        b.set_field(c, zero[(id(b), c)])
    for b, c, o, m in layout:
        shp = b.shape(c)
        for q in range(m):
            u = np.zeros(m)
            u[q] = 1.0
            b.set_field(c, u.reshape(shp))
            oracle.rhs(blocks)
            col = np.concatenate([bb.rhs(cc).reshape(-1) for bb, cc, _, _ in layout])
            M[:, o + q] = col
        b.set_field(c, zero[(id(b), c)])
    return M


def weights_1d(n, plus, h):
    return h * (appendix.p_plus(n) if plus else appendix.p_minus(n))


def p3(blk, comp):
    """P''' of Eq. (EP_1) for one component: P_z (x) P_y (x) P_x, from the printed norms."""
    w = [weights_1d(blk.n[a], oracle.ON_PLUS[comp][a], blk.h[a]) for a in range(3)]
    return np.kron(w[2], np.kron(w[1], w[0]))


def energy_matrix(blocks, eps_r=1.0, mu_r=1.0):
    """Diagonal of the energy norm of Eq. (16): eps P''' on E, mu P''' on H (uniform media)."""
    d = []
    for b in blocks:
        for c in range(6):
            m = EPS0 * eps_r if c < 3 else MU0 * mu_r
            d.append(m * p3(b, c))
    return np.concatenate(d)


def kron_axis(op, axis, ext):
    """Extend a 1D operator along axis to 3D with identities of the given (x, y, z) extents (ED_1-3)."""
    mats = [np.eye(ext[0]), np.eye(ext[1]), np.eye(ext[2])]
    mats[axis] = op
    return np.kron(mats[2], np.kron(mats[1], mats[0]))


# Eqs. (7)-(12): component -> ((sign, partner, axis), (sign, partner, axis))
CURL = {
    0: ((+1, 5, 1), (-1, 4, 2)),
    1: ((+1, 3, 2), (-1, 5, 0)),
    2: ((+1, 4, 0), (-1, 3, 1)),
    3: ((+1, 1, 2), (-1, 2, 1)),
    4: ((+1, 2, 0), (-1, 0, 2)),
    5: ((+1, 0, 1), (-1, 1, 0)),
}


def kronecker_operator(blk, faces):
    """Expected M for one vacuum block with PEC/PMC faces, built from the printed Q, P:
    PEC ends replace Q- by Q- - B^T on the H equations, PMC ends replace Q+ by Q+ - B on
    the E equations (the closed forms the SATs of Eqs. (13)-(15), (19)-(21) produce)."""
    sz = sizes(blk)
    offs = np.concatenate([[0], np.cumsum(sz)])
    M = np.zeros((offs[-1], offs[-1]))
    for c in range(6):
        ext_c = oracle.extents(blk.n, c)
        for sgn, u, a in CURL[c]:
            n, h = blk.n[a], blk.h[a]
            if c < 3:   # E equation, D+ on the plus grid
                Q = appendix.q_plus(n).copy()
                if faces[2 * a] == oracle.PMC:
                    Q[0, 0] += 1.0            # - B_low, B_low = -1 at (0, 0)
                if faces[2 * a + 1] == oracle.PMC:
                    Q[n, n + 1] -= 1.0        # - B_high, B_high = +1 at (n, n+1)
                op = np.linalg.solve(np.diag(appendix.p_plus(n)), Q) / h / EPS0
            else:       # H equation, D- on the minus grid
                Q = appendix.q_minus(n).copy()
                if faces[2 * a] == oracle.PEC:
                    Q[0, 0] += 1.0
                if faces[2 * a + 1] == oracle.PEC:
                    Q[n + 1, n] -= 1.0
                op = np.linalg.solve(np.diag(appendix.p_minus(n)), Q) / h / MU0
            K = kron_axis(op, a, ext_c)
            M[offs[c]:offs[c + 1], offs[u]:offs[u + 1]] += sgn * K
    return M
