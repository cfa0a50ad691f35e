"""Dense SBP matrices built from the closure blocks printed in the Appendix.

The blocks come from ``tests/golden/appendix_operators.txt`` (typed from the
paper); the interior rows follow the printed band pattern (-1, 1).  Nothing
here calls the oracle, so these matrices pin the oracle's operator tables.
"""
import os
from fractions import Fraction

import numpy as np

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "appendix_operators.txt")


def _load():
    blocks = {}
    ends = {}
    with open(_GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0].endswith("_end"):
                ends[parts[0]] = [float(Fraction(v)) for v in parts[1:]]
            else:
                blocks.setdefault(parts[0], []).append((int(parts[1]), int(parts[2]), float(Fraction(parts[3]))))
    return blocks, ends


_BLOCKS, _ENDS = _load()


def _fill(M, name_top, name_bot):
    R, Cn = M.shape
    for r, c, v in _BLOCKS[name_top]:
        M[r, c] = v
    for r, c, v in _BLOCKS[name_bot]:
        M[R + r, Cn + c] = v


def q_plus(n):
    """Q+ of size (n+1) x (n+2)."""
    M = np.zeros((n + 1, n + 2))
    for r in range(2, n - 1):            # interior rows: -1 at column r, +1 at column r+1
        M[r, r], M[r, r + 1] = -1.0, 1.0
    _fill(M, "Qp_top", "Qp_bot")
    return M


def q_minus(n):
    """Q- of size (n+2) x (n+1)."""
    M = np.zeros((n + 2, n + 1))
    for r in range(3, n - 1):            # interior rows: -1 at column r-1, +1 at column r
        M[r, r - 1], M[r, r] = -1.0, 1.0
    _fill(M, "Qm_top", "Qm_bot")
    return M


def d_plus_printed(n):
    M = np.zeros((n + 1, n + 2))
    for r in range(2, n - 1):
        M[r, r], M[r, r + 1] = -1.0, 1.0
    _fill(M, "Dp_top", "Dp_bot")
    return M


def d_minus_printed(n):
    M = np.zeros((n + 2, n + 1))
    for r in range(3, n - 1):
        M[r, r - 1], M[r, r] = -1.0, 1.0
    _fill(M, "Dm_top", "Dm_bot")
    return M


def p_plus(n):
    e = _ENDS["Pp_end"]
    p = np.ones(n + 1)
    p[0] = p[-1] = e[0]
    return p


def p_minus(n):
    e = _ENDS["Pm_end"]
    p = np.ones(n + 2)
    p[0:3] = e
    p[-3:] = e[::-1]
    return p


def boundary_b(n):
    """B of Eq. (4): -1 at (0, 0), +1 at (n, n+1), size (n+1) x (n+2)."""
    B = np.zeros((n + 1, n + 2))
    B[0, 0] = -1.0
    B[n, n + 1] = 1.0
    return B
