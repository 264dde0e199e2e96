"""Ghost-cell averages beyond a grid-aligned wall (Sec. 4.1, Fig. 2).

Beyond an extendable face two ghost cells are filled so that a quartic
polynomial, fixed by the four interior cell averages nearest the wall and by
the boundary datum on the face, has those averages (Sec. 4.1, the two ghost
formulas for Dirichlet and for Neumann data).  The paper prints the Dirichlet
and Neumann coefficients; it gives none for Robin data.  This module derives
all three cases from that one defining property, by solving the 5 x 5 fit
exactly, so that the printed numbers serve as an independent pin.

Coordinates: s is the signed distance from the wall in units of h, positive
outward.  Interior cell k (k = 0 nearest the wall) covers s in [-k-1, -k];
ghost m (m = 1, 2) covers [m-1, m].  The outward normal derivative on the
face is (1/h) d/ds.
"""
from __future__ import annotations

import numpy as np

from workloads import DIRICHLET, NEUMANN, ROBIN


def _avg_monomial(q: int, s0: float, s1: float) -> float:
    """Average of s**q over [s0, s1]."""
    return (s1 ** (q + 1) - s0 ** (q + 1)) / ((q + 1) * (s1 - s0))


def ghost_coefficients(kind: int, alpha1: float, alpha2: float, h: float):
    """Return G, a 2 x 5 array: ghost_m = G[m-1, :4] . (U_0..U_3) + G[m-1, 4] * g.

    U_k is the average over interior cell k (k = 0 touches the wall) and g the
    face average of N u, N = alpha1 + alpha2 d/dn (Dirichlet: alpha1=1,
    alpha2=0; Neumann: alpha1=0, alpha2=1).
    """
    if kind == DIRICHLET:
        alpha1, alpha2 = 1.0, 0.0
    elif kind == NEUMANN:
        alpha1, alpha2 = 0.0, 1.0
    elif kind != ROBIN:
        raise ValueError("unknown boundary kind")
    # Rows: 4 interior averages, then the boundary functional at s = 0.
    M = np.zeros((5, 5))
    for k in range(4):
        for q in range(5):
            M[k, q] = _avg_monomial(q, -k - 1.0, -float(k))
    # p(0) = a_0 ; p'(0) = a_1 ; N p = alpha1 a_0 + alpha2 a_1 / h
    M[4, 0] = alpha1
    M[4, 1] = alpha2 / h
    Minv = np.linalg.inv(M)           # coefficients a = Minv @ [U0..U3, g]
    G = np.zeros((2, 5))
    for m in (1, 2):
        row = np.array([_avg_monomial(q, m - 1.0, float(m)) for q in range(5)])
        G[m - 1] = row @ Minv
    return G


def extrapolation_coefficients():
    """Return E, a 2 x 5 array: the averages over the cells at depth m = 1, 2
    beyond a wall of the quartic that has the averages U_0..U_4 of the five
    cells nearest the wall (no boundary datum).  Used for the corner ghosts
    that the cross term needs where two walls meet."""
    M = np.zeros((5, 5))
    for k in range(5):
        for q in range(5):
            M[k, q] = _avg_monomial(q, -k - 1.0, -float(k))
    Minv = np.linalg.inv(M)
    E = np.zeros((2, 5))
    for m in (1, 2):
        row = np.array([_avg_monomial(q, m - 1.0, float(m)) for q in range(5)])
        E[m - 1] = row @ Minv
    return E
