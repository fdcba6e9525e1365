"""A second, independent statement of one RK stage with the three-dimensional
reconstruction and Simpson face quadrature, in NumPy, for the pins.

Written from the reading of the scheme (PPM along the face normal gives face
averages; the limited tensor-product parabola through the 3 x 3 neighbouring
face averages, first along the face's first transverse axis, then along its
second, gives the values at the 3 x 3 Simpson points; the central-upwind flux
at each point; the Simpson weights (1, 4, 1)/6 along each axis, outer points
first), on the GLOBAL array of a periodic box: every neighbour is a
`np.roll`, so there are no sub-grids, ghost cells or neighbour tables at all,
which is where the oracle's indexing could go wrong.  One numpy operation per
rounding, in the definition's order, so results can be compared with the
oracle to the last bits.  Test infrastructure only.
"""
import numpy as np

from tests import numpy_stage as NS

# axes of G[f][z][y][x]: the normal of direction d and its first and second
# transverse axes (x-faces: y then z; y-faces: x then z; z-faces: x then y)
NORMAL = {0: 3, 1: 2, 2: 1}
TRANSVERSE = {0: (2, 1), 1: (3, 1), 2: (3, 2)}


def ppm_faces(q, ax):
    """Left and right face values (aL, aR) of every cell of the periodic array
    q along axis ax: MC-limited slopes, the fourth-order interpolant, the
    parabola limiter."""
    qm, qp = np.roll(q, 1, ax), np.roll(q, -1, ax)
    dl, dr = q - qm, qp - q
    delta = 0.5 * (qp - qm)
    mag = np.minimum(np.minimum(np.abs(delta), 2.0 * np.abs(dl)), 2.0 * np.abs(dr))
    dm = np.where(dl * dr <= 0.0, 0.0, np.where(delta > 0.0, mag, -mag))
    face = 0.5 * (q + qp) - (np.roll(dm, -1, ax) - dm) / 6.0     # at i + 1/2
    a, l, r = q, np.roll(face, 1, ax), face
    flat = (r - a) * (a - l) <= 0.0
    da = r - l
    lhs = da * (a - 0.5 * (l + r))
    rhs = da * da / 6.0
    move_l = ~flat & (lhs > rhs)
    move_r = ~flat & ~move_l & (-rhs > lhs)
    aL = np.where(flat, a, np.where(move_l, 3.0 * a - 2.0 * r, l))
    aR = np.where(flat, a, np.where(move_r, 3.0 * a - 2.0 * l, r))
    return aL, aR


def transverse(A, ax):
    """Values at -1/2, 0, +1/2 of every cell's limited parabola through the
    averages A of it and its two neighbours along axis ax."""
    am, a0, ap = np.roll(A, 1, ax), A, np.roll(A, -1, ax)
    flat = (ap - a0) * (a0 - am) <= 0.0
    d1 = ap - am
    d2 = (ap + am) - 2.0 * a0
    l = (a0 + d2 / 12.0) - d1 / 4.0
    h = (a0 + d2 / 12.0) + d1 / 4.0
    c = a0 - d2 / 24.0
    outside = ((l - am) * (a0 - l) < 0.0) | ((h - a0) * (ap - h) < 0.0) | ((c - l) * (h - c) < 0.0)
    dl, dr = a0 - am, ap - a0
    delta = 0.5 * (ap - am)
    mag = np.minimum(np.minimum(np.abs(delta), 2.0 * np.abs(dl)), 2.0 * np.abs(dr))
    sl = np.where(dl * dr <= 0.0, 0.0, np.where(delta > 0.0, mag, -mag))
    lo = np.where(flat, a0, np.where(outside, a0 - 0.5 * sl, l))
    mid = np.where(flat | outside, a0, c)
    hi = np.where(flat, a0, np.where(outside, a0 + 0.5 * sl, h))
    return lo, mid, hi


def point_states(A, d):
    """The 3 x 3 point states P[q2][q1] of the faces whose averages are A[11, ...]."""
    t1, t2 = TRANSVERSE[d]
    rows = transverse(A, t1)
    P = [[None] * 3 for _ in range(3)]
    for q1 in range(3):
        lo, mid, hi = transverse(rows[q1], t2)
        P[0][q1], P[1][q1], P[2][q1] = lo, mid, hi
    return P


def face_fluxes(G, d, gamma, eta):
    """Simpson fluxes F[11, ...] of the faces i + 1/2 along d (indexed by the
    cell i on their left) and the largest point speed."""
    ax = NORMAL[d]
    aL, aR = ppm_faces(G, ax)
    UL, UR = aR, np.roll(aL, -1, ax)
    PL, PR = point_states(UL, d), point_states(UR, d)
    Fq = [[None] * 3 for _ in range(3)]
    amax = 0.0
    for q2 in range(3):
        for q1 in range(3):
            Fq[q2][q1], sp = NS.flux(PL[q2][q1], PR[q2][q1], d, gamma, eta)
            amax = max(amax, float(sp.max()))
    rows = [((Fq[q2][0] + Fq[q2][2]) + 4.0 * Fq[q2][1]) / 6.0 for q2 in range(3)]
    return ((rows[0] + rows[2]) + 4.0 * rows[1]) / 6.0, amax


def stage(G, dx, dt, gamma=5.0 / 3.0, eta=1e-3, G0=None, beta=1.0):
    """One stage of the periodic global state G[11, Z, Y, X]: returns
    (G_out, max_speed)."""
    F = {}
    amax = 0.0
    for d in range(3):
        F[d], a = face_fluxes(G, d, gamma, eta)
        amax = max(amax, a)
    diff = [np.roll(F[d], 1, NORMAL[d]) - F[d] for d in range(3)]
    dU = (diff[0] + diff[1]) + diff[2]
    lam = dt / dx
    Us = G + lam * dU
    out = Us if beta == 1.0 else G0 + beta * (Us - G0)
    return out, amax
