"""A second, independent statement of one RK stage in NumPy, for the pins.

Written from the scheme's definition (Colella-Woodward PPM with MC-limited
slopes and the parabola limiter, face EOS with the dual-energy switch, the
Kurganov-Noelle-Petrova central-upwind flux, the flux-divergence update and
the Shu-Osher blend), vectorized over whole arrays of pencils rather than
looping cell by cell, for same-level grids (no coarse-fine faces).  Input: the
padded state of a grid whose ghosts are filled; only interiors are written.
Operations are written in the order the definition states them, one
numpy operation per rounding, so results can be compared with the oracle to
the last bits.  Test infrastructure only.
"""
import numpy as np

NX, NG, NP, NF = 8, 3, 14, 11


def _slopes(q):
    """Monotonized-central slopes of q[..., 14] at positions 1..12 (array of 14, ends unused)."""
    dm = np.zeros_like(q)
    qm, q0, qp = q[..., 0:12], q[..., 1:13], q[..., 2:14]
    dl = q0 - qm
    dr = qp - q0
    delta = 0.5 * (qp - qm)
    mag = np.minimum(np.minimum(np.abs(delta), 2.0 * np.abs(dl)), 2.0 * np.abs(dr))
    lim = np.where(delta > 0.0, mag, -mag)
    dm[..., 1:13] = np.where(dl * dr <= 0.0, 0.0, lim)
    return dm


def ppm(q):
    """Face states of q[..., 14]: (aL, aR) arrays of 14, valid at positions 2..11."""
    dm = _slopes(q)
    face = np.zeros_like(q)   # face[m]: interpolant at m + 1/2, m = 1..11
    face[..., 1:12] = 0.5 * (q[..., 1:12] + q[..., 2:13]) - (dm[..., 2:13] - dm[..., 1:12]) / 6.0
    a = q[..., 2:12]
    l = face[..., 1:11].copy()
    r = face[..., 2:12].copy()
    flat = (r - a) * (a - l) <= 0.0
    da = r - l
    lhs = da * (a - 0.5 * (l + r))
    rhs = da * da / 6.0
    move_l = ~flat & (lhs > rhs)
    move_r = ~flat & ~move_l & (-rhs > lhs)
    nl = np.where(move_l, 3.0 * a - 2.0 * r, l)
    nr = np.where(move_r, 3.0 * a - 2.0 * l, r)
    aL = np.zeros_like(q)
    aR = np.zeros_like(q)
    aL[..., 2:12] = np.where(flat, a, nl)
    aR[..., 2:12] = np.where(flat, a, nr)
    return aL, aR


def _eos(U, d, gamma, eta):
    """u, p, c of face states U[11, ...] for direction d."""
    rho = U[0]
    u = U[1 + d] / rho
    ek = 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho
    ei = U[4] - ek
    if eta > 0.0:
        ei = np.where(ei < eta * U[4], np.power(U[5], gamma), ei)
    p = (gamma - 1.0) * ei
    c = np.sqrt(gamma * p / rho)
    return u, p, c


def flux(UL, UR, d, gamma, eta):
    """Central-upwind numerical flux F[11, ...] and speeds max(a+, -a-) of faces with states UL, UR [11, ...]."""
    uL, pL, cL = _eos(UL, d, gamma, eta)
    uR, pR, cR = _eos(UR, d, gamma, eta)
    ap = np.maximum(np.maximum(uL + cL, uR + cR), 0.0)
    am = np.minimum(np.minimum(uL - cL, uR - cR), 0.0)

    def phys(U, u, p):
        F = U * u
        F[1 + d] = U[1 + d] * u + p
        F[4] = (U[4] + p) * u
        return F
    FL, FR = phys(UL, uL, pL), phys(UR, uR, pR)
    den = ap - am
    central = ~(den > 1e-300)
    safe = np.where(central, 1.0, den)
    F = ((ap * FL - am * FR) + ap * am * (UR - UL)) / safe
    F = np.where(central, 0.5 * (FL + FR), F)
    return F, np.maximum(ap, -am)


def stage(U, dx, dt, gamma=5.0 / 3.0, eta=1e-3, U0=None, beta=1.0):
    """One stage on every sub-grid of the padded state U[n, 11, 14, 14, 14]
    (ghosts filled); returns (U_out with interiors written, amax [n])."""
    n = U.shape[0]
    out = U.copy()
    dU = np.zeros((n, NF, NX, NX, NX))
    amax = np.zeros(n)
    I = slice(NG, NG + NX)
    for d in range(3):
        # pencils along axis d: move it last, keep the transverse interior
        if d == 0:
            P = U[:, :, I, I, :]                    # [n, f, k, j, m]
        elif d == 1:
            P = np.swapaxes(U[:, :, I, :, I], 3, 4)  # [n, f, k, i, m]
        else:
            P = np.moveaxis(U[:, :, :, I, I], 2, 4)  # [n, f, j, i, m]
        aL, aR = ppm(np.ascontiguousarray(P))
        UL = np.moveaxis(aR[..., 2:11], 1, 0)     # right edge of cell m, faces m + 1/2, m = 2..10
        UR = np.moveaxis(aL[..., 3:12], 1, 0)     # left edge of cell m + 1
        F, sp = flux(UL, UR, d, gamma, eta)
        amax = np.maximum(amax, sp.reshape(n, -1).max(axis=1))
        diff = np.moveaxis(F[..., 0:8] - F[..., 1:9], 0, 1)   # lower minus upper face of each interior cell
        if d == 0:
            term = diff                              # [n, f, k, j, i]
        elif d == 1:
            term = np.swapaxes(diff, 3, 4)           # [n, f, k, i, j] -> [n, f, k, j, i]
        else:
            term = np.moveaxis(diff, 4, 2)           # [n, f, j, i, k] -> [n, f, k, j, i]
        dU = term if d == 0 else dU + term
    lam = (dt / np.asarray(dx, np.float64))[:, None, None, None, None]
    Us = U[:, :, I, I, I] + lam * dU
    out[:, :, I, I, I] = Us if beta == 1.0 else U0[:, :, I, I, I] + beta * (Us - U0[:, :, I, I, I])
    return out, amax
