"""Per-cell relative error metric of the parity tests and the sweep.

For a field f over the compared interior cells,

    err_f = max_cells |x - r| / max(|r|, 1e-8 * ||r_f||_inf),

so every cell is measured against its own value, down to a floor of 1e-8 of
the field's largest magnitude (a field that is identically zero in the
reference must be exactly zero).  ||r_f||_inf is taken over the compared cells.

Margin cells: interior cells near a branch decision of the scheme (the oracle's
`margin_cells`, tests within 64 eps of their threshold, spread 3 cells along the
pencil).  Two kinds are told apart:
  * the PPM tests (slope extremum, parabola extremum, overshoot) choose between
    outcomes that meet at the threshold, so taking them the other way moves a
    face value by about the rounding that put the test near its threshold; those
    cells stay in the gate and are only counted;
  * the dual-energy test switches between two pressures that need not agree,
    and the CW84 flattening and steepening tests (when enabled) switch a
    coefficient on or off; those cells (and their stencil) are left out of the
    gate, counted, and their error is reported separately.
No solver arithmetic lives here.
"""
import numpy as np

FLOOR = 1e-8
EPS = {"fp64": 2.0 ** -53, "mixed": 2.0 ** -24}
M_SLOPE, M_EXTREMUM, M_OVERSHOOT, M_DUAL, M_CW84, M_RECON3D = 1, 2, 4, 8, 16, 32
M_SWITCH = M_DUAL | M_CW84 | M_RECON3D   # tests whose two outcomes need not meet at the threshold
SL = (slice(None), slice(None), slice(3, 11), slice(3, 11), slice(3, 11))


def interiors(U):
    """[m, 11, 14, 14, 14] padded states -> [m, 11, 8, 8, 8] interiors (views pass through)."""
    return U[SL] if U.shape[-1] == 14 else U


def cell_errors(x, r):
    """Per-cell errors e[m, 11, 8, 8, 8] and the per-field norms ||r_f||_inf."""
    xi, ri = interiors(x), interiors(r)
    d = np.abs(xi - ri)
    norm = np.abs(ri).max(axis=(0, 2, 3, 4))
    den = np.maximum(np.abs(ri), FLOOR * norm[None, :, None, None, None])
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d == 0, 0.0, np.inf))
    e = np.where(np.isnan(xi) & ~np.isnan(ri), np.inf, e)
    return e, norm


def r12(x, r, margin=None):
    """Errors of x against r (padded [m,11,14,14,14] or interiors [m,11,8,8,8]).

    margin: optional uint8 [m, 8, 8, 8] of MARGIN_* bits.  Returns a dict:
      err        per-field max error over the gated cells (all cells but the
                 dual-energy margin cells),
      err_margin per-field max error over the dual-energy margin cells (0 if none),
      err_all    per-field max error over every cell,
      n_cells, n_margin (dual-energy margin cells), n_near_ppm (cells near a
      PPM test only: counted, still gated), worst (index of the worst gated cell
      of the worst field, as (m, f, k, j, i)).
    """
    e, norm = cell_errors(x, r)
    m = e.shape[0]
    if margin is None:
        margin = np.zeros((m, 8, 8, 8), np.uint8)
    dual = (margin & M_SWITCH) != 0
    ppm = ((margin & (M_SLOPE | M_EXTREMUM | M_OVERSHOOT)) != 0) & ~dual
    gated = np.where(dual[:, None], 0.0, e)
    out = {
        "err": gated.max(axis=(0, 2, 3, 4)),
        "err_margin": np.where(dual[:, None], e, 0.0).max(axis=(0, 2, 3, 4)),
        "err_all": e.max(axis=(0, 2, 3, 4)),
        "n_cells": int(m * 512),
        "n_margin": int(dual.sum()),
        "n_near_ppm": int(ppm.sum()),
        "norm": norm,
    }
    out["worst"] = tuple(int(v) for v in np.unravel_index(np.argmax(gated), gated.shape))
    return out


def summary(res):
    """One-line text of r12's result for assertion messages."""
    return ("R12 err per field %s; margin cells %d of %d (their err %s); cells near PPM tests %d; worst cell %s"
            % (np.array2string(res["err"], precision=2), res["n_margin"], res["n_cells"],
               np.array2string(res["err_margin"], precision=2), res["n_near_ppm"], res["worst"]))


def margin_union(oracle_obj, states, eps, ids=None):
    """Union of the oracle's margin cells over the input states of the stages
    compared (the stage input alone, or U, U1, U2 of an RK3 step)."""
    mask = None
    for U in states:
        mask, _ = oracle_obj.margin_cells(U, eps, ids=ids, mask=mask)
    return mask


def momentum_scaled(x, r, gamma=5.0 / 3.0, margin=None):
    """Per field of the three momenta, the largest per-cell error measured
    against the cell's own momentum-density scale:
        max_cells |x - r| / max(|r|, rho c, 1e-8 ||r_f||_inf),
    rho c from the reference cell (c = sqrt(gamma p / rho), p = (gamma - 1)
    (E - |s|^2 / 2 rho), clipped at 0).  It reads like R12 wherever a cell moves
    faster than sound and like an error relative to rho c in near-static cells,
    where the momentum one stage makes is a difference of face pressures far
    below the pressure itself.  margin (optional, as for r12): cells with an
    M_SWITCH bit are left out.  Returns an array of 3."""
    xi, ri = interiors(x), interiors(r)
    rho = ri[:, 0]
    s2 = ri[:, 1] ** 2 + ri[:, 2] ** 2 + ri[:, 3] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        p = (gamma - 1.0) * np.maximum(ri[:, 4] - 0.5 * s2 / rho, 0.0)
        rc = np.sqrt(gamma * rho * p)
    out = np.zeros(3)
    for k, f in enumerate((1, 2, 3)):
        d = np.abs(xi[:, f] - ri[:, f])
        sc = np.maximum(np.maximum(np.abs(ri[:, f]), rc), FLOOR * np.abs(ri[:, f]).max())
        with np.errstate(divide="ignore", invalid="ignore"):
            e = np.where(sc > 0, d / np.where(sc > 0, sc, 1.0), np.where(d == 0, 0.0, np.inf))
        if margin is not None:
            e = np.where((margin & M_SWITCH) != 0, 0.0, e)
        out[k] = e.max()
    return out
