/* hydro_oracle.c -- plain FP64 CPU oracle for the batched octree hydro step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the CUDA library.
 *
 * The paper (Section IV-C) names the method: inviscid Euler equations solved
 * with a finite-volume central scheme (Kurganov-Tadmor) on an octree of N^3
 * sub-grids, N = 8; Section V-B.1 names the two GPU kernels it profiles: a PPM
 * reconstruction kernel and a flux kernel, inside the Runge-Kutta sub-step
 * driver compute_fluxes that also reduces the global time-step.  The paper
 * prints no formulas, so each function below follows the published method the
 * paper cites, step by step, in the order those methods state them:
 *   - PPM face interpolant and limiter: Colella & Woodward (1984), eqs. 1.6-1.10;
 *   - central-upwind flux: Kurganov, Noelle & Petrova (2001), with the central
 *     Kurganov-Tadmor (2000) flux as the a+ = -a- special case;
 *   - Shu-Osher SSP-RK3 stage blend U0 + beta (U* - U0), beta supplied by the
 *     caller (alpha = 1 - beta; the form keeps a uniform state exactly);
 *   - Neumaier compensated summation for the totals;
 *   - the three-dimensional reconstruction with Simpson face quadrature that
 *     Sections IV-C and V-B.1 name, for grids of one level, in the reading
 *     stated where it is defined (oracle_stage3d).
 * Readings where the paper is silent are listed with the design notes.
 *
 * Build: -O2 -ffp-contract=off, no -ffast-math, optional -fopenmp.
 */
#include "hydro_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { NX = 8, NG = 3, NP = 14, NF = 11, NFACE = 9 };
enum { F_RHO = 0, F_SX = 1, F_EGAS = 4, F_TAU = 5 };

static size_t at(int s, int f, int k, int j, int i) {
  return ((((size_t)s * NF + f) * NP + k) * NP + j) * NP + i;
}

/* Cell (k,j,i) of the pencil along direction d at position m, transverse
 * interior coordinates (t1, t2): x-pencils (t1,t2) = (j,k), y: (i,k), z: (i,j). */
static size_t pencil_at(int s, int f, int d, int t1, int t2, int m) {
  if (d == 0) return at(s, f, t2, t1, m);
  if (d == 1) return at(s, f, t2, m, t1);
  return at(s, f, m, t2, t1);
}

/* ------------------------------------------------------------------------- */
/* PPM reconstruction (Colella & Woodward 1984)                               */
/* ------------------------------------------------------------------------- */

/* Monotonized-central limited slope of cell with neighbours qm, q0, qp:
 * delta = (qp - qm)/2; limited to min(|delta|, 2|q0-qm|, 2|qp-q0|) with the
 * sign of delta when q0 is not a local extremum, else zero (CW84 eq. 1.8). */
static double limited_slope(double qm, double q0, double qp) {
  double dl = q0 - qm;
  double dr = qp - q0;
  if (dl * dr <= 0.0) return 0.0;
  double delta = 0.5 * (qp - qm);
  double m = fabs(delta);
  double l = 2.0 * fabs(dl);
  double r = 2.0 * fabs(dr);
  if (l < m) m = l;
  if (r < m) m = r;
  return delta > 0.0 ? m : -m;
}

/* CW84 eq. 1.10: flatten at a local extremum, else pull the far face in so
 * that the parabola has no interior extremum. */
static void parabola_limit(double a, double *lp, double *rp) {
  double l = *lp, r = *rp;
  if ((r - a) * (a - l) <= 0.0) {
    l = a;
    r = a;
  } else {
    double da = r - l;
    double lhs = da * (a - 0.5 * (l + r));
    double rhs = da * da / 6.0;
    if (lhs > rhs)
      l = 3.0 * a - 2.0 * r;
    else if (-rhs > lhs)
      r = 3.0 * a - 2.0 * l;
  }
  *lp = l;
  *rp = r;
}

void oracle_ppm_pencil(const double *q, double *aL, double *aR) {
  double dm[NP];
  double face[NP]; /* face[m] is the interpolant at face m + 1/2 */
  for (int m = 1; m <= 12; ++m) dm[m] = limited_slope(q[m - 1], q[m], q[m + 1]);
  /* CW84 eq. 1.6 with limited slopes: a_{m+1/2} = (q_m + q_{m+1})/2 - (dm_{m+1} - dm_m)/6 */
  for (int m = 1; m <= 11; ++m) face[m] = 0.5 * (q[m] + q[m + 1]) - (dm[m + 1] - dm[m]) / 6.0;
  for (int m = 2; m <= 11; ++m) {
    double l = face[m - 1];
    double r = face[m];
    parabola_limit(q[m], &l, &r);
    aL[m] = l;
    aR[m] = r;
  }
}

/* ------------------------------------------------------------------------- */
/* CW84 shock flattening and contact steepening                               */
/* ------------------------------------------------------------------------- */

/* Flattening coefficients f[m] of cells m = 2..11 of a pencil (CW84 Section 4,
 * eqs. 4.1-4.5, constants epsilon = 0.33, omega1 = 0.75, omega2 = 10): with
 * P[m + 1] = p_m for m = -1..14 (the pressure of cell m; m = -1 and 14 are the
 * fourth ghost layer) and u[m] the velocity along the pencil (m = 0..13),
 *   ft_m = max(0, min(1, omega2 ((p_{m+1} - p_{m-1}) / (p_{m+2} - p_{m-2}) - omega1)))
 * where cell m sees a shock, |p_{m+1} - p_{m-1}| > epsilon min(p_{m+1}, p_{m-1})
 * and u_{m-1} - u_{m+1} > 0, else ft_m = 0 (m = 1..12); then
 *   f_m = max(ft_m, ft_{m - sigma_m}),  sigma_m = sgn(p_{m+1} - p_{m-1}),
 * the larger of the cell's own and its upstream neighbour's. */
static void flattening_candidates(const double *P, const double *u, double *ft) {
  for (int m = 0; m < NP; ++m) ft[m] = 0.0;
  for (int m = 1; m <= 12; ++m) {
    const double pm1 = P[m], pp1 = P[m + 2], pm2 = P[m - 1], pp2 = P[m + 3];
    const double dp = pp1 - pm1;
    const double pmin = pp1 < pm1 ? pp1 : pm1;
    ft[m] = 0.0;
    if (fabs(dp) > 0.33 * pmin && u[m - 1] - u[m + 1] > 0.0) {
      const double t = 10.0 * (dp / (pp2 - pm2) - 0.75);
      double v = t > 1.0 ? 1.0 : t;
      ft[m] = v > 0.0 ? v : 0.0;
    }
  }
}

static void flattening(const double *P, const double *u, double *f) {
  double ft[NP];
  flattening_candidates(P, u, ft);
  for (int m = 2; m <= 11; ++m) {
    const double dp = P[m + 2] - P[m];
    const int up = dp > 0.0 ? m - 1 : (dp < 0.0 ? m + 1 : m);
    f[m] = ft[up] > ft[m] ? ft[up] : ft[m];
  }
}

/* Contact steepening coefficient eta of cell m from the density r (CW84 eqs.
 * 1.14-1.17 on a uniform pencil, constants eta1 = 20, eta2 = 0.05,
 * epsilon = 0.01, K0 = 0.1): with d2_k = (r_{k+1} + r_{k-1}) - 2 r_k,
 *   etat = -(d2_{m+1} - d2_{m-1}) / (6 (r_{m+1} - r_{m-1}))
 * where d2_{m+1} d2_{m-1} < 0, |r_{m+1} - r_{m-1}| - epsilon min(|r_{m+1}|, |r_{m-1}|) > 0
 * and the jump is a contact, gamma K0 |r_{m+1} - r_{m-1}| / min(r_{m+1}, r_{m-1}) >=
 * |p_{m+1} - p_{m-1}| / min(p_{m+1}, p_{m-1}); else etat = 0;
 *   eta = max(0, min(eta1 (etat - eta2), 1)). */
static double steepening(const double *r, const double *P, double gamma, int m) {
  const double d2p = (r[m + 2] + r[m]) - 2.0 * r[m + 1];
  const double d2m = (r[m] + r[m - 2]) - 2.0 * r[m - 1];
  const double dr = r[m + 1] - r[m - 1];
  const double a1 = fabs(r[m + 1]), a0 = fabs(r[m - 1]);
  const double amin = a1 < a0 ? a1 : a0;
  double etat = 0.0;
  if (d2p * d2m < 0.0 && fabs(dr) - 0.01 * amin > 0.0) {
    const double rmin = r[m + 1] < r[m - 1] ? r[m + 1] : r[m - 1];
    const double pp1 = P[m + 2], pm1 = P[m];
    const double pmin = pp1 < pm1 ? pp1 : pm1;
    if (gamma * 0.1 * fabs(dr) / rmin >= fabs(pp1 - pm1) / pmin) etat = -(d2p - d2m) / (6.0 * dr);
  }
  const double t = 20.0 * (etat - 0.05);
  const double e = t > 1.0 ? 1.0 : t;
  return e > 0.0 ? e : 0.0;
}

/* PPM of the NF fields of one pencil with the CW84 extensions of `flags`
 * (bit 0 flattening, bit 1 contact steepening), in CW84's order: interpolant
 * (eq. 1.6), steepening, flattening, parabola limiter (eq. 1.10).  P and u as
 * for flattening().  Both coefficients are properties of the cell, applied to
 * every conserved field: the flattening one from the pressure and velocity,
 * the steepening one detected on the density; with conserved variables this
 * keeps a contact (velocity and pressure uniform, every field affine in the
 * density) consistent, where steepening the density alone would not.  The
 * steepened faces are l -> l (1 - eta) + (q_{m-1} + dm_{m-1}/2) eta and
 * r -> r (1 - eta) + (q_{m+1} - dm_{m+1}/2) eta, dm the limited slopes of eq.
 * 1.8; the flattened ones l -> f q_m + (1 - f) l, r -> f q_m + (1 - f) r. */
static void ppm_pencil_cw84(double q[NF][NP], const double *P, const double *u, double gamma, int flags,
                            double aL[NF][NP], double aR[NF][NP]) {
  double fl[NP], st[NP];
  for (int m = 0; m < NP; ++m) fl[m] = st[m] = 0.0;
  if (flags & 1) flattening(P, u, fl);
  if (flags & 2)
    for (int m = 2; m <= 11; ++m) st[m] = steepening(q[F_RHO], P, gamma, m);
  for (int f = 0; f < NF; ++f) {
    double dm[NP], face[NP];
    for (int m = 1; m <= 12; ++m) dm[m] = limited_slope(q[f][m - 1], q[f][m], q[f][m + 1]);
    for (int m = 1; m <= 11; ++m) face[m] = 0.5 * (q[f][m] + q[f][m + 1]) - (dm[m + 1] - dm[m]) / 6.0;
    for (int m = 2; m <= 11; ++m) {
      const double a = q[f][m];
      double l = face[m - 1], r = face[m];
      if (st[m] > 0.0) {
        l = l * (1.0 - st[m]) + (q[f][m - 1] + 0.5 * dm[m - 1]) * st[m];
        r = r * (1.0 - st[m]) + (q[f][m + 1] - 0.5 * dm[m + 1]) * st[m];
      }
      if (fl[m] > 0.0) {
        l = fl[m] * a + (1.0 - fl[m]) * l;
        r = fl[m] * a + (1.0 - fl[m]) * r;
      }
      parabola_limit(a, &l, &r);
      aL[f][m] = l;
      aR[f][m] = r;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Face EOS and numerical flux                                                */
/* ------------------------------------------------------------------------- */

void oracle_face_eos(const double *U, int d, double gamma, double eta, double *u, double *p, double *c) {
  double rho = U[F_RHO];
  double sx = U[F_SX], sy = U[F_SX + 1], sz = U[F_SX + 2];
  double E = U[F_EGAS];
  *u = U[F_SX + d] / rho;
  double ek = 0.5 * (sx * sx + sy * sy + sz * sz) / rho;
  double ei = E - ek;
  /* dual-energy switch: when the internal energy is a small fraction of the
   * total, take it from the entropy tracer, e_i = tau^gamma */
  if (eta > 0.0 && ei < eta * E) ei = pow(U[F_TAU], gamma);
  *p = (gamma - 1.0) * ei;
  *c = sqrt(gamma * *p / rho);
}

/* Physical flux along d: every field is carried with velocity u; the normal
 * momentum adds p and the energy adds p*u. */
static void physical_flux(const double *U, int d, double u, double p, double *F) {
  for (int f = 0; f < NF; ++f) F[f] = U[f] * u;
  F[F_SX + d] = U[F_SX + d] * u + p;
  F[F_EGAS] = (U[F_EGAS] + p) * u;
}

double oracle_face_flux(const double *UL, const double *UR, int d, double gamma, double eta, int form,
                        double *F) {
  double uL, pL, cL, uR, pR, cR;
  oracle_face_eos(UL, d, gamma, eta, &uL, &pL, &cL);
  oracle_face_eos(UR, d, gamma, eta, &uR, &pR, &cR);
  double ap, am;
  if (form == 1) { /* Kurganov-Tadmor: one local speed a, a+ = a, a- = -a */
    double a = fabs(uL) + cL;
    double b = fabs(uR) + cR;
    ap = a > b ? a : b;
    am = -ap;
  } else { /* Kurganov-Noelle-Petrova one-sided local speeds */
    ap = uL + cL;
    if (uR + cR > ap) ap = uR + cR;
    if (0.0 > ap) ap = 0.0;
    am = uL - cL;
    if (uR - cR < am) am = uR - cR;
    if (0.0 < am) am = 0.0;
  }
  double FL[NF], FR[NF];
  physical_flux(UL, d, uL, pL, FL);
  physical_flux(UR, d, uR, pR, FR);
  double den = ap - am;
  if (den > 1e-300) {
    for (int f = 0; f < NF; ++f) F[f] = ((ap * FL[f] - am * FR[f]) + ap * am * (UR[f] - UL[f])) / den;
  } else {
    for (int f = 0; f < NF; ++f) F[f] = 0.5 * (FL[f] + FR[f]);
  }
  return ap > -am ? ap : -am;
}

/* ------------------------------------------------------------------------- */
/* One RK stage on one sub-grid                                               */
/* ------------------------------------------------------------------------- */

typedef struct {
  double flux[3][NF][NX][NX][NFACE]; /* [d][f][t2][t1][face], face m+1/2 for m = 2..10 */
} work_t;

/* Face fluxes of every pencil of sub-grid s into w->flux; returns the largest
 * face speed. */
static double ghost_value(const oracle_grid *g, const double *U, int s, int a, int side, int ga, int c1, int c2,
                          int f);

static double flux_subgrid(const oracle_grid *g, int s, const double *Uin, work_t *w) {
  double q[NF][NP], aL[NF][NP], aR[NF][NP];
  double UL[NF], UR[NF], F[NF];
  double amax = 0.0;
  for (int d = 0; d < 3; ++d) {
    for (int t2 = NG; t2 < NG + NX; ++t2) {
      for (int t1 = NG; t1 < NG + NX; ++t1) {
        for (int f = 0; f < NF; ++f)
          for (int m = 0; m < NP; ++m) q[f][m] = Uin[pencil_at(s, f, d, t1, t2, m)];
        if (g->cw84) {
          /* cell pressures along the pencil, m = -1..14 (the fourth ghost
           * layer from the neighbours' interiors by the ghost-fill rules), and
           * the velocities along it, m = 0..13 */
          double P[NP + 2], u[NP], cell[NF], c;
          for (int m = -1; m <= NP; ++m) {
            if (m < 0 || m == NP) {
              const int side = m < 0 ? 0 : 1;
              for (int f = 0; f < NF; ++f)
                cell[f] = ghost_value(g, Uin, s, d, side, side ? NX + NG : -1 - NG, t1 - NG, t2 - NG, f);
            } else {
              for (int f = 0; f < NF; ++f) cell[f] = q[f][m];
            }
            double um;
            oracle_face_eos(cell, d, g->gamma, g->de_switch, &um, &P[m + 1], &c);
            if (m >= 0 && m < NP) u[m] = um;
          }
          ppm_pencil_cw84(q, P, u, g->gamma, g->cw84, aL, aR);
        } else {
          for (int f = 0; f < NF; ++f) oracle_ppm_pencil(q[f], aL[f], aR[f]);
        }
        for (int m = 2; m <= 10; ++m) {
          for (int f = 0; f < NF; ++f) {
            UL[f] = aR[f][m];     /* right edge of cell m */
            UR[f] = aL[f][m + 1]; /* left edge of cell m+1 */
          }
          double a = oracle_face_flux(UL, UR, d, g->gamma, g->de_switch, g->flux_form, F);
          if (a != a || a > amax) amax = a; /* a NaN speed sticks */
          for (int f = 0; f < NF; ++f) w->flux[d][f][t2 - NG][t1 - NG][m - 2] = F[f];
        }
      }
    }
  }
  return amax;
}

/* Coarse-fine flux correction (paper Section V-B.1: compute_fluxes corrects the
 * fluxes on coarse-fine boundaries).  On every face of sub-grid s whose
 * neighbours are finer, the flux of each coarse boundary face is replaced by
 * the mean of the four fine fluxes over it, as the fine neighbour computes
 * them on its own boundary face:
 *   F = ((F(0,0) + F(1,0)) + (F(0,1) + F(1,1))) * 1/4,
 * (a, b) the fine offsets along the face's first and second transverse axes.
 * The fine side loses exactly what the coarse side gains, so the AMR step
 * conserves to round-off.  Only fine neighbours advanced in the same call
 * (listed in `in_batch`, or all when it is NULL) count; elsewhere the coarse
 * flux stays.  w2 is scratch for the neighbours' fluxes. */
static void correct_fluxes(const oracle_grid *g, int s, const double *Uin, const unsigned char *in_batch, work_t *w,
                           work_t *w2) {
  for (int face = 0; face < 6; ++face) {
    if (g->neighbor_rel[s * 6 + face] != 1) continue;
    const int d = face / 2, side = face % 2;
    const int32_t *nb = g->neighbor + ((size_t)s * 6 + face) * 4;
    const int mine = side ? NFACE - 1 : 0, theirs = side ? 0 : NFACE - 1;
    for (int q = 0; q < 4; ++q) {
      const int q1 = q & 1, q2 = q >> 1;
      if (in_batch && !in_batch[nb[q]]) continue;
      flux_subgrid(g, nb[q], Uin, w2);
      for (int c2 = 4 * q2; c2 < 4 * q2 + 4; ++c2)
        for (int c1 = 4 * q1; c1 < 4 * q1 + 4; ++c1) {
          const int f1 = 2 * (c1 - 4 * q1), f2 = 2 * (c2 - 4 * q2);
          for (int f = 0; f < NF; ++f) {
            const double a00 = w2->flux[d][f][f2][f1][theirs], a10 = w2->flux[d][f][f2][f1 + 1][theirs];
            const double a01 = w2->flux[d][f][f2 + 1][f1][theirs], a11 = w2->flux[d][f][f2 + 1][f1 + 1][theirs];
            w->flux[d][f][c2][c1][mine] = ((a00 + a10) + (a01 + a11)) * 0.25;
          }
        }
    }
  }
}

static int update_subgrid(const oracle_grid *g, int s, const double *Uin, const double *U0, double beta,
                          double dt, double *Uout, const work_t *w);

static int stage_subgrid(const oracle_grid *g, int s, const double *Uin, const double *U0, double beta,
                         double dt, double *Uout, double *amax_s, const unsigned char *in_batch, work_t *w,
                         work_t *w2) {
  *amax_s = flux_subgrid(g, s, Uin, w);
  if (g->reflux) correct_fluxes(g, s, Uin, in_batch, w, w2);
  return update_subgrid(g, s, Uin, U0, beta, dt, Uout, w);
}

/* Uout = U0 + beta (Uin + dt/dx dU - U0) of sub-grid s from the face fluxes in w. */
static int update_subgrid(const oracle_grid *g, int s, const double *Uin, const double *U0, double beta,
                          double dt, double *Uout, const work_t *w) {
  double lam = dt / g->dx[s];
  int bad = 0;
  for (int k = NG; k < NG + NX; ++k) {
    for (int j = NG; j < NG + NX; ++j) {
      for (int i = NG; i < NG + NX; ++i) {
        int ii = i - NG, jj = j - NG, kk = k - NG;
        for (int f = 0; f < NF; ++f) {
          /* cell i has faces i-1/2 (stored index i-3) and i+1/2 (index i-2) */
          double fxl = w->flux[0][f][kk][jj][ii], fxh = w->flux[0][f][kk][jj][ii + 1];
          double fyl = w->flux[1][f][kk][ii][jj], fyh = w->flux[1][f][kk][ii][jj + 1];
          double fzl = w->flux[2][f][jj][ii][kk], fzh = w->flux[2][f][jj][ii][kk + 1];
          double dU = ((fxl - fxh) + (fyl - fyh)) + (fzl - fzh);
          size_t o = at(s, f, k, j, i);
          double Us = Uin[o] + lam * dU;
          double v = (beta == 1.0) ? Us : U0[o] + beta * (Us - U0[o]);
          Uout[o] = v;
          if (!isfinite(v) || (f == F_RHO && !(v > 0.0))) bad = 1;
        }
      }
    }
  }
  return bad;
}

int oracle_stage(const oracle_grid *g, const int32_t *ids, int32_t n_ids, const double *Uin, const double *U0,
                 double beta, double dt, double *Uout, double *max_speed, double *sub_amax, int nthreads,
                 int batch_all) {
  if (!g || !Uin || !Uout || !max_speed || n_ids < 0) return ORACLE_ERR_INVALID;
  if (beta != 1.0 && !U0) return ORACLE_ERR_INVALID;
  int n = ids ? n_ids : g->n;
  double amax = 0.0, amax_dx = 0.0;
  int bad = 0;
  unsigned char *in_batch = NULL;
  if (ids && !batch_all) {
    in_batch = (unsigned char *)calloc((size_t)g->n, 1);
    for (int t = 0; t < n_ids; ++t)
      if (ids[t] >= 0 && ids[t] < g->n) in_batch[ids[t]] = 1;
  }
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(max : amax, amax_dx) reduction(| : bad)
#endif
  {
    work_t *w = (work_t *)malloc(sizeof(work_t));
    work_t *w2 = (work_t *)malloc(sizeof(work_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (int t = 0; t < n; ++t) {
      int s = ids ? ids[t] : t;
      double a = 0.0;
      bad |= stage_subgrid(g, s, Uin, U0, beta, dt, Uout, &a, in_batch, w, w2);
      if (sub_amax) sub_amax[s] = a;
      if (a != a) bad = 1;
      if (a > amax) amax = a;
      if (a / g->dx[s] > amax_dx) amax_dx = a / g->dx[s];
    }
    free(w);
    free(w2);
  }
  (void)nthreads;
  free(in_batch);
  max_speed[0] = amax;
  max_speed[1] = amax_dx;
  return bad ? ORACLE_ERR_NONFINITE : ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Margin cells of the error metric: interior cells near a branch decision     */
/* ------------------------------------------------------------------------- */

/* The scheme above takes discrete decisions: the slope's extremum test
 * (dl dr <= 0), the parabola's extremum test ((r - a)(a - l) <= 0), its two
 * overshoot tests (lhs > rhs, -rhs > lhs), and the dual-energy test at every
 * face side (e_i < eta E).  An implementation that rounds differently (another
 * precision, another operation order) may decide such a test the other way
 * when its operands are within rounding of the threshold.  A test counts as
 * "near" when its distance from the threshold is at most tol times the
 * magnitude its operands are computed from:
 *   slope:     0 < |dl| <= tol S or 0 < |dr| <= tol S,  S = max |q| of the 3 cells;
 *   extremum:  0 < |r - a| <= tol S or 0 < |a - l| <= tol S,  S = max(|a|, |l|, |r|);
 *   overshoot: |lhs -+ rhs| <= tol |r - l| S;
 *   dual energy: |e_i - eta E| <= tol (|E| + e_k).
 * Differences that are exactly zero are not near: equal inputs stay equal in
 * any precision.  A near test at pencil position m marks the interior cells of
 * that pencil within 3 cells of m (the update stencil's reach along the pencil);
 * a near face test marks those around both of its cells.  mask[s][512]
 * ((k*8 + j)*8 + i) is OR-ed, for the listed sub-grids, with one bit per kind
 * of test (MARGIN_* in the header); returns the number of near tests found.
 * The three PPM tests decide between outcomes that meet where the test is
 * exactly at its threshold (the limited slope and the pulled faces tend to the
 * unlimited ones), so a decision taken the other way there moves a face value
 * by about the distance from the threshold; the dual-energy test switches
 * between two pressures that differ wherever tau^gamma and E - e_k disagree. */
static int near_zero(double v, double tol_scale) { return v != 0.0 && fabs(v) <= tol_scale; }

static double max3(double a, double b, double c) {
  double m = fabs(a);
  if (fabs(b) > m) m = fabs(b);
  if (fabs(c) > m) m = fabs(c);
  return m;
}

static void mark_pencil(unsigned char *mask, int d, int t1, int t2, int m, unsigned char bit) {
  for (int c = m - 3; c <= m + 3; ++c) {
    if (c < NG || c >= NG + NX) continue;
    int i, j, k;
    if (d == 0) { i = c; j = t1; k = t2; }
    else if (d == 1) { i = t1; j = c; k = t2; }
    else { i = t1; j = t2; k = c; }
    mask[((k - NG) * NX + (j - NG)) * NX + (i - NG)] |= bit;
  }
}

static int dual_energy_near(const double *U, double eta, double tol) {
  double rho = U[F_RHO], sx = U[F_SX], sy = U[F_SX + 1], sz = U[F_SX + 2], E = U[F_EGAS];
  double ek = 0.5 * (sx * sx + sy * sy + sz * sz) / rho;
  double ei = E - ek;
  return eta > 0.0 && fabs(ei - eta * E) <= tol * (fabs(E) + fabs(ek));
}

/* The CW84 tests of one pencil near their thresholds, counted only where
 * taking the test the other way would change the coefficient: each detector
 * fires when all of its tests pass, so a test near its threshold matters only
 * where the detector's other tests pass and its value would be positive
 * (flattening: shock and compression tests, candidate clamp(omega2 (ratio -
 * omega1)) > 0, and the sign of its denominator p_{m+2} - p_{m-2}, across
 * which the candidate jumps between 0 and 1; the sign of dp that picks the
 * upstream neighbour, where the two
 * neighbours' candidates differ; steepening: curvature, jump and contact
 * tests, clamp(eta1 (etat - eta2)) > 0 for the unconditioned etat).  Each of
 * these switches between outcomes that do not meet at the threshold.  A
 * pressure enters with the relative uncertainty of its own evaluation: tol
 * times (|E| + e_k) / |e_i| (the cancellation in e_i = E - e_k), 16 tol on the
 * tau^gamma branch, and 1 where the dual-energy test itself is near its
 * threshold (either branch may be taken). */
static long cw84_margins(const oracle_grid *g, const double *U, int s, int d, int t1, int t2, double tol,
                         unsigned char *ms) {
  double P[NP + 2], K[NP + 2], u[NP], r[NP], cell[NF], c, ft[NP];
  long found = 0;
  for (int m = -1; m <= NP; ++m) {
    if (m < 0 || m == NP) {
      const int side = m < 0 ? 0 : 1;
      for (int f = 0; f < NF; ++f)
        cell[f] = ghost_value(g, U, s, d, side, side ? NX + NG : -1 - NG, t1 - NG, t2 - NG, f);
    } else {
      for (int f = 0; f < NF; ++f) cell[f] = U[pencil_at(s, f, d, t1, t2, m)];
      r[m] = cell[F_RHO];
    }
    double um;
    oracle_face_eos(cell, d, g->gamma, g->de_switch, &um, &P[m + 1], &c);
    if (m >= 0 && m < NP) u[m] = um;
    /* relative uncertainty of the pressure (K[m + 1] * |p|) */
    const double E = cell[F_EGAS];
    const double ek = 0.5 * (cell[F_SX] * cell[F_SX] + cell[F_SX + 1] * cell[F_SX + 1] +
                             cell[F_SX + 2] * cell[F_SX + 2]) / cell[F_RHO];
    const double ei = E - ek;
    if (dual_energy_near(cell, g->de_switch, tol))
      K[m + 1] = 1.0;
    else if (g->de_switch > 0.0 && ei < g->de_switch * E)
      K[m + 1] = 16.0 * tol;
    else
      K[m + 1] = ei != 0.0 ? tol * (fabs(E) + fabs(ek)) / fabs(ei) : 1.0;
    if (K[m + 1] > 1.0) K[m + 1] = 1.0;
  }
  if (g->cw84 & 1) flattening_candidates(P, u, ft);
  for (int m = 1; m <= 12; ++m) {
    const double pm1 = P[m], pp1 = P[m + 2], pm2 = P[m - 1], pp2 = P[m + 3];
    const double S = fabs(pp1) > fabs(pm1) ? fabs(pp1) : fabs(pm1);
    const double pmin = pp1 < pm1 ? pp1 : pm1;
    const double dp = pp1 - pm1;
    const double up = K[m] * fabs(pm1) + K[m + 2] * fabs(pp1); /* uncertainty of dp */
    int near = 0;
    if (g->cw84 & 1) {
      const double t = 10.0 * (dp / (pp2 - pm2) - 0.75);
      {
        const int shock = fabs(dp) > 0.33 * pmin, comp = u[m - 1] - u[m + 1] > 0.0;
        const double S2 = fabs(pp2) > fabs(pm2) ? fabs(pp2) : fabs(pm2);
        const double up2 = K[m - 1] * fabs(pm2) + K[m + 3] * fabs(pp2);
        near = shock && comp && near_zero(pp2 - pm2, tol * S2 + up2);
      }
      if (t > 0.0) {
        const double us = fabs(u[m - 1]) > fabs(u[m + 1]) ? fabs(u[m - 1]) : fabs(u[m + 1]);
        const int shock = fabs(dp) > 0.33 * pmin, comp = u[m - 1] - u[m + 1] > 0.0;
        const int near_shock = fabs(fabs(dp) - 0.33 * pmin) <= tol * S + up;
        const int near_comp = near_zero(u[m - 1] - u[m + 1], tol * us);
        near = near || (near_shock && comp) || (near_comp && shock);
      }
      if (m >= 2 && m <= 11 && ft[m - 1] != ft[m + 1]) near = near || near_zero(dp, tol * S + up);
    }
    if ((g->cw84 & 2) && m >= 2 && m <= 11) {
      const double d2p = (r[m + 2] + r[m]) - 2.0 * r[m + 1];
      const double d2m = (r[m] + r[m - 2]) - 2.0 * r[m - 1];
      const double dr = r[m + 1] - r[m - 1];
      if (dr != 0.0 && 20.0 * (-(d2p - d2m) / (6.0 * dr) - 0.05) > 0.0) {
        const double R = max3(r[m - 1], r[m], r[m + 1]);
        const double a1 = fabs(r[m + 1]), a0 = fabs(r[m - 1]);
        const double amin = a1 < a0 ? a1 : a0;
        const double rmin = r[m + 1] < r[m - 1] ? r[m + 1] : r[m - 1];
        const int curv = d2p * d2m < 0.0, jump = fabs(dr) - 0.01 * amin > 0.0;
        int contact = 0, near_contact = 0;
        if (rmin > 0.0 && pmin > 0.0) {
          const double lhs = g->gamma * 0.1 * fabs(dr) / rmin, rhs = fabs(dp) / pmin;
          contact = lhs >= rhs;
          near_contact = fabs(lhs - rhs) <= tol * (fabs(lhs) + fabs(rhs)) + (up / fabs(dp != 0.0 ? dp : 1.0) + K[m] + K[m + 2]) * rhs;
        }
        const int near_curv = near_zero(d2p, tol * R) || near_zero(d2m, tol * R);
        const int near_jump = fabs(fabs(dr) - 0.01 * amin) <= tol * R;
        near = near || (near_curv && jump && contact) || (near_jump && curv && contact) ||
               (near_contact && curv && jump);
      }
    }
    if (near) {
      mark_pencil(ms, d, t1, t2, m, MARGIN_CW84);
      ++found;
    }
  }
  return found;
}

long oracle_margin_cells(const oracle_grid *g, const int32_t *ids, int32_t n_ids, const double *U, double tol,
                         unsigned char *mask) {
  int n = ids ? n_ids : g->n;
  long found = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : found)
#endif
  for (int t = 0; t < n; ++t) {
    int s = ids ? ids[t] : t;
    unsigned char *ms = mask + (size_t)s * NX * NX * NX;
    for (int d = 0; d < 3; ++d)
      for (int t2 = NG; t2 < NG + NX; ++t2)
        for (int t1 = NG; t1 < NG + NX; ++t1) {
          double aL[NF][NP], aR[NF][NP];
          for (int f = 0; f < NF; ++f) {
            double q[NP], face[NP];
            for (int m = 0; m < NP; ++m) q[m] = U[pencil_at(s, f, d, t1, t2, m)];
            for (int m = 1; m <= 12; ++m) {
              double S = max3(q[m - 1], q[m], q[m + 1]);
              if (near_zero(q[m] - q[m - 1], tol * S) || near_zero(q[m + 1] - q[m], tol * S)) {
                mark_pencil(ms, d, t1, t2, m, MARGIN_SLOPE);
                ++found;
              }
            }
            /* the face values before the limiter, as the PPM above forms them */
            double dm[NP];
            for (int m = 1; m <= 12; ++m) dm[m] = limited_slope(q[m - 1], q[m], q[m + 1]);
            for (int m = 1; m <= 11; ++m) face[m] = 0.5 * (q[m] + q[m + 1]) - (dm[m + 1] - dm[m]) / 6.0;
            for (int m = 2; m <= 11; ++m) {
              double a = q[m], l = face[m - 1], r = face[m];
              double S = max3(a, l, r);
              if (near_zero(r - a, tol * S) || near_zero(a - l, tol * S)) {
                mark_pencil(ms, d, t1, t2, m, MARGIN_EXTREMUM);
                ++found;
              }
              if (!((r - a) * (a - l) <= 0.0)) {
                double da = r - l;
                double lhs = da * (a - 0.5 * (l + r)), rhs = da * da / 6.0;
                if (fabs(lhs - rhs) <= tol * fabs(da) * S || fabs(lhs + rhs) <= tol * fabs(da) * S) {
                  mark_pencil(ms, d, t1, t2, m, MARGIN_OVERSHOOT);
                  ++found;
                }
              }
            }
            oracle_ppm_pencil(q, aL[f], aR[f]);
          }
          for (int m = 2; m <= 10; ++m) {
            double UL[NF], UR[NF];
            for (int f = 0; f < NF; ++f) {
              UL[f] = aR[f][m];
              UR[f] = aL[f][m + 1];
            }
            if (dual_energy_near(UL, g->de_switch, tol) || dual_energy_near(UR, g->de_switch, tol)) {
              mark_pencil(ms, d, t1, t2, m, MARGIN_DUAL_ENERGY);
              mark_pencil(ms, d, t1, t2, m + 1, MARGIN_DUAL_ENERGY);
              ++found;
            }
          }
          if (g->cw84) found += cw84_margins(g, U, s, d, t1, t2, tol, ms);
        }
  }
  return found;
}

/* ------------------------------------------------------------------------- */
/* Ghost fill                                                                 */
/* ------------------------------------------------------------------------- */

/* padded coordinate array p[3] = (i, j, k) */
static size_t at3(int s, int f, const int *p) { return at(s, f, p[2], p[1], p[0]); }

static const int T1[3] = {1, 0, 0}; /* first transverse axis of a face normal to axis a */
static const int T2[3] = {2, 2, 1}; /* second transverse axis */

static int floor_half(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }

/* The value of field f of the ghost cell of sub-grid s across the face of
 * axis a on `side`, at interior coordinate ga along a (-1, -2, ... on the low
 * side; 8, 9, ... on the high side) and interior coordinates (c1, c2) along the
 * face's transverse axes, from the current interiors. */
static double ghost_value(const oracle_grid *g, const double *U, int s, int a, int side, int ga, int c1, int c2,
                          int f) {
  const int face = 2 * a + side;
  const int b1 = T1[a], b2 = T2[a];
  const int rel = g->neighbor_rel[s * 6 + face];
  const int32_t *nb = g->neighbor + ((size_t)s * 6 + face) * 4;
  int dst[3];
  dst[a] = ga + NG;
  dst[b1] = c1 + NG;
  dst[b2] = c2 + NG;
  if (nb[0] < 0) { /* outflow: nearest interior cell */
    int src[3] = {dst[0], dst[1], dst[2]};
    src[a] = side ? NG + NX - 1 : NG;
    return U[at3(s, f, src)];
  }
  if (rel == 0) { /* same level: the neighbour's interior cell */
    int src[3] = {dst[0], dst[1], dst[2]};
    src[a] = (side ? ga - NX : ga + NX) + NG;
    return U[at3(nb[0], f, src)];
  }
  if (rel < 0) {
    /* coarser neighbour: value of the coarse cell that contains the centre of
     * the fine ghost cell.  In coarse-cell units relative to the neighbour's
     * interior origin, this sub-grid's origin is at 8 (neighbour on the low
     * side) or -4 (high side) along a, and at 4*octant bit along each
     * transverse axis. */
    int oct = g->octant[s];
    int src[3];
    src[a] = (side ? -4 : 8) + floor_half(ga) + NG;
    src[b1] = 4 * ((oct >> b1) & 1) + floor_half(c1) + NG;
    src[b2] = 4 * ((oct >> b2) & 1) + floor_half(c2) + NG;
    return U[at3(nb[0], f, src)];
  }
  /* finer neighbours: mean of the 2x2x2 fine cells covering the coarse ghost
   * cell, summed in (k, j, i) order */
  int q1 = c1 >> 2, q2 = c2 >> 2;
  int fs = nb[q1 + 2 * q2];
  int base[3];
  base[a] = 2 * (side ? ga - NX : ga + 4);
  base[b1] = 2 * (c1 - 4 * q1);
  base[b2] = 2 * (c2 - 4 * q2);
  double sum = 0.0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        int src[3] = {base[0] + di + NG, base[1] + dj + NG, base[2] + dk + NG};
        sum += U[at3(fs, f, src)];
      }
  return sum * 0.125;
}

double oracle_ghost_cell(const oracle_grid *g, const double *U, int s, int face, int ga, int c1, int c2, int f) {
  return ghost_value(g, U, s, face / 2, face % 2, ga, c1, c2, f);
}

int oracle_fill_ghosts(const oracle_grid *g, double *U) {
  for (int s = 0; s < g->n; ++s)
    for (int face = 0; face < 6; ++face) {
      const int a = face / 2, side = face % 2;
      const int b1 = T1[a], b2 = T2[a];
      for (int f = 0; f < NF; ++f)
        for (int layer = 0; layer < NG; ++layer) {
          /* interior coordinate of the ghost cell along a: -1,-2,-3 or 8,9,10 */
          const int ga = side ? NX + layer : -1 - layer;
          for (int c2 = 0; c2 < NX; ++c2)
            for (int c1 = 0; c1 < NX; ++c1) {
              int dst[3];
              dst[a] = ga + NG;
              dst[b1] = c1 + NG;
              dst[b2] = c2 + NG;
              U[at3(s, f, dst)] = ghost_value(g, U, s, a, side, ga, c1, c2, f);
            }
        }
    }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Totals                                                                     */
/* ------------------------------------------------------------------------- */

/* Neumaier's improved Kahan summation: add x to (sum, comp). */
static void neumaier_add(double *sum, double *comp, double x) {
  double t = *sum + x;
  if (fabs(*sum) >= fabs(x))
    *comp += (*sum - t) + x;
  else
    *comp += (x - t) + *sum;
  *sum = t;
}

void oracle_totals(const oracle_grid *g, const double *U, double *totals) {
  for (int f = 0; f < NF; ++f) {
    double S = 0.0, C = 0.0;
    for (int s = 0; s < g->n; ++s) {
      double ss = 0.0, sc = 0.0;
      for (int k = NG; k < NG + NX; ++k)
        for (int j = NG; j < NG + NX; ++j)
          for (int i = NG; i < NG + NX; ++i) neumaier_add(&ss, &sc, U[at(s, f, k, j, i)]);
      double vol = g->dx[s] * g->dx[s] * g->dx[s];
      neumaier_add(&S, &C, vol * ss);
      neumaier_add(&S, &C, vol * sc);
    }
    totals[f] = S + C;
  }
}

/* ------------------------------------------------------------------------- */
/* Diagnostics (paper Section V-B.1, diagnostics task: total mass, total     */
/* angular momentum, centre of mass of each star of a binary).               */
/*                                                                           */
/* Per interior cell of sub-grid s, centre (x, y, z) = origin_s + (i + 1/2,  */
/* j + 1/2, k + 1/2) dx_s, each coordinate rounded as o + ((c + 1/2) * dx):  */
/*   q0 = rho,                                    total mass M                */
/*   q1..q3 = r x s = (y sz - z sy, z sx - x sz, x sy - y sx), angular        */
/*            momentum about the origin, each product rounded separately;     */
/*   q4 = rho X1, q5..q7 = rho X1 * (x, y, z)      star 1 (scalar field 6)     */
/*   q8 = rho X2, q9..q11 = rho X2 * (x, y, z)     star 2 (scalar field 7)     */
/* Q_q = sum_s dx_s^3 sum_cells q (Neumaier, in sub-grid order), then         */
/* out = {M, Lx, Ly, Lz, M1, X1, Y1, Z1, M2, X2, Y2, Z2}, the centres being    */
/* Q_{5..7} / Q_4 and Q_{9..11} / Q_8 (0 where the star mass is 0).           */
/* ------------------------------------------------------------------------- */

enum { NQ = 12 };

static void cell_quantities(const double *U, int s, int k, int j, int i, const double *o, double dx, double *q) {
  const double x = o[0] + (i + 0.5) * dx, y = o[1] + (j + 0.5) * dx, z = o[2] + (k + 0.5) * dx;
  const int K = k + NG, J = j + NG, I = i + NG;
  const double rho = U[at(s, F_RHO, K, J, I)];
  const double sx = U[at(s, F_SX, K, J, I)], sy = U[at(s, F_SX + 1, K, J, I)], sz = U[at(s, F_SX + 2, K, J, I)];
  const double m1 = U[at(s, 6, K, J, I)], m2 = U[at(s, 7, K, J, I)];
  q[0] = rho;
  q[1] = y * sz - z * sy;
  q[2] = z * sx - x * sz;
  q[3] = x * sy - y * sx;
  q[4] = m1;
  q[5] = m1 * x;
  q[6] = m1 * y;
  q[7] = m1 * z;
  q[8] = m2;
  q[9] = m2 * x;
  q[10] = m2 * y;
  q[11] = m2 * z;
}

void oracle_diagnostics(const oracle_grid *g, const double *U, const double *origin, double *out) {
  double S[NQ], C[NQ];
  for (int q = 0; q < NQ; ++q) S[q] = C[q] = 0.0;
  for (int s = 0; s < g->n; ++s) {
    double ss[NQ], sc[NQ], v[NQ];
    for (int q = 0; q < NQ; ++q) ss[q] = sc[q] = 0.0;
    for (int k = 0; k < NX; ++k)
      for (int j = 0; j < NX; ++j)
        for (int i = 0; i < NX; ++i) {
          cell_quantities(U, s, k, j, i, origin + 3 * (size_t)s, g->dx[s], v);
          for (int q = 0; q < NQ; ++q) neumaier_add(&ss[q], &sc[q], v[q]);
        }
    const double vol = g->dx[s] * g->dx[s] * g->dx[s];
    for (int q = 0; q < NQ; ++q) {
      neumaier_add(&S[q], &C[q], vol * ss[q]);
      neumaier_add(&S[q], &C[q], vol * sc[q]);
    }
  }
  double T[NQ];
  for (int q = 0; q < NQ; ++q) T[q] = S[q] + C[q];
  out[0] = T[0];
  out[1] = T[1];
  out[2] = T[2];
  out[3] = T[3];
  for (int star = 0; star < 2; ++star) {
    const double m = T[4 + 4 * star];
    out[4 + 4 * star] = m;
    for (int c = 0; c < 3; ++c) out[5 + 4 * star + c] = m != 0.0 ? T[5 + 4 * star + c] / m : 0.0;
  }
}

/* ------------------------------------------------------------------------- */
/* Dual-energy resynchronisation of the entropy tracer (the paper is silent on */
/* the EOS; a reading that completes the face EOS switch above).              */
/* Per interior cell, with the same kinetic and internal energies as the face */
/* EOS:                                                                       */
/*   e_k = (sx^2 + sy^2 + sz^2) / 2 rho,   e_i = E - e_k;                      */
/* where the switch takes e_i from the total energy (eta > 0, e_i > 0 and     */
/* e_i >= eta E: the complement of the face EOS test e_i < eta E), the tracer */
/* is reset to the value that reproduces it, tau = e_i^(1/gamma); every other */
/* cell and field is left as it is.  Returns the number of cells reset.       */
/* ------------------------------------------------------------------------- */

long oracle_tau_resync(const oracle_grid *g, double *U) {
  const double eta = g->de_switch;
  if (!(eta > 0.0)) return 0;
  const double inv_gamma = 1.0 / g->gamma;
  long reset = 0;
  for (int s = 0; s < g->n; ++s)
    for (int k = 0; k < NX; ++k)
      for (int j = 0; j < NX; ++j)
        for (int i = 0; i < NX; ++i) {
          const double rho = U[at(s, F_RHO, k + NG, j + NG, i + NG)];
          const double sx = U[at(s, F_SX, k + NG, j + NG, i + NG)];
          const double sy = U[at(s, F_SX + 1, k + NG, j + NG, i + NG)];
          const double sz = U[at(s, F_SX + 2, k + NG, j + NG, i + NG)];
          const double E = U[at(s, F_EGAS, k + NG, j + NG, i + NG)];
          const double ek = 0.5 * (sx * sx + sy * sy + sz * sz) / rho;
          const double ei = E - ek;
          if (ei > 0.0 && ei >= eta * E) {
            U[at(s, F_TAU, k + NG, j + NG, i + NG)] = pow(ei, inv_gamma);
            ++reset;
          }
        }
  return reset;
}

/* ------------------------------------------------------------------------- */
/* Three-dimensional reconstruction with Simpson face quadrature             */
/* ------------------------------------------------------------------------- */

/* The paper (Section IV-C) names a full three-dimensional reconstruction and
 * (Section V-B.1) a flux kernel that applies a Newton-Cotes quadrature over
 * each face, without stating either.  The reading built here, for grids of one
 * level:
 *   1. PPM along the face normal (oracle_ppm_pencil) gives the left and right
 *      states of every face as averages over the face;
 *   2. across the face, the face averages of the 3 x 3 faces around it (same
 *      plane, neighbouring pencils) determine, per state and field, the
 *      tensor product of the parabolas whose averages over three cells are
 *      the three given ones; evaluated at the 3 x 3 Simpson points of the face
 *      (transverse offsets -1/2, 0, +1/2 of the face width);
 *   3. each parabola is limited to stay monotone: at a local extremum of the
 *      three averages the face value is constant; where the parabola's edge
 *      values leave the range of the neighbouring averages, or its centre
 *      value leaves the range of its edge values, it is replaced by the line
 *      with the monotonized-central slope;
 *   4. the numerical flux at each of the 9 points from the two point states,
 *      combined with the Simpson weights (1, 4, 1)/6 in each transverse
 *      direction, row by row.
 * It is exact for states quadratic across the face (the face average of the
 * flux of transverse quadratics), where point values of one-dimensional PPM
 * along the 13 lines through a cell are not. */

/* Point values at -1/2, 0, +1/2 of the centre cell of the limited parabola
 * whose averages over three cells are am, a0, ap. */
static void transverse_points(double am, double a0, double ap, double *lo, double *mid, double *hi) {
  if ((ap - a0) * (a0 - am) <= 0.0) {
    *lo = a0;
    *mid = a0;
    *hi = a0;
    return;
  }
  const double d1 = ap - am;
  const double d2 = (ap + am) - 2.0 * a0;
  double l = (a0 + d2 / 12.0) - d1 / 4.0;
  double h = (a0 + d2 / 12.0) + d1 / 4.0;
  double c = a0 - d2 / 24.0;
  const int outside = (l - am) * (a0 - l) < 0.0 || (h - a0) * (ap - h) < 0.0 || (c - l) * (h - c) < 0.0;
  if (outside) {
    const double sl = limited_slope(am, a0, ap);
    l = a0 - 0.5 * sl;
    h = a0 + 0.5 * sl;
    c = a0;
  }
  *lo = l;
  *mid = c;
  *hi = h;
}

/* Whether a test of transverse_points(am, a0, ap) sits within t = tol S of its
 * threshold (S the largest magnitude of the three averages and the parabola's
 * three values) where taking it the other way would move a point value by
 * more than t:
 *   the extremum test, when a0 - am or ap - a0 is non-zero and at most t: the
 *     other outcome is the parabola (or, if a range test holds, the line,
 *     whose half-slope is at most that small difference);
 *   the range tests, once the extremum test passes, when one of lo - am,
 *     a0 - lo, hi - a0, ap - hi, mid - lo, hi - mid is non-zero and at most t
 *     while no other range test holds by more than t: the outcomes are the
 *     parabola and the line a0 -+ sl/2. */
static int transverse_near(double am, double a0, double ap, double tol) {
  const double d1 = ap - am;
  const double d2 = (ap + am) - 2.0 * a0;
  const double l = (a0 + d2 / 12.0) - d1 / 4.0;
  const double h = (a0 + d2 / 12.0) + d1 / 4.0;
  const double c = a0 - d2 / 24.0;
  double S = max3(am, a0, ap);
  const double S2 = max3(l, h, c);
  if (S2 > S) S = S2;
  const double t = tol * S;
  /* the line of the limiter as if the extremum test passed */
  double m = fabs(0.5 * d1);
  if (2.0 * fabs(a0 - am) < m) m = 2.0 * fabs(a0 - am);
  if (2.0 * fabs(ap - a0) < m) m = 2.0 * fabs(ap - a0);
  const double half = 0.5 * (d1 > 0.0 ? m : -m);
  const double jump_line = fmax(fmax(fabs(l - (a0 - half)), fabs(c - a0)), fabs(h - (a0 + half)));
  const double a[3] = {l - am, h - a0, c - l}, b[3] = {a0 - l, ap - h, h - c};
  int near_range = 0, clear_out = 0;
  for (int k = 0; k < 3; ++k) {
    const int nk = near_zero(a[k], t) || near_zero(b[k], t);
    if (nk) near_range = 1;
    else if (a[k] * b[k] < 0.0) clear_out = 1;
  }
  if (near_zero(ap - a0, t) || near_zero(a0 - am, t)) {
    const double jump = clear_out ? fabs(half) : fmax(fmax(fabs(l - a0), fabs(c - a0)), fabs(h - a0));
    if (jump > t) return 1;
  }
  if ((ap - a0) * (a0 - am) <= 0.0) return 0;
  return near_range && !clear_out && jump_line > t;
}

/* The value of field f at padded cell (i, j, k) of sub-grid s, for any cell of
 * the 14^3 padded cube of a grid of one level: each coordinate outside the
 * interior moves to the neighbour across that face (outflow: the nearest
 * interior cell), faces, edges and corners alike. */
static double full_cell(const oracle_grid *g, const double *U, int s, int i, int j, int k, int f) {
  int c[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (c[a] >= NG && c[a] < NG + NX) continue;
    const int side = c[a] >= NG + NX ? 1 : 0;
    const int nb = g->neighbor[((size_t)s * 6 + 2 * a + side) * 4];
    if (nb < 0) {
      c[a] = side ? NG + NX - 1 : NG;
    } else {
      s = nb;
      c[a] += side ? -NX : NX;
    }
  }
  return U[at(s, f, c[2], c[1], c[0])];
}

static int single_level(const oracle_grid *g) {
  for (int s = 0; s < g->n; ++s) {
    if (g->dx[s] != g->dx[0]) return 0;
    for (int f = 0; f < 6; ++f)
      if (g->neighbor_rel[s * 6 + f] != 0) return 0;
  }
  return 1;
}

int oracle_fill_ghosts_full(const oracle_grid *g, double *U) {
  if (!single_level(g)) return ORACLE_ERR_INVALID;
  for (int s = 0; s < g->n; ++s)
    for (int f = 0; f < NF; ++f)
      for (int k = 0; k < NP; ++k)
        for (int j = 0; j < NP; ++j)
          for (int i = 0; i < NP; ++i) {
            const int inside = i >= NG && i < NG + NX && j >= NG && j < NG + NX && k >= NG && k < NG + NX;
            if (!inside) U[at(s, f, k, j, i)] = full_cell(g, U, s, i, j, k, f);
          }
  return ORACLE_OK;
}

typedef struct {
  double aL[NX + 2][NX + 2][NF][NP], aR[NX + 2][NX + 2][NF][NP]; /* [t2 + 1][t1 + 1]: pencils -1..8 */
} face_avg_t;

/* Steps 2-4 for one face normal to d: AL, AR [b2][b1][f] are the left and
 * right face-average states of the 3 x 3 faces around it (b = 0, 1, 2 for
 * offsets -1, 0, +1 along the face's first and second transverse axes); F[f]
 * the Simpson flux; returns the largest point signal speed. */
/* Steps 2-3 for one state of one face: A [b2][b1][f] the face averages of
 * the 3 x 3 faces around it -> P [q2][q1][f] the point states; with near !=
 * NULL, *near is set when one of the parabolas has a test near its threshold
 * (transverse_near). */
static void point_states(const double *A, double (*P)[3][NF], double tol, int *near) {
  for (int f = 0; f < NF; ++f) {
    double rows[3][3]; /* [b2][q1] */
    for (int b2 = 0; b2 < 3; ++b2) {
      const double am = A[(b2 * 3 + 0) * NF + f], a0 = A[(b2 * 3 + 1) * NF + f], ap = A[(b2 * 3 + 2) * NF + f];
      transverse_points(am, a0, ap, &rows[b2][0], &rows[b2][1], &rows[b2][2]);
      if (near && transverse_near(am, a0, ap, tol)) *near = 1;
    }
    for (int q1 = 0; q1 < 3; ++q1) {
      transverse_points(rows[0][q1], rows[1][q1], rows[2][q1], &P[0][q1][f], &P[1][q1][f], &P[2][q1][f]);
      if (near && transverse_near(rows[0][q1], rows[1][q1], rows[2][q1], tol)) *near = 1;
    }
  }
}

double oracle_simpson_flux(const double *AL, const double *AR, int d, double gamma, double eta, int form, double *F) {
  double PL[3][3][NF], PR[3][3][NF]; /* [q2][q1][f] point states */
  point_states(AL, PL, 0.0, NULL);
  point_states(AR, PR, 0.0, NULL);
  double Fq[3][3][NF];
  double amax = 0.0;
  for (int q2 = 0; q2 < 3; ++q2)
    for (int q1 = 0; q1 < 3; ++q1) {
      const double a = oracle_face_flux(PL[q2][q1], PR[q2][q1], d, gamma, eta, form, Fq[q2][q1]);
      if (a != a || a > amax) amax = a;
    }
  /* weights (1, 4, 1)/6, the two outer points added first so that mirror
   * images of a face give the same sum bit for bit */
  for (int f = 0; f < NF; ++f) {
    double row[3];
    for (int q2 = 0; q2 < 3; ++q2) row[q2] = ((Fq[q2][0][f] + Fq[q2][2][f]) + 4.0 * Fq[q2][1][f]) / 6.0;
    F[f] = ((row[0] + row[2]) + 4.0 * row[1]) / 6.0;
  }
  return amax;
}

/* Face fluxes of sub-grid s (every cell of its padded cube filled) by the 3D
 * reconstruction and the Simpson rule, into w->flux; returns the largest
 * point signal speed. */
static double flux3d_subgrid(const oracle_grid *g, int s, const double *Uin, work_t *w, face_avg_t *fa) {
  double amax = 0.0;
  for (int d = 0; d < 3; ++d) {
    /* step 1: PPM along d for the 10 x 10 pencils around the sub-grid */
    for (int t2 = NG - 1; t2 <= NG + NX; ++t2)
      for (int t1 = NG - 1; t1 <= NG + NX; ++t1)
        for (int f = 0; f < NF; ++f) {
          double q[NP];
          for (int m = 0; m < NP; ++m) q[m] = Uin[pencil_at(s, f, d, t1, t2, m)];
          oracle_ppm_pencil(q, fa->aL[t2 - NG + 1][t1 - NG + 1][f], fa->aR[t2 - NG + 1][t1 - NG + 1][f]);
        }
    /* steps 2-4 for every face of the sub-grid */
    for (int t2 = 0; t2 < NX; ++t2)
      for (int t1 = 0; t1 < NX; ++t1)
        for (int m = 2; m <= 10; ++m) {
          double AL[3][3][NF], AR[3][3][NF], F[NF];
          for (int b2 = 0; b2 < 3; ++b2)
            for (int b1 = 0; b1 < 3; ++b1)
              for (int f = 0; f < NF; ++f) {
                AL[b2][b1][f] = fa->aR[t2 + b2][t1 + b1][f][m];     /* right edge of cell m */
                AR[b2][b1][f] = fa->aL[t2 + b2][t1 + b1][f][m + 1]; /* left edge of cell m + 1 */
              }
          const double a = oracle_simpson_flux(&AL[0][0][0], &AR[0][0][0], d, g->gamma, g->de_switch, g->flux_form, F);
          if (a != a || a > amax) amax = a;
          for (int f = 0; f < NF; ++f) w->flux[d][f][t2][t1][m - 2] = F[f];
        }
  }
  return amax;
}

/* Margin cells of the 3D reconstruction: per face, a transverse test of its
 * point states within tol of its threshold (transverse_near) or the
 * dual-energy test at one of its 18 point states (dual_energy_near) marks
 * the two cells beside the face (their update is the only one that face's
 * flux enters).  The transverse tests switch between outcomes that do not
 * meet at the threshold (a parabola against a constant or a line), as the
 * dual-energy test does.  U: every ghost cell filled
 * (oracle_fill_ghosts_full); mask as for oracle_margin_cells, OR-ed with
 * MARGIN_RECON3D and MARGIN_DUAL_ENERGY; returns the number of marked faces,
 * or ORACLE_ERR_INVALID on a grid of several levels. */
static void mark_cell(unsigned char *mask, int d, int t1, int t2, int c, unsigned char bit) {
  if (c < NG || c >= NG + NX) return;
  int i, j, k;
  if (d == 0) { i = c; j = t1; k = t2; }
  else if (d == 1) { i = t1; j = c; k = t2; }
  else { i = t1; j = t2; k = c; }
  mask[((k - NG) * NX + (j - NG)) * NX + (i - NG)] |= bit;
}

long oracle_margin_cells3d(const oracle_grid *g, const double *U, double tol, unsigned char *mask) {
  if (!g || !U || !mask || !single_level(g)) return ORACLE_ERR_INVALID;
  long found = 0;
#ifdef _OPENMP
#pragma omp parallel reduction(+ : found)
#endif
  {
    face_avg_t *fa = (face_avg_t *)malloc(sizeof(face_avg_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (int s = 0; s < g->n; ++s) {
      unsigned char *ms = mask + (size_t)s * NX * NX * NX;
      for (int d = 0; d < 3; ++d) {
        for (int t2 = NG - 1; t2 <= NG + NX; ++t2)
          for (int t1 = NG - 1; t1 <= NG + NX; ++t1)
            for (int f = 0; f < NF; ++f) {
              double q[NP];
              for (int m = 0; m < NP; ++m) q[m] = U[pencil_at(s, f, d, t1, t2, m)];
              oracle_ppm_pencil(q, fa->aL[t2 - NG + 1][t1 - NG + 1][f], fa->aR[t2 - NG + 1][t1 - NG + 1][f]);
            }
        for (int t2 = 0; t2 < NX; ++t2)
          for (int t1 = 0; t1 < NX; ++t1)
            for (int m = 2; m <= 10; ++m) {
              double AL[3][3][NF], AR[3][3][NF], PL[3][3][NF], PR[3][3][NF];
              for (int b2 = 0; b2 < 3; ++b2)
                for (int b1 = 0; b1 < 3; ++b1)
                  for (int f = 0; f < NF; ++f) {
                    AL[b2][b1][f] = fa->aR[t2 + b2][t1 + b1][f][m];
                    AR[b2][b1][f] = fa->aL[t2 + b2][t1 + b1][f][m + 1];
                  }
              int near = 0, dual = 0;
              point_states(&AL[0][0][0], PL, tol, &near);
              point_states(&AR[0][0][0], PR, tol, &near);
              for (int q2 = 0; q2 < 3; ++q2)
                for (int q1 = 0; q1 < 3; ++q1)
                  if (dual_energy_near(PL[q2][q1], g->de_switch, tol) || dual_energy_near(PR[q2][q1], g->de_switch, tol))
                    dual = 1;
              if (!near && !dual) continue;
              const unsigned char bit = (unsigned char)((near ? MARGIN_RECON3D : 0) | (dual ? MARGIN_DUAL_ENERGY : 0));
              mark_cell(ms, d, t1 + NG, t2 + NG, m, bit);
              mark_cell(ms, d, t1 + NG, t2 + NG, m + 1, bit);
              ++found;
            }
      }
    }
    free(fa);
  }
  return found;
}

int oracle_stage3d(const oracle_grid *g, const double *Uin, const double *U0, double beta, double dt, double *Uout,
                   double *max_speed, int nthreads) {
  if (!g || !Uin || !Uout || !max_speed) return ORACLE_ERR_INVALID;
  if (beta != 1.0 && !U0) return ORACLE_ERR_INVALID;
  if (!single_level(g)) return ORACLE_ERR_INVALID;
  double amax = 0.0, amax_dx = 0.0;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(max : amax, amax_dx) reduction(| : bad)
#endif
  {
    work_t *w = (work_t *)malloc(sizeof(work_t));
    face_avg_t *fa = (face_avg_t *)malloc(sizeof(face_avg_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (int s = 0; s < g->n; ++s) {
      const double a = flux3d_subgrid(g, s, Uin, w, fa);
      bad |= update_subgrid(g, s, Uin, U0, beta, dt, Uout, w);
      if (a != a) bad = 1;
      if (a > amax) amax = a;
      if (a / g->dx[s] > amax_dx) amax_dx = a / g->dx[s];
    }
    free(w);
    free(fa);
  }
  (void)nthreads;
  max_speed[0] = amax;
  max_speed[1] = amax_dx;
  return bad ? ORACLE_ERR_NONFINITE : ORACLE_OK;
}
