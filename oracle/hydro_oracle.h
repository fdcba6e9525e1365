/* hydro_oracle.h -- plain FP64 CPU oracle for the batched octree hydro step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * What it computes (paper Section IV-C: inviscid Euler equations, finite-volume
 * central scheme, octree of 8^3 sub-grids; Section V-B.1: PPM reconstruction
 * kernel and flux kernel; Section V-B.1 compute_fluxes: one Runge-Kutta
 * sub-step with a global time-step reduction; diagnostics: grid totals):
 *
 *   stage:  per sub-grid, per direction, PPM (Colella-Woodward) reconstruction
 *           of the 11 conserved fields on the 9 faces of every pencil, face EOS
 *           with dual-energy switch, central-upwind (Kurganov-Noelle-Petrova)
 *           or central (Kurganov-Tadmor) flux, the coarse-fine flux
 *           correction (coarse boundary faces take the mean of the four fine
 *           fluxes), flux-divergence update and Shu-Osher RK blend; the
 *           maximum signal speed over all faces.
 *   ghosts: fill of the 6 face ghost slabs (3 layers) from neighbours: copy,
 *           coarse-to-fine injection, fine-to-coarse 2x2x2 mean, outflow.
 *   totals: Neumaier-compensated grid totals of the 11 fields;
 *   diagnostics: total mass, angular momentum, centre of mass of each star;
 *   resync: dual-energy reset of the entropy tracer tau from the internal energy.
 *
 * Layout: U[s][f][k][j][i], 14^3 padded cells per field, interior 3..10.
 * Compile with -O2 -ffp-contract=off (no fused multiply-add, no fast-math).
 */
#ifndef HYDRO_ORACLE_H
#define HYDRO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n;                   /* number of sub-grids */
  double gamma;                /* ideal-gas adiabatic index */
  double de_switch;            /* dual-energy eta; <= 0 disables the switch */
  int32_t flux_form;           /* 0 central-upwind (KNP), 1 central (KT) */
  const double *dx;            /* [n] cell width */
  const int32_t *neighbor;     /* [n][6][4] face neighbours, see workloads */
  const int8_t *neighbor_rel;  /* [n][6] level(neighbour) - level(self) */
  const int8_t *octant;        /* [n] position in the parent: bit0 x, bit1 y, bit2 z */
  int32_t reflux;              /* 1: coarse-fine flux correction (the default), 0: none */
  int32_t cw84;                /* PPM extensions of Colella & Woodward (1984): bit 0 shock flattening
                                  (Section 4), bit 1 contact steepening of the density (eqs. 1.14-1.17);
                                  0 (the default): neither */
} oracle_grid;

/* status codes */
#define ORACLE_OK 0
#define ORACLE_ERR_NONFINITE (-4)
#define ORACLE_ERR_INVALID (-1)

/* PPM on one pencil of 14 values: fills aL[m], aR[m] for m = 2..11. */
void oracle_ppm_pencil(const double *q, double *aL, double *aR);

/* Face EOS on one side: returns pressure p and sound speed c, velocity along d. */
void oracle_face_eos(const double *U, int d, double gamma, double eta, double *u, double *p, double *c);

/* Numerical flux F[11] through a face normal to d from the left/right states.
 * Returns the face signal speed max(a+, -a-). */
double oracle_face_flux(const double *UL, const double *UR, int d, double gamma, double eta, int form,
                        double *F);

/* One RK stage on the listed sub-grids (ids == NULL: all).  Writes only the
 * interior of Uout for those sub-grids:
 *   U* = Uin + (dt/dx) dU,   Uout = U0 + beta (U* - U0)   (Uout = U* if beta == 1)
 * i.e. the Shu-Osher convex blend alpha U0 + beta U* with alpha = 1 - beta.
 * U0 may be NULL when beta == 1.
 * max_speed[0] = max amax_s, max_speed[1] = max amax_s/dx_s over the listed
 * sub-grids; sub_amax (optional, [n]) receives amax_s.  nthreads <= 0 uses the
 * OpenMP default.  Returns ORACLE_ERR_NONFINITE if an output is not finite or
 * a density is not positive (outputs are still written).
 * batch_all: the coarse-fine flux correction counts every sub-grid as advanced
 * by this call (a batch that lists all of them, of which only `ids` are
 * computed here); 0: only the listed ones. */
int oracle_stage(const oracle_grid *g, const int32_t *ids, int32_t n_ids, const double *Uin, const double *U0,
                 double beta, double dt, double *Uout, double *max_speed, double *sub_amax, int nthreads,
                 int batch_all);

/* Margin cells of the error metric (interior cells near a branch decision of
 * the scheme, see the definition beside the function): OR-s one MARGIN_* bit
 * per kind of decision into mask[s][512] ((k*8 + j)*8 + i) for the listed
 * sub-grids (ids == NULL: all) of the padded state U (ghosts filled);
 * tol = 64 eps of the compared precision.  Returns the number of near
 * decisions found. */
#define MARGIN_SLOPE 1       /* the slope's extremum test */
#define MARGIN_EXTREMUM 2    /* the parabola's extremum test */
#define MARGIN_OVERSHOOT 4   /* the parabola's two overshoot tests */
#define MARGIN_DUAL_ENERGY 8 /* the dual-energy test at a face side */
#define MARGIN_CW84 16       /* a test of the CW84 flattening or steepening (when enabled) */
#define MARGIN_RECON3D 32    /* a transverse test of the 3D reconstruction (oracle_margin_cells3d) */
long oracle_margin_cells(const oracle_grid *g, const int32_t *ids, int32_t n_ids, const double *U, double tol,
                         unsigned char *mask);

/* Fill the six face ghost slabs of every sub-grid from the interiors. */
int oracle_fill_ghosts(const oracle_grid *g, double *U);

/* The ghost value of field f of sub-grid s across `face` (0..5 = -x,+x,-y,+y,
 * -z,+z) at interior coordinate ga along the face's axis (-1, -2, ... low side;
 * 8, 9, ... high side) and interior transverse coordinates (c1, c2), by the
 * ghost-fill rules, from the interiors of U; any depth (the CW84 flattening
 * reads the fourth layer). */
double oracle_ghost_cell(const oracle_grid *g, const double *U, int s, int face, int ga, int c1, int c2, int f);

/* Three-dimensional reconstruction with Simpson face quadrature (grids of one
 * level only; see the definition): fill every ghost cell of the padded cube,
 * faces, edges and corners (ORACLE_ERR_INVALID on a grid of several levels),
 * and one RK stage of every sub-grid, as oracle_stage with the face fluxes
 * of that reconstruction (no coarse-fine faces, no correction). */
int oracle_fill_ghosts_full(const oracle_grid *g, double *U);
/* The Simpson flux of one face from the face averages of the 3 x 3 faces
 * around it (AL, AR: [b2][b1][f], the left and right states); returns the
 * largest point signal speed. */
double oracle_simpson_flux(const double *AL, const double *AR, int d, double gamma, double eta, int form, double *F);
int oracle_stage3d(const oracle_grid *g, const double *Uin, const double *U0, double beta, double dt, double *Uout,
                   double *max_speed, int nthreads);
/* Margin cells of the 3D reconstruction (see the definition): U with every
 * ghost cell filled; mask [n][512] OR-ed with MARGIN_RECON3D and
 * MARGIN_DUAL_ENERGY; returns the number of marked faces, ORACLE_ERR_INVALID
 * on a grid of several levels. */
long oracle_margin_cells3d(const oracle_grid *g, const double *U, double tol, unsigned char *mask);

/* Grid totals T_f = sum_s dx_s^3 sum_cells U_f, Neumaier-compensated, fixed order. */
void oracle_totals(const oracle_grid *g, const double *U, double *totals);

/* Diagnostics (Section V-B.1 diagnostics task): out[12] = {M, Lx, Ly, Lz, M1,
 * X1, Y1, Z1, M2, X2, Y2, Z2}: total mass, angular momentum about the origin,
 * mass and centre of mass of star 1 (scalar field 6) and star 2 (field 7).
 * origin[n][3] is the lower corner of each sub-grid's interior. */
void oracle_diagnostics(const oracle_grid *g, const double *U, const double *origin, double *out);

/* Dual-energy resynchronisation of the entropy tracer: tau = e_i^(1/gamma) in
 * every interior cell where e_i = E - |s|^2 / 2 rho > 0 and e_i >= eta E
 * (eta = de_switch; nothing when eta <= 0).  Returns the number of cells reset. */
long oracle_tau_resync(const oracle_grid *g, double *U);

#ifdef __cplusplus
}
#endif
#endif
