/* hydro.h -- C ABI of the batched octree hydro step for GB300 (sm_103a).
 *
 * The library advances the inviscid Euler equations of an ideal gas on many
 * 8^3 sub-grids of an octree with a finite-volume central scheme: PPM
 * reconstruction of the conserved fields on the cell faces, a central-upwind
 * (Kurganov-Tadmor-type) flux with a maximum-signal-speed reduction, and the
 * flux-divergence update inside a Runge-Kutta sub-step.  This is the hydro
 * solver the paper profiles: Section IV-C names the equations (inviscid Euler,
 * solved by a finite-volume central scheme) and the octree of N^3 sub-grids
 * with N = 8; Section V-B.1 names the reconstruct (PPM) and flux CUDA kernels
 * and the compute_fluxes task, which drives one Runge-Kutta substep, reduces
 * the global time-step and updates the hydrodynamic variables, and the
 * diagnostics task that forms grid totals; Section VI covers the hydro
 * ghost-cell exchange.
 *
 * Data layout (all state arrays are caller-owned DEVICE memory, float64):
 *   U[s][f][k][j][i], s < n_subgrids, f < 11, k, j, i < 14 (x fastest);
 *   each sub-grid is an 8^3 interior (indices 3..10) padded by 3 ghost layers.
 *   Fields: 0 rho, 1 sx, 2 sy, 3 sz (momentum density), 4 egas (total energy
 *   density), 5 tau (entropy tracer, e_int = tau^gamma), 6..10 rho*X_k.
 *   Base pointers must be 16-byte aligned.
 *
 * Calls are stream-ordered and asynchronous.  Host-detectable errors (null
 * pointers, bad sizes or values) are returned at once and nothing is
 * launched.  Errors found on the device (a non-finite output or a density that
 * is not positive, a sub-grid id out of range) set a device error word that
 * the next hydro_sync() returns and clears.  No call aborts the process or
 * traps the GPU.
 */
#ifndef GB300_HYDRO_H
#define GB300_HYDRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HYDRO_OK = 0,
  HYDRO_ERR_INVALID = -1,   /* bad argument (host) or bad sub-grid id (device) */
  HYDRO_ERR_CUDA = -2,      /* a CUDA runtime call failed; see hydro_last_error */
  HYDRO_ERR_NOMEM = -3,     /* device or host allocation failed in hydro_create (or hydro_set_param) */
  HYDRO_ERR_NONFINITE = -4, /* an updated value is not finite, or a density <= 0 */
  HYDRO_ERR_TIMEOUT = -5,   /* a bounded device wait gave up (HYDRO_PARAM_WAIT_LIMIT) */
  HYDRO_ERR_STATE = -6      /* call not valid in the handle's current state */
} hydro_status;

typedef enum {
  HYDRO_FP64 = 0,  /* every step of the path in float64 */
  HYDRO_MIXED = 1  /* reconstruction and flux in float32; accumulation of the
                      conserved variables, the speed reduction and totals in
                      float64-accurate arithmetic */
} hydro_precision;

typedef enum {
  HYDRO_FLUX_KNP = 0, /* central-upwind, one-sided speeds a+ >= 0 >= a- */
  HYDRO_FLUX_KT = 1   /* central Kurganov-Tadmor, a+ = -a- = max |u| + c */
} hydro_flux_form;

/* Grid descriptor.  All arrays are HOST memory, read and copied to the device
 * by hydro_create (the caller may free them afterwards).
 *   neighbor[s][face][q], faces ordered -x,+x,-y,+y,-z,+z:
 *     neighbor_rel == 0 : q = 0 is the same-level neighbour (periodic wrap is
 *                         expressed here), or -1 for a domain boundary, which
 *                         is filled as outflow (copy of the nearest interior
 *                         cell);
 *     neighbor_rel == -1: q = 0 is the one-level-coarser neighbour; octant[s]
 *                         gives this sub-grid's position in its parent (bit0 x,
 *                         bit1 y, bit2 z);
 *     neighbor_rel == +1: q = t1 + 2*t2 are the four one-level-finer
 *                         neighbours across the face, t1/t2 their offsets
 *                         along the first/second transverse axis (x-face: y,z;
 *                         y-face: x,z; z-face: x,y).
 * The octree must be 2:1 balanced across faces. */
typedef struct {
  int32_t n_subgrids;          /* >= 1 */
  int32_t n_fields;            /* must be 11 */
  int32_t nx;                  /* interior cells per edge, must be 8 */
  int32_t ghost;               /* ghost layers, must be 3 */
  double gamma;                /* adiabatic index, > 1 (5/3 in the workloads) */
  double de_switch;            /* dual-energy switch eta in [0, 1); 0 disables */
  int32_t precision;           /* hydro_precision */
  int32_t flux_form;           /* hydro_flux_form */
  const double *dx;            /* [n_subgrids] cell width, > 0 */
  const int32_t *neighbor;     /* [n_subgrids][6][4] */
  const int8_t *neighbor_rel;  /* [n_subgrids][6], values -1, 0, +1 */
  const int8_t *octant;        /* [n_subgrids], 0..7 */
} hydro_grid_desc;

/* A list of sub-grids to advance, cut into batches (the uneven leaf batches of
 * the octree).  All batches of one call are processed by one persistent
 * launch that pulls sub-grids from a device work queue. */
typedef struct {
  const int32_t *subgrid_ids;   /* DEVICE [n_items], ids in [0, n_subgrids), unique; an id
                                   or-ed with HYDRO_ITEM_FLUX_ONLY is not advanced: its
                                   coarse-fine boundary fluxes are only computed and
                                   exported for the correction of its coarser neighbours
                                   in the same call (a proxy of a sub-grid that another
                                   grid partition advances) */
  int32_t n_items;              /* >= 0 */
  const int32_t *batch_offsets; /* HOST [n_batches + 1], non-decreasing, 0 .. n_items;
                                   may be NULL (one batch) */
  int32_t n_batches;            /* >= 0 */
} hydro_batch;

/* Batch id flag: export the sub-grid's coarse-fine boundary fluxes, do not
 * advance it (see hydro_batch.subgrid_ids). */
#define HYDRO_ITEM_FLUX_ONLY 0x40000000

typedef struct hydro_handle hydro_handle;

/* Create a handle for one grid on the current CUDA device: validates and
 * copies the descriptor, allocates the handle's device scratch (work-queue
 * counter, error word, reduction partials).  Returns HYDRO_OK and *out, or an
 * error with *out = NULL. */
int hydro_create(const hydro_grid_desc *desc, hydro_handle **out);

/* One Runge-Kutta stage on the batch (Section V-B.1: reconstruct, flux,
 * global speed reduction, update), for each listed sub-grid s:
 *   U* = U_in + (dt/dx_s) * dU,
 *   dU = ((Fx(i-1/2) - Fx(i+1/2)) + (Fy(j-1/2) - Fy(j+1/2))) + (Fz(k-1/2) - Fz(k+1/2)),
 *   U_out = U0 + beta * (U* - U0)      (U_out = U* when beta == 1),
 * which is the Shu-Osher blend (1 - beta) U0 + beta U*.  SSP-RK3 uses
 * beta = 1, 1/4, 2/3 with U0 the state at the start of the step.
 *   U_in   DEVICE padded state; only interior cells are read: each face
 *          halo is gathered from the neighbours' interiors by the rules of
 *          hydro_fill_ghosts, so the ghost cells of U_in need not be filled;
 *   U0     DEVICE padded state, read at interior cells; may be NULL iff beta == 1;
 *   U_out  DEVICE padded state; only the interiors of the listed sub-grids are
 *          written; must not alias U_in; may alias U0;
 *   dt     >= 0 and finite; beta in (0, 1];
 *   d_max_speed  DEVICE double[2], overwritten with the maximum over the
 *          listed sub-grids and their faces of max(a+, -a-) (the CFL signal
 *          speed of the INPUT state) and of that speed divided by dx_s;
 *   stream cudaStream_t (NULL = legacy default stream).
 * A mixed-precision handle first writes the FP32 shadow of U_in into its own
 * buffer: of the listed sub-grids and the face neighbours their halos read
 * when the batch lists fewer than an eighth of the sub-grids, else of all of
 * them (hydro_shadow); hydro_step_shadowed skips that pass when the caller
 * already holds the shadow.
 * Coarse-fine flux correction (Section V-B.1: compute_fluxes corrects the
 * fluxes on coarse-fine boundaries; HYDRO_PARAM_REFLUX, on by default): where
 * a listed sub-grid meets four finer neighbours, each coarse boundary face
 * takes the flux ((F00 + F10) + (F01 + F11)) / 4 of the fine faces over it, as
 * the fine neighbours computed them in the same call, so an AMR step conserves
 * to round-off; a quadrant whose fine neighbour is not listed keeps the coarse
 * flux.  FP64 handles correct inside the stage kernel, before the flux
 * differences, as the plain statement does: the stage takes the listed
 * sub-grids finest level first (a one-CTA pass orders the batch), each fine
 * sub-grid publishes its boundary fluxes with a flag, and a coarse one waits
 * for them (bounded by HYDRO_PARAM_WAIT_LIMIT; HYDRO_ERR_TIMEOUT from
 * hydro_sync when a wait runs out).  With every operation rounded as written
 * (no contraction, IEEE quotients), an FP64 stage equals a plain FP64
 * evaluation of the scheme bit for bit, except at faces where the dual-energy
 * switch evaluates tau^gamma (pow, correctly rounded by no math library).
 * Mixed-precision handles correct in a second launch after the stage kernel,
 * adding the exact float-pair difference (mean - own flux) to what the stage
 * wrote. */
int hydro_step(hydro_handle *h, const hydro_batch *batch, const double *U_in, const double *U0, double beta,
               double dt, double *U_out, double *d_max_speed, void *stream);

/* FP32 shadow of the interiors of every sub-grid of U, the input the
 * mixed-precision reconstruction reads (the paper has no counterpart; it is
 * the GB300 layout of the float32 reconstruction inputs).  Per sub-grid s and
 * field f, 576 floats:
 *   S[s][f][(k*8 + j)*8 + i] = r(U[s][f][k+3][j+3][i+3]), k, j, i < 8, with r
 *     the rounding to the nearest float32 (ties away from zero; magnitudes
 *     below the float32 normal range become signed zero, finite values beyond
 *     it infinity);
 *   S[s][f][512 + (K*4 + J)*4 + I] = the float32 sum of the eight rounded cells
 *     c(dk,dj,di) = (2K+dk, 2J+dj, 2I+di), added pairwise as
 *     ((c000 + c001) + (c010 + c011)) + ((c100 + c101) + (c110 + c111)),
 *     times 1/8: the restriction a coarser neighbour reads as its halo.
 *   U DEVICE padded state; S DEVICE float[n_subgrids][11][576], 16-byte
 *   aligned.  Works with either precision of handle. */
int hydro_shadow(hydro_handle *h, const double *U, float *S, void *stream);

/* hydro_step for a mixed-precision handle whose caller keeps the shadows:
 *   S_in   DEVICE shadow of U_in (as hydro_shadow writes it) for every
 *          sub-grid; the reconstruction reads it in place of U_in's interiors
 *          (finer neighbours' 2x2x2 means are still formed from U_in);
 *   S_out  DEVICE shadow buffer or NULL; when given, the shadow of U_out is
 *          written for the listed sub-grids; must not alias S_in.
 * Other arguments as hydro_step.  A FP64 handle returns HYDRO_ERR_STATE. */
int hydro_step_shadowed(hydro_handle *h, const hydro_batch *batch, const double *U_in, const float *S_in,
                        const double *U0, double beta, double dt, double *U_out, float *S_out, double *d_max_speed,
                        void *stream);

/* Packed interiors, for moving states between host and device without their
 * ghost cells (5.36x fewer bytes than the padded layout; the paper has no
 * counterpart):
 *   P[s][f][(k*8 + j)*8 + i] = U[s][f][k+3][j+3][i+3],  P DEVICE double[n][11][512].
 * hydro_pack_interiors writes P from U; hydro_unpack_interiors writes the
 * interiors of U from P and leaves its ghost cells untouched.  Both pointers
 * 16-byte aligned. */
int hydro_pack_interiors(hydro_handle *h, const double *U, double *P, void *stream);
int hydro_unpack_interiors(hydro_handle *h, const double *P, double *U, void *stream);

/* The same for the sub-grids first .. first + count - 1 only (U and P are the
 * whole arrays), so that the packing of one slice can overlap the host copies
 * of others.  0 <= first, 0 <= count, first + count <= n_subgrids, else
 * HYDRO_ERR_INVALID; count == 0 launches nothing. */
int hydro_pack_interiors_range(hydro_handle *h, const double *U, double *P, int32_t first, int32_t count,
                               void *stream);
int hydro_unpack_interiors_range(hydro_handle *h, const double *P, double *U, int32_t first, int32_t count,
                                 void *stream);

/* Fill the six face ghost slabs (3 layers each) of every sub-grid of U from
 * the neighbours' interiors (Section VI: hydro boundary exchange): copy from a
 * same-level neighbour; coarse neighbour: value of the coarse cell containing
 * the ghost-cell centre; fine neighbours: mean of the 2x2x2 fine cells, summed
 * in (k, j, i) order and scaled by 1/8; domain boundary: copy of the nearest
 * interior cell.  Edge and corner ghost cells are left untouched. */
int hydro_fill_ghosts(hydro_handle *h, double *U, void *stream);

/* One SSP-RK3 step (three stages, Section I: three hydro iterations per
 * time-step), replayed from a CUDA graph that the handle captures on first use
 * for each (batch, U, scratch) combination.  The stages gather their halos
 * from the neighbours' interiors, so no ghost fill runs between stages.  The
 * batch must list every sub-grid once (n_items == n_subgrids, any order and
 * batch cut), since later stages read the neighbours' intermediate states;
 * otherwise HYDRO_ERR_INVALID.  FP64: the Shu-Osher stages of hydro_step
 * (beta = 1, 1/4, 2/3), scratch1 and scratch2 holding U1 and U2.  Mixed
 * precision evaluates the same step in increment form, with L_k = dt/dx *
 * dU(U_k): U1 = U + L0, U2 = U + (L0 + L1)/4, U_new = U + 2/3 ((L0 + L1)/4 + L2);
 * the increments are kept as float pairs (about 48 bits) in scratch1 and
 * scratch2, and U is changed once, by two FP64 additions per value.  The
 * graph writes the FP32 shadow of U once; each stage writes the shadow of its
 * state for the next (stages 1 and 2 as RN32(RN32(U) + increment), within one
 * float32 ulp of the rounded state).
 * HYDRO_PARAM_FUSED_RK3 runs the three stages as ONE persistent kernel launch
 * (Section VI: neighbours' data read in place, no exchange step between
 * stages): one work queue of the three stages' items, in stage order; the
 * stage-k item of a sub-grid starts once the sub-grid and the face neighbours
 * its halo reads have completed stage k - 1 (per-sub-grid completion counters,
 * release/acquire), and in mixed precision the coarse-fine correction of a
 * coarse sub-grid runs inside the launch as soon as it and its finer
 * neighbours are done, applied by the CTA that completes the last of them.
 * The results are bit-identical to the three-launch form.  Every wait is
 * bounded by HYDRO_PARAM_WAIT_LIMIT; one that runs out makes the launch stop
 * taking work and hydro_sync return HYDRO_ERR_TIMEOUT (the state is then
 * undefined).  The one-launch form needs mutual neighbour tables (every
 * sub-grid whose halo reads s is read by s, as on an octree); handles whose
 * tables are not mutual use the three-launch form.
 *   U        DEVICE padded state; its interior is overwritten by the new state
 *            (ghost cells are neither read nor updated: call hydro_fill_ghosts
 *            when they are wanted);
 *   scratch1, scratch2  DEVICE arrays of the size of a padded state
 *            (contents destroyed);
 *   d_max_speed DEVICE double[2]: the max speeds of the first stage, i.e. of
 *            the state at the start of the step. */
int hydro_rk3_step(hydro_handle *h, const hydro_batch *batch, double *U, double *scratch1, double *scratch2,
                   double dt, double *d_max_speed, void *stream);

/* As hydro_rk3_step, with the time step chosen on the device from the CFL
 * condition (the paper's global time-step reduction, Section V-B.1):
 *   dt = cfl / d_max_speed[1]
 * where d_max_speed holds, on entry, the speeds of the previous step's first
 * stage (or of a dry hydro_step with dt = 0 before the first step); on exit it
 * holds this step's first-stage speeds, so successive calls chain without a
 * host round trip.  If d_dt_out is not NULL the dt used is written there
 * (DEVICE double).  cfl in (0, 1]. */
int hydro_rk3_step_cfl(hydro_handle *h, const hydro_batch *batch, double *U, double *scratch1, double *scratch2,
                       double cfl, double *d_max_speed, double *d_dt_out, void *stream);

/* n_steps successive SSP-RK3 steps in one call, each exactly as
 * hydro_rk3_step_cfl followed by hydro_totals, replayed from one CUDA graph:
 * step k takes dt = cfl / d_max_speed[1] from the speeds left by step k-1 (or
 * by the caller on entry), writes it to d_dt_out[k] if d_dt_out is not NULL,
 * and writes the totals of its new state to d_totals[11*k .. 11*k+10] if
 * d_totals is not NULL (DEVICE double[n_steps][11]).  The results are
 * bit-identical to n_steps separate calls; a mixed-precision handle writes
 * the FP32 shadow of U once per call instead of once per step (the last
 * stage of each step writes the next step's shadow).
 *   n_steps in [1, HYDRO_RK3_RUN_MAX_STEPS]; other arguments as
 *   hydro_rk3_step_cfl.  One graph is kept per (batch, buffers, n_steps,
 *   cfl, output pointers) combination. */
#define HYDRO_RK3_RUN_MAX_STEPS 1024
int hydro_rk3_run_cfl(hydro_handle *h, const hydro_batch *batch, double *U, double *scratch1, double *scratch2,
                      double cfl, int32_t n_steps, double *d_max_speed, double *d_dt_out, double *d_totals,
                      void *stream);

/* Capture (and cache) the graph hydro_rk3_run_cfl would replay for these
 * arguments without launching anything, so that a later call starts at once.
 * Same validation and return codes as hydro_rk3_run_cfl. */
int hydro_rk3_run_prepare(hydro_handle *h, const hydro_batch *batch, double *U, double *scratch1, double *scratch2,
                          double cfl, int32_t n_steps, double *d_max_speed, double *d_dt_out, double *d_totals);

/* Grid totals (diagnostics): d_totals[f] = sum_s dx_s^3 * sum_interior U_f,
 * compensated and in a fixed order, so the result is deterministic.
 *   U DEVICE padded state; d_totals DEVICE double[11]. */
int hydro_totals(hydro_handle *h, const double *U, double *d_totals, void *stream);

/* Diagnostics (Section V-B.1, the diagnostics task: total mass, total angular
 * momentum and the centre of mass of each star of a binary), deterministic
 * like hydro_totals:
 *   d_out[0]     M  = sum dx^3 rho
 *   d_out[1..3]  L  = sum dx^3 (r x s), about the coordinate origin
 *   d_out[4]     M1 = sum dx^3 rho X1   (star 1: scalar field 6)
 *   d_out[5..7]  R1 = sum dx^3 rho X1 r / M1   (0 when M1 == 0)
 *   d_out[8..11] M2, R2 likewise for star 2 (scalar field 7)
 * with r the cell centre, each coordinate rounded as o + ((c + 1/2) * dx), and
 * each product of r x s and rho X r rounded on its own.
 *   U DEVICE padded state; d_origin DEVICE double[n_subgrids][3], the lower
 *   corner of each sub-grid's interior; d_out DEVICE double[12]. */
int hydro_diagnostics(hydro_handle *h, const double *U, const double *d_origin, double *d_out, void *stream);

/* Dual-energy reset of the entropy tracer (the paper is silent on the EOS;
 * this completes the dual-energy switch of the face EOS).  In every interior cell where the internal
 * energy e_i = E - (sx^2 + sy^2 + sz^2) / (2 rho) is positive and at least
 * eta E (eta = the handle's de_switch; the complement of the face EOS test
 * that takes e_i = tau^gamma), set tau = e_i^(1/gamma); every other cell and
 * field is unchanged, and nothing happens when de_switch <= 0.  e_k and e_i
 * are formed in FP64 on both handles; the power is FP64 on an FP64 handle and
 * FP32 (powf, about 1 ulp) on a mixed one.
 *   U  DEVICE padded state (interior tau overwritten in place; 16-byte aligned);
 *   S  optional DEVICE FP32 shadow of U (layout of hydro_shadow, mixed handles
 *      only, else HYDRO_ERR_INVALID): its tau field and tau restriction are
 *      rewritten from the new state, as hydro_shadow would write them.
 * With HYDRO_PARAM_TAU_RESYNC set, the RK3 entry points apply the same reset
 * at the end of every step (before the totals of hydro_rk3_run_cfl).
 * Returns HYDRO_OK, HYDRO_ERR_INVALID or HYDRO_ERR_CUDA. */
int hydro_tau_resync(hydro_handle *h, double *U, float *S, void *stream);

/* Allocation-free variant of hydro_totals for callers that cannot allocate
 * device memory (no cudaMalloc available to them: an allocator callback, a
 * framework that owns all device memory, a process with its memory reserved up
 * front).  The paper has no counterpart of this entry point.
 *   U         DEVICE padded state of n_subgrids sub-grids (16-byte aligned);
 *   d_dx      DEVICE double[n_subgrids], the cell width of each sub-grid;
 *   d_totals  DEVICE double[11], receives the same totals as hydro_totals;
 *   n_subgrids in [1, HYDRO_TOTALS_NOALLOC_MAX_SUBGRIDS]; a larger value is
 *             rejected with HYDRO_ERR_INVALID before anything is launched.
 * Needs no handle and allocates nothing: the partial sums live in one fixed
 * device array inside the library (HYDRO_TOTALS_NOALLOC_MAX_SUBGRIDS * 11 * 3
 * words of 8 bytes, 17.3 MB, held on every GPU that loads the library until
 * the process exits).  Each call looks up that array's device address on the
 * current device; a call made while its stream is being captured reuses the
 * address found by the last uncaptured call on that device instead, so make
 * one call on each device before capturing it.  A device reset (or any other
 * unload of the module) moves the array: the next uncaptured call finds the
 * new address, while a graph captured before the reset keeps the old one and
 * must be captured again.
 * All calls share the array: calls whose work overlaps on the GPU (different
 * streams, or the same stream from several threads without ordering) race and
 * must not be issued.  Returns HYDRO_OK, HYDRO_ERR_INVALID or HYDRO_ERR_CUDA. */
#define HYDRO_TOTALS_NOALLOC_MAX_SUBGRIDS 65536
int hydro_totals_noalloc(const double *U, const double *d_dx, int32_t n_subgrids, double *d_totals, void *stream);

/* Wait for the handle's work on the stream of its last call, then return and
 * clear the device error word: HYDRO_OK, HYDRO_ERR_NONFINITE or
 * HYDRO_ERR_INVALID (bad sub-grid id), or HYDRO_ERR_CUDA. */
int hydro_sync(hydro_handle *h);

/* Text of the last error on this handle (static storage of the handle). */
const char *hydro_last_error(const hydro_handle *h);

/* Number of kernel launches issued by this handle so far (instrumentation). */
int64_t hydro_launch_count(const hydro_handle *h);

/* Set a tuning parameter (see hydro_param); returns HYDRO_ERR_INVALID for an
 * unknown key or value out of range. */
int hydro_set_param(hydro_handle *h, int32_t key, int32_t value);

typedef enum {
  HYDRO_PARAM_STAGE_CTAS_PER_SM = 0, /* persistent CTAs per SM for the stage kernel, 1..8 (0 = auto) */
  HYDRO_PARAM_GHOST_THREADS = 1,     /* threads per CTA of the ghost-fill kernel, 64..1024 */
  HYDRO_PARAM_REFLUX = 2,            /* coarse-fine flux correction: 1 (default) or 0 */
  HYDRO_PARAM_TAU_RESYNC = 3,        /* dual-energy tracer reset after every RK3 step: 0 (default) or 1 */
  HYDRO_PARAM_WAIT_LIMIT = 4,        /* clock cycles a stage CTA waits for a finer neighbour's fluxes, >= 1
                                        (default 2^31 - 1, about a second); a wait that runs out makes the
                                        stage stop taking work and hydro_sync return HYDRO_ERR_TIMEOUT */
  HYDRO_PARAM_QUEUE_ORDER = 5,       /* 0 (default): stages take finer levels first; 1: the batch's own order
                                        (waits may then be for sub-grids not yet taken) */
  HYDRO_PARAM_STAGE_GRID = 6,        /* stage kernel CTAs in total, >= 1 (0 = the default from the occupancy) */
  HYDRO_PARAM_PREFETCH_PASS = 7,     /* direction pass (0 x, 1 y (default), 2 z) in which a stage pulls the rows
                                        its update reads into L2: the prefetch distance */
  HYDRO_PARAM_REFLUX_SHAPE = 8,      /* launch shape of the mixed correction pass: 0 (default) 256 threads x 3
                                        items, 1: 128 x 3, 2: 256 x 2, 3: 512 x 3 */
  HYDRO_PARAM_FUSED_RK3 = 9,         /* RK3 steps: 0 (default) three stage launches (and, mixed, three
                                        correction passes); 1 one persistent launch per step; 2 one launch whose queue
                                        interleaves the stages of each sub-grid, which cannot complete while a
                                        CTA holds a later stage whose inputs are queued behind it: its bounded
                                        waits give up (HYDRO_ERR_TIMEOUT), which is all it is for */
  HYDRO_PARAM_CW84 = 10,             /* PPM extensions of Colella & Woodward (1984), both 0 by default: bit 0
                                        shock flattening (their Section 4; reads the pressure one cell beyond
                                        the three ghost layers, from the neighbours' interiors), bit 1 contact
                                        steepening (their eqs. 1.14-1.17, detected on the density); both
                                        coefficients apply to every conserved field.  Stages and RK3 steps
                                        then use a stage kernel built with them (RK3 steps in three launches) */
  HYDRO_PARAM_RECON3D = 11           /* face fluxes: 0 (default) the face-centre flux of the states that PPM
                                        along the face normal gives; 1 the three-dimensional reconstruction
                                        with Simpson face quadrature (Section IV-C names a full 3D
                                        reconstruction, Section V-B.1 a Newton-Cotes rule over each face):
                                        the left and right face averages of the 3 x 3 faces around a face
                                        determine, per field, the tensor product of the parabolas with those
                                        three-cell averages across the face (first along the face's first
                                        transverse axis, then its second), limited to stay monotone (constant
                                        at a local extremum of the three averages; the monotonized-central
                                        line where an edge value leaves the neighbouring averages' range or
                                        the centre value the edge values' range); its values at the 3 x 3
                                        Simpson points (offsets -1/2, 0, +1/2 of the face width) give nine
                                        central-upwind fluxes, combined with the weights (1, 4, 1)/6 along
                                        each transverse axis (outer points added first).  Grids of one
                                        level (one cell width, no coarse-fine faces) only, without CW84
                                        extensions, else HYDRO_ERR_INVALID; enabling it allocates 627 kB of
                                        device scratch per sub-grid (HYDRO_ERR_NOMEM when that fails).
                                        Stages (at most n_subgrids items) and RK3 steps (three launches,
                                        Shu-Osher stages in both precisions, scratch1/scratch2 holding U1
                                        and U2) then run three kernels per stage: face averages (halos read
                                        from face, edge and corner neighbours of the FP64 state), Simpson
                                        fluxes, update.  FP64 handles: results equal a plain FP64
                                        evaluation bit for bit, with the same exception as hydro_step
                                        (tau^gamma).  Mixed handles: the state rounded to FP32 as for the
                                        shadows, reconstruction, transverse parabolas, point fluxes and
                                        Simpson sums in FP32, flux differences and update in FP64;
                                        hydro_step_shadowed returns HYDRO_ERR_STATE */
} hydro_param;

/* Release the handle and its device scratch (waits for its work first). */
void hydro_destroy(hydro_handle *h);

#ifdef __cplusplus
}
#endif
#endif
