// hydro_internal.cuh -- shared definitions of the CUDA library (not part of the ABI).
//
// Sub-grid layout (identical to the ABI): U[s][f][k][j][i], 14^3 padded cells
// per field, interior 3..10, 11 fields (rho, sx, sy, sz, egas, tau, rhoX1..5).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace hydro {

constexpr int NX = 8;            // interior cells per edge
constexpr int NG = 3;            // ghost layers
constexpr int NP = NX + 2 * NG;  // padded edge (14)
constexpr int NP2 = NP * NP;
constexpr int NP3 = NP * NP * NP;
constexpr int NF = 11;           // conserved fields
constexpr int NFACE = 9;         // faces per pencil that the update needs (2+1/2 .. 10+1/2)
constexpr int NPEN = NX * NX;    // pencils per direction
constexpr int FACES_DIR = NPEN * NFACE;  // 576
constexpr int CELLS = NX * NX * NX;      // 512
constexpr int F_RHO = 0, F_SX = 1, F_EGAS = 4, F_TAU = 5;

// A batch id with this bit set names a sub-grid whose coarse-fine boundary
// fluxes are exported (and, FP64, published) for the correction of its coarser
// neighbours, without updating it (the ABI's HYDRO_ITEM_FLUX_ONLY).
constexpr int ITEM_FLUX_ONLY = 0x40000000;

// device error word bits
constexpr int ERRBIT_NONFINITE = 1;
constexpr int ERRBIT_BAD_ID = 2;
constexpr int ERRBIT_TIMEOUT = 4;   // a bounded wait for a neighbour's exported fluxes gave up

__host__ __device__ inline size_t field_offset(int s, int f) { return ((size_t)s * NF + f) * NP3; }

struct StageArgs {
  // TMA descriptors of Uin and U0 viewed as [n*11][14][14][14] doubles with a
  // box of 10 x 8 x 8 x 11 (i = 2..11, j, k = 3..10, all fields of one
  // sub-grid); the kernel prefetches each sub-grid's box into L2 ahead of its
  // update.  Zero-filled when not used.
  CUtensorMap tm_in;  // 128-byte aligned by its type
  CUtensorMap tm_u0;
  const double* Uin;
  const double* U0;     // nullptr when beta == 1
  double* Uout;
  const float* Sin;     // mixed path: FP32 interior shadow of Uin, [n][11][512]
  float* Sout;          // mixed path: shadow of Uout to write (may be null)
  const int32_t* ids;
  int32_t n_items;
  int32_t n_sub;
  const double* dx;
  const double* inv_dx;  // [n] 1/dx
  const int32_t* nb;   // [n][6][4] face neighbours
  const int8_t* rel;   // [n][6]
  const int8_t* oct;   // [n]
  double beta;
  double dt;
  const double* dt_dev;  // when non-null, dt is read from device memory
  double gamma;
  double eta;
  int32_t form;          // 0 KNP, 1 KT
  unsigned int* queue;   // work-queue counter, zero at launch
  int* err;
  unsigned long long* max_speed;  // [2] ordered bits of non-negative doubles
  int32_t has_tm;        // bit 0: tm_in valid; bit 1: tm_u0 valid and read by the update
  // Mixed-precision RK3 in increment form (mode 1..3; 0 = the Shu-Osher stage
  // U_out = U0 + beta (U* - U0) above).  Stage k's increment L_k = lam * dU_k
  // is kept as a float pair (hi word, lo word of an 8-byte slot of the padded
  // layout); Uin is always the state U at the start of the step:
  //   mode 1: Dout = L0,                     Sout ~ shadow of U + L0;
  //   mode 2: Dout = (Din + L1) / 4,         Sout ~ shadow of U + Dout;
  //   mode 3: Uout = U + 2/3 (Din + L2) (FP64), Sout (optional) = its shadow.
  // Modes 1 and 2 take RN32(U) of their own cells from S0, the shadow of U
  // (in mode 1 that is Sin itself), and read no FP64 state.
  int32_t mode;
  const double* Din;     // increments as float pairs, packed interiors [s][f][512]
  double* Dout;
  const float* S0;
  // Coarse-fine flux correction (when fb is set).
  // Mixed precision: every sub-grid stamps fb_stamp[s] = call_id and stores
  // its fluxes on every coarse-fine face, fb[(s*6 + face)][f][pencil] (T),
  // pencil = t2*8 + t1 across the face; a separate pass (reflux_kernel)
  // corrects the coarse side after the stage.
  // FP64: the correction runs inside the stage.  A sub-grid
  // with a coarser face neighbour stores that face's fluxes,
  // fb[(s*6 + face)][f][pencil] (T), pencil = t2*8 + t1 across the face, and
  // after each direction d's faces raises cf_flag[s] to 3 call_id + d + 1
  // (release).  A sub-grid with finer face neighbours waits (acquire, bounded
  // by wait_limit clock cycles) until each fine neighbour advanced by this call
  // has exported direction d, then takes the mean of the four fine fluxes over
  // each coarse boundary face.  The queue lists finer sub-grids first, so a
  // wait is only ever for an item taken earlier by a running CTA.  member[s] ==
  // call_id marks the sub-grids of the call (member == nullptr: all of them).
  // A wait that gives up sets ERRBIT_TIMEOUT and *abort_word, after which
  // every CTA stops taking work.  (The queue order of a whole-grid stage is
  // by level, finest first: measured faster than a Morton order that moves
  // each sub-grid's finer neighbours just before it, whose waits are longer.)
  void* fb;
  int32_t* fb_stamp;     // mixed precision only
  int32_t* cf_flag;      // FP64 only (also member, abort_word, wait_limit)
  const int32_t* member;
  int* abort_word;
  long long wait_limit;
  int32_t call_id;
  int32_t flag_base;     // FP64: cf_flag values are flag_base + d + 1 (stage k of a one-launch RK3 step: 3k)
  int32_t cw84;          // CW84 PPM extensions: bit 0 shock flattening, bit 1 contact steepening (0: neither)
  int32_t pf_pass;       // the direction pass (0 x, 1 y, 2 z) that prefetches the update's rows into L2
};

// Coarse-fine flux correction after a mixed-precision stage (one CTA per
// coarse sub-grid of `list`): each coarse boundary face flux is replaced by the
// mean of the four fine fluxes over it, for the finer neighbours advanced by
// the same call.  One record per coarse sub-grid with at least one finer face
// neighbour: its id, then for each face and quadrant (face * 4 + q) the fine
// neighbour's id, -1 where the face does not meet finer sub-grids.
constexpr int CF_ENTRY = 25;

struct RefluxArgs {
  const int32_t* cf;     // [n_list][CF_ENTRY]
  int32_t n_list;
  const void* fb;        // stage flux export (see StageArgs)
  const int32_t* fb_stamp;
  int32_t call_id;
  const double* inv_dx;
  double dt;
  const double* dt_dev;
  int32_t mode;          // the stage's mode (StageArgs)
  double beta;           // mode 0
  double* U;             // mode 0 and 3: the stage's FP64 output
  double* D;             // modes 1, 2: the stage's increment output (packed interiors [s][f][512])
  const float* S0;       // modes 1, 2: shadow of the step's input state
  float* Sout;           // the stage's shadow output, refreshed where corrected (may be null)
  int* err;
  int32_t shape;         // launch shape (REFLUX_SHAPES): threads per CTA and items per thread
};

// Launch shapes of the correction pass: {threads per CTA, items per thread}.
constexpr int REFLUX_SHAPES = 4;

// One SSP-RK3 step (three stages over every sub-grid) in one persistent
// launch.  One work queue of 3 n tickets, stage-major (order 0) or
// stage-interleaved (order 1, which cannot finish once a CTA holds a later
// stage of an item whose neighbours' earlier stages are queued behind it: its
// bounded waits give up, which is what it exists to show).  The stage-k item
// of sub-grid s starts once s and every face neighbour whose interior its halo
// gather reads have completed stage k - 1 (done[x] >= k; release / acquire;
// a wait bounded by st[0].wait_limit cycles that sets ERRBIT_TIMEOUT and
// *st[0].abort_word when it gives up).  FP64 corrects the coarse-fine fluxes
// inside the stage (cf_flag, flag_base = 3k; the queue of each stage lists
// finer sub-grids first).  Mixed precision: the correction of a coarse
// sub-grid with finer face neighbours (row r of rf[k].cf) runs once its own
// stage-k item and those of its finer neighbours are done: each of them adds
// one to arrive[r], and the one that brings it to (k + 1) * cf_target[r]
// applies the correction and then marks the coarse sub-grid complete.
struct FusedArgs {
  StageArgs st[3];
  RefluxArgs rf[3];          // mixed: the correction of each stage (rf[k].cf: the coarse sub-grids)
  int32_t* done;             // [n] stages completed in this launch, zero at launch
  int32_t* arrive;           // [n_cf_list] arrivals, zero at launch
  const int32_t* cf_slot;    // [n] row of the sub-grid in rf[k].cf, -1 if it has no finer face neighbour
  const int32_t* cf_target;  // [n_cf_list] 1 + the number of finer face neighbours
  int32_t n;                 // items per stage (every sub-grid)
  int32_t order;
};

// Encode the TMA descriptor of a padded state (n sub-grids) used by
// StageArgs::tm_in / tm_u0; returns false if cuTensorMapEncodeTiled refuses it.
bool encode_state_map(CUtensorMap* tm, const double* U, int n);

struct GhostArgs {
  double* U;
  int32_t n_sub;
  const int32_t* nb;   // [n][6][4]
  const int8_t* rel;   // [n][6]
  const int8_t* oct;   // [n]
};

// FP32 shadow of a sub-grid field: the 8^3 interior [k][j][i], then its 4^3
// restriction [K][J][I] (FP32 mean of the 2x2x2 rounded cells, summed
// pairwise: in i, then j, then k), which a coarser neighbour reads as its halo.
constexpr int SHADOW_COARSE = CELLS;            // offset of the restriction
constexpr int SHADOW_FIELD = CELLS + CELLS / 8;  // 576 floats per field

// launchers (defined in the .cu files)
cudaError_t launch_shadow(const double* U, float* S, int n, cudaStream_t st);
// The shadows of the batch's sub-grids and of the face neighbours their halos
// read (one CTA per item; for batches small against the grid).
cudaError_t launch_shadow_ids(const double* U, float* S, const int32_t* ids, int n_items, int n, const int32_t* nb,
                              const int8_t* rel, cudaStream_t st);
// Dual-energy tracer reset of every sub-grid of U (and the tau field of its
// shadow S when mixed and S is not null); nothing when eta <= 0.
cudaError_t launch_tau_resync(double* U, float* S, int n, double gamma, double eta, bool mixed, cudaStream_t st);
cudaError_t launch_reflux_mixed(const RefluxArgs& r, cudaStream_t st);
// The work queue of a stage over a batch: the batch's ids ordered finest
// level first (level_rank[s], 0 = finest; ids outside [0, n) first), into
// `order`, and member[id] = call_id for every valid id.  One CTA.
cudaError_t launch_order_batch(const int32_t* ids, int n_items, int n_sub, const int8_t* level_rank, int n_levels,
                               int32_t* order, int32_t* member, int32_t call_id, cudaStream_t st);
cudaError_t launch_pack(const double* U, double* P, int n, cudaStream_t st);
cudaError_t launch_unpack(const double* P, double* U, int n, cudaStream_t st);
cudaError_t launch_stage_fp64(const StageArgs& a, int grid, cudaStream_t st);
cudaError_t launch_stage_mixed(const StageArgs& a, int grid, cudaStream_t st);
cudaError_t launch_rk3_fp64(const FusedArgs& f, int grid, cudaStream_t st);
cudaError_t launch_rk3_mixed(const FusedArgs& f, int grid, cudaStream_t st);
int stage_blocks_per_sm_fp64();
int stage_blocks_per_sm_mixed();
int rk3_blocks_per_sm_fp64();
int rk3_blocks_per_sm_mixed();
int cw_blocks_per_sm_fp64();
int cw_blocks_per_sm_mixed();
cudaError_t launch_ghost_fill(const GhostArgs& a, int threads, cudaStream_t st);
// scratch doubles needed by launch_totals for n sub-grids
size_t totals_scratch_doubles(int n);
// Diagnostics sums into sums[12] (device scratch) and the results into out[12].
cudaError_t launch_diagnostics(const double* U, const double* origin, int n, const double* dx, double* scratch,
                               double* sums, double* out, cudaStream_t st);
cudaError_t launch_totals(const double* U, int n, const double* dx, double* scratch, double* totals,
                          cudaStream_t st);

}  // namespace hydro
