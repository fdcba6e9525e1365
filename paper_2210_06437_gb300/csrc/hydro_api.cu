// hydro_api.cu -- the C ABI declared in include/hydro.h.
//
// Host side: validates every argument before anything is launched, owns the
// device copy of the grid descriptor and the handle's scratch (work-queue
// counters, error word, totals partials, per-stage speed scratch), sizes the
// persistent stage launch from the occupancy of the kernel, and replays a full
// SSP-RK3 step from a CUDA graph captured once per (batch, buffers) set.
// Mixed-precision handles also own two FP32 shadows of the interiors, which
// the RK3 graph passes from stage to stage (each stage reads its input's shadow
// and writes its output's).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "hydro.h"
#include "hydro_internal.cuh"
#include "hydro_recon3d.cuh"

using namespace hydro;

namespace {

// What a captured RK3 graph depends on: the batch ids and buffers it was
// captured with, and, for a multi-step run, the step count and the per-step
// outputs (0 steps: the single-step graph, whose dt is set before each launch).
struct GraphKey {
  const int32_t* ids;
  int32_t n_items;
  double* U;
  double* s1;
  double* s2;
  double* dms;
  int32_t n_steps;
  double cfl;
  double* dt_out;
  double* totals;
  bool operator==(const GraphKey& o) const {
    return ids == o.ids && n_items == o.n_items && U == o.U && s1 == o.s1 && s2 == o.s2 && dms == o.dms &&
           n_steps == o.n_steps && cfl == o.cfl && dt_out == o.dt_out && totals == o.totals;
  }
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
  int kernels;
};

}  // namespace

struct hydro_handle {
  int n = 0;
  int precision = 0;
  int form = 0;
  double gamma = 5.0 / 3.0;
  double eta = 1e-3;
  int device = 0;
  int sm_count = 0;
  int ctas_per_sm = 0;
  int occupancy = 1;  // resident stage CTAs per SM for this precision
  int ghost_threads = 256;
  double* d_dx = nullptr;
  double* d_inv_dx = nullptr;
  int32_t* d_nb = nullptr;
  int8_t* d_rel = nullptr;
  int8_t* d_oct = nullptr;
  unsigned int* d_queue = nullptr;     // [4] work-queue counters
  int* d_err = nullptr;                // device error word
  double* d_partial = nullptr;         // totals scratch (per-sub-grid and per-chunk partials)
  double* d_dt = nullptr;              // [1] time step read by graph replays
  double* d_diag = nullptr;            // [12] diagnostics sums
  unsigned long long* d_ms_tmp = nullptr;  // [2] speeds of RK stages 2 and 3
  float* d_shadow[3] = {nullptr, nullptr, nullptr};  // mixed precision: FP32 shadows [n][NF][576]
  // coarse-fine flux correction: FP64 inside the stage kernel, mixed precision
  // in a pass after it
  int tau_resync = 0;                  // dual-energy tracer reset after every RK3 step
  int reflux = 1;
  int n_cf = 0;                        // faces onto a finer neighbour
  int n_cf_list = 0;                   // mixed: coarse sub-grids with a finer face neighbour
  int32_t* d_cf = nullptr;             // mixed: [n_cf_list][CF_ENTRY] correction records
  int32_t* d_fb_stamp = nullptr;       // mixed: [n] call id of the last stage that advanced the sub-grid
  int n_levels = 1;                    // distinct cell widths
  int queue_order = 0;                 // 0: finest level first; 1: the batch's own order
  int grid_cap = 0;                    // stage CTAs (0: from the occupancy)
  int pf_pass = 1;                     // direction pass that prefetches the update's rows
  int reflux_shape = 0;                // launch shape of the mixed correction pass
  long long wait_limit = 0x7fffffffll;  // clock cycles a CTA waits for a neighbour's fluxes
  int8_t* d_level = nullptr;           // [n] level rank, 0 = finest
  int32_t* d_order_all = nullptr;      // [n] every sub-grid, finest level first
  int32_t* d_order = nullptr;          // [n] the current batch, finest level first
  int32_t* d_member = nullptr;         // [n] call id of the last batch listing the sub-grid
  void* d_fb = nullptr;                // [n][6][NF][64] exported boundary fluxes (T)
  int32_t* d_cf_flag = nullptr;        // [n] export progress of the current stage
  int* d_abort = nullptr;              // a bounded wait gave up during the current stage
  // one-launch RK3 step
  int fused = 0;                       // 0: three stage launches (and correction passes); 1: one launch; 2: the
                                       // stage-interleaved queue (its waits give up: for tests of the bound)
  int fused_ok = 0;                    // the neighbour tables are mutual (the one-launch step relies on it)
  int occupancy_fused = 1;             // resident CTAs per SM of the one-launch kernel
  int occupancy_cw = 1;                // resident CTAs per SM of the stage kernel with the CW84 extensions
  int cw84 = 0;                        // CW84 PPM extensions: bit 0 flattening, bit 1 contact steepening
  int single_level = 0;                // one cell width and no coarse-fine faces
  int recon3d = 0;                     // stages by the 3D reconstruction with Simpson face quadrature
  double* d_r3_fa = nullptr;           // its scratch: face averages and face fluxes of n items
  double* d_r3_fl = nullptr;
  int32_t* d_done = nullptr;           // [n] stages completed in the current launch
  int32_t* d_arrive = nullptr;         // mixed: [n_cf_list] arrivals at each coarse sub-grid
  int32_t* d_cf_slot = nullptr;        // mixed: [n] row in d_cf, -1 if none
  int32_t* d_cf_target = nullptr;      // mixed: [n_cf_list] 1 + finer face neighbours
  int32_t call_counter = 0;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  int64_t launches = 0;
  std::vector<GraphEntry> graphs;
  char msg[512] = {0};
};

namespace {

int fail(hydro_handle* h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_fail(hydro_handle* h, cudaError_t e, const char* what) {
  return fail(h, HYDRO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(h, expr)                                   \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr);  \
  } while (0)

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

void free_all(hydro_handle* h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  cudaFree(h->d_dx);
  cudaFree(h->d_inv_dx);
  cudaFree(h->d_nb);
  cudaFree(h->d_rel);
  cudaFree(h->d_oct);
  cudaFree(h->d_queue);
  cudaFree(h->d_err);
  cudaFree(h->d_partial);
  cudaFree(h->d_dt);
  cudaFree(h->d_diag);
  cudaFree(h->d_ms_tmp);
  for (float* p : h->d_shadow) cudaFree(p);
  cudaFree(h->d_cf);
  cudaFree(h->d_fb_stamp);
  cudaFree(h->d_level);
  cudaFree(h->d_order_all);
  cudaFree(h->d_order);
  cudaFree(h->d_member);
  cudaFree(h->d_fb);
  cudaFree(h->d_cf_flag);
  cudaFree(h->d_abort);
  cudaFree(h->d_done);
  cudaFree(h->d_arrive);
  cudaFree(h->d_cf_slot);
  cudaFree(h->d_cf_target);
  cudaFree(h->d_r3_fa);
  cudaFree(h->d_r3_fl);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
}

__global__ void set_scalar(double* p, double v) { *p = v; }

// dt = cfl / max(a/dx) of the previous first stage; a zero or non-finite speed
// gives dt = 0 (no motion) rather than an infinite step.
__global__ void cfl_dt(double* dt, const double* max_speed, double cfl, double* dt_out) {
  const double m = max_speed[1];
  const double v = (m > 0.0 && m <= 1.7976931348623157e308) ? cfl / m : 0.0;
  *dt = v;
  if (dt_out) *dt_out = v;
}

int check_batch(hydro_handle* h, const hydro_batch* b) {
  if (!b) return fail(h, HYDRO_ERR_INVALID, "batch is NULL");
  if (b->n_items < 0) return fail(h, HYDRO_ERR_INVALID, "batch n_items < 0");
  if (b->n_items > 0 && !b->subgrid_ids) return fail(h, HYDRO_ERR_INVALID, "batch subgrid_ids is NULL");
  if (b->batch_offsets) {
    if (b->n_batches < 1) return fail(h, HYDRO_ERR_INVALID, "batch_offsets given with n_batches < 1");
    if (b->batch_offsets[0] != 0 || b->batch_offsets[b->n_batches] != b->n_items)
      return fail(h, HYDRO_ERR_INVALID, "batch_offsets must run from 0 to n_items");
    for (int i = 0; i < b->n_batches; ++i)
      if (b->batch_offsets[i + 1] < b->batch_offsets[i])
        return fail(h, HYDRO_ERR_INVALID, "batch_offsets decrease at %d", i);
  } else if (b->n_batches < 0) {
    return fail(h, HYDRO_ERR_INVALID, "n_batches < 0");
  }
  return HYDRO_OK;
}

int stage_grid(hydro_handle* h, int n_items) {
  const int occ = h->cw84 ? h->occupancy_cw : h->occupancy;
  int per_sm = h->ctas_per_sm > 0 ? std::min(h->ctas_per_sm, occ) : occ;
  int grid = h->grid_cap > 0 ? h->grid_cap : h->sm_count * per_sm;
  return n_items < grid ? (n_items > 0 ? n_items : 1) : grid;
}

// Enqueue one stage (no validation).  queue_slot selects the counter.
// mode 0: Shu-Osher stage; 1..3: mixed RK3 in increment form (Din / Dout the
// increment pairs, see StageArgs)
// The arguments of one stage that do not depend on how it is launched.
void fill_stage(hydro_handle* h, StageArgs& a, const int32_t* ids, int n_items, const double* Uin, const float* Sin,
                const double* U0, double beta, double dt, const double* dt_dev, double* Uout, float* Sout,
                unsigned long long* ms, int queue_slot, int mode, const double* Din, double* Dout, const float* S0) {
  std::memset(&a, 0, sizeof(a));
  // the padded FP64 arrays the update reads, prefetched by tensor map: Uin
  // (and U0) in mode 0, U in mode 3 (the increments, packed, are prefetched
  // as plain blocks)
  const double* first = mode == 0 || mode == 3 ? Uin : nullptr;
  const double* second = mode == 0 ? U0 : nullptr;
  if (first && encode_state_map(&a.tm_in, first, h->n)) {
    a.has_tm = 1;
    if (second && encode_state_map(&a.tm_u0, second, h->n)) a.has_tm |= 2;
  }
  a.mode = mode;
  a.Din = Din;
  a.Dout = Dout;
  a.S0 = S0;
  a.Uin = Uin;
  a.U0 = U0;
  a.Uout = Uout;
  a.Sin = Sin;
  a.Sout = Sout;
  a.n_items = n_items;
  a.n_sub = h->n;
  a.dx = h->d_dx;
  a.inv_dx = h->d_inv_dx;
  a.nb = h->d_nb;
  a.rel = h->d_rel;
  a.oct = h->d_oct;
  a.beta = beta;
  a.dt = dt;
  a.dt_dev = dt_dev;
  a.gamma = h->gamma;
  a.eta = h->eta;
  a.form = h->form;
  a.queue = h->d_queue + queue_slot;
  a.err = h->d_err;
  a.max_speed = ms;
  a.pf_pass = h->pf_pass;
  a.cw84 = h->cw84;
  a.ids = ids;
}

// The mixed correction of the stage described by a (its call id set).
void fill_reflux(hydro_handle* h, RefluxArgs& r, const StageArgs& a) {
  std::memset(&r, 0, sizeof(r));
  r.cf = h->d_cf;
  r.n_list = h->n_cf_list;
  r.fb = h->d_fb;
  r.fb_stamp = h->d_fb_stamp;
  r.call_id = a.call_id;
  r.inv_dx = h->d_inv_dx;
  r.dt = a.dt;
  r.dt_dev = a.dt_dev;
  r.mode = a.mode;
  r.beta = a.beta;
  r.U = a.Uout;
  r.D = a.Dout;
  r.S0 = a.S0;
  r.Sout = a.Sout;
  r.err = h->d_err;
  r.shape = h->reflux_shape;
}

// One stage by the 3D reconstruction (the handle's parameter checks made it a
// grid of one level); the batch may list at most n items.
int enqueue_recon3d(hydro_handle* h, const int32_t* ids, int n_items, const double* Uin, const double* U0,
                    double beta, double dt, const double* dt_dev, double* Uout, unsigned long long* ms,
                    cudaStream_t st) {
  if (n_items > h->n) return fail(h, HYDRO_ERR_INVALID, "the 3D reconstruction takes at most n items per stage");
  Recon3dArgs r;
  std::memset(&r, 0, sizeof(r));
  r.Uin = Uin;
  r.U0 = U0;
  r.Uout = Uout;
  r.ids = ids;
  r.n_items = n_items;
  r.n_sub = h->n;
  r.dx = h->d_dx;
  r.nb = h->d_nb;
  r.beta = beta;
  r.dt = dt;
  r.dt_dev = dt_dev;
  r.gamma = h->gamma;
  r.eta = h->eta;
  r.form = h->form;
  r.mixed = h->precision == HYDRO_MIXED ? 1 : 0;
  r.fa = h->d_r3_fa;
  r.fl = h->d_r3_fl;
  r.max_speed = ms;
  r.err = h->d_err;
  cudaError_t e = launch_recon3d(r, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "3D reconstruction kernel launch");
  h->launches += 3;
  return HYDRO_OK;
}

int enqueue_stage(hydro_handle* h, const int32_t* ids, int n_items, const double* Uin, const float* Sin,
                  const double* U0, double beta, double dt, const double* dt_dev, double* Uout, float* Sout,
                  unsigned long long* ms, int queue_slot, cudaStream_t st, int mode = 0, const double* Din = nullptr,
                  double* Dout = nullptr, const float* S0 = nullptr, bool all_items = false) {
  CUDA_TRY(h, cudaMemsetAsync(ms, 0, 2 * sizeof(unsigned long long), st));
  if (n_items == 0) return HYDRO_OK;
  if (h->recon3d) return enqueue_recon3d(h, ids, n_items, Uin, U0, beta, dt, dt_dev, Uout, ms, st);
  CUDA_TRY(h, cudaMemsetAsync(h->d_queue + queue_slot, 0, sizeof(unsigned int), st));
  StageArgs a;
  fill_stage(h, a, ids, n_items, Uin, Sin, U0, beta, dt, dt_dev, Uout, Sout, ms, queue_slot, mode, Din, Dout, S0);
  const bool mixed = h->precision == HYDRO_MIXED;
  const bool correct = h->reflux && h->n_cf > 0;
  if (correct && mixed) {
    // the stage exports its coarse-fine fluxes; a pass after it corrects
    a.fb = h->d_fb;
    a.fb_stamp = h->d_fb_stamp;
    a.call_id = ++h->call_counter;
  } else if (correct) {
    // FP64: the correction runs inside the stage: a queue in level order
    // (finest first), the batch's members, fresh export flags
    CUDA_TRY(h, cudaMemsetAsync(h->d_cf_flag, 0, sizeof(int32_t) * (size_t)h->n, st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_abort, 0, sizeof(int), st));
    a.call_id = ++h->call_counter;
    if (all_items) {
      a.member = nullptr;  // the batch lists every sub-grid
      if (h->queue_order == 0) ids = h->d_order_all;
    } else {
      cudaError_t e = launch_order_batch(ids, n_items, h->n, h->d_level, h->n_levels, h->d_order, h->d_member,
                                         a.call_id, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "queue order kernel launch");
      h->launches += 1;
      a.member = h->d_member;
      if (h->queue_order == 0) ids = h->d_order;
    }
    a.fb = h->d_fb;
    a.cf_flag = h->d_cf_flag;
    a.abort_word = h->d_abort;
    a.wait_limit = h->wait_limit;
  }
  a.ids = ids;
  const int grid = stage_grid(h, n_items);
  cudaError_t e = mixed ? launch_stage_mixed(a, grid, st) : launch_stage_fp64(a, grid, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage kernel launch");
  h->launches += 1;
  if (correct && mixed) {
    RefluxArgs r;
    fill_reflux(h, r, a);
    e = launch_reflux_mixed(r, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "flux correction kernel launch");
    h->launches += 1;
  }
  return HYDRO_OK;
}

int enqueue_tau_resync(hydro_handle* h, double* U, float* S, cudaStream_t st) {
  if (!(h->eta > 0.0)) return HYDRO_OK;
  cudaError_t e = launch_tau_resync(U, S, h->n, h->gamma, h->eta, h->precision == HYDRO_MIXED, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "tau resync kernel launch");
  h->launches += 1;
  return HYDRO_OK;
}

int enqueue_shadow(hydro_handle* h, const double* U, float* S, cudaStream_t st) {
  cudaError_t e = launch_shadow(U, S, h->n, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "shadow kernel launch");
  h->launches += 1;
  return HYDRO_OK;
}

int enqueue_ghosts(hydro_handle* h, double* U, cudaStream_t st) {
  GhostArgs g;
  g.U = U;
  g.n_sub = h->n;
  g.nb = h->d_nb;
  g.rel = h->d_rel;
  g.oct = h->d_oct;
  cudaError_t e = launch_ghost_fill(g, h->ghost_threads, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "ghost kernel launch");
  h->launches += 1;
  return HYDRO_OK;
}

}  // namespace

extern "C" {

int hydro_create(const hydro_grid_desc* d, hydro_handle** out) {
  if (!out) return HYDRO_ERR_INVALID;
  *out = nullptr;
  if (!d) return HYDRO_ERR_INVALID;
  if (d->n_subgrids < 1 || d->n_fields != NF || d->nx != NX || d->ghost != NG) return HYDRO_ERR_INVALID;
  if (!(d->gamma > 1.0) || !std::isfinite(d->gamma)) return HYDRO_ERR_INVALID;
  if (!(d->de_switch >= 0.0 && d->de_switch < 1.0)) return HYDRO_ERR_INVALID;
  if (d->precision != HYDRO_FP64 && d->precision != HYDRO_MIXED) return HYDRO_ERR_INVALID;
  if (d->flux_form != HYDRO_FLUX_KNP && d->flux_form != HYDRO_FLUX_KT) return HYDRO_ERR_INVALID;
  if (!d->dx || !d->neighbor || !d->neighbor_rel || !d->octant) return HYDRO_ERR_INVALID;
  const int n = d->n_subgrids;
  for (int s = 0; s < n; ++s) {
    if (!(d->dx[s] > 0.0) || !std::isfinite(d->dx[s])) return HYDRO_ERR_INVALID;
    if (d->octant[s] < 0 || d->octant[s] > 7) return HYDRO_ERR_INVALID;
    for (int f = 0; f < 6; ++f) {
      const int rel = d->neighbor_rel[s * 6 + f];
      const int32_t* nb = d->neighbor + ((size_t)s * 6 + f) * 4;
      if (rel < -1 || rel > 1) return HYDRO_ERR_INVALID;
      if (nb[0] < -1 || nb[0] >= n) return HYDRO_ERR_INVALID;
      if (rel != 0 && nb[0] < 0) return HYDRO_ERR_INVALID;
      if (rel == 1)
        for (int q = 1; q < 4; ++q)
          if (nb[q] < 0 || nb[q] >= n) return HYDRO_ERR_INVALID;
    }
  }
  {
    // the queue orders sub-grids by cell width: at most 32 distinct widths
    std::vector<double> widths(d->dx, d->dx + n);
    std::sort(widths.begin(), widths.end());
    if (std::unique(widths.begin(), widths.end()) - widths.begin() > 32) return HYDRO_ERR_INVALID;
  }
  hydro_handle* h = new (std::nothrow) hydro_handle();
  if (!h) return HYDRO_ERR_NOMEM;
  h->n = n;
  h->precision = d->precision;
  h->form = d->flux_form;
  h->gamma = d->gamma;
  h->eta = d->de_switch;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    delete h;
    return HYDRO_ERR_CUDA;
  }
  bool ok = true;
  ok = ok && cudaMalloc(&h->d_dx, sizeof(double) * n) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_inv_dx, sizeof(double) * n) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_nb, sizeof(int32_t) * n * 24) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_rel, n * 6) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_oct, n) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_queue, 4 * sizeof(unsigned int)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_err, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_partial, sizeof(double) * totals_scratch_doubles(n)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_dt, sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_diag, 12 * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_ms_tmp, 2 * sizeof(unsigned long long)) == cudaSuccess;
  std::vector<int8_t> level(n);
  std::vector<int32_t> order(n);
  std::vector<int32_t> cf;
  std::vector<int32_t> cf_slot, cf_target;
  // the one-launch RK3 step needs mutual neighbour tables: every sub-grid whose
  // halo reads s is read by s (a stage-3 output overwrites what stage-1 halos
  // read, and a sub-grid waits only for those it reads)
  {
    auto reads = [&](int s, int x) {
      for (int f = 0; f < 6; ++f) {
        const int rel = d->neighbor_rel[s * 6 + f];
        for (int q = 0; q < (rel == 1 ? 4 : 1); ++q)
          if (d->neighbor[((size_t)s * 6 + f) * 4 + q] == x) return true;
      }
      return false;
    };
    bool mutual = true;
    for (int s = 0; s < n && mutual; ++s)
      for (int f = 0; f < 6 && mutual; ++f) {
        const int rel = d->neighbor_rel[s * 6 + f];
        for (int q = 0; q < (rel == 1 ? 4 : 1); ++q) {
          const int x = d->neighbor[((size_t)s * 6 + f) * 4 + q];
          if (x >= 0 && x != s && !reads(x, s)) mutual = false;
        }
      }
    h->fused_ok = mutual ? 1 : 0;
  }
  {
    // level ranks from the cell widths (0 = finest) and the queue of every
    // sub-grid in level order, for the in-stage coarse-fine correction
    for (int s = 0; s < n; ++s)
      for (int f = 0; f < 6; ++f) h->n_cf += d->neighbor_rel[s * 6 + f] == 1 ? 1 : 0;
    std::vector<double> widths(d->dx, d->dx + n);
    std::sort(widths.begin(), widths.end());
    widths.erase(std::unique(widths.begin(), widths.end()), widths.end());
    h->n_levels = (int)widths.size();
    bool same = h->n_levels == 1;
    for (int s = 0; s < n * 6 && same; ++s) same = d->neighbor_rel[s] == 0;
    h->single_level = same ? 1 : 0;
    for (int s = 0; s < n; ++s)
      level[s] = (int8_t)(std::lower_bound(widths.begin(), widths.end(), d->dx[s]) - widths.begin());
    // the queue of a whole-grid stage: every sub-grid, finest level first
    // (ids ascending within a level)
    for (int s = 0; s < n; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return level[x] < level[y]; });
    if (h->n_cf > 0 && d->precision == HYDRO_MIXED) {
      for (int s = 0; s < n; ++s) {
        bool any = false;
        for (int f = 0; f < 6; ++f) any = any || d->neighbor_rel[s * 6 + f] == 1;
        if (!any) continue;
        cf.push_back(s);
        for (int f = 0; f < 6; ++f)
          for (int q = 0; q < 4; ++q)
            cf.push_back(d->neighbor_rel[s * 6 + f] == 1 ? d->neighbor[(s * 6 + f) * 4 + q] : -1);
      }
      h->n_cf_list = (int)(cf.size() / CF_ENTRY);
      // the one-launch step's arrival targets: the coarse sub-grid itself and
      // every finer sub-grid that names it as the neighbour of a coarser face
      cf_slot.assign(n, -1);
      cf_target.assign(h->n_cf_list, 1);
      for (int r = 0; r < h->n_cf_list; ++r) cf_slot[cf[(size_t)r * CF_ENTRY]] = r;
      for (int s = 0; s < n; ++s)
        for (int f = 0; f < 6; ++f)
          if (d->neighbor_rel[s * 6 + f] == -1) {
            const int r = cf_slot[d->neighbor[((size_t)s * 6 + f) * 4]];
            if (r < 0)
              h->fused_ok = 0;  // a coarser neighbour without finer ones: not a mutual table
            else
              ++cf_target[r];
          }
      for (int r = 0; r < h->n_cf_list; ++r) {
        int fine = 0;
        for (int e = 1; e < CF_ENTRY; ++e) fine += cf[(size_t)r * CF_ENTRY + e] >= 0 ? 1 : 0;
        if (cf_target[r] != 1 + fine) h->fused_ok = 0;
      }
      ok = ok && cudaMalloc(&h->d_cf, sizeof(int32_t) * cf.size()) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_cf_slot, sizeof(int32_t) * n) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_cf_target, sizeof(int32_t) * h->n_cf_list) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_arrive, sizeof(int32_t) * h->n_cf_list) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_order_all, sizeof(int32_t) * n) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_fb, sizeof(float) * (size_t)n * 6 * NF * NPEN) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_fb_stamp, sizeof(int32_t) * n) == cudaSuccess;
    } else if (h->n_cf > 0) {
      const size_t tsize = sizeof(double);
      ok = ok && cudaMalloc(&h->d_level, n) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_order_all, sizeof(int32_t) * n) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_order, sizeof(int32_t) * n) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_member, sizeof(int32_t) * n) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_fb, tsize * (size_t)n * 6 * NF * NPEN) == cudaSuccess;
      ok = ok && cudaMalloc(&h->d_cf_flag, sizeof(int32_t) * n) == cudaSuccess;
    }
  }
  ok = ok && cudaMalloc(&h->d_abort, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->d_done, sizeof(int32_t) * n) == cudaSuccess;
  if (d->precision == HYDRO_MIXED)
    for (int b = 0; b < 3; ++b)
      ok = ok && cudaMalloc(&h->d_shadow[b], sizeof(float) * (size_t)n * NF * SHADOW_FIELD) == cudaSuccess;
  if (!ok) {
    free_all(h);
    delete h;
    cudaGetLastError();
    return HYDRO_ERR_NOMEM;
  }
  ok = ok && cudaMemcpy(h->d_dx, d->dx, sizeof(double) * n, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) {
    std::vector<double> inv(n);
    for (int s = 0; s < n; ++s) inv[s] = 1.0 / d->dx[s];
    ok = cudaMemcpy(h->d_inv_dx, inv.data(), sizeof(double) * n, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  ok = ok && cudaMemcpy(h->d_nb, d->neighbor, sizeof(int32_t) * n * 24, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(h->d_rel, d->neighbor_rel, n * 6, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(h->d_oct, d->octant, n, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemset(h->d_err, 0, sizeof(int)) == cudaSuccess;
  if (h->n_cf > 0 && d->precision == HYDRO_MIXED) {
    ok = ok && cudaMemcpy(h->d_cf, cf.data(), sizeof(int32_t) * cf.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_cf_slot, cf_slot.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_cf_target, cf_target.data(), sizeof(int32_t) * h->n_cf_list,
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(h->d_fb_stamp, 0, sizeof(int32_t) * n) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_order_all, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice) == cudaSuccess;
  } else if (h->n_cf > 0) {
    ok = ok && cudaMemcpy(h->d_level, level.data(), n, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_order_all, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(h->d_member, 0, sizeof(int32_t) * n) == cudaSuccess;
    ok = ok && cudaMemset(h->d_cf_flag, 0, sizeof(int32_t) * n) == cudaSuccess;
  }
  ok = ok && cudaMemset(h->d_abort, 0, sizeof(int)) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  h->occupancy = h->precision == HYDRO_MIXED ? stage_blocks_per_sm_mixed() : stage_blocks_per_sm_fp64();
  h->occupancy_fused = h->precision == HYDRO_MIXED ? rk3_blocks_per_sm_mixed() : rk3_blocks_per_sm_fp64();
  h->occupancy_cw = h->precision == HYDRO_MIXED ? cw_blocks_per_sm_mixed() : cw_blocks_per_sm_fp64();
  if (!ok) {
    free_all(h);
    delete h;
    return HYDRO_ERR_CUDA;
  }
  *out = h;
  return HYDRO_OK;
}

}  // extern "C"

namespace {

int check_step(hydro_handle* h, const hydro_batch* batch, const double* U_in, const double* U0, double beta,
               double dt, const double* U_out, const double* d_max_speed) {
  int rc = check_batch(h, batch);
  if (rc) return rc;
  if (!U_in || !U_out || !d_max_speed) return fail(h, HYDRO_ERR_INVALID, "NULL state or speed pointer");
  if (U_in == U_out) return fail(h, HYDRO_ERR_INVALID, "U_out must not alias U_in");
  if (!aligned(U_in, 16) || !aligned(U_out, 16) || (U0 && !aligned(U0, 16)) || !aligned(d_max_speed, 8))
    return fail(h, HYDRO_ERR_INVALID, "misaligned pointer");
  if (!(beta > 0.0 && beta <= 1.0)) return fail(h, HYDRO_ERR_INVALID, "beta must be in (0, 1]");
  if (beta != 1.0 && !U0) return fail(h, HYDRO_ERR_INVALID, "U0 is required when beta != 1");
  if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(h, HYDRO_ERR_INVALID, "dt must be finite and >= 0");
  return HYDRO_OK;
}

}  // namespace

extern "C" {

int hydro_step(hydro_handle* h, const hydro_batch* batch, const double* U_in, const double* U0, double beta,
               double dt, double* U_out, double* d_max_speed, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  int rc = check_step(h, batch, U_in, U0, beta, dt, U_out, d_max_speed);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  const float* S = nullptr;
  if (h->precision == HYDRO_MIXED && !h->recon3d && batch->n_items > 0) {
    // the shadows the stage reads: of the batch and its face neighbours when
    // the batch is small against the grid, else of the whole grid in one pass
    if ((int64_t)batch->n_items * 8 < (int64_t)h->n) {
      cudaError_t e = launch_shadow_ids(U_in, h->d_shadow[0], batch->subgrid_ids, batch->n_items, h->n, h->d_nb,
                                        h->d_rel, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "shadow kernel launch");
      h->launches += 1;
    } else {
      rc = enqueue_shadow(h, U_in, h->d_shadow[0], st);
      if (rc) return rc;
    }
    S = h->d_shadow[0];
  }
  return enqueue_stage(h, batch->subgrid_ids, batch->n_items, U_in, S, beta == 1.0 ? nullptr : U0, beta, dt,
                       nullptr, U_out, nullptr, reinterpret_cast<unsigned long long*>(d_max_speed), 0, st);
}

int hydro_shadow(hydro_handle* h, const double* U, float* S, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !S || !aligned(U, 16) || !aligned(S, 16)) return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned pointer");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return enqueue_shadow(h, U, S, st);
}

int hydro_pack_interiors(hydro_handle* h, const double* U, double* P, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !P || !aligned(U, 16) || !aligned(P, 16)) return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned pointer");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  cudaError_t e = launch_pack(U, P, h->n, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "pack kernel launch");
  h->launches += 1;
  return HYDRO_OK;
}

int hydro_unpack_interiors(hydro_handle* h, const double* P, double* U, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !P || !aligned(U, 16) || !aligned(P, 16)) return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned pointer");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  cudaError_t e = launch_unpack(P, U, h->n, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "unpack kernel launch");
  h->launches += 1;
  return HYDRO_OK;
}

int hydro_pack_interiors_range(hydro_handle* h, const double* U, double* P, int32_t first, int32_t count,
                               void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !P || !aligned(U, 16) || !aligned(P, 16)) return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned pointer");
  if (first < 0 || count < 0 || (int64_t)first + count > h->n) return fail(h, HYDRO_ERR_INVALID, "range out of bounds");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  if (count == 0) return HYDRO_OK;
  cudaError_t e = launch_pack(U + (size_t)first * NF * NP3, P + (size_t)first * NF * CELLS, count, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "pack kernel launch");
  h->launches += 1;
  return HYDRO_OK;
}

int hydro_unpack_interiors_range(hydro_handle* h, const double* P, double* U, int32_t first, int32_t count,
                                 void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !P || !aligned(U, 16) || !aligned(P, 16)) return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned pointer");
  if (first < 0 || count < 0 || (int64_t)first + count > h->n) return fail(h, HYDRO_ERR_INVALID, "range out of bounds");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  if (count == 0) return HYDRO_OK;
  cudaError_t e = launch_unpack(P + (size_t)first * NF * CELLS, U + (size_t)first * NF * NP3, count, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "unpack kernel launch");
  h->launches += 1;
  return HYDRO_OK;
}

int hydro_step_shadowed(hydro_handle* h, const hydro_batch* batch, const double* U_in, const float* S_in,
                        const double* U0, double beta, double dt, double* U_out, float* S_out, double* d_max_speed,
                        void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (h->precision != HYDRO_MIXED) return fail(h, HYDRO_ERR_STATE, "hydro_step_shadowed needs a mixed-precision handle");
  if (h->recon3d) return fail(h, HYDRO_ERR_STATE, "the 3D reconstruction reads no shadow");
  int rc = check_step(h, batch, U_in, U0, beta, dt, U_out, d_max_speed);
  if (rc) return rc;
  if (!S_in || !aligned(S_in, 16) || (S_out && !aligned(S_out, 16)))
    return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned shadow pointer");
  if (S_out == S_in) return fail(h, HYDRO_ERR_INVALID, "S_out must not alias S_in");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return enqueue_stage(h, batch->subgrid_ids, batch->n_items, U_in, S_in, beta == 1.0 ? nullptr : U0, beta, dt,
                       nullptr, U_out, S_out, reinterpret_cast<unsigned long long*>(d_max_speed), 0, st);
}

int hydro_fill_ghosts(hydro_handle* h, double* U, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !aligned(U, 16)) return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned state");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return enqueue_ghosts(h, U, st);
}

}  // extern "C"

namespace {

int check_rk3(hydro_handle* h, const hydro_batch* batch, double* U, double* scratch1, double* scratch2,
              double* d_max_speed, double* d_dt_out) {
  int rc = check_batch(h, batch);
  if (rc) return rc;
  if (!U || !scratch1 || !scratch2 || !d_max_speed) return fail(h, HYDRO_ERR_INVALID, "NULL pointer");
  if (U == scratch1 || U == scratch2 || scratch1 == scratch2)
    return fail(h, HYDRO_ERR_INVALID, "U, scratch1, scratch2 must be distinct");
  if (!aligned(U, 16) || !aligned(scratch1, 16) || !aligned(scratch2, 16) || !aligned(d_max_speed, 8) ||
      (d_dt_out && !aligned(d_dt_out, 8)))
    return fail(h, HYDRO_ERR_INVALID, "misaligned pointer");
  if (batch->n_items != h->n)
    return fail(h, HYDRO_ERR_INVALID, "an RK3 step advances every sub-grid: n_items must equal n_subgrids");
  return HYDRO_OK;
}

// Enqueue the three stages of one RK3 step on cs.  FP64: the Shu-Osher stages
// U1 = U*(U), U2 = U + 1/4 (U*(U1) - U), U3 = U + 2/3 (U*(U2) - U) through
// scratch1 and scratch2.  Mixed: the same step in increment form (modes 1..3),
// scratch1 and scratch2 holding the increment pairs, U changed once at the
// end; shadow buffers A = shadow of U (kept for the whole step), B = stage 1's
// state, C = stage 2's; with write_next, stage 3 writes the new U's shadow into A.
// The same step in one persistent launch (rk3_kernel, see FusedArgs): the
// three stages' arguments as the separate launches take them, one queue, the
// completion counters zeroed first.
int enqueue_rk3_fused(hydro_handle* h, const int32_t* ids, int ni, double* U, double* s1, double* s2,
                      unsigned long long* ms, bool write_next, cudaStream_t cs) {
  FusedArgs F;
  std::memset(&F, 0, sizeof(F));
  const bool mixed = h->precision == HYDRO_MIXED;
  const bool correct = h->reflux && h->n_cf > 0;
  const double* dtd = h->d_dt;
  unsigned long long* mt = h->d_ms_tmp;
  // each stage's queue lists finer sub-grids first: FP64, the in-stage
  // correction waits for them; mixed, a coarse sub-grid then completes (its
  // finer neighbours have arrived) when its own item ends
  const int32_t* q = correct && h->queue_order == 0 ? h->d_order_all : ids;
  if (mixed) {
    float *A = h->d_shadow[0], *B = h->d_shadow[1], *C = h->d_shadow[2];
    fill_stage(h, F.st[0], q, ni, U, A, nullptr, 1.0, 0.0, dtd, nullptr, B, ms, 0, 1, nullptr, s1, A);
    fill_stage(h, F.st[1], q, ni, U, B, nullptr, 1.0, 0.0, dtd, nullptr, C, mt, 0, 2, s1, s2, A);
    fill_stage(h, F.st[2], q, ni, U, C, nullptr, 1.0, 0.0, dtd, U, write_next ? A : nullptr, mt, 0, 3, s2, nullptr, A);
  } else {
    fill_stage(h, F.st[0], q, ni, U, nullptr, nullptr, 1.0, 0.0, dtd, s1, nullptr, ms, 0, 0, nullptr, nullptr, nullptr);
    fill_stage(h, F.st[1], q, ni, s1, nullptr, U, 0.25, 0.0, dtd, s2, nullptr, mt, 0, 0, nullptr, nullptr, nullptr);
    fill_stage(h, F.st[2], q, ni, s2, nullptr, U, 2.0 / 3.0, 0.0, dtd, U, nullptr, mt, 0, 0, nullptr, nullptr,
               nullptr);
  }
  for (int k = 0; k < 3; ++k) {
    StageArgs& a = F.st[k];
    a.abort_word = h->d_abort;
    a.wait_limit = h->wait_limit;
    if (!correct) continue;
    a.fb = h->d_fb;
    a.call_id = ++h->call_counter;
    if (mixed) {
      a.fb_stamp = h->d_fb_stamp;
      fill_reflux(h, F.rf[k], a);
    } else {
      a.cf_flag = h->d_cf_flag;
      a.member = nullptr;  // every sub-grid
      a.flag_base = 3 * k;
    }
  }
  F.done = h->d_done;
  F.arrive = h->d_arrive;
  F.cf_slot = h->d_cf_slot;
  F.cf_target = h->d_cf_target;
  F.n = ni;
  F.order = h->fused == 2 ? 1 : 0;
  CUDA_TRY(h, cudaMemsetAsync(ms, 0, 2 * sizeof(unsigned long long), cs));
  CUDA_TRY(h, cudaMemsetAsync(mt, 0, 2 * sizeof(unsigned long long), cs));
  CUDA_TRY(h, cudaMemsetAsync(h->d_queue, 0, sizeof(unsigned int), cs));
  CUDA_TRY(h, cudaMemsetAsync(h->d_done, 0, sizeof(int32_t) * (size_t)h->n, cs));
  CUDA_TRY(h, cudaMemsetAsync(h->d_abort, 0, sizeof(int), cs));
  if (correct && mixed) CUDA_TRY(h, cudaMemsetAsync(h->d_arrive, 0, sizeof(int32_t) * (size_t)h->n_cf_list, cs));
  if (correct && !mixed) CUDA_TRY(h, cudaMemsetAsync(h->d_cf_flag, 0, sizeof(int32_t) * (size_t)h->n, cs));
  const int per_sm = h->ctas_per_sm > 0 ? std::min(h->ctas_per_sm, h->occupancy_fused) : h->occupancy_fused;
  int grid = h->grid_cap > 0 ? h->grid_cap : h->sm_count * per_sm;
  grid = std::max(1, std::min(grid, 3 * ni));
  cudaError_t e = mixed ? launch_rk3_mixed(F, grid, cs) : launch_rk3_fp64(F, grid, cs);
  if (e != cudaSuccess) return cuda_fail(h, e, "one-launch RK3 kernel launch");
  h->launches += 1;
  return HYDRO_OK;
}

int enqueue_rk3_stages(hydro_handle* h, const int32_t* ids, int ni, double* U, double* s1, double* s2,
                       unsigned long long* ms, bool write_next, cudaStream_t cs) {
  int rc;
  if (h->fused && h->fused_ok && !h->cw84 && !h->recon3d && ni == h->n) {
    rc = enqueue_rk3_fused(h, ids, ni, U, s1, s2, ms, write_next, cs);
    if (!rc && h->tau_resync)
      rc = enqueue_tau_resync(h, U, h->precision == HYDRO_MIXED && write_next ? h->d_shadow[0] : nullptr, cs);
    return rc;
  }
  if (h->precision == HYDRO_MIXED && !h->recon3d) {
    float *A = h->d_shadow[0], *B = h->d_shadow[1], *C = h->d_shadow[2];
    rc = enqueue_stage(h, ids, ni, U, A, nullptr, 1.0, 0.0, h->d_dt, nullptr, B, ms, 0, cs, 1, nullptr, s1, A, true);
    if (!rc)
      rc = enqueue_stage(h, ids, ni, U, B, nullptr, 1.0, 0.0, h->d_dt, nullptr, C, h->d_ms_tmp, 1, cs, 2, s1, s2, A,
                         true);
    if (!rc)
      rc = enqueue_stage(h, ids, ni, U, C, nullptr, 1.0, 0.0, h->d_dt, U, write_next ? A : nullptr, h->d_ms_tmp, 2,
                         cs, 3, s2, nullptr, A, true);
    if (!rc && h->tau_resync) rc = enqueue_tau_resync(h, U, write_next ? A : nullptr, cs);
    return rc;
  }
  rc = enqueue_stage(h, ids, ni, U, nullptr, nullptr, 1.0, 0.0, h->d_dt, s1, nullptr, ms, 0, cs, 0, nullptr, nullptr,
                     nullptr, true);
  if (!rc)
    rc = enqueue_stage(h, ids, ni, s1, nullptr, U, 0.25, 0.0, h->d_dt, s2, nullptr, h->d_ms_tmp, 1, cs, 0, nullptr,
                       nullptr, nullptr, true);
  if (!rc)
    rc = enqueue_stage(h, ids, ni, s2, nullptr, U, 2.0 / 3.0, 0.0, h->d_dt, U, nullptr, h->d_ms_tmp, 2, cs, 0, nullptr,
                       nullptr, nullptr, true);
  if (!rc && h->tau_resync) rc = enqueue_tau_resync(h, U, nullptr, cs);
  return rc;
}

// Find or capture the graph of key k.  n_steps == 0: one RK3 step whose dt the
// caller sets in h->d_dt before each launch.  n_steps >= 1: that many steps,
// each with dt = cfl / d_max_speed[1] chosen on the device and the totals of
// the new state, the shadow written once and then chained from step to step.
int get_graph(hydro_handle* h, const GraphKey& k, GraphEntry** out) {
  for (auto& e : h->graphs)
    if (e.key == k) {
      *out = &e;
      return HYDRO_OK;
    }
  const int64_t before = h->launches;
  CUDA_TRY(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaStream_t cs = h->cap_stream;
  unsigned long long* ms = reinterpret_cast<unsigned long long*>(k.dms);
  // the stage kernel gathers halos from the neighbours' interiors itself, so
  // no ghost fill is needed between stages; in mixed precision each stage
  // reads the shadow of its input and writes the shadow of its output
  // (the 3D reconstruction reads the FP64 state in both precisions)
  const bool mixed = h->precision == HYDRO_MIXED && !h->recon3d;
  int rc = mixed ? enqueue_shadow(h, k.U, h->d_shadow[0], cs) : HYDRO_OK;
  if (k.n_steps == 0) {
    if (!rc) rc = enqueue_rk3_stages(h, k.ids, k.n_items, k.U, k.s1, k.s2, ms, false, cs);
  } else {
    for (int step = 0; step < k.n_steps && !rc; ++step) {
      cfl_dt<<<1, 1, 0, cs>>>(h->d_dt, k.dms, k.cfl, k.dt_out ? k.dt_out + step : nullptr);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        rc = cuda_fail(h, e, "cfl_dt launch");
        break;
      }
      h->launches += 1;
      // stage 3 leaves the new state's shadow where the next step reads it
      rc = enqueue_rk3_stages(h, k.ids, k.n_items, k.U, k.s1, k.s2, ms, mixed && step + 1 < k.n_steps, cs);
      if (!rc && k.totals) {
        e = launch_totals(k.U, h->n, h->d_dx, h->d_partial, k.totals + (size_t)step * NF, cs);
        if (e != cudaSuccess)
          rc = cuda_fail(h, e, "totals kernel launch");
        else
          h->launches += 3;
      }
    }
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  const int kernels = (int)(h->launches - before);
  h->launches = before;
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  GraphEntry ne;
  ne.key = k;
  ne.kernels = kernels;
  e = cudaGraphInstantiate(&ne.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  if (h->graphs.size() >= 16) {
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(ne);
  *out = &h->graphs.back();
  return HYDRO_OK;
}

int rk3_common(hydro_handle* h, const hydro_batch* batch, double* U, double* scratch1, double* scratch2,
               double dt, double cfl, double* d_max_speed, double* d_dt_out, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  int rc = check_rk3(h, batch, U, scratch1, scratch2, d_max_speed, d_dt_out);
  if (rc) return rc;
  if (cfl > 0.0) {
    if (!(cfl <= 1.0)) return fail(h, HYDRO_ERR_INVALID, "cfl must be in (0, 1]");
  } else if (!(dt >= 0.0) || !std::isfinite(dt)) {
    return fail(h, HYDRO_ERR_INVALID, "dt must be finite and >= 0");
  }
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  GraphKey k{batch->subgrid_ids, batch->n_items, U, scratch1, scratch2, d_max_speed, 0, 0.0, nullptr, nullptr};
  GraphEntry* g = nullptr;
  rc = get_graph(h, k, &g);
  if (rc) return rc;
  if (cfl > 0.0)
    cfl_dt<<<1, 1, 0, st>>>(h->d_dt, d_max_speed, cfl, d_dt_out);
  else
    set_scalar<<<1, 1, 0, st>>>(h->d_dt, dt);
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaGraphLaunch(g->exec, st));
  h->launches += 1 + g->kernels;
  return HYDRO_OK;
}

}  // namespace

extern "C" {

int hydro_rk3_step(hydro_handle* h, const hydro_batch* batch, double* U, double* scratch1, double* scratch2,
                   double dt, double* d_max_speed, void* stream) {
  return rk3_common(h, batch, U, scratch1, scratch2, dt, 0.0, d_max_speed, nullptr, stream);
}

int hydro_rk3_step_cfl(hydro_handle* h, const hydro_batch* batch, double* U, double* scratch1, double* scratch2,
                       double cfl, double* d_max_speed, double* d_dt_out, void* stream) {
  if (!(cfl > 0.0)) return h ? fail(h, HYDRO_ERR_INVALID, "cfl must be in (0, 1]") : HYDRO_ERR_INVALID;
  return rk3_common(h, batch, U, scratch1, scratch2, 0.0, cfl, d_max_speed, d_dt_out, stream);
}

}  // extern "C"

namespace {

int run_graph(hydro_handle* h, const hydro_batch* batch, double* U, double* scratch1, double* scratch2, double cfl,
              int32_t n_steps, double* d_max_speed, double* d_dt_out, double* d_totals, GraphEntry** g) {
  int rc = check_rk3(h, batch, U, scratch1, scratch2, d_max_speed, d_dt_out);
  if (rc) return rc;
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(h, HYDRO_ERR_INVALID, "cfl must be in (0, 1]");
  if (n_steps < 1 || n_steps > HYDRO_RK3_RUN_MAX_STEPS)
    return fail(h, HYDRO_ERR_INVALID, "n_steps must be in [1, %d]", HYDRO_RK3_RUN_MAX_STEPS);
  if (d_totals && !aligned(d_totals, 8)) return fail(h, HYDRO_ERR_INVALID, "misaligned pointer");
  GraphKey k{batch->subgrid_ids, batch->n_items, U, scratch1, scratch2, d_max_speed, n_steps, cfl, d_dt_out,
             d_totals};
  return get_graph(h, k, g);
}

}  // namespace

extern "C" {

int hydro_rk3_run_cfl(hydro_handle* h, const hydro_batch* batch, double* U, double* scratch1, double* scratch2,
                      double cfl, int32_t n_steps, double* d_max_speed, double* d_dt_out, double* d_totals,
                      void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  GraphEntry* g = nullptr;
  int rc = run_graph(h, batch, U, scratch1, scratch2, cfl, n_steps, d_max_speed, d_dt_out, d_totals, &g);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  CUDA_TRY(h, cudaGraphLaunch(g->exec, st));
  h->launches += g->kernels;
  return HYDRO_OK;
}

int hydro_rk3_run_prepare(hydro_handle* h, const hydro_batch* batch, double* U, double* scratch1, double* scratch2,
                          double cfl, int32_t n_steps, double* d_max_speed, double* d_dt_out, double* d_totals) {
  if (!h) return HYDRO_ERR_INVALID;
  GraphEntry* g = nullptr;
  return run_graph(h, batch, U, scratch1, scratch2, cfl, n_steps, d_max_speed, d_dt_out, d_totals, &g);
}

int hydro_totals(hydro_handle* h, const double* U, double* d_totals, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !d_totals || !aligned(U, 16) || !aligned(d_totals, 8))
    return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned pointer");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  cudaError_t e = launch_totals(U, h->n, h->d_dx, h->d_partial, d_totals, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "totals kernel launch");
  h->launches += 3;
  return HYDRO_OK;
}

int hydro_diagnostics(hydro_handle* h, const double* U, const double* d_origin, double* d_out, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !d_origin || !d_out || !aligned(U, 16) || !aligned(d_origin, 8) || !aligned(d_out, 8))
    return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned pointer");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  cudaError_t e = launch_diagnostics(U, d_origin, h->n, h->d_dx, h->d_partial, h->d_diag, d_out, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics kernel launch");
  h->launches += 4;
  return HYDRO_OK;
}

int hydro_tau_resync(hydro_handle* h, double* U, float* S, void* stream) {
  if (!h) return HYDRO_ERR_INVALID;
  if (!U || !aligned(U, 16) || (S && !aligned(S, 16))) return fail(h, HYDRO_ERR_INVALID, "NULL or misaligned pointer");
  if (S && h->precision != HYDRO_MIXED) return fail(h, HYDRO_ERR_INVALID, "a shadow needs a mixed-precision handle");
  cudaStream_t st = (cudaStream_t)stream;
  h->last_stream = st;
  return enqueue_tau_resync(h, U, S, st);
}

int hydro_sync(hydro_handle* h) {
  if (!h) return HYDRO_ERR_INVALID;
  CUDA_TRY(h, cudaStreamSynchronize(h->last_stream));
  int err = 0;
  CUDA_TRY(h, cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(h, cudaMemset(h->d_err, 0, sizeof(int)));
  if (err & ERRBIT_TIMEOUT)
    return fail(h, HYDRO_ERR_TIMEOUT, "a stage gave up waiting for a finer neighbour's exported fluxes");
  if (err & ERRBIT_BAD_ID) return fail(h, HYDRO_ERR_INVALID, "a sub-grid id was out of range");
  if (err & ERRBIT_NONFINITE) return fail(h, HYDRO_ERR_NONFINITE, "non-finite value or non-positive density");
  return HYDRO_OK;
}

const char* hydro_last_error(const hydro_handle* h) { return h ? h->msg : "NULL handle"; }

int64_t hydro_launch_count(const hydro_handle* h) { return h ? h->launches : 0; }

int hydro_set_param(hydro_handle* h, int32_t key, int32_t value) {
  if (!h) return HYDRO_ERR_INVALID;
  if (key == HYDRO_PARAM_STAGE_CTAS_PER_SM) {
    if (value < 0 || value > 8) return fail(h, HYDRO_ERR_INVALID, "ctas per SM out of range");
    h->ctas_per_sm = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_REFLUX) {
    if (value != 0 && value != 1) return fail(h, HYDRO_ERR_INVALID, "reflux must be 0 or 1");
    h->reflux = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_TAU_RESYNC) {
    if (value != 0 && value != 1) return fail(h, HYDRO_ERR_INVALID, "tau resync must be 0 or 1");
    h->tau_resync = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_WAIT_LIMIT) {
    if (value < 1) return fail(h, HYDRO_ERR_INVALID, "wait limit must be >= 1 clock cycle");
    h->wait_limit = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_QUEUE_ORDER) {
    if (value != 0 && value != 1) return fail(h, HYDRO_ERR_INVALID, "queue order must be 0 or 1");
    h->queue_order = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_STAGE_GRID) {
    if (value < 0) return fail(h, HYDRO_ERR_INVALID, "stage grid must be >= 0");
    h->grid_cap = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_PREFETCH_PASS) {
    if (value < 0 || value > 2) return fail(h, HYDRO_ERR_INVALID, "prefetch pass must be 0, 1 or 2");
    h->pf_pass = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_REFLUX_SHAPE) {
    if (value < 0 || value >= REFLUX_SHAPES) return fail(h, HYDRO_ERR_INVALID, "correction shape out of range");
    h->reflux_shape = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_FUSED_RK3) {
    if (value < 0 || value > 2) return fail(h, HYDRO_ERR_INVALID, "one-launch RK3 mode must be 0, 1 or 2");
    h->fused = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_CW84) {
    if (value < 0 || value > 3) return fail(h, HYDRO_ERR_INVALID, "CW84 flags must be in 0..3");
    if (value && h->recon3d) return fail(h, HYDRO_ERR_INVALID, "CW84 extensions with the 3D reconstruction");
    h->cw84 = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_RECON3D) {
    if (value != 0 && value != 1) return fail(h, HYDRO_ERR_INVALID, "3D reconstruction must be 0 or 1");
    if (value) {
      if (!h->single_level) return fail(h, HYDRO_ERR_INVALID, "the 3D reconstruction needs a grid of one level");
      if (h->cw84) return fail(h, HYDRO_ERR_INVALID, "the 3D reconstruction with CW84 extensions");
      cudaError_t e = recon3d_prepare();
      if (e != cudaSuccess) return cuda_fail(h, e, "3D reconstruction kernel attributes");
      if (!h->d_r3_fa) {
        if (cudaMalloc(&h->d_r3_fa, recon3d_scratch_doubles(h->n, 0) * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->d_r3_fl, recon3d_scratch_doubles(h->n, 1) * sizeof(double)) != cudaSuccess) {
          cudaGetLastError();
          cudaFree(h->d_r3_fa);
          h->d_r3_fa = nullptr;
          h->d_r3_fl = nullptr;
          return fail(h, HYDRO_ERR_NOMEM, "3D reconstruction scratch allocation");
        }
      }
    }
    h->recon3d = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  if (key == HYDRO_PARAM_GHOST_THREADS) {
    if (value < 64 || value > 1024 || value % 32) return fail(h, HYDRO_ERR_INVALID, "ghost threads out of range");
    h->ghost_threads = value;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return HYDRO_OK;
  }
  return fail(h, HYDRO_ERR_INVALID, "unknown parameter %d", key);
}

void hydro_destroy(hydro_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->last_stream);
  free_all(h);
  delete h;
}

}  // extern "C"
