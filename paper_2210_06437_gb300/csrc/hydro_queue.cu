// hydro_queue.cu -- the work queue of one stage over a batch.
//
// The stage kernel corrects the fluxes of a coarse sub-grid's faces onto finer
// neighbours while it runs (paper Section V-B.1: compute_fluxes corrects the
// fluxes on coarse-fine boundaries), waiting for those neighbours to export
// theirs.  Taking the finer levels first makes every such wait one for an
// item that a running CTA already holds.  This pass orders the batch's ids by
// level (a counting sort: finest level first; the order inside a level does
// not matter, every sub-grid's result depends on its inputs only) and marks
// the batch's members with the call's id.
#include "hydro_internal.cuh"

namespace hydro {
namespace {

constexpr int QT = 1024;
constexpr int MAX_LEVELS = 32;

__global__ void __launch_bounds__(QT) order_batch_kernel(const int32_t* __restrict__ ids, int n_items, int n_sub,
                                                         const int8_t* __restrict__ level_rank, int n_levels,
                                                         int32_t* __restrict__ order, int32_t* __restrict__ member,
                                                         int32_t call_id) {
  __shared__ int cnt[MAX_LEVELS + 1];
  const int tid = threadIdx.x;
  if (tid <= MAX_LEVELS) cnt[tid] = 0;
  __syncthreads();
  // bucket 0: ids outside [0, n) (the stage reports them); bucket 1 + L: level rank L
  for (int t = tid; t < n_items; t += QT) {
    const int s = ids[t] >= 0 ? ids[t] & ~ITEM_FLUX_ONLY : ids[t];  // a flux-only item counts as advanced
    const bool ok = s >= 0 && s < n_sub;
    atomicAdd(&cnt[ok ? 1 + level_rank[s] : 0], 1);
    if (ok) member[s] = call_id;
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int b = 0; b <= n_levels; ++b) {
      const int c = cnt[b];
      cnt[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int t = tid; t < n_items; t += QT) {
    const int raw = ids[t];
    const int s = raw >= 0 ? raw & ~ITEM_FLUX_ONLY : raw;
    const bool ok = s >= 0 && s < n_sub;
    order[atomicAdd(&cnt[ok ? 1 + level_rank[s] : 0], 1)] = raw;
  }
}

}  // namespace

cudaError_t launch_order_batch(const int32_t* ids, int n_items, int n_sub, const int8_t* level_rank, int n_levels,
                               int32_t* order, int32_t* member, int32_t call_id, cudaStream_t st) {
  if (n_levels < 1 || n_levels > MAX_LEVELS) return cudaErrorInvalidValue;
  if (n_items < 1) return cudaSuccess;
  order_batch_kernel<<<1, QT, 0, st>>>(ids, n_items, n_sub, level_rank, n_levels, order, member, call_id);
  return cudaGetLastError();
}

}  // namespace hydro
