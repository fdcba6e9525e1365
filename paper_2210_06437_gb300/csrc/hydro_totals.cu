// hydro_totals.cu -- grid totals T_f = sum_s dx_s^3 sum_interior U_f
// (paper Section V-B.1, diagnostics_actions_type: total mass and other grid
// sums), compensated and deterministic.
//
// Pass 1: one CTA per sub-grid; each thread sums two cells per field with
// Neumaier's compensation, then a fixed-shape tree merges (sum, comp) pairs
// with an error-free TwoSum; the partial dx^3 * (sum, comp) goes to scratch.
// Pass 2: one CTA per field sums the partials of all sub-grids in a fixed
// order (strided per thread, then a fixed tree).  No atomics, so the result
// is bit-reproducible.
#include "hydro_internal.cuh"

namespace hydro {
namespace {

constexpr int TT = 256;

struct Pair {
  double s, c;
};

__device__ __forceinline__ void neumaier(Pair& p, double x) {
  double t = p.s + x;
  if (fabs(p.s) >= fabs(x))
    p.c += (p.s - t) + x;
  else
    p.c += (x - t) + p.s;
  p.s = t;
}

__device__ __forceinline__ Pair merge(Pair a, Pair b) {
  double s = a.s + b.s;
  double bp = s - a.s;
  double e = (a.s - (s - bp)) + (b.s - bp);
  Pair r;
  r.s = s;
  r.c = (a.c + b.c) + e;
  return r;
}

__device__ __forceinline__ Pair block_merge(Pair p, Pair* sh) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Pair q;
    q.s = __shfl_down_sync(0xffffffffu, p.s, o);
    q.c = __shfl_down_sync(0xffffffffu, p.c, o);
    p = merge(p, q);
  }
  if ((tid & 31) == 0) sh[tid >> 5] = p;
  __syncthreads();
  if (tid < 32) {
    p = tid < TT / 32 ? sh[tid] : Pair{0.0, 0.0};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Pair q;
      q.s = __shfl_down_sync(0xffffffffu, p.s, o);
      q.c = __shfl_down_sync(0xffffffffu, p.c, o);
      p = merge(p, q);
    }
  }
  __syncthreads();
  return p;  // valid in thread 0
}

__global__ void __launch_bounds__(TT) totals_partial(const double* __restrict__ U, const double* __restrict__ dx,
                                                     double* __restrict__ partial) {
  __shared__ Pair sh[TT / 32];
  const int s = blockIdx.x;
  const double vol = dx[s] * dx[s] * dx[s];
  for (int f = 0; f < NF; ++f) {
    Pair p{0.0, 0.0};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int c = threadIdx.x + r * TT;
      const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
      neumaier(p, U[field_offset(s, f) + (size_t)(k + NG) * NP2 + (j + NG) * NP + (i + NG)]);
    }
    p = block_merge(p, sh);
    if (threadIdx.x == 0) {
      partial[((size_t)s * NF + f) * 2 + 0] = vol * p.s;
      partial[((size_t)s * NF + f) * 2 + 1] = vol * p.c;
    }
  }
}

__global__ void __launch_bounds__(TT) totals_final(const double* __restrict__ partial, int n,
                                                   double* __restrict__ totals) {
  __shared__ Pair sh[TT / 32];
  const int f = blockIdx.x;
  Pair p{0.0, 0.0};
  for (int s = threadIdx.x; s < n; s += TT) {
    neumaier(p, partial[((size_t)s * NF + f) * 2 + 0]);
    neumaier(p, partial[((size_t)s * NF + f) * 2 + 1]);
  }
  p = block_merge(p, sh);
  if (threadIdx.x == 0) totals[f] = p.s + p.c;
}

}  // namespace

cudaError_t launch_totals(const double* U, int n, const double* dx, double* partial, double* totals,
                          cudaStream_t st) {
  totals_partial<<<n, TT, 0, st>>>(U, dx, partial);
  totals_final<<<NF, TT, 0, st>>>(partial, n, totals);
  return cudaGetLastError();
}

}  // namespace hydro
