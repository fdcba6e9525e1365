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

// ---------------------------------------------------------------------------
// Allocation-free totals.
//
// Some callers cannot allocate device memory: code running where cudaMalloc is
// unavailable or forbidden, such as inside a host allocator callback, a
// framework that owns every device allocation, or a process whose memory is
// fully reserved up front.  hydro_totals_noalloc serves them: the caller passes
// the state, the cell widths and the output, and the per-sub-grid partial sums
// live in the fixed array below, which is part of the loaded module (every
// GPU that loads the library holds its 11.5 MB until the process exits).
// ---------------------------------------------------------------------------

#include <mutex>

#include "hydro.h"

namespace {

static __device__ __align__(256) double g_noalloc_partial[(size_t)HYDRO_TOTALS_NOALLOC_MAX_SUBGRIDS * hydro::NF * 2];

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int hydro_totals_noalloc(const double* U, const double* d_dx, int32_t n_subgrids, double* d_totals,
                                    void* stream) {
  if (!U || !d_dx || !d_totals) return HYDRO_ERR_INVALID;
  if (((uintptr_t)U % 16) || ((uintptr_t)d_dx % 8) || ((uintptr_t)d_totals % 8)) return HYDRO_ERR_INVALID;
  if (n_subgrids < 1 || n_subgrids > HYDRO_TOTALS_NOALLOC_MAX_SUBGRIDS) return HYDRO_ERR_INVALID;
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return HYDRO_ERR_CUDA;
  // every partial the final pass reads is written first by the partial pass,
  // so the stale contents of the shared array never reach the result
  if (hydro::launch_totals(U, n_subgrids, d_dx, scratch, d_totals, (cudaStream_t)stream) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  return HYDRO_OK;
}
