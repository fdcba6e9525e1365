// hydro_totals.cu -- grid totals T_f = sum_s dx_s^3 sum_interior U_f
// (paper Section V-B.1: the diagnostics task forms total mass and other grid
// sums), exact per sub-grid and deterministic.
//
// GB300 runs FP64 arithmetic at about 2 operations per clock per SM, so the
// bulk of the summation uses integer operations instead:
//   pass 1: one warp per (sub-grid, field) reads the 512 interior values,
//           finds their largest binary exponent E and adds the significands
//           as signed 128-bit fixed-point numbers with 63 guard bits below the
//           last bit of a value of exponent E (values more than 63 binades
//           below E keep their leading bits only).  The integer sum is exact
//           and independent of order; it is stored with E (integer work only);
//   pass 2: per field and chunk of sub-grids, one thread per sub-grid turns
//           the integer sum into a double-double scaled by dx^3 (the FP64
//           work, every lane busy), then a Neumaier-compensated sum of these
//           partials in a fixed order;
//   pass 3: per field, the chunk sums combined in a fixed order.
// No atomics anywhere, so the result is bit-reproducible.
#include "hydro_internal.cuh"

namespace hydro {
namespace {

constexpr int TT = 256;
constexpr int CHUNKS = 128;  // sub-grid chunks of pass 2

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

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  double bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

__device__ __forceinline__ Pair merge(Pair a, Pair b) {
  Pair r;
  double e;
  two_sum(a.s, b.s, r.s, e);
  r.c = (a.c + b.c) + e;
  return r;
}

__device__ __forceinline__ Pair warp_merge(Pair p) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Pair q;
    q.s = __shfl_down_sync(0xffffffffu, p.s, o);
    q.c = __shfl_down_sync(0xffffffffu, p.c, o);
    p = merge(p, q);
  }
  return p;  // valid in lane 0
}

// exact value of a signed 128-bit integer times 2^e2 as a double-double
__device__ __forceinline__ void i128_to_dd(__int128 v, int e2, double& hi, double& lo) {
  const bool neg = v < 0;
  const unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const double w3 = ldexp((double)(unsigned)(a >> 96), 96 + e2);
  const double w2 = ldexp((double)(unsigned)(a >> 64), 64 + e2);
  const double w1 = ldexp((double)(unsigned)(a >> 32), 32 + e2);
  const double w0 = ldexp((double)(unsigned)a, e2);
  double s, e1, e2s, e3;
  two_sum(w3, w2, s, e1);
  two_sum(s, w1, s, e2s);
  two_sum(s, w0, s, e3);
  double l = (e1 + e2s) + e3;
  hi = s + l;
  lo = l - (hi - s);
  if (neg) {
    hi = -hi;
    lo = -lo;
  }
}

// pass 1 output per (sub-grid, field): the 128-bit sum (low, high word) and E
// (0x7ff: a value is not finite).
constexpr int PARTIAL_WORDS = 3;

__global__ void __launch_bounds__(TT) totals_subgrid(const double* __restrict__ U, int n,
                                                     unsigned long long* __restrict__ partial) {
  const int gw = blockIdx.x * (TT / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= n * NF) return;
  const int s = gw / NF, f = gw - s * NF;
  const double* base = U + field_offset(s, f) + NG * NP2 + NG * NP + NG;
  unsigned long long b[16];
  unsigned emax = 1;  // zero and subnormals count as exponent 1
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int c = lane + 32 * r;
    b[r] = (unsigned long long)__double_as_longlong(base[(c >> 6) * NP2 + ((c >> 3) & 7) * NP + (c & 7)]);
    const unsigned e = (unsigned)(b[r] >> 52) & 0x7ffu;
    emax = e > emax ? e : emax;
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  __int128 acc = 0;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    unsigned e = (unsigned)(b[r] >> 52) & 0x7ffu;
    unsigned long long m = b[r] & 0x000fffffffffffffull;
    if (e)
      m |= 0x0010000000000000ull;
    else
      e = 1;
    const int sh = 63 - (int)(emax - e);  // bit position of the significand's last bit
    unsigned __int128 F;
    if (sh >= 0)
      F = (unsigned __int128)m << sh;
    else
      F = sh > -64 ? (unsigned __int128)(m >> (-sh)) : (unsigned __int128)0;
    acc += (b[r] >> 63) ? -(__int128)F : (__int128)F;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)acc, o);
    const unsigned long long hi = __shfl_down_sync(0xffffffffu, (unsigned long long)((unsigned __int128)acc >> 64), o);
    acc += (__int128)(((unsigned __int128)hi << 64) | lo);
  }
  if (lane == 0) {
    unsigned long long* o = partial + ((size_t)s * NF + f) * PARTIAL_WORDS;
    o[0] = (unsigned long long)acc;
    o[1] = (unsigned long long)((unsigned __int128)acc >> 64);
    o[2] = emax;
  }
}

// Sub-grid partial dx^3 * sum as a double pair (p, e), p + e the exact value
// rounded to about 2^-106.
__device__ __forceinline__ void subgrid_partial(const unsigned long long* w, double dx, double& p, double& e) {
  const unsigned emax = (unsigned)w[2];
  if (emax == 0x7ffu) {  // a non-finite value: make the total non-finite
    p = __longlong_as_double(0x7ff8000000000000ll);
    e = 0.0;
    return;
  }
  const __int128 acc = (__int128)(((unsigned __int128)w[1] << 64) | w[0]);
  double hi, lo;
  i128_to_dd(acc, (int)emax - 1075 - 63, hi, lo);
  const double v = dx * dx * dx;
  p = hi * v;
  e = fma(hi, v, -p) + lo * v;
}

// pass 2: block (f, chunk) sums the partials of its contiguous range of sub-grids
__global__ void __launch_bounds__(TT) totals_chunks(const unsigned long long* __restrict__ partial,
                                                    const double* __restrict__ dx, int n, double* __restrict__ chunk) {
  __shared__ Pair sh[TT / 32];
  const int f = blockIdx.x, ch = blockIdx.y;
  const int a = (int)((long long)n * ch / CHUNKS), b = (int)((long long)n * (ch + 1) / CHUNKS);
  Pair p{0.0, 0.0};
  for (int s = a + (int)threadIdx.x; s < b; s += TT) {
    double ps, pe;
    subgrid_partial(partial + ((size_t)s * NF + f) * PARTIAL_WORDS, dx[s], ps, pe);
    neumaier(p, ps);
    neumaier(p, pe);
  }
  p = warp_merge(p);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    Pair q = sh[0];
    for (int w = 1; w < TT / 32; ++w) q = merge(q, sh[w]);
    chunk[((size_t)f * CHUNKS + ch) * 2 + 0] = q.s;
    chunk[((size_t)f * CHUNKS + ch) * 2 + 1] = q.c;
  }
}

// pass 3: one warp per field combines the chunk sums
__global__ void totals_final(const double* __restrict__ chunk, double* __restrict__ totals) {
  const int f = blockIdx.x;
  Pair p{0.0, 0.0};
  for (int c = (int)threadIdx.x; c < CHUNKS; c += 32) {
    neumaier(p, chunk[((size_t)f * CHUNKS + c) * 2 + 0]);
    neumaier(p, chunk[((size_t)f * CHUNKS + c) * 2 + 1]);
  }
  p = warp_merge(p);
  if (threadIdx.x == 0) totals[f] = p.s + p.c;
}

}  // namespace

size_t totals_scratch_doubles(int n) { return (size_t)n * NF * PARTIAL_WORDS + (size_t)NF * CHUNKS * 2; }

cudaError_t launch_totals(const double* U, int n, const double* dx, double* scratch, double* totals,
                          cudaStream_t st) {
  unsigned long long* partial = reinterpret_cast<unsigned long long*>(scratch);
  double* chunk = scratch + (size_t)n * NF * PARTIAL_WORDS;
  const int warps = n * NF;
  totals_subgrid<<<(warps + TT / 32 - 1) / (TT / 32), TT, 0, st>>>(U, n, partial);
  totals_chunks<<<dim3(NF, CHUNKS), TT, 0, st>>>(partial, dx, n, chunk);
  totals_final<<<NF, 32, 0, st>>>(chunk, totals);
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
// GPU that loads the library holds its 17.3 MB until the process exits).
// ---------------------------------------------------------------------------

#include <mutex>

#include "hydro.h"

namespace {

static __device__ __align__(256) double g_noalloc_partial[(size_t)HYDRO_TOTALS_NOALLOC_MAX_SUBGRIDS * hydro::NF * 3 +
                                                          (size_t)hydro::NF * 128 * 2];

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
