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
#include "hydro_sums.cuh"

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
// (0x7ff: a value is not finite), see hydro_sums.cuh.

// Per-cell quantity q of sub-grid s at interior cell c = (k*8 + j)*8 + i.
// Totals: the 11 fields.
struct FieldQ {
  static constexpr int NQ = NF;
  const double* U;
  __device__ __forceinline__ double operator()(int s, int q, int c) const {
    return U[field_offset(s, q) + (size_t)((c >> 6) + NG) * NP2 + (((c >> 3) & 7) + NG) * NP + ((c & 7) + NG)];
  }
};

// Diagnostics (the paper's diagnostics task, Section V-B.1): with the cell
// centre x = o + (i + 1/2) dx (each coordinate rounded as o + ((i + 1/2) * dx)),
//   q0 rho; q1..3 r x s (each product rounded on its own); q4 rho X1 and
//   q5..7 rho X1 * (x, y, z) (star 1, scalar field 6); q8..11 likewise for
//   star 2 (field 7).
struct DiagQ {
  static constexpr int NQ = 12;
  const double* U;
  const double* origin;  // [n][3]
  const double* dx;
  __device__ __forceinline__ double at(int s, int f, int c) const {
    return U[field_offset(s, f) + (size_t)((c >> 6) + NG) * NP2 + (((c >> 3) & 7) + NG) * NP + ((c & 7) + NG)];
  }
  __device__ __forceinline__ double coord(int s, int a, int ic) const {
    return __dadd_rn(origin[3 * (size_t)s + a], __dmul_rn((double)ic + 0.5, dx[s]));
  }
  __device__ __forceinline__ double operator()(int s, int q, int c) const {
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    if (q == 0) return at(s, F_RHO, c);
    if (q <= 3) {
      const int a = q - 1, b = (a + 1) % 3, e = (a + 2) % 3;  // (r x s)_a = r_b s_e - r_e s_b
      const int ib = b == 0 ? i : (b == 1 ? j : k), ie = e == 0 ? i : (e == 1 ? j : k);
      return __dsub_rn(__dmul_rn(coord(s, b, ib), at(s, F_SX + e, c)), __dmul_rn(coord(s, e, ie), at(s, F_SX + b, c)));
    }
    const int star = (q - 4) >> 2, m = (q - 4) & 3;
    const double w = at(s, 6 + star, c);
    if (m == 0) return w;
    const int a = m - 1, ia = a == 0 ? i : (a == 1 ? j : k);
    return __dmul_rn(w, coord(s, a, ia));
  }
};

template <class Q>
__global__ void __launch_bounds__(TT) totals_subgrid(const Q Qf, int n, unsigned long long* __restrict__ partial) {
  constexpr int NQ = Q::NQ;
  const int gw = blockIdx.x * (TT / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= n * NQ) return;
  const int s = gw / NQ, f = gw - s * NQ;
  warp_exact_sum([&](int r) { return Qf(s, f, lane + 32 * r); }, partial + ((size_t)s * NQ + f) * PARTIAL_WORDS);
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
                                                    const double* __restrict__ dx, int n, int nq,
                                                    double* __restrict__ chunk) {
  __shared__ Pair sh[TT / 32];
  const int f = blockIdx.x, ch = blockIdx.y;
  const int a = (int)((long long)n * ch / CHUNKS), b = (int)((long long)n * (ch + 1) / CHUNKS);
  Pair p{0.0, 0.0};
  for (int s = a + (int)threadIdx.x; s < b; s += TT) {
    double ps, pe;
    subgrid_partial(partial + ((size_t)s * nq + f) * PARTIAL_WORDS, dx[s], ps, pe);
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

// diagnostics: centres of mass from the 12 sums (0 where a star has no mass)
__global__ void diag_finish(const double* __restrict__ T, double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= DiagQ::NQ) return;
  if (q < 4 || q == 4 || q == 8) {
    out[q] = T[q];
  } else {
    const double m = T[q < 8 ? 4 : 8];
    out[q] = m != 0.0 ? __ddiv_rn(T[q], m) : 0.0;
  }
}

template <class Q>
void enqueue_sums(const Q& Qf, int n, const double* dx, double* scratch, double* sums, cudaStream_t st) {
  constexpr int NQ = Q::NQ;
  unsigned long long* partial = reinterpret_cast<unsigned long long*>(scratch);
  double* chunk = scratch + (size_t)n * NQ * PARTIAL_WORDS;
  const int warps = n * NQ;
  totals_subgrid<Q><<<(warps + TT / 32 - 1) / (TT / 32), TT, 0, st>>>(Qf, n, partial);
  totals_chunks<<<dim3(NQ, CHUNKS), TT, 0, st>>>(partial, dx, n, NQ, chunk);
  totals_final<<<NQ, 32, 0, st>>>(chunk, sums);
}

}  // namespace

size_t totals_scratch_doubles(int n) {
  return (size_t)n * DiagQ::NQ * PARTIAL_WORDS + (size_t)DiagQ::NQ * CHUNKS * 2;  // enough for either
}

cudaError_t launch_totals(const double* U, int n, const double* dx, double* scratch, double* totals,
                          cudaStream_t st) {
  enqueue_sums(FieldQ{U}, n, dx, scratch, totals, st);
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(const double* U, const double* origin, int n, const double* dx, double* scratch,
                               double* sums, double* out, cudaStream_t st) {
  enqueue_sums(DiagQ{U, origin, dx}, n, dx, scratch, sums, st);
  diag_finish<<<1, 32, 0, st>>>(sums, out);
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

// Device address of the scratch array on the current device.  The host-side
// name of the array is only a stand-in, so the address is looked up with the
// device current.  It is looked up again on every call whose stream is not
// being captured (cheap, and correct after a device reset reloads the module);
// a captured call reuses the last address found on that device.
cudaError_t noalloc_scratch(cudaStream_t st, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_noalloc_ptr[dev]) {
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
  if (noalloc_scratch((cudaStream_t)stream, &scratch) != cudaSuccess) return HYDRO_ERR_CUDA;
  // every partial the final pass reads is written first by the partial pass,
  // so the stale contents of the shared array never reach the result
  if (hydro::launch_totals(U, n_subgrids, d_dx, scratch, d_totals, (cudaStream_t)stream) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  return HYDRO_OK;
}
