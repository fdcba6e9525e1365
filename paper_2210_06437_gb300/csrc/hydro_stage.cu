// hydro_stage.cu -- one Runge-Kutta stage of the octree hydro step on GB300.
//
// Persistent kernel: CTAs pull sub-grid ids from a device work queue (one
// atomic counter per launch), so any number of uneven leaf batches runs in
// one launch.  Per sub-grid and per direction d:
//   A. PPM (Colella & Woodward 1984) of every field along each of the 64
//      pencils, sliding window in registers: one task = (field, pencil);
//      writes the left/right face states of the 9 faces the update needs;
//   B. one task per face: face EOS with dual-energy switch, one-sided
//      (central-upwind, Kurganov-Noelle-Petrova) or symmetric (Kurganov-
//      Tadmor) signal speeds, numerical flux of the 11 fields;
//   C. every thread owns two interior cells and accumulates the flux
//      difference of direction d, in x, y, z order.
// Then U* = U + dt/dx dU and U_out = U0 + beta (U* - U0).  The face signal
// speeds are reduced with warp shuffles and one ordered-bits atomicMax per
// sub-grid (paper Section V-B.1: reconstruct kernel, flux kernel, and the
// global time-step reduction of compute_fluxes).
//
// Two instantiations: T = double (all FP64) and T = float (mixed: FP32
// reconstruction and flux; flux differences accumulated exactly as a float
// pair and the conserved update done in FP64).
#include <cmath>

#include "hydro_internal.cuh"

namespace hydro {
namespace {

constexpr int THREADS = 256;

template <typename T>
struct Arith;

template <>
struct Arith<double> {
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double from64(double x) { return x; }
  static constexpr double tiny = 1e-300;
};

template <>
struct Arith<float> {
  static __device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float pow_(float x, float y) { return __powf(x, y); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float from64(double x) { return __double2float_rn(x); }
  static constexpr float tiny = 1e-30f;
};

// ---------------------------------------------------------------------------
// PPM
// ---------------------------------------------------------------------------

// Monotonized-central slope: (qp - qm)/2 limited by twice the one-sided
// differences, zero at a local extremum (CW84 eq. 1.8).
template <typename T>
__device__ __forceinline__ T limited_slope(T qm, T q0, T qp) {
  T dl = q0 - qm;
  T dr = qp - q0;
  T delta = T(0.5) * (qp - qm);
  T m = fabs(delta);
  T l = T(2) * fabs(dl);
  T r = T(2) * fabs(dr);
  m = (l < m) ? l : m;
  m = (r < m) ? r : m;
  T res = (delta > T(0)) ? m : -m;
  return (dl * dr <= T(0)) ? T(0) : res;
}

// CW84 eq. 1.10: flatten at an extremum, else move the far face so that the
// parabola has no interior extremum.
template <typename T>
__device__ __forceinline__ void parabola_limit(T a, T& l, T& r) {
  bool flat = (r - a) * (a - l) <= T(0);
  T da = r - l;
  T lhs = da * (a - T(0.5) * (l + r));
  T rhs = da * da * T(1.0 / 6.0);
  bool lo = lhs > rhs;
  bool hi = (!lo) && (-rhs > lhs);
  T nl = lo ? T(3) * a - T(2) * r : l;
  T nr = hi ? T(3) * a - T(2) * l : r;
  l = flat ? a : nl;
  r = flat ? a : nr;
}

// One pencil of 14 values -> face states of faces m+1/2, m = 2..10:
// ul[m-2] = right edge of cell m, ur[m-2] = left edge of cell m+1.
template <typename T>
__device__ __forceinline__ void ppm_pencil(const T (&q)[NP], T (&ul)[NFACE], T (&ur)[NFACE]) {
  T dm[NP];
#pragma unroll
  for (int m = 1; m <= 12; ++m) dm[m] = limited_slope(q[m - 1], q[m], q[m + 1]);
  T face[NP];
#pragma unroll
  for (int m = 1; m <= 11; ++m) face[m] = T(0.5) * (q[m] + q[m + 1]) - (dm[m + 1] - dm[m]) * T(1.0 / 6.0);
#pragma unroll
  for (int m = 2; m <= 11; ++m) {
    T l = face[m - 1], r = face[m];
    parabola_limit(q[m], l, r);
    if (m <= 10) ul[m - 2] = r;
    if (m >= 3) ur[m - 3] = l;
  }
}

// ---------------------------------------------------------------------------
// face EOS and flux
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void face_eos(const T (&U)[NF], int d, T gamma, T eta, T& u, T& p, T& c) {
  T inv = Arith<T>::rcp(U[F_RHO]);
  T sx = U[F_SX], sy = U[F_SX + 1], sz = U[F_SX + 2];
  u = U[F_SX + d] * inv;
  T ek = T(0.5) * ((sx * sx + sy * sy) + sz * sz) * inv;
  T ei = U[F_EGAS] - ek;
  if (eta > T(0) && ei < eta * U[F_EGAS]) ei = Arith<T>::pow_(U[F_TAU], gamma);
  p = (gamma - T(1)) * ei;
  c = Arith<T>::sqrt_(gamma * p * inv);
}

// Numerical flux written as F = wl*UL + wr*UR for every field plus pressure
// terms on the normal momentum and the energy; algebraically the central-
// upwind flux ((a+ FL - a- FR) + a+ a- (UR - UL)) / (a+ - a-).  Products are
// rounded separately (no contraction) so that mirrored faces give exactly
// negated or equal fluxes.
template <typename T>
__device__ __forceinline__ T face_flux(const T (&UL)[NF], const T (&UR)[NF], int d, T gamma, T eta, int form,
                                       T (&F)[NF]) {
  using A = Arith<T>;
  T uL, pL, cL, uR, pR, cR;
  face_eos(UL, d, gamma, eta, uL, pL, cL);
  face_eos(UR, d, gamma, eta, uR, pR, cR);
  T ap, am;
  if (form == 1) {
    T a = fmax(fabs(uL) + cL, fabs(uR) + cR);
    ap = a;
    am = -a;
  } else {
    ap = fmax(fmax(uL + cL, uR + cR), T(0));
    am = fmin(fmin(uL - cL, uR - cR), T(0));
  }
  T den = ap - am;
  T wl, wr, pm, pe;
  if (den > A::tiny) {
    T r = A::rcp(den);
    wl = A::mul(A::mul(ap, uL - am), r);
    wr = A::mul(A::mul(am, ap - uR), r);
    pm = A::mul(A::add(A::mul(ap, pL), -A::mul(am, pR)), r);
    pe = A::mul(A::add(A::mul(ap, A::mul(pL, uL)), -A::mul(am, A::mul(pR, uR))), r);
  } else {
    wl = T(0.5) * uL;
    wr = T(0.5) * uR;
    pm = T(0.5) * (pL + pR);
    pe = T(0.5) * A::add(A::mul(pL, uL), A::mul(pR, uR));
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) F[f] = A::add(A::mul(wl, UL[f]), A::mul(wr, UR[f]));
  F[F_SX + d] = A::add(F[F_SX + d], pm);
  F[F_EGAS] = A::add(F[F_EGAS], pe);
  return fmax(ap, -am);
}

// ---------------------------------------------------------------------------
// accumulators
// ---------------------------------------------------------------------------

template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double v;
  __device__ __forceinline__ void set_diff(double lo, double hi) { v = lo - hi; }
  __device__ __forceinline__ void add_diff(double lo, double hi) { v = v + (lo - hi); }
  __device__ __forceinline__ double value() const { return v; }
};

// Float pair (hi + lo) carrying the flux-difference sum exactly enough for
// conservation to FP64 round-off: error-free TwoSum (Knuth) of each term.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bp = __fadd_rn(s, -a);
  float ap = __fadd_rn(s, -bp);
  e = __fadd_rn(__fadd_rn(a, -ap), __fadd_rn(b, -bp));
}

template <>
struct Acc<float> {
  float hi, lo;
  __device__ __forceinline__ void set_diff(float a, float b) { two_sum(a, -b, hi, lo); }
  __device__ __forceinline__ void add_diff(float a, float b) {
    float d, e, s, t;
    two_sum(a, -b, d, e);
    two_sum(hi, d, s, t);
    t = __fadd_rn(t, __fadd_rn(lo, e));
    hi = __fadd_rn(s, t);
    lo = __fadd_rn(t, -__fadd_rn(hi, -s));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ bool finite64(double v) {
  return (((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (w > v || w != w) ? w : v;
  }
  return v;
}

template <typename T>
__global__ void __launch_bounds__(THREADS, 2) stage_kernel(const StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* fsl = reinterpret_cast<T*>(smem_raw);  // [NF][576] left states, then fluxes
  T* fsr = fsl + NF * FACES_DIR;             // [NF][576] right states
  __shared__ int s_item;
  __shared__ double s_red[THREADS / 32];

  const int tid = threadIdx.x;
  const T gamma = T(a.gamma), eta = T(a.eta);
  const double dt = a.dt_dev ? *a.dt_dev : a.dt;
  int bad = 0;

  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= a.n_items) break;
    const int s = a.ids[item];
    if (s < 0 || s >= a.n_sub) {
      if (tid == 0) atomicOr(a.err, ERRBIT_BAD_ID);
      __syncthreads();
      continue;
    }
    const double* Us = a.Uin + field_offset(s, 0);
    Acc<T> acc[2][NF];
    T amax = T(0);

#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      // pencil p = t2*8 + t1 -> (i,j,k) strides of the transverse and normal axes
      const int sn = d == 0 ? 1 : (d == 1 ? NP : NP2);
      const int s1 = d == 0 ? NP : 1;
      const int s2 = d == 2 ? NP : NP2;
      // A: PPM, one (field, pencil) task per thread iteration
#pragma unroll 1
      for (int task = tid; task < NF * NPEN; task += THREADS) {
        const int f = task / NPEN, p = task % NPEN;
        const double* src = Us + (size_t)f * NP3 + (NG + (p & 7)) * s1 + (NG + (p >> 3)) * s2;
        T q[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) q[m] = Arith<T>::from64(src[m * sn]);
        T ul[NFACE], ur[NFACE];
        ppm_pencil(q, ul, ur);
#pragma unroll
        for (int m = 0; m < NFACE; ++m) {
          fsl[f * FACES_DIR + p * NFACE + m] = ul[m];
          fsr[f * FACES_DIR + p * NFACE + m] = ur[m];
        }
      }
      __syncthreads();
      // B: one face per thread iteration
#pragma unroll 1
      for (int fc = tid; fc < FACES_DIR; fc += THREADS) {
        T UL[NF], UR[NF], F[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          UL[f] = fsl[f * FACES_DIR + fc];
          UR[f] = fsr[f * FACES_DIR + fc];
        }
        T sp = face_flux(UL, UR, d, gamma, eta, a.form, F);
        amax = (sp > amax || sp != sp) ? sp : amax;
#pragma unroll
        for (int f = 0; f < NF; ++f) fsl[f * FACES_DIR + fc] = F[f];
      }
      __syncthreads();
      // C: flux differences of direction d for the two owned cells
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int c = tid + r * THREADS;
        const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
        const int p = d == 0 ? (k * 8 + j) : (d == 1 ? (k * 8 + i) : (j * 8 + i));
        const int id = d == 0 ? i : (d == 1 ? j : k);
        const int base = p * NFACE + id;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          T lo = fsl[f * FACES_DIR + base], hi = fsl[f * FACES_DIR + base + 1];
          if (d == 0)
            acc[r][f].set_diff(lo, hi);
          else
            acc[r][f].add_diff(lo, hi);
        }
      }
      __syncthreads();
    }

    // update of the owned cells
    const double lam = dt / a.dx[s];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int c = tid + r * THREADS;
      const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
      const size_t cell = (size_t)(k + NG) * NP2 + (j + NG) * NP + (i + NG);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const size_t o = field_offset(s, f) + cell;
        double ustar = fma(lam, acc[r][f].value(), a.Uin[o]);
        double v = ustar;
        if (a.beta != 1.0) {
          double u0 = a.U0[o];
          v = fma(a.beta, ustar - u0, u0);
        }
        a.Uout[o] = v;
        bad |= !finite64(v) || (f == F_RHO && !(v > 0.0));
      }
    }

    // max signal speed of this sub-grid
    double m = warp_max((double)amax);
    if ((tid & 31) == 0) s_red[tid >> 5] = m;
    __syncthreads();
    if (tid < 32) {
      double v = tid < THREADS / 32 ? s_red[tid] : 0.0;
      v = warp_max(v);
      if (tid == 0) {
        const unsigned long long mask = 0x7fffffffffffffffull;
        atomicMax(&a.max_speed[0], (unsigned long long)__double_as_longlong(v) & mask);
        atomicMax(&a.max_speed[1], (unsigned long long)__double_as_longlong(v / a.dx[s]) & mask);
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(a.err, ERRBIT_NONFINITE);
}

template <typename T>
size_t stage_smem() {
  return sizeof(T) * 2 * NF * FACES_DIR;
}

template <typename T>
cudaError_t launch(const StageArgs& a, int grid, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)stage_smem<T>());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  stage_kernel<T><<<grid, THREADS, stage_smem<T>(), st>>>(a);
  return cudaGetLastError();
}

template <typename T>
int blocks_per_sm() {
  int n = 0;
  cudaFuncSetAttribute(stage_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_smem<T>());
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<T>, THREADS, stage_smem<T>()) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace

cudaError_t launch_stage_fp64(const StageArgs& a, int grid, cudaStream_t st) { return launch<double>(a, grid, st); }
cudaError_t launch_stage_mixed(const StageArgs& a, int grid, cudaStream_t st) { return launch<float>(a, grid, st); }
int stage_blocks_per_sm_fp64() { return blocks_per_sm<double>(); }
int stage_blocks_per_sm_mixed() { return blocks_per_sm<float>(); }

}  // namespace hydro
