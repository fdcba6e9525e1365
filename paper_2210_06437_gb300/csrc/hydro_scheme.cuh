// hydro_scheme.cuh -- the arithmetic of the finite-volume scheme shared by the
// stage kernels (hydro_stage.cu) and the three-dimensional reconstruction
// (hydro_recon3d.cu): precision traits, FP64 quotients in the plain
// evaluation's rounding, the PPM reconstruction (Colella & Woodward 1984) and
// the central-upwind face flux (Kurganov, Noelle & Petrova 2001).
#pragma once
#include <cuda_runtime.h>

#include "hydro_fp.cuh"
#include "hydro_internal.cuh"

namespace hydro {
namespace {

// ---------------------------------------------------------------------------
// precision traits
// ---------------------------------------------------------------------------

template <typename T>
struct Arith;

template <>
struct Arith<double> {
  // 1/x by Newton-Raphson from the hardware's approximate FP64 reciprocal:
  // r <- r + r (1 - x r) squares the relative error each step, so three
  // steps take even a coarse seed below the final rounding; two FP64 FMAs per
  // step instead of a full IEEE division.  Used for densities
  // and positive signal-speed sums only (finite, normal, non-zero).
  static __device__ __forceinline__ double rcp(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
  }
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
  static __device__ __forceinline__ float from64(double x) { return f64_to_f32(x); }
  static constexpr float tiny = 1e-30f;
};

// ---------------------------------------------------------------------------
// FP64 arithmetic in the reference order.  The FP64 stage evaluates every
// expression of the scheme with the operations, operand order and roundings
// of its plain statement (no contraction into FMAs, IEEE quotients), so its
// results equal those of a straightforward FP64 evaluation bit for bit.  The
// quotients use a correctly rounded reciprocal y = RN(1/b) and Markstein's
// correction q = RN(q0 + RN(a - b q0) y), q0 = RN(a y): the remainder is exact
// in an FMA, and with y within half an ulp of 1/b and q0 within one ulp of a/b
// the corrected q is the correctly rounded a/b (Markstein 1990).  For normal
// operands this is the IEEE quotient at 3 FP64 operations once y is known.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double div_by(double a, double b, double y) {  // RN(a / b), y = RN(1 / b)
  const double q0 = __dmul_rn(a, y);
  const double r = __fma_rn(-q0, b, a);
  return __fma_rn(r, y, q0);
}

template <int C>
__device__ __forceinline__ double div_const(double a) {  // RN(a / C); RN(1 / C) rounded by the compiler
  constexpr double c = (double)C, y = 1.0 / (double)C;
  return div_by(a, c, y);
}

// (a * b) <= 0 as an FP64 product test decides it: from the sign bits, with the
// product formed only where it could underflow to zero (both factors tiny).
__device__ __forceinline__ bool prod_nonpos(double a, double b) {
  constexpr long long MAG = 0x7fffffffffffffffLL;
  const long long ba = __double_as_longlong(a), bb = __double_as_longlong(b);
  const bool by_sign = ((ba & MAG) == 0) || ((bb & MAG) == 0) || ((ba ^ bb) < 0);
  const int ea = (int)((ba >> 52) & 0x7ff), eb = (int)((bb >> 52) & 0x7ff);
  if (!by_sign && ea + eb < 1100) return __dmul_rn(a, b) <= 0.0;
  return by_sign;
}

// x > y for a non-negative, non-NaN y, on the bit patterns (non-negative
// doubles order as their bits; a negative x is never greater)
__device__ __forceinline__ bool gt_nonneg(double x, double y) {
  const long long bx = __double_as_longlong(x);
  return bx >= 0 && bx > __double_as_longlong(y);
}
// -y > x for a non-negative, non-NaN y
__device__ __forceinline__ bool lt_neg(double x, double y) {
  const long long bx = __double_as_longlong(x);
  return bx < 0 && (bx & 0x7fffffffffffffffLL) > __double_as_longlong(y);
}

// ---------------------------------------------------------------------------
// PPM
// ---------------------------------------------------------------------------

// Twice the monotonized-central slope: (qp - qm) limited by four times the
// one-sided differences, zero at a local extremum (CW84 eq. 1.8, scaled by 2,
// which is exact in binary floating point).
template <typename T>
__device__ __forceinline__ T limited_slope2(T qm, T q0, T qp) {
  T dl = q0 - qm;
  T dr = qp - q0;
  T delta = qp - qm;
  if constexpr (sizeof(T) == 4) {
    T m = fabs(delta);
    T l = T(4) * fabs(dl);
    T r = T(4) * fabs(dr);
    m = (l < m) ? l : m;
    m = (r < m) ? r : m;
    // same sign for dl and dr (else 0); then delta has it too (a zero dl or
    // dr already made m zero)
    const unsigned sl = __float_as_uint(dl), sr = __float_as_uint(dr);
    const unsigned keep = ~(unsigned)((int)(sl ^ sr) >> 31);
    return __uint_as_float((__float_as_uint(m) | (sl & 0x80000000u)) & keep);
  } else {
    // FP64 is scarce: the magnitudes are compared as integers (non-negative
    // doubles order as their bit patterns), the sign is taken from the bits and
    // the extremum test dl dr <= 0 from the sign bits (prod_nonpos), leaving
    // three FP64 operations (two differences and 4 dr; 4 dl is the previous
    // cell's 4 dr); every value is exactly twice the plain evaluation's
    // (scaling by 2 commutes with rounding)
    constexpr long long MAG = 0x7fffffffffffffffLL;
    long long m = __double_as_longlong(delta) & MAG;
    const long long l = __double_as_longlong(__dmul_rn(T(4), dl)) & MAG;
    const long long r = __double_as_longlong(__dmul_rn(T(4), dr)) & MAG;
    m = l < m ? l : m;
    m = r < m ? r : m;
    if (prod_nonpos(dl, dr)) return T(0);
    return __longlong_as_double(m | (__double_as_longlong(dl) & ~MAG));
  }
}

// CW84 eq. 1.10: flatten at an extremum, else move the far face so that the
// parabola has no interior extremum.
// FP32: in the differences u = r - a, w = a - l: flat where u w <= 0; with
// D = u + w (= r - l) and E = w - u (= 2 (a - (l + r)/2)), the tests
// (r - l)(a - (l + r)/2) > (r - l)^2 / 6 and its mirror become 3 D E > D^2 and
// -D^2 > 3 D E, and the moved faces are 3a - 2r = a - 2u and 3a - 2l = a + 2w.
// Mirroring (l <-> r) maps (u, w) to (-w, -u): D changes sign, E and D^2 do
// not, so the two tests swap exactly.
// FP64: the plain statement, (r - a)(a - l) <= 0; da = r - l,
// lhs = da (a - (l + r)/2), rhs = da^2 / 6; lhs > rhs moves l to 3a - 2r, else
// -rhs > lhs moves r to 3a - 2l, each operation rounded as written (the sign
// and comparison tests on the bits, rhs >= 0).
template <typename T>
__device__ __forceinline__ void parabola_limit(T a, T& l, T& r) {
  if constexpr (sizeof(T) == 4) {
    const T u = r - a, w = a - l;
    const bool flat = u * w <= T(0);
    const T D = u + w, E = w - u;
    const T X = T(3) * (D * E), Y = D * D;
    const bool lo = X > Y;
    const bool hi = (!lo) && (-Y > X);
    const T nl = lo ? a - T(2) * u : l;
    const T nr = hi ? a + T(2) * w : r;
    l = flat ? a : nl;
    r = flat ? a : nr;
  } else {
    const double u = __dsub_rn(r, a), w = __dsub_rn(a, l);
    if (prod_nonpos(u, w)) {
      l = a;
      r = a;
      return;
    }
    const double da = __dsub_rn(r, l);
    const double lhs = __dmul_rn(da, __dsub_rn(a, __dmul_rn(0.5, __dadd_rn(l, r))));
    const double rhs = div_const<6>(__dmul_rn(da, da));
    const double a3 = __dmul_rn(3.0, a);
    if (gt_nonneg(lhs, rhs))
      l = __dsub_rn(a3, __dmul_rn(2.0, r));
    else if (lt_neg(lhs, rhs))
      r = __dsub_rn(a3, __dmul_rn(2.0, l));
  }
}

// One pencil of 14 values -> face states of faces m+1/2, m = 2..10:
// ul[m-2] = right edge of cell m, ur[m-2] = left edge of cell m+1.
template <typename T>
__device__ __forceinline__ void ppm_pencil(const T (&q)[NP], T (&ul)[NFACE], T (&ur)[NFACE]) {
  T dm[NP];
#pragma unroll
  for (int m = 1; m <= 12; ++m) dm[m] = limited_slope2(q[m - 1], q[m], q[m + 1]);  // 2 x slope
  T face[NP];
  // CW84 eq. 1.6 with limited slopes: (q_m + q_{m+1})/2 - (dm_{m+1} - dm_m)/6;
  // dm holds twice the slopes, so FP64 divides their difference by 12, which
  // rounds as the plain quotient by 6 of the halved difference
#pragma unroll
  for (int m = 1; m <= 11; ++m) {
    if constexpr (sizeof(T) == 4)
      face[m] = T(0.5) * (q[m] + q[m + 1]) - (dm[m + 1] - dm[m]) * T(1.0 / 12.0);
    else
      face[m] = __dsub_rn(__dmul_rn(0.5, __dadd_rn(q[m], q[m + 1])), div_const<12>(__dsub_rn(dm[m + 1], dm[m])));
  }
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

// FP64: u = s_d / rho, e_k = (1/2 ((sx^2 + sy^2) + sz^2)) / rho, e_i = E - e_k
// (tau^gamma below the dual-energy switch), p = (gamma - 1) e_i,
// c = sqrt((gamma p) / rho), every operation rounded as written.
__device__ __forceinline__ void face_eos64(const double (&U)[NF], int d, double gamma, double eta, double& u,
                                           double& p, double& c) {
  const double rho = U[F_RHO], y = __drcp_rn(rho);
  const double sx = U[F_SX], sy = U[F_SX + 1], sz = U[F_SX + 2], E = U[F_EGAS];
  u = div_by(U[F_SX + d], rho, y);
  const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)), __dmul_rn(sz, sz));
  const double ek = div_by(__dmul_rn(0.5, s2), rho, y);
  double ei = __dsub_rn(E, ek);
  if (eta > 0.0 && ei < __dmul_rn(eta, E)) ei = pow(U[F_TAU], gamma);
  p = __dmul_rn(__dsub_rn(gamma, 1.0), ei);
  c = __dsqrt_rn(div_by(__dmul_rn(gamma, p), rho, y));
}

// FP64 numerical flux as the central-upwind formula states it:
// F = ((a+ FL - a- FR) + (a+ a-)(UR - UL)) / (a+ - a-) with the physical
// fluxes FL = U_L u_L (+ p_L on the normal momentum, (E_L + p_L) u_L for the
// energy), the central average (FL + FR)/2 when a+ - a- <= 1e-300.
__device__ __forceinline__ double face_flux64(const double (&UL)[NF], const double (&UR)[NF], int d, double gamma,
                                              double eta, int form, double (&F)[NF]) {
  double uL, pL, cL, uR, pR, cR;
  face_eos64(UL, d, gamma, eta, uL, pL, cL);
  face_eos64(UR, d, gamma, eta, uR, pR, cR);
  double ap, am;
  if (form == 1) {
    const double a = __dadd_rn(fabs(uL), cL), b = __dadd_rn(fabs(uR), cR);
    ap = a > b ? a : b;
    am = -ap;
  } else {
    ap = __dadd_rn(uL, cL);
    const double bp = __dadd_rn(uR, cR);
    if (bp > ap) ap = bp;
    if (0.0 > ap) ap = 0.0;
    am = __dsub_rn(uL, cL);
    const double bm = __dsub_rn(uR, cR);
    if (bm < am) am = bm;
    if (0.0 < am) am = 0.0;
  }
  const double den = __dsub_rn(ap, am);
  const bool central = !(den > 1e-300);
  const double y = central ? 1.0 : __drcp_rn(den);
  const double apam = __dmul_rn(ap, am);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    double fl, fr;
    if (f == F_EGAS) {
      fl = __dmul_rn(__dadd_rn(UL[f], pL), uL);
      fr = __dmul_rn(__dadd_rn(UR[f], pR), uR);
    } else {
      fl = __dmul_rn(UL[f], uL);
      fr = __dmul_rn(UR[f], uR);
      if (f == F_SX + d) {
        fl = __dadd_rn(fl, pL);
        fr = __dadd_rn(fr, pR);
      }
    }
    if (central)
      F[f] = __dmul_rn(0.5, __dadd_rn(fl, fr));
    else
      F[f] = div_by(__dadd_rn(__dsub_rn(__dmul_rn(ap, fl), __dmul_rn(am, fr)),
                              __dmul_rn(apam, __dsub_rn(UR[f], UL[f]))),
                    den, y);
  }
  return ap > -am ? ap : -am;
}

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
// terms on the normal momentum and the energy: algebraically the central-
// upwind flux ((a+ FL - a- FR) + a+ a- (UR - UL)) / (a+ - a-).  Products are
// rounded separately (no contraction) so that mirrored faces give exactly
// negated or equal fluxes.  Returns max(a+, -a-).
template <typename T>
__device__ __forceinline__ T face_flux(const T (&UL)[NF], const T (&UR)[NF], int d, T gamma, T eta, int form,
                                       T (&F)[NF]) {
  if constexpr (sizeof(T) == 8) return face_flux64(UL, UR, d, gamma, eta, form, F);
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

}  // namespace
}  // namespace hydro
