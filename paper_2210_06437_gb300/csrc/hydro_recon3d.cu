// hydro_recon3d.cu -- one Runge-Kutta stage with the three-dimensional
// reconstruction and Simpson face quadrature (grids of one level; FP64, and
// mixed precision).
//
// The paper names a full three-dimensional reconstruction (Section IV-C) and a
// flux kernel that integrates over each face with a Newton-Cotes rule
// (Section V-B.1), printing neither.  The reading built here:
//   1. PPM along the face normal gives, for every face, its left and right
//      states as averages over the face (the stage kernel's reconstruction);
//   2. across the face, the face averages of the 3 x 3 faces around it give,
//      per state and field, the tensor product of the parabolas with those
//      three-cell averages (first along the face's first transverse axis, then
//      along its second), evaluated at the 3 x 3 Simpson points (transverse
//      offsets -1/2, 0, +1/2 of the face width);
//   3. each parabola is limited: constant at a local extremum of its three
//      averages; the line with the monotonized-central slope where an edge
//      value leaves the range of the neighbouring averages or the centre value
//      the range of the edge values;
//   4. the central-upwind flux at each point, combined with the Simpson
//      weights (1, 4, 1)/6 along each transverse axis, outer points first.
// T = double: every operation is rounded as the plain FP64 statement rounds it
// (no contraction, correctly rounded quotients), so the stage equals a plain
// evaluation of that reading bit for bit.  T = float (mixed precision): the
// FP64 state rounded to FP32 as for the shadows, the reconstruction, the
// transverse parabolas, the point fluxes and the Simpson sums in FP32, the
// flux differences as exact FP32 pairs and the update in FP64.
//
// Three launches per stage, each with one CTA per (item, direction[, plane]):
//   faces   PPM of the 10 x 10 pencils along d around the sub-grid (their
//           cells read from the sub-grid and its face, edge and corner
//           neighbours, found by hopping across faces in x, y, z order;
//           outflow at the domain boundary) -> face averages in scratch;
//   flux    per face plane: point states (step 2-3) in shared memory, the 9
//           point fluxes, the Simpson sums -> face fluxes in scratch, and the
//           plane's largest point speed -> the global maximum;
//   update  U* = U_in + dt/dx dU, U_out = U0 + beta (U* - U0).
// Scratch (per item): face averages [3][2][11][9][100], fluxes [3][11][9][64].
#include <mutex>

#include "hydro_internal.cuh"
#include "hydro_recon3d.cuh"
#include "hydro_scheme.cuh"

namespace hydro {
namespace {

constexpr int R3_THREADS = 128;
constexpr int TP = NX + 2;           // pencils per transverse axis around a sub-grid (-1 .. 8)
constexpr int NPEN3 = TP * TP;       // 100
constexpr int QS = NP + 1;           // shared-memory stride of a pencil
constexpr int NQ = 9;                // Simpson points per face
constexpr size_t FA_DIR = (size_t)2 * NF * NFACE * NPEN3;
constexpr size_t FL_DIR = (size_t)NF * NFACE * NPEN;

// The cell at padded coordinates (i, j, k) of sub-grid s, for any cell of the
// padded cube: each coordinate outside the interior moves to the neighbour
// across that face (x, then y, then z), or to the nearest interior cell at the
// domain boundary.  Returns the element offset of field 0 of that cell.
__device__ __forceinline__ long long full_cell_offset(const int32_t* __restrict__ nb, int s, int i, int j, int k) {
  int c[3] = {i, j, k};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (c[a] >= NG && c[a] < NG + NX) continue;
    const int side = c[a] >= NG + NX ? 1 : 0;
    const int n = __ldg(nb + ((size_t)s * 6 + 2 * a + side) * 4);
    if (n < 0) {
      c[a] = side ? NG + NX - 1 : NG;
    } else {
      s = n;
      c[a] += side ? -NX : NX;
    }
  }
  return (long long)s * NF * NP3 + (c[2] * NP + c[1]) * NP + c[0];
}

// Step 1: face averages of the pencils along d.  fa[item][d][side][f][m][p]:
// side 0 the right edge of cell m + 2 (the left state of face m + 2 + 1/2),
// side 1 the left edge of cell m + 3; p = (t2 + 1) * 10 + (t1 + 1) for the
// pencils at interior transverse coordinates t1, t2 = -1 .. 8.
// (Loading field f + 1 into registers during field f's PPM was measured: on
// the L2-resident 64^3 box it was slower, 129 against 118 us, its registers
// lowering the occupancy; on the 128^3 box the mixed stage took 3.11 against
// 3.19 ms, within the run-to-run spread.  The simpler form stays.)
template <typename T>
__global__ void __launch_bounds__(R3_THREADS) recon3d_faces(Recon3dArgs a) {
  __shared__ T q[NPEN3 * QS];
  __shared__ long long src[NPEN3 * NP];
  const int t = blockIdx.x, d = blockIdx.y, tid = threadIdx.x;
  const int s = a.ids ? (a.ids[t] & ~ITEM_FLUX_ONLY) : t;
  if (s < 0 || s >= a.n_sub) {
    if (tid == 0) atomicOr(a.err, ERRBIT_BAD_ID);
    return;
  }
  for (int e = tid; e < NPEN3 * NP; e += R3_THREADS) {
    const int p = e / NP, m = e - p * NP;
    const int a1 = p % TP + NG - 1, a2 = p / TP + NG - 1;
    const int i = d == 0 ? m : a1, j = d == 1 ? m : (d == 0 ? a1 : a2), k = d == 2 ? m : a2;
    src[e] = full_cell_offset(a.nb, s, i, j, k);
  }
  T* out = reinterpret_cast<T*>(a.fa) + (size_t)t * 3 * FA_DIR + d * FA_DIR;
  for (int f = 0; f < NF; ++f) {
    __syncthreads();  // src written / the previous field's pencils read
    for (int e = tid; e < NPEN3 * NP; e += R3_THREADS) {
      const int p = e / NP, m = e - p * NP;
      q[p * QS + m] = Arith<T>::from64(__ldg(a.Uin + src[e] + (long long)f * NP3));
    }
    __syncthreads();
    if (tid < NPEN3) {
      T v[NP], ul[NFACE], ur[NFACE];
#pragma unroll
      for (int m = 0; m < NP; ++m) v[m] = q[tid * QS + m];
      ppm_pencil<T>(v, ul, ur);
#pragma unroll
      for (int m = 0; m < NFACE; ++m) {
        out[((size_t)(0 * NF + f) * NFACE + m) * NPEN3 + tid] = ul[m];
        out[((size_t)(1 * NF + f) * NFACE + m) * NPEN3 + tid] = ur[m];
      }
    }
  }
}

// a * b < 0 for finite a, b, as the FP64 product decides it: from the sign
// bits (different signs, neither zero), with the product formed only where it
// could underflow to zero (both factors tiny).
__device__ __forceinline__ bool prod_neg(double a, double b) {
  constexpr long long MAG = 0x7fffffffffffffffLL;
  const long long ba = __double_as_longlong(a), bb = __double_as_longlong(b);
  if ((ba ^ bb) >= 0 || (ba & MAG) == 0 || (bb & MAG) == 0) return false;
  const int ea = (int)((ba >> 52) & 0x7ff), eb = (int)((bb >> 52) & 0x7ff);
  if (ea + eb < 1100) return __dmul_rn(a, b) < 0.0;
  return true;
}

// Step 2-3 for three averages am, a0, ap of neighbouring cells (width 1):
// the limited parabola's values at -1/2, 0, +1/2 of the centre cell.
//   parabola: d1 = ap - am, d2 = (ap + am) - 2 a0,
//     lo = (a0 + d2/12) - d1/4, hi = (a0 + d2/12) + d1/4, mid = a0 - d2/24;
//   constant a0 where (ap - a0)(a0 - am) <= 0;
//   the line a0 -+ sl/2 (sl the monotonized-central slope: sign of a0 - am,
//     magnitude min(|d1|/2, 2|a0 - am|, 2|ap - a0|)) where
//     (lo - am)(a0 - lo) < 0, (hi - a0)(ap - hi) < 0 or (mid - lo)(hi - mid) < 0.
// This form rounds every operation as written; the fast form below calls it
// only for values near the bottom of the normal range.
__device__ __noinline__ void transverse_points_plain(double am, double a0, double ap, double& lo, double& mid,
                                                     double& hi) {
  if (__dmul_rn(__dsub_rn(ap, a0), __dsub_rn(a0, am)) <= 0.0) {
    lo = a0;
    mid = a0;
    hi = a0;
    return;
  }
  const double d1 = __dsub_rn(ap, am);
  const double d2 = __dsub_rn(__dadd_rn(ap, am), __dmul_rn(2.0, a0));
  const double base = __dadd_rn(a0, div_const<12>(d2));
  const double q4 = __dmul_rn(d1, 0.25);
  double l = __dsub_rn(base, q4);
  double h = __dadd_rn(base, q4);
  double c = __dsub_rn(a0, div_const<24>(d2));
  const bool outside = __dmul_rn(__dsub_rn(l, am), __dsub_rn(a0, l)) < 0.0 ||
                       __dmul_rn(__dsub_rn(h, a0), __dsub_rn(ap, h)) < 0.0 ||
                       __dmul_rn(__dsub_rn(c, l), __dsub_rn(h, c)) < 0.0;
  if (outside) {
    const double half = __dmul_rn(0.5, __dmul_rn(0.5, limited_slope2<double>(am, a0, ap)));
    l = __dsub_rn(a0, half);
    h = __dadd_rn(a0, half);
    c = a0;
  }
  lo = l;
  mid = c;
  hi = h;
}

// The same values with the tests on the bits (off the FP64 pipe), every
// candidate formed and the result selected (the lanes of a warp do not
// diverge), and two exact rewritings while d1/4 and d2/12 are well inside the
// normal range (else, or for a zero d2/12 from a non-zero d2, the plain form):
//   d2/24 = RN(d2/12) / 2, and
//   sl/2 = min(|d1|/4, |a0 - am|, |ap - a0|) with the sign of a0 - am, d1/4
//   being the quarter that the parabola already uses.
__device__ __forceinline__ void transverse_points(double am, double a0, double ap, double& lo, double& mid,
                                                  double& hi) {
  constexpr long long MAG = 0x7fffffffffffffffLL;
  const double dl = __dsub_rn(a0, am), dr = __dsub_rn(ap, a0);
  const double d1 = __dsub_rn(ap, am);
  const double d2 = __dsub_rn(__dadd_rn(ap, am), __dmul_rn(2.0, a0));
  const double q12 = div_const<12>(d2);
  const double q4 = __dmul_rn(d1, 0.25);
  const long long b12 = __double_as_longlong(q12), b4 = __double_as_longlong(q4);
  const bool ok12 = ((b12 >> 52) & 0x7ff) > 2 || (__double_as_longlong(d2) & MAG) == 0;
  const bool ok4 = ((b4 >> 52) & 0x7ff) > 2 || (__double_as_longlong(d1) & MAG) == 0;
  if (!(ok12 && ok4)) {
    transverse_points_plain(am, a0, ap, lo, mid, hi);
    return;
  }
  const double base = __dadd_rn(a0, q12);
  const double l = __dsub_rn(base, q4);
  const double h = __dadd_rn(base, q4);
  const double c = __dsub_rn(a0, __dmul_rn(q12, 0.5));
  const bool outside = prod_neg(__dsub_rn(l, am), __dsub_rn(a0, l)) || prod_neg(__dsub_rn(h, a0), __dsub_rn(ap, h)) ||
                       prod_neg(__dsub_rn(c, l), __dsub_rn(h, c));
  long long m = b4 & MAG;
  const long long ml = __double_as_longlong(dl) & MAG, mr = __double_as_longlong(dr) & MAG;
  m = ml < m ? ml : m;
  m = mr < m ? mr : m;
  const double half = __longlong_as_double(m | (__double_as_longlong(dl) & ~MAG));
  const bool flat = prod_nonpos(dr, dl);
  lo = flat ? a0 : (outside ? __dsub_rn(a0, half) : l);
  hi = flat ? a0 : (outside ? __dadd_rn(a0, half) : h);
  mid = (flat || outside) ? a0 : c;
}

// FP32 (mixed precision): the same limited parabola, each product and sum
// rounded separately (no contraction, so mirror images stay exact), d2/12 and
// d2/24 as products with the rounded reciprocals, the half-slope as
// min(|d1|/4, |a0 - am|, |ap - a0|) with the sign of a0 - am.
__device__ __forceinline__ void transverse_points(float am, float a0, float ap, float& lo, float& mid, float& hi) {
  const float dl = __fsub_rn(a0, am), dr = __fsub_rn(ap, a0);
  const float d1 = __fsub_rn(ap, am);
  const float d2 = __fsub_rn(__fadd_rn(ap, am), __fmul_rn(2.0f, a0));
  const float q12 = __fmul_rn(d2, 1.0f / 12.0f);
  const float q4 = __fmul_rn(d1, 0.25f);
  const float base = __fadd_rn(a0, q12);
  const float l = __fsub_rn(base, q4);
  const float h = __fadd_rn(base, q4);
  const float c = __fsub_rn(a0, __fmul_rn(d2, 1.0f / 24.0f));
  const bool outside = __fmul_rn(__fsub_rn(l, am), __fsub_rn(a0, l)) < 0.0f ||
                       __fmul_rn(__fsub_rn(h, a0), __fsub_rn(ap, h)) < 0.0f ||
                       __fmul_rn(__fsub_rn(c, l), __fsub_rn(h, c)) < 0.0f;
  const float mag = fminf(fabsf(q4), fminf(fabsf(dl), fabsf(dr)));
  const float half = copysignf(mag, dl);
  const bool flat = __fmul_rn(dr, dl) <= 0.0f;
  lo = flat ? a0 : (outside ? __fsub_rn(a0, half) : l);
  hi = flat ? a0 : (outside ? __fadd_rn(a0, half) : h);
  mid = (flat || outside) ? a0 : c;
}

// The Simpson sum ((F0 + F2) + 4 F1) / 6: FP64 with the correctly rounded
// quotient, FP32 with the product by the rounded reciprocal.
__device__ __forceinline__ double simpson(double f0, double f1, double f2) {
  return div_const<6>(__dadd_rn(__dadd_rn(f0, f2), __dmul_rn(4.0, f1)));
}
__device__ __forceinline__ float simpson(float f0, float f1, float f2) {
  return __fmul_rn(__fadd_rn(__fadd_rn(f0, f2), __fmul_rn(4.0f, f1)), 1.0f / 6.0f);
}

template <typename T>
struct FluxSmem {
  T P[2][NPEN][NQ][NF];  // point states [side][face][q2 * 3 + q1][f]; then the point fluxes in P[0]
  unsigned long long red[R3_THREADS / 32];
};

// Steps 2-4 for the 64 faces of plane m (faces m + 2 + 1/2 along D) of item t.
template <typename T, int D>
__device__ __forceinline__ void flux_plane(const Recon3dArgs& a, FluxSmem<T>& sm, int t, int s, int m) {
  constexpr int d = D;
  const int tid = threadIdx.x;
  const T* fa = reinterpret_cast<const T*>(a.fa) + (size_t)t * 3 * FA_DIR + d * FA_DIR;
  // point states: one unit per (side, field, t1, half of the face column):
  // the row parabolas (along t1) of the 6 pencil rows that the 4 faces
  // t2 = 4 half .. 4 half + 3 read, then each face's 3 column parabolas
  for (int e = tid; e < 2 * NF * NX * 2; e += R3_THREADS) {
    const int t1 = e & 7, half = (e >> 3) & 1, sf = e >> 4, f = sf % NF, side = sf / NF;
    const T* A = fa + ((size_t)(side * NF + f) * NFACE + m) * NPEN3 + 4 * half * TP + t1;
    T rows[6][3];  // [row - 4 half][q1]
#pragma unroll
    for (int r = 0; r < 6; ++r)
      transverse_points(__ldg(A + r * TP), __ldg(A + r * TP + 1), __ldg(A + r * TP + 2), rows[r][0], rows[r][1],
                        rows[r][2]);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int p = (4 * half + c) * NX + t1;
#pragma unroll
      for (int q1 = 0; q1 < 3; ++q1) {
        T lo, mid, hi;
        transverse_points(rows[c][q1], rows[c + 1][q1], rows[c + 2][q1], lo, mid, hi);
        sm.P[side][p][0 * 3 + q1][f] = lo;
        sm.P[side][p][1 * 3 + q1][f] = mid;
        sm.P[side][p][2 * 3 + q1][f] = hi;
      }
    }
  }
  __syncthreads();
  // point fluxes: one unit per (face, point); the flux overwrites the left state
  T amax = T(0);
  for (int e = tid; e < NPEN * NQ; e += R3_THREADS) {
    const int p = e / NQ, qq = e - p * NQ;
    T UL[NF], UR[NF], F[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      UL[f] = sm.P[0][p][qq][f];
      UR[f] = sm.P[1][p][qq][f];
    }
    const T sp = face_flux<T>(UL, UR, d, T(a.gamma), T(a.eta), a.form, F);
    amax = (sp > amax || sp != sp) ? sp : amax;  // a NaN speed sticks
#pragma unroll
    for (int f = 0; f < NF; ++f) sm.P[0][p][qq][f] = F[f];
  }
  __syncthreads();
  // Simpson sums: one unit per (field, face)
  T* fl = reinterpret_cast<T*>(a.fl) + (size_t)t * 3 * FL_DIR + d * FL_DIR;
  for (int e = tid; e < NF * NPEN; e += R3_THREADS) {
    const int p = e & (NPEN - 1), f = e >> 6;
    T row[3];
#pragma unroll
    for (int q2 = 0; q2 < 3; ++q2)
      row[q2] = simpson(sm.P[0][p][q2 * 3 + 0][f], sm.P[0][p][q2 * 3 + 1][f], sm.P[0][p][q2 * 3 + 2][f]);
    fl[((size_t)f * NFACE + m) * NPEN + p] = simpson(row[0], row[1], row[2]);
  }
  // the plane's largest point speed (non-negative values order as their bits)
  unsigned long long bits = (unsigned long long)__double_as_longlong((double)amax) & 0x7fffffffffffffffull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = w > bits ? w : bits;
  }
  if ((tid & 31) == 0) sm.red[tid >> 5] = bits;
  __syncthreads();
  if (tid == 0) {
    unsigned long long b = 0;
#pragma unroll
    for (int w = 0; w < R3_THREADS / 32; ++w) b = sm.red[w] > b ? sm.red[w] : b;
    const double v = __longlong_as_double((long long)b);
    const unsigned long long mask = 0x7fffffffffffffffull;
    atomicMax(&a.max_speed[0], b);
    atomicMax(&a.max_speed[1], (unsigned long long)__double_as_longlong(__ddiv_rn(v, __ldg(a.dx + s))) & mask);
  }
}

template <typename T>
__global__ void __launch_bounds__(R3_THREADS) recon3d_flux(Recon3dArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FluxSmem<T>& sm = *reinterpret_cast<FluxSmem<T>*>(smem_raw);
  const int t = blockIdx.x, m = blockIdx.z;
  const int s = a.ids ? (a.ids[t] & ~ITEM_FLUX_ONLY) : t;
  if (s < 0 || s >= a.n_sub) return;  // reported by recon3d_faces
  if (blockIdx.y == 0)
    flux_plane<T, 0>(a, sm, t, s, m);
  else if (blockIdx.y == 1)
    flux_plane<T, 1>(a, sm, t, s, m);
  else
    flux_plane<T, 2>(a, sm, t, s, m);
}

// dU = ((fxl - fxh) + (fyl - fyh)) + (fzl - fzh) of one cell and field.
// FP64: as written.  FP32 fluxes (mixed): each difference exactly as a float
// pair (TwoSum), the three pairs summed by a TwoSum cascade (about 48 bits),
// then widened, so that the scarce FP64 pipe sees one addition instead of the
// six conversions and five operations of the FP64 form.
__device__ __forceinline__ double divergence(double fxl, double fxh, double fyl, double fyh, double fzl, double fzh) {
  return __dadd_rn(__dadd_rn(__dsub_rn(fxl, fxh), __dsub_rn(fyl, fyh)), __dsub_rn(fzl, fzh));
}
__device__ __forceinline__ double divergence(float fxl, float fxh, float fyl, float fyh, float fzl, float fzh) {
  float sx, ex, sy, ey, sz, ez;
  two_sum1(fxl, -fxh, sx, ex);
  two_sum1(fyl, -fyh, sy, ey);
  two_sum1(fzl, -fzh, sz, ez);
  float h, l;
  two_sum1(sx, sy, h, l);
  l = __fadd_rn(l, __fadd_rn(ex, ey));
  float h2, l2;
  two_sum1(h, sz, h2, l2);
  l2 = __fadd_rn(l2, __fadd_rn(l, ez));
  return __dadd_rn(f32_to_f64(h2), f32_to_f64(l2));
}

// The update of one item, one thread per (field, cell) unit:
//   dU = ((Fx(i-1/2) - Fx(i+1/2)) + (Fy(j-1/2) - Fy(j+1/2))) + (Fz(k-1/2) - Fz(k+1/2)),
//   U* = U_in + (dt/dx) dU, U_out = U0 + beta (U* - U0) (U* when beta == 1).
template <typename T>
__global__ void __launch_bounds__(256) recon3d_update(Recon3dArgs a) {
  const int t = blockIdx.x;
  const int id = a.ids ? a.ids[t] : t;
  const int s = id & ~ITEM_FLUX_ONLY;
  if (s < 0 || s >= a.n_sub || (id & ITEM_FLUX_ONLY)) return;
  const double dt = a.dt_dev ? *a.dt_dev : a.dt;
  const double lam = __ddiv_rn(dt, __ldg(a.dx + s));
  const T* fl = reinterpret_cast<const T*>(a.fl) + (size_t)t * 3 * FL_DIR;
  bool bad = false;
  for (int e = threadIdx.x; e < NF * CELLS; e += 256) {
    const int f = e / CELLS, c = e - f * CELLS;
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const T* fx = fl + 0 * FL_DIR + (size_t)f * NFACE * NPEN;
    const T* fy = fl + 1 * FL_DIR + (size_t)f * NFACE * NPEN;
    const T* fz = fl + 2 * FL_DIR + (size_t)f * NFACE * NPEN;
    const T fxl = fx[i * NPEN + k * 8 + j], fxh = fx[(i + 1) * NPEN + k * 8 + j];
    const T fyl = fy[j * NPEN + k * 8 + i], fyh = fy[(j + 1) * NPEN + k * 8 + i];
    const T fzl = fz[k * NPEN + j * 8 + i], fzh = fz[(k + 1) * NPEN + j * 8 + i];
    const double dU = divergence(fxl, fxh, fyl, fyh, fzl, fzh);
    const size_t o = field_offset(s, f) + ((k + NG) * NP + (j + NG)) * NP + (i + NG);
    const double us = __dadd_rn(__ldg(a.Uin + o), __dmul_rn(lam, dU));
    double v = us;
    if (a.beta != 1.0) {
      const double u0 = __ldg(a.U0 + o);
      v = __dadd_rn(u0, __dmul_rn(a.beta, __dsub_rn(us, u0)));
    }
    a.Uout[o] = v;
    bad |= !isfinite(v) || (f == F_RHO && !(v > 0.0));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(a.err, ERRBIT_NONFINITE);
}

}  // namespace

size_t recon3d_scratch_doubles(int n_items, int which) {
  return (size_t)n_items * 3 * (which == 0 ? FA_DIR : FL_DIR);
}

// The flux kernel's shared-memory limit is an attribute of the function on
// each device: set once per device, under a lock.
cudaError_t recon3d_prepare() {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    e = cudaFuncSetAttribute(recon3d_flux<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(FluxSmem<double>));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(recon3d_flux<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(FluxSmem<float>));
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}

cudaError_t launch_recon3d(const Recon3dArgs& a, cudaStream_t st) {
  if (a.n_items <= 0) return cudaSuccess;
  const cudaError_t e = recon3d_prepare();
  if (e != cudaSuccess) return e;
  if (a.mixed) {
    recon3d_faces<float><<<dim3(a.n_items, 3), R3_THREADS, 0, st>>>(a);
    recon3d_flux<float><<<dim3(a.n_items, 3, NFACE), R3_THREADS, sizeof(FluxSmem<float>), st>>>(a);
    recon3d_update<float><<<a.n_items, 256, 0, st>>>(a);
  } else {
    recon3d_faces<double><<<dim3(a.n_items, 3), R3_THREADS, 0, st>>>(a);
    recon3d_flux<double><<<dim3(a.n_items, 3, NFACE), R3_THREADS, sizeof(FluxSmem<double>), st>>>(a);
    recon3d_update<double><<<a.n_items, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace hydro
