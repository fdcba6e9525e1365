// hydro_stage.cu -- one Runge-Kutta stage of the octree hydro step on GB300.
//
// Persistent kernel: CTAs pull sub-grid ids from a device work queue (one
// atomic counter per launch), so every uneven leaf batch of a call runs in one
// launch.  For each sub-grid:
//   * the 8^3 interior of the 11 fields is staged once into shared memory;
//   * for each direction d the two 3-layer halo slabs are gathered straight
//     from the neighbours' interiors (same level: asynchronous cp.async copies
//     issued while the previous direction computes; coarser neighbour:
//     injection; finer neighbours: 2x2x2 mean; domain boundary: outflow copy)
//     -- the on-device form of the paper's direct neighbour access for the
//     hydro boundary exchange (Section VI), so no ghost-fill pass is needed
//     between stages and ghost cells of the input are never read;
//   * PPM (Colella & Woodward 1984) per (field, pencil), sliding window in
//     registers, writes the 9 face states of each pencil (Section V-B.1
//     reconstruct kernel);
//   * one thread per face: EOS with dual-energy switch, central-upwind or
//     central speeds, numerical flux of all fields (flux kernel);
//   * each thread owns two cells and sums their flux differences in x, y, z
//     order;
// then U* = U + dt/dx dU, U_out = U0 + beta (U* - U0), and the sub-grid's
// largest face speed joins the global maximum (compute_fluxes' time-step
// reduction) through one ordered-bits atomicMax.
//
// T = double: every step in FP64 (tests and reciprocals kept off the scarce
// FP64 pipe where integer operations or a Newton-Raphson refinement do).
// T = float (mixed): FP64 inputs are rounded to FP32 once, by integer
// operations (GB300 runs FP64 and f32<->f64 conversions at about 2 per clock
// per SM, the FP32/INT pipes at 128), into FP32 shadows the stage reads its
// interior and halos from; the reconstruction and flux run in FP32, the six
// flux terms of every cell are summed error-free as a float pair (TwoSum
// cascade), and the conserved update is done in FP64.  The SSP-RK3 step runs
// in increment form (modes 1..3, see update_inc): the increments stay float
// pairs in packed scratch arrays and the FP64 state changes once per step.
// Stages on coarse-fine faces also export their boundary fluxes for the
// correction pass (hydro_reflux.cu).  The scheme's arithmetic (PPM, face flux,
// FP64 quotients) lives in hydro_scheme.cuh.
#include <cmath>
#include <mutex>

#include "hydro_fp.cuh"
#include "hydro_internal.cuh"
#include "hydro_reflux.cuh"
#include "hydro_scheme.cuh"

namespace hydro {
namespace {

constexpr int THREADS = 256;
constexpr int SJ = 9, SK = 72;   // shared-memory strides of the interior tile (2-way bank conflicts at most)
constexpr int ISZ = 8 * SK;      // elements per field of the interior tile
constexpr int HALO = 3 * NPEN;   // cells per halo slab (3 layers x 64 pencils)

// ---------------------------------------------------------------------------
// accumulators and update
// ---------------------------------------------------------------------------

// Packed FP32 pairs: lane x is the thread's first owned cell, lane y its second.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// Error-free sums (Knuth's TwoSum) on both lanes: s + e == a + b exactly.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bp = sub2(s, a);
  const float2 ap = sub2(s, bp);
  e = add2(sub2(a, ap), sub2(b, bp));
}
// the same for a - b (bit-identical to two_sum2(a, -b))
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2& s, float2& e) {
  s = sub2(a, b);
  const float2 bp = sub2(s, a);
  const float2 ap = sub2(s, bp);
  e = sub2(sub2(a, ap), add2(b, bp));
}

// RN64(s + c) for a float pair with |c| <= ulp(s)/2, by integer operations.
// The exact sum has the bits of s followed, after a gap, by those of c; it is
// exact in FP64 when c starts at most 29 binades below the end of s, and is
// rounded to nearest (ties to even) otherwise.
__device__ __forceinline__ double pair_to_f64(float s, float c) {
  const unsigned bs = __float_as_uint(s), bc = __float_as_uint(c);
  const int es = (int)((bs >> 23) & 0xffu), ec = (int)((bc >> 23) & 0xffu);
  if (es == 0 || es == 0xff || ec == 0) return f32_to_f64(s);  // zero/subnormal/non-finite s, or c ~ 0
  // significands as integers in units of 2^(es-150) (s) and 2^(ec-150) (c)
  const unsigned long long ms = (unsigned long long)((bs & 0x7fffffu) | 0x800000u);
  const unsigned long long mc = (unsigned long long)((bc & 0x7fffffu) | 0x800000u);
  const int gap = es - ec;  // >= 24 for a normalized pair
  // value / 2^(es-150) = ms + sign*mc*2^-gap; scale by 2^39 to keep 63 bits:
  // A = ms << 39 (at most 2^63), B = mc << 39 >> gap (with sticky bit)
  unsigned long long A = ms << 39;
  unsigned long long B;
  if (gap >= 63) {
    B = 1;  // only a sticky bit survives
  } else {
    const unsigned long long full = mc << 39;
    B = full >> gap;
    if ((B << gap) != full) B |= 1;  // sticky
  }
  const bool same = ((bs ^ bc) & 0x80000000u) == 0;
  unsigned long long M = same ? A + B : A - B;  // A > B always
  int e = es;  // M is in units of 2^(es-150-39) = 2^(es-189)
  // normalize M so that its leading bit is bit 63 or 62
  const int lz = __clzll((long long)M);
  M <<= lz;
  e -= lz;  // now M in units of 2^(e-189), leading bit at 63
  // round to 53 bits: keep bits 63..11, rounding bits 10..0
  const unsigned long long rem = M & 0x7ffull;
  unsigned long long m53 = M >> 11;
  if (rem > 0x400ull || (rem == 0x400ull && (m53 & 1ull))) ++m53;
  if (m53 >> 53) {  // rounding carried out
    m53 >>= 1;
    ++e;
  }
  // value = m53 * 2^(e-189+11) with m53 in [2^52, 2^53): biased FP64 exponent
  const long long e64 = (long long)e - 189 + 11 + 52 + 1023;
  const unsigned long long bits =
      ((unsigned long long)(bs & 0x80000000u) << 32) | ((unsigned long long)e64 << 52) | (m53 & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// Flux-difference accumulator of one field for the thread's two owned cells.
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double v0, v1;
  __device__ __forceinline__ void set_diff(double lo0, double hi0, double lo1, double hi1) {
    v0 = __dsub_rn(lo0, hi0);
    v1 = __dsub_rn(lo1, hi1);
  }
  __device__ __forceinline__ void add_diff(double lo0, double hi0, double lo1, double hi1) {
    v0 = __dadd_rn(v0, __dsub_rn(lo0, hi0));
    v1 = __dadd_rn(v1, __dsub_rn(lo1, hi1));
  }
  // U* = u + lam dU of cell r, rounded as written (no contraction)
  __device__ __forceinline__ double advance(int r, double u, double lam) const {
    return __dadd_rn(u, __dmul_rn(lam, r ? v1 : v0));
  }
};

// Float pair (s + c) per cell holding the running flux-difference sum: the
// difference of a direction's two face fluxes is formed exactly first (so a
// mirrored cell, which sees the two terms swapped and negated, gets the same
// pair), then added through an error-free TwoSum; the six-term sum is exact to
// about 2^-48.  Both cells advance together in packed FP32x2 operations.
template <>
struct Acc<float> {
  float2 s, c;
  __device__ __forceinline__ void set_diff(float lo0, float hi0, float lo1, float hi1) {
    two_diff2(make_float2(lo0, lo1), make_float2(hi0, hi1), s, c);
  }
  __device__ __forceinline__ void add_diff(float lo0, float hi0, float lo1, float hi1) {
    float2 d, e, t, e2;
    two_diff2(make_float2(lo0, lo1), make_float2(hi0, hi1), d, e);
    two_sum2(s, d, t, e2);
    s = t;
    c = add2(c, add2(e, e2));
  }
  // U* = u + lam (s + c): both terms widen exactly to FP64 (integer
  // operations), the small one is added first; two FP64 operations.
  __device__ __forceinline__ double advance(int r, double u, double lam) const {
    const double sd = f32_to_f64(r ? s.y : s.x), cd = f32_to_f64(r ? c.y : c.x);
    return fma(lam, sd, fma(lam, cd, u));
  }
  // The same with one FP64 operation: dU = RN64(s + c) assembled by integer
  // operations after renormalizing the pair (for the blended stages, whose two
  // further FP64 operations keep the FP64 pipe busier than the integer pipes).
  __device__ __forceinline__ double advance_one_fma(int r, double u, double lam) const {
    const float sv = r ? s.y : s.x, cv = r ? c.y : c.x;
    const float hi = __fadd_rn(sv, cv);  // renormalize: |lo| <= ulp(hi)/2
    const float lo = __fadd_rn(cv, -__fadd_rn(hi, -sv));
    return fma(lam, pair_to_f64(hi, lo), u);
  }
};

__device__ __forceinline__ bool bad64(double v, bool density) {
  const unsigned hi = (unsigned)__double2hiint(v);
  const bool nonfinite = (hi & 0x7ff00000u) == 0x7ff00000u;
  const bool nonpos = density && (((int)hi < 0) || ((hi | (unsigned)__double2loint(v)) == 0u));
  return nonfinite || nonpos;
}

// Bit 31 of the result is set iff v is not finite: the exponent field plus one
// overflows into it only for the all-ones exponent.  OR-ed over many values.
__device__ __forceinline__ unsigned nonfinite_bit(double v) {
  return ((unsigned)__double2hiint(v) & 0x7ff00000u) + 0x00100000u;
}

// ---------------------------------------------------------------------------
// flags of the in-stage coarse-fine flux correction
// ---------------------------------------------------------------------------

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// ---------------------------------------------------------------------------
// halo gather
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {  // 8-byte global -> shared copy
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {  // 16-byte global -> shared copy
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(src));
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {  // 4-byte global -> shared copy
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(src));
}

struct Nbr {
  int32_t id[6][4];
  int rel[6];
  int oct;
};

__device__ __forceinline__ int pad_offset(int i, int j, int k) { return k * NP2 + j * NP + i; }

// Offset within a field of padded cell coordinates given along (D, b1, b2).
template <int D>
__device__ __forceinline__ int offset_dbb(int cd, int c1, int c2) {
  return D == 0 ? pad_offset(cd, c1, c2) : (D == 1 ? pad_offset(c1, cd, c2) : pad_offset(c1, c2, cd));
}

// Gather the two halo slabs of direction D of sub-grid s into halo[f][side][l*64 + p]
// (FP64); l is the slab layer (pencil position m = l or 11 + l), p = t2*8 + t1.
// 192 threads each own one (l, p) and walk the 11 fields of both slabs;
// every copy of a single cell (same level, coarser neighbour, outflow) is an
// asynchronous cp.async, the 2x2x2 means are computed in place.
template <int D>
__device__ __forceinline__ void gather_halo(const double* __restrict__ U, int s, const Nbr& nb, double* halo) {
  // threads 64..255: they have one face task fewer than threads 0..63
  const int q = (int)threadIdx.x - (THREADS - HALO);
  if (q < 0) return;
  int l, p;
  if (D == 0) {  // x slabs: consecutive threads walk the 3 contiguous cells of a row
    p = q / 3;
    l = q - 3 * p;
  } else {
    l = q >> 6;
    p = q & 63;
  }
  const int t1 = p & 7, t2 = p >> 3;
  const int b1 = D == 0 ? 1 : 0;
  const int b2 = D == 2 ? 1 : 2;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int face = 2 * D + side;
    const int ga = side ? NX + l : l - NG;  // interior coordinate of the ghost cell along D
    double* dst = halo + side * HALO + l * NPEN + p;
    const int n0 = nb.id[face][0];
    const int rel = nb.rel[face];
    if (rel <= 0) {
      // one source cell per ghost cell: copy
      int src_s, off;
      if (n0 >= 0 && rel == 0) {
        src_s = n0;
        off = offset_dbb<D>((side ? ga - NX : ga + NX) + NG, t1 + NG, t2 + NG);
      } else if (n0 < 0) {
        src_s = s;
        off = offset_dbb<D>(side ? NG + NX - 1 : NG, t1 + NG, t2 + NG);
      } else {
        const int fa = ga >= 0 ? ga / 2 : -((1 - ga) / 2);
        src_s = n0;
        off = offset_dbb<D>((side ? -4 : 8) + fa + NG, 4 * ((nb.oct >> b1) & 1) + (t1 >> 1) + NG,
                            4 * ((nb.oct >> b2) & 1) + (t2 >> 1) + NG);
      }
      const double* src = U + field_offset(src_s, 0) + off;
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async8(dst + f * 2 * HALO, src + (size_t)f * NP3);
    } else {
      // finer neighbours: mean of the 2x2x2 fine cells, summed in (k, j, i) order
      const int q1 = t1 >> 2, q2 = t2 >> 2;
      const int fs = nb.id[face][q1 + 2 * q2];
      const int cd = 2 * (side ? ga - NX : ga + 4) + NG;
      const int c1 = 2 * (t1 - 4 * q1) + NG, c2 = 2 * (t2 - 4 * q2) + NG;
      int c[3];
      c[D] = cd;
      c[b1] = c1;
      c[b2] = c2;
      const double* src = U + field_offset(fs, 0) + pad_offset(c[0], c[1], c[2]);
#pragma unroll 4
      for (int f = 0; f < NF; ++f) {
        const double* g = src + (size_t)f * NP3;
        double sum = 0.0;
#pragma unroll
        for (int dk = 0; dk < 2; ++dk)
#pragma unroll
          for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int di = 0; di < 2; ++di) sum = __dadd_rn(sum, g[dk * NP2 + dj * NP + di]);
        dst[f * 2 * HALO] = __dmul_rn(sum, 0.125);
      }
    }
  }
}

__device__ __forceinline__ int shadow_index(int i, int j, int k) { return (k * NX + j) * NX + i; }

template <int D>
__device__ __forceinline__ int shadow_dbb(int cd, int c1, int c2) {
  return D == 0 ? shadow_index(cd, c1, c2) : (D == 1 ? shadow_index(c1, cd, c2) : shadow_index(c1, c2, cd));
}

// Mixed path: the same gather from the FP32 shadow (interior at
// (k*8 + j)*8 + i, 4^3 restriction after it): every ghost cell is one 4-byte
// asynchronous copy, a finer neighbour's from its restriction.
template <int D>
__device__ __forceinline__ void gather_halo_shadow(const float* __restrict__ S, int s, const Nbr& nb, float* halo) {
  const int q = (int)threadIdx.x - (THREADS - HALO);
  if (q < 0) return;
  if constexpr (D == 0) {
    // x slabs: threads q < 128 take one (side, pencil) each and all 11 fields,
    // into the pencil's 16-byte chunk: side 0 holds i = 4..7 of the low
    // neighbour's row (elements 1..3 are the ghost layers -3..-1), side 1
    // holds i = 0..3 of the high one (elements 0..2 are layers 8..10)
    if (q >= 2 * NPEN) return;
    const int p = q & 63, side = q >> 6;
    const int t1 = p & 7, t2 = p >> 3;  // (j, k)
    float* dst = halo + (side * NPEN + p) * 4;
    constexpr int DF = 2 * NPEN * 4;  // per field
    constexpr size_t FS = SHADOW_FIELD;
    const int n0 = nb.id[side][0];
    const int rel = nb.rel[side];
    if (rel >= 0 && n0 >= 0) {
      const float* src;
      if (rel == 0) {
        src = S + (size_t)n0 * NF * FS + shadow_index(side ? 0 : 4, t1, t2);
      } else {
        const int q1 = t1 >> 2, q2 = t2 >> 2;
        src = S + (size_t)nb.id[side][q1 + 2 * q2] * NF * FS + SHADOW_COARSE + ((t2 - 4 * q2) * 4 + (t1 - 4 * q1)) * 4;
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async16(dst + f * DF, src + f * FS);
    } else {
      int off[NG];
      const float* base = S + (size_t)(n0 >= 0 ? n0 : s) * NF * FS;
#pragma unroll
      for (int l = 0; l < NG; ++l) {
        const int ga = side ? NX + l : l - NG;
        const int fa = ga >= 0 ? ga / 2 : -((1 - ga) / 2);
        off[l] = n0 < 0 ? shadow_index(side ? NX - 1 : 0, t1, t2)
                        : shadow_index((side ? -4 : 8) + fa, 4 * ((nb.oct >> 1) & 1) + (t1 >> 1),
                                       4 * ((nb.oct >> 2) & 1) + (t2 >> 1));
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int l = 0; l < NG; ++l) cp_async4(dst + f * DF + (side ? l : l + 1), base + f * FS + off[l]);
    }
    return;
  } else {
    // y, z slabs: thread q takes one (field parity, side, layer, row t2, half)
    // of 4 consecutive cells t1 = half*4 .. +3; same level, outflow and finer
    // neighbours are one 16-byte copy per field, a coarser one four 4-byte
    // copies
    constexpr int b1 = 0, b2 = D == 2 ? 1 : 2;
    constexpr size_t FS = SHADOW_FIELD;
    const int half = q & 1, t2 = (q >> 1) & 7, rest = q >> 4;  // rest = f0 * 6 + side * 3 + layer
    const int f0 = rest / (2 * NG), side = (rest % (2 * NG)) / NG, l = rest % NG;
    const int face = 2 * D + side;
    const int ga = side ? NX + l : l - NG;
    float* dst = halo + side * HALO + l * NPEN + t2 * 8 + half * 4;
    constexpr int DF = 2 * HALO;
    const int n0 = nb.id[face][0];
    const int rel = nb.rel[face];
    if (rel >= 0) {
      const float* src;
      if (rel == 0) {
        const int src_s = n0 >= 0 ? n0 : s;
        const int cd = n0 >= 0 ? (side ? ga - NX : ga + NX) : (side ? NX - 1 : 0);
        src = S + (size_t)src_s * NF * FS + shadow_dbb<D>(cd, half * 4, t2);
      } else {
        const int q2 = t2 >> 2;
        const int cdc = side ? ga - NX : ga + 4;
        const int rr = t2 - 4 * q2;
        src = S + (size_t)nb.id[face][half + 2 * q2] * NF * FS + SHADOW_COARSE +
              (D == 1 ? (rr * 4 + cdc) * 4 : (cdc * 4 + rr) * 4);
      }
#pragma unroll
      for (int f = f0; f < NF; f += 2) cp_async16(dst + f * DF, src + f * FS);
    } else {
      const int fa = ga >= 0 ? ga / 2 : -((1 - ga) / 2);
      const float* base = S + (size_t)n0 * NF * FS;
      int off[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        off[e] = shadow_dbb<D>((side ? -4 : 8) + fa, 4 * ((nb.oct >> b1) & 1) + ((half * 4 + e) >> 1),
                               4 * ((nb.oct >> b2) & 1) + (t2 >> 1));
#pragma unroll
      for (int f = f0; f < NF; f += 2)
#pragma unroll
        for (int e = 0; e < 4; ++e) cp_async4(dst + f * DF + e, base + f * FS + off[e]);
    }
  }
}

// Cell r (0, 1) owned by this thread in the flux accumulation and the update:
// the k-pair (2*(tid/64) + r) at (i, j) = (tid % 8, tid / 8 % 8), so that a
// 2x2x2 block lies in one thread pair in k and lanes ^1, ^8, ^9 of one warp.
__device__ __forceinline__ int owned_cell(int r) {
  const int tid = threadIdx.x;
  return ((tid >> 6) * 2 + r) * 64 + (tid & 63);
}

// interior tile index of pencil position n (0..7) of pencil p in direction d
__device__ __forceinline__ int tile_index(int d, int p, int n) {
  const int t1 = p & 7, t2 = p >> 3;
  return d == 0 ? t2 * SK + t1 * SJ + n : (d == 1 ? t2 * SK + n * SJ + t1 : n * SK + t2 * SJ + t1);
}

template <typename T>
struct StageSmem {
  static constexpr size_t interior = sizeof(T) * NF * ISZ;
  // FP32: the x slabs as one 16-byte chunk per (field, side, pencil), which is
  // larger than the y/z layout [NF][2][HALO]
  static constexpr size_t halo = sizeof(T) * (sizeof(T) == 4 ? NF * 2 * NPEN * 4 : NF * 2 * HALO);
  static constexpr size_t faces = sizeof(T) * 2 * NF * FACES_DIR;
  static constexpr size_t total = interior + halo + faces;
};

template <typename T>
struct Shared {
  T* tile;  // [NF][ISZ] interior
  T* halo;  // [NF][2][HALO] current direction's halo slabs
  T* fsl;        // [NF][576] left face states, then fluxes
  T* fsr;        // [NF][576] right face states
};

template <typename T, int D>
__device__ __forceinline__ void gather(const StageArgs& a, int s, const Nbr& nb, T* halo) {
  if constexpr (sizeof(T) == 4)
    gather_halo_shadow<D>(a.Sin, s, nb, halo);
  else
    gather_halo<D>(a.Uin, s, nb, halo);
}

// The array a stage's halos and (mixed) interiors are read from.
template <typename T>
__device__ __forceinline__ const T* stage_src(const StageArgs& a) {
  if constexpr (sizeof(T) == 4)
    return a.Sin;
  else
    return a.Uin;
}

// The source array of the stage of an item fetched ahead (one-launch step:
// any of the three; read from the parameters with constant offsets).
template <typename T, bool FUSED>
__device__ __forceinline__ const T* next_src(const StageArgs* st, int k) {
  if constexpr (FUSED)
    return k == 0 ? stage_src<T>(st[0]) : (k == 1 ? stage_src<T>(st[1]) : stage_src<T>(st[2]));
  else
    return stage_src<T>(st[0]);
}

// Mixed path: asynchronous copy of sub-grid s's interior (all fields) from the
// shadow into the tile; consecutive threads take consecutive cells.
__device__ __forceinline__ void stage_interior_async(const float* __restrict__ S, int s, float* tile) {
  const float* src = S + (size_t)s * NF * SHADOW_FIELD;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int c = threadIdx.x + r * THREADS;
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int t = k * SK + j * SJ + i;
#pragma unroll
    for (int f = 0; f < NF; ++f) cp_async4(tile + f * ISZ + t, src + f * SHADOW_FIELD + c);
  }
}

// Start the copies of the first direction's halo (and, mixed, of the interior)
// of sub-grid s from src.
template <typename T>
__device__ __forceinline__ void start_item(const T* src, int s, const Nbr& nb, T* tile, T* halo) {
  if constexpr (sizeof(T) == 4) {
    stage_interior_async(src, s, tile);
    gather_halo_shadow<0>(src, s, nb, halo);
  } else {
    gather_halo<0>(src, s, nb, halo);
  }
}

// Pull what the update of sub-grid s will read into L2 ahead of time: the
// previous increment (packed, one 4 KB bulk prefetch per field), and the
// 10 x 8 x 8 x 11 box around the interior rows of the padded FP64 arrays it
// reads (U_in, and U0 in the blended stages): one TMA tensor prefetch per
// array (the box starts at i = 2, a 16-byte boundary).
__device__ __forceinline__ void prefetch_update_rows(const StageArgs& a, int s) {
  if (a.Din && threadIdx.x < NF) {  // the previous increment: one 4 KB block per field
    const double* p = a.Din + ((size_t)s * NF + threadIdx.x) * CELLS;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((unsigned)(CELLS * sizeof(double)))
                 : "memory");
  }
  if (threadIdx.x != 0 || !(a.has_tm & 1)) return;
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(&a.tm_in), "r"(NG - 1),
               "r"(NG), "r"(NG), "r"(s * NF)
               : "memory");
  if (a.has_tm & 2)
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(&a.tm_u0),
                 "r"(NG - 1), "r"(NG), "r"(NG), "r"(s * NF)
                 : "memory");
}

// Work item and what its processing needs: sub-grid id (-1: queue exhausted,
// -2: bad id), whether it only exports its coarse-fine fluxes (an id with
// ITEM_FLUX_ONLY: a proxy of a sharded grid, read by the correction of a
// coarser neighbour but advanced elsewhere), neighbour table, dt/dx.
struct Meta {
  Nbr nb;
  int item;
  int s;
  int flux_only;
  double lam;    // FP64: dt / dx, the IEEE quotient; mixed: dt * (1/dx)
  double sdx;    // the factor of the speed per cell width: FP64 dx (a quotient), mixed 1/dx (a product)
  float lh, ll;  // lam split into two floats (lh + ll = lam to about 2^-48)
  int stage;     // one-launch RK3 step: the item's stage (0..2); else 0
  int ready;     // one-launch RK3 step: its inputs were complete when it was fetched
};

// The next work item as warp 7 (threads 224..255, one PPM task fewer than
// threads 0..191) fetches it while the current one is processed: the queue
// ticket after the x PPM, the sub-grid id after the y PPM, the neighbour table
// loads before the z PPM (into registers) and their store after it, so that
// each dependent load has a whole phase to arrive.
struct Pf {
  int item;   // queue ticket (lane 0 until shuffled)
  int s;      // its sub-grid id, -1 past the end of the queue, -2 bad id
  int nbv;    // lane l < 24: neighbour entry l of s
  int relv;   // lane l < 6: level relation of face l
  int octv;   // lane 0: octant
  double dx;  // lane 0: dx (FP64) or 1/dx (mixed)
  int fo;     // the item only exports fluxes
  int stage;  // its stage (one-launch RK3 step)
};

// The queue: n_total tickets.  A stage launch hands out its batch's items; the
// one-launch RK3 step (FUSED) hands out 3 n tickets, stage-major (ticket t is
// item t - k n of stage k = t / n) or, with order 1, stage-interleaved (stage
// t % 3 of item t / 3).  Once a bounded wait has given up anywhere, the queue
// counts as empty.
__device__ __forceinline__ void pf_ticket(const StageArgs& a0, int n_total, Pf& pf) {
  if ((threadIdx.x & 31) == 0)
    pf.item = (a0.abort_word && ld_volatile(a0.abort_word)) ? n_total : (int)atomicAdd(a0.queue, 1u);
}

template <bool FUSED>
__device__ __forceinline__ void pf_id(const StageArgs* st, const FusedArgs* fx, int n_total, Pf& pf) {
  pf.item = __shfl_sync(0xffffffffu, pf.item, 0);
  pf.stage = 0;
  if (pf.item >= n_total) {
    pf.s = -1;
  } else if constexpr (FUSED) {
    const int n = fx->n;
    pf.stage = fx->order ? pf.item % 3 : pf.item / n;
    const int idx = fx->order ? pf.item / 3 : pf.item - pf.stage * n;
    const int32_t* ids = pf.stage == 0 ? st[0].ids : (pf.stage == 1 ? st[1].ids : st[2].ids);
    pf.s = ids[idx];
  } else {
    pf.s = st[0].ids[pf.item];
  }
}

// Whether the stage-k item of sub-grid s may start: s and every face
// neighbour whose interior its halo gather reads (the neighbour of a same-level
// or coarser face, the four of a finer one) have completed stage k - 1
// (done >= k).  One warp: lane l < 24 takes neighbour entry l (id, and the
// relation of its face), lane 24 takes s; acquire loads, so that the halo
// copies issued after the CTA barrier that follows see the neighbours' outputs.
__device__ __forceinline__ bool stage_ready(const int32_t* done, int s, int k, int id, int rel) {
  const int lane = threadIdx.x & 31;
  int x = -1;
  if (lane < 24) {
    if (((lane & 3) == 0 || rel == 1) && id >= 0) x = id;
  } else if (lane == 24) {
    x = s;
  }
  const bool ok = x < 0 || ld_acquire(done + x) >= k;
  return __all_sync(0xffffffffu, ok);
}

// Check the fetched id and issue the loads of its neighbour table.
// exact_quotients (FP64): dt/dx and speed/dx as IEEE quotients, as the plain
// statement has them; the mixed path multiplies by 1/dx (one FP64 division
// per sub-grid sits on its critical path, measured 1 % of the step).
template <bool exact_quotients>
__device__ __forceinline__ void pf_load(const StageArgs& a, int n_total, Pf& pf) {
  const int lane = threadIdx.x & 31;
  int s = -1;
  pf.fo = 0;
  if (pf.item < n_total) {
    s = pf.s;
    if (s >= 0 && (s & ITEM_FLUX_ONLY)) {
      pf.fo = 1;
      s &= ~ITEM_FLUX_ONLY;
    }
    if (s < 0 || s >= a.n_sub) {
      if (lane == 0) atomicOr(a.err, ERRBIT_BAD_ID);
      s = -2;
    }
  }
  pf.s = s;
  if (s >= 0) {
    if (lane < 24) pf.nbv = a.nb[(size_t)s * 24 + lane];
    if (lane < 6) pf.relv = a.rel[s * 6 + lane];
    if (lane == 0) {
      pf.octv = a.oct[s];
      pf.dx = exact_quotients ? a.dx[s] : a.inv_dx[s];
    }
  }
}

// Store the fetched item into m.
template <bool exact_quotients>
__device__ __forceinline__ void pf_store(double dt, const Pf& pf, Meta& m) {
  const int lane = threadIdx.x & 31;
  if (pf.s >= 0) {
    if (lane < 24) m.nb.id[lane >> 2][lane & 3] = pf.nbv;
    if (lane < 6) m.nb.rel[lane] = pf.relv;
    if (lane == 0) {
      m.nb.oct = pf.octv;
      const double lam = exact_quotients ? __ddiv_rn(dt, pf.dx) : dt * pf.dx;
      m.lam = lam;
      m.sdx = pf.dx;
      m.lh = (float)lam;
      m.ll = (float)(lam - (double)m.lh);
    }
  }
  if (lane == 0) {
    m.item = pf.item;
    m.s = pf.s;
    m.flux_only = pf.fo;
    m.stage = pf.stage;
  }
}

// One-launch RK3 step: whether the fetched item's inputs are complete (stage 0
// items always are); warp-uniform, every lane of the warp calls it.
template <bool FUSED>
__device__ __forceinline__ void pf_ready(const FusedArgs* fx, const Pf& pf, Meta& m) {
  if constexpr (FUSED) {
    const int lane = threadIdx.x & 31;
    const int rel = __shfl_sync(0xffffffffu, pf.relv, (lane >> 2) & 7);
    bool r = true;
    if (pf.s >= 0 && pf.stage > 0) r = stage_ready(fx->done, pf.s, pf.stage, lane < 24 ? pf.nbv : -1, rel);
    if (lane == 0) m.ready = r;
  } else {
    if ((threadIdx.x & 31) == 0) m.ready = 1;
  }
}

// All three steps at once (loop prologue and after a bad id).
template <bool exact_quotients, bool FUSED>
__device__ __forceinline__ void prefetch_meta(const StageArgs* st, const FusedArgs* fx, int n_total, double dt,
                                              Meta& m) {
  Pf pf;
  pf_ticket(st[0], n_total, pf);
  pf_id<FUSED>(st, fx, n_total, pf);
  pf_load<exact_quotients>(st[0], n_total, pf);
  pf_store<exact_quotients>(dt, pf, m);
  pf_ready<FUSED>(fx, pf, m);
}

// Coarse side of the in-stage flux correction.  Thread 0 waits until every
// finer face neighbour across the sides `corr` of direction D that this call
// advances has exported its direction-D fluxes (cf_flag >= D + 1), bounded by
// wait_limit cycles; a wait that runs out (or finds another one given up)
// records ERRBIT_TIMEOUT / raises abort_word and returns false.
template <int D>
__device__ bool wait_fine(const StageArgs& a, const Nbr& nb, unsigned corr) {
  const long long t0 = clock64();
  for (int side = 0; side < 2; ++side) {
    if (!((corr >> side) & 1u)) continue;
    for (int q = 0; q < 4; ++q) {
      const int fs = nb.id[2 * D + side][q];
      if (a.member && a.member[fs] != a.call_id) continue;  // not advanced by this call
      while (ld_acquire(a.cf_flag + fs) < a.flag_base + D + 1) {
        if (ld_volatile(a.abort_word)) return false;
        if (clock64() - t0 > a.wait_limit) {
          atomicOr(a.err, ERRBIT_TIMEOUT);
          atomicExch(a.abort_word, 1);
          return false;
        }
        __nanosleep(100);
      }
    }
  }
  return true;
}

// The correction itself (after the wait, FP64): every coarse boundary face
// flux of the sides `corr` whose fine neighbour this call advances becomes
//   ((F(0,0) + F(1,0)) + (F(0,1) + F(1,1))) / 4
// of the four fine faces over it, as the fine neighbour exported them
// ((a, b) the fine offsets along the face's first and second transverse
// axes), in place, before the flux differences are taken.
template <typename T, int D>
__device__ __forceinline__ void correct_faces(const Shared<T>& sh, const StageArgs& a, const Nbr& nb, unsigned corr) {
  static_assert(sizeof(T) == 8, "the FP32 stage corrects in a separate pass");
  const double* __restrict__ fb = static_cast<const double*>(a.fb);
  for (int e = threadIdx.x; e < 2 * NF * NPEN; e += THREADS) {
    const int side = e >= NF * NPEN ? 1 : 0;
    if (!((corr >> side) & 1u)) continue;
    const int rem = e - side * NF * NPEN, f = rem >> 6, p = rem & 63, t1 = p & 7, t2 = p >> 3;
    const int face = 2 * D + side;
    const int fs = nb.id[face][(t1 >> 2) + 2 * (t2 >> 2)];
    if (a.member && a.member[fs] != a.call_id) continue;  // not advanced by this call: keep the coarse flux
    const double* fine = fb + ((size_t)fs * 6 + (face ^ 1)) * NF * NPEN + f * NPEN + (2 * (t2 & 3)) * NX + 2 * (t1 & 3);
    const double a00 = __ldcg(fine), a10 = __ldcg(fine + 1), a01 = __ldcg(fine + NX), a11 = __ldcg(fine + NX + 1);
    sh.fsl[f * FACES_DIR + p * NFACE + (side ? NFACE - 1 : 0)] =
        __dmul_rn(__dadd_rn(__dadd_rn(a00, a10), __dadd_rn(a01, a11)), 0.25);
  }
}

// CW84 flattening and steepening (optional): hydro_cw84.cuh, which uses the
// tile layout and the PPM helpers above.
#include "hydro_cw84.cuh"

// One direction of the stage: PPM of every (field, pencil), the next
// direction's halo gather (issued once the halo buffer is free; after z, the
// next sub-grid's x halo), the face fluxes, the coarse-fine correction of the
// faces onto finer neighbours, the flux differences of the two owned cells,
// and the export of the faces onto a coarser neighbour.  Warp 7 also fetches
// the next work item, one step per pass.  Returns whether fluxes were exported
// (for x and y the export flag is raised here; z's after the update).
template <typename T, int D, bool FUSED, bool CW>
__device__ __forceinline__ bool direction_pass(const Shared<T>& sh, const StageArgs* st, const FusedArgs* fx,
                                               int n_total, const StageArgs& a, const Meta& cur, Meta& nxt, Pf& pf,
                                               double dt, Acc<T> (&acc)[NF], T& amax, T gamma, T eta) {
  const int tid = threadIdx.x;
  if constexpr (CW) cw84_coefficients<T, D>(sh, a, cur.s, cur.nb, gamma, eta);
  if (D == a.pf_pass) prefetch_update_rows(a, cur.s);  // the prefetch distance: a tuning parameter
  if (D == 2 && (tid >> 5) == THREADS / 32 - 1) pf_load<sizeof(T) == 8>(st[0], n_total, pf);
  // A: PPM, one (field, pencil) task per iteration
#pragma unroll 1
  for (int task = tid; task < NF * NPEN; task += THREADS) {
    const int f = task >> 6, p = task & 63;
    T q[NP];
    if constexpr (sizeof(T) == 4 && D == 0) {
      const float4* hx = reinterpret_cast<const float4*>(sh.halo) + (f * 2) * NPEN + p;
      const float4 h0 = hx[0], h1 = hx[NPEN];
      q[0] = h0.y, q[1] = h0.z, q[2] = h0.w;
      q[11] = h1.x, q[12] = h1.y, q[13] = h1.z;
    } else {
      const T* hl = sh.halo + (f * 2) * HALO + p;
#pragma unroll
      for (int m = 0; m < NG; ++m) q[m] = hl[m * NPEN];
#pragma unroll
      for (int m = 0; m < NG; ++m) q[NG + NX + m] = hl[HALO + m * NPEN];
    }
#pragma unroll
    for (int n = 0; n < NX; ++n) q[NG + n] = sh.tile[f * ISZ + tile_index(D, p, n)];
    T ul[NFACE], ur[NFACE];
    if constexpr (CW)
      ppm_pencil_cw(q, cw_smem<T>().coef[p], cw_smem<T>().coef[NPEN + p], ul, ur);
    else
      ppm_pencil(q, ul, ur);
#pragma unroll
    for (int m = 0; m < NFACE; ++m) {
      sh.fsl[f * FACES_DIR + p * NFACE + m] = ul[m];
      sh.fsr[f * FACES_DIR + p * NFACE + m] = ur[m];
    }
  }
  if ((tid >> 5) == THREADS / 32 - 1) {
    if (D == 0) pf_ticket(st[0], n_total, pf);
    if (D == 1) pf_id<FUSED>(st, fx, n_total, pf);
    if (D == 2) {
      pf_store<sizeof(T) == 8>(dt, pf, nxt);
      pf_ready<FUSED>(fx, pf, nxt);
    }
  }
  __syncthreads();
  // the halo buffer is free: start gathering the next slabs; after z the tile
  // is free too, and the mixed path starts copying the next interior (an item
  // of the one-launch RK3 step whose inputs are not complete yet is gathered
  // at the loop head instead, after its wait)
  if (D < 2) {
    gather<T, (D < 2 ? D + 1 : 2)>(a, cur.s, cur.nb, sh.halo);
    if constexpr (CW) cw84_prefetch_layer4<T, (D < 2 ? D + 1 : 2)>(a, cur.s, cur.nb);
  } else if (nxt.s >= 0 && nxt.ready) {
    start_item<T>(next_src<T, FUSED>(st, nxt.stage), nxt.s, nxt.nb, sh.tile, sh.halo);
    if constexpr (CW) cw84_prefetch_layer4<T, 0>(st[0], nxt.s, nxt.nb);
  }
  // B: one face per iteration
#pragma unroll 1
  for (int fc = tid; fc < FACES_DIR; fc += THREADS) {
    T UL[NF], UR[NF], F[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      UL[f] = sh.fsl[f * FACES_DIR + fc];
      UR[f] = sh.fsr[f * FACES_DIR + fc];
    }
    T sp = face_flux(UL, UR, D, gamma, eta, a.form, F);
    amax = (sp > amax || sp != sp) ? sp : amax;
#pragma unroll
    for (int f = 0; f < NF; ++f) sh.fsl[f * FACES_DIR + fc] = F[f];
  }
  __syncthreads();
  // FP64: faces of direction D onto finer neighbours wait for the fine
  // neighbours' exported fluxes, then take their means (correct_faces)
  if constexpr (sizeof(T) == 8) {
    unsigned corr = 0;
    if (a.fb && !cur.flux_only) corr = (cur.nb.rel[2 * D] == 1 ? 1u : 0u) | (cur.nb.rel[2 * D + 1] == 1 ? 2u : 0u);
    if (corr) {
      __shared__ int s_ok;
      if (tid == 0) s_ok = wait_fine<D>(a, cur.nb, corr);
      __syncthreads();
      if (s_ok) correct_faces<T, D>(sh, a, cur.nb, corr);
      __syncthreads();
    }
  }
  // C: flux differences of direction D for the two owned cells (k and k+1:
  // same pencil for x and y, adjacent faces of one pencil for z)
  {
    const int c = owned_cell(0);
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int p0 = D == 0 ? (k * 8 + j) : (D == 1 ? (k * 8 + i) : (j * 8 + i));
    const int p1 = D == 2 ? p0 : p0 + 8;
    const int id0 = D == 0 ? i : (D == 1 ? j : k);
    const int id1 = D == 2 ? k + 1 : id0;
    const int b0 = p0 * NFACE + id0, b1 = p1 * NFACE + id1;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const T* F = sh.fsl + f * FACES_DIR;
      const T lo0 = F[b0], hi0 = F[b0 + 1], lo1 = F[b1], hi1 = F[b1 + 1];
      if (D == 0)
        acc[f].set_diff(lo0, hi0, lo1, hi1);
      else
        acc[f].add_diff(lo0, hi0, lo1, hi1);
    }
  }
  // export this direction's coarse-fine boundary fluxes: FP64, the faces onto
  // a coarser neighbour, for its in-stage correction (after the barrier that
  // follows, one thread fences and raises the flag: the barrier orders the
  // CTA's stores before its fence, whose release covers them); FP32, the
  // faces of both sides, for the correction pass after the stage
  bool exported = false;
  if (a.fb) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (sizeof(T) == 8 ? cur.nb.rel[2 * D + side] != -1 : cur.nb.rel[2 * D + side] == 0) continue;
      T* dst = static_cast<T*>(a.fb) + ((size_t)cur.s * 6 + 2 * D + side) * NF * NPEN;
      const int m = side ? NFACE - 1 : 0;
      for (int e = tid; e < NF * NPEN; e += THREADS) dst[e] = sh.fsl[(e >> 6) * FACES_DIR + (e & 63) * NFACE + m];
      exported = true;
    }
  }
  // the next direction's halo is in place and the face buffers are free (after
  // z, the loop head's barrier does both for the next sub-grid)
  if (D < 2) {
    cp_async_wait_all();
    __syncthreads();
    if (sizeof(T) == 8 && exported && tid == 0) {
      __threadfence();
      st_release(a.cf_flag + cur.s, a.flag_base + D + 1);
    }
  }
  return exported;
}

// ---------------------------------------------------------------------------
// Mixed-precision SSP-RK3 in increment form.  With L_k = lam * dU(U_k) the
// stages are U1 = U + L0, U2 = U + (L0 + L1)/4, U3 = U + 2/3 ((L0 + L1)/4 + L2),
// algebraically the Shu-Osher stages.  The increments stay float pairs (about
// 48 bits; error-free TwoSums and products); the FP64 state is read by every
// stage but changed only once, by two FP64 additions in stage 3.  Stages 1
// and 2 write the shadow of their state as RN32(RN32(RN32(U) + D_hi) + D_lo),
// about one FP32 ulp from the rounded state, taking RN32(U) from the shadow of
// U, so they read no FP64 state at all.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// (h, l) = (ah + al) * (bh + bl) to about 2^-46, both cells packed
__device__ __forceinline__ void pair_mul(float2 ah, float2 al, float2 bh, float2 bl, float2& h, float2& l) {
  h = mul2(ah, bh);
  const float2 e = fma2(ah, bh, neg2(h));
  l = fma2(ah, bl, fma2(al, bh, e));
}

// (h, l) = (ah + al) + (bh + bl)
__device__ __forceinline__ void pair_add(float2 ah, float2 al, float2 bh, float2 bl, float2& h, float2& l) {
  float2 e;
  two_sum2(ah, bh, h, e);
  l = add2(e, add2(al, bl));
}

__device__ __forceinline__ double pack_pair(float h, float l) {
  return __hiloint2double(__float_as_int(h), __float_as_int(l));
}
__device__ __forceinline__ float pair_hi(double d) { return __int_as_float(__double2hiint(d)); }
__device__ __forceinline__ float pair_lo(double d) { return __int_as_float(__double2loint(d)); }

// Shadow output of one field (the two owned cells x0, x1) and its restriction.
__device__ __forceinline__ void write_shadow(float* So, int c0, float x0, float x1) {
  const int tid = threadIdx.x;
  So[c0] = x0;
  So[c0 + 64] = x1;
  // pairs in i (lane ^ 1), then in j (lane ^ 8), both cells of the k-pair at once
  const float2 xi = make_float2(x0, x1);
  const float2 p = add2(xi, make_float2(__shfl_xor_sync(0xffffffffu, x0, 1), __shfl_xor_sync(0xffffffffu, x1, 1)));
  const float2 t = add2(p, make_float2(__shfl_xor_sync(0xffffffffu, p.x, 8), __shfl_xor_sync(0xffffffffu, p.y, 8)));
  const int cc = (tid >> 6) * 16 + ((tid >> 4) & 3) * 4 + ((tid >> 1) & 3);
  if ((tid & 9) == 0) So[SHADOW_COARSE + cc] = __fmul_rn(__fadd_rn(t.x, t.y), 0.125f);  // i and j even
}

// The increments live in the scratch arrays as packed interiors, one float
// pair per 8-byte slot at [s][f][(k*8 + j)*8 + i]: 64-byte rows on 64-byte
// boundaries (the padded layout's rows start 24 bytes into a 32-byte sector,
// so every row write there also read back two partial sectors).
__device__ __forceinline__ size_t inc_offset(int s, int f) { return ((size_t)s * NF + f) * CELLS; }

// Fields [F0, F1) of update_inc below.
template <int MODE, bool SHADOW, int F0, int F1>
__device__ __forceinline__ unsigned update_inc_fields(const StageArgs& a, int s, const Acc<float> (&acc)[NF],
                                                      float lh, float ll, size_t cell0, int c0, unsigned& nf) {
  constexpr bool READ_D = MODE >= 2;
  unsigned bad = 0;
  double u0v[MODE == 3 ? F1 - F0 : 1][2], dv[READ_D ? F1 - F0 : 1][2];
  float s0v[MODE < 3 ? F1 - F0 : 1][2];
#pragma unroll
  for (int f = F0; f < F1; ++f)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const size_t o = field_offset(s, f) + cell0 + (size_t)r * NP2;
      if constexpr (MODE == 3)
        u0v[f - F0][r] = a.Uin[o];
      else
        s0v[f - F0][r] = a.S0[((size_t)s * NF + f) * SHADOW_FIELD + c0 + r * 64];
      if constexpr (READ_D) dv[f - F0][r] = a.Din[inc_offset(s, f) + c0 + r * 64];
    }
  const float2 lh2 = make_float2(lh, lh), ll2 = make_float2(ll, ll);
#pragma unroll
  for (int f = F0; f < F1; ++f) {
    float2 Lh, Ll;  // L = lam * (s + c) for both cells
    pair_mul(acc[f].s, acc[f].c, lh2, ll2, Lh, Ll);
    float2 Dh, Dl;  // the new increment
    if constexpr (MODE == 1) {
      Dh = Lh, Dl = Ll;
    } else {
      const float2 ph = make_float2(pair_hi(dv[f - F0][0]), pair_hi(dv[f - F0][1]));
      const float2 pl = make_float2(pair_lo(dv[f - F0][0]), pair_lo(dv[f - F0][1]));
      pair_add(ph, pl, Lh, Ll, Dh, Dl);
      if constexpr (MODE == 2) {
        Dh = mul2(Dh, make_float2(0.25f, 0.25f));
        Dl = mul2(Dl, make_float2(0.25f, 0.25f));
      } else {
        constexpr float ch = (float)(2.0 / 3.0), cl = (float)(2.0 / 3.0 - (double)(float)(2.0 / 3.0));
        pair_mul(Dh, Dl, make_float2(ch, ch), make_float2(cl, cl), Dh, Dl);
      }
    }
    float x[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const size_t o = field_offset(s, f) + cell0 + (size_t)r * NP2;
      const float dh = r ? Dh.y : Dh.x, dl = r ? Dl.y : Dl.x;
      if constexpr (MODE == 3) {
        const double v = __dadd_rn(__dadd_rn(u0v[f - F0][r], f32_to_f64(dh)), f32_to_f64(dl));
        a.Uout[o] = v;
        nf |= nonfinite_bit(v);
        if (f == F_RHO) bad |= bad64(v, true);
        x[r] = f64_to_f32(v);
      } else {
        a.Dout[inc_offset(s, f) + c0 + r * 64] = pack_pair(dh, dl);
        // both parts of the pair: a corrected increment may be unnormalized
        // (its low part above half an ulp of its high part) after the
        // correction pass, and the shadow of the next stage reads this value
        x[r] = __fadd_rn(__fadd_rn(s0v[f - F0][r], dh), dl);
        nf |= (__float_as_uint(x[r]) & 0x7f800000u) == 0x7f800000u ? 0x80000000u : 0u;
        if (f == F_RHO) bad |= !(x[r] > 0.0f);
      }
    }
    if constexpr (SHADOW) write_shadow(a.Sout + ((size_t)s * NF + f) * SHADOW_FIELD, c0, x[0], x[1]);
  }
  return bad;
}

// The update of mode 1..3 for the two owned cells of sub-grid s (loads in one
// group in mode 1, two when the previous increment is read as well).
template <int MODE, bool SHADOW>
__device__ __forceinline__ unsigned update_inc(const StageArgs& a, int s, const Acc<float> (&acc)[NF], float lh,
                                               float ll) {
  const int c0 = owned_cell(0);
  const size_t cell0 = (size_t)((c0 >> 6) + NG) * NP2 + (((c0 >> 3) & 7) + NG) * NP + ((c0 & 7) + NG);
  unsigned nf = 0, bad = 0;
  if constexpr (MODE >= 2) {
    bad |= update_inc_fields<MODE, SHADOW, 0, 6>(a, s, acc, lh, ll, cell0, c0, nf);
    bad |= update_inc_fields<MODE, SHADOW, 6, NF>(a, s, acc, lh, ll, cell0, c0, nf);
  } else {
    bad |= update_inc_fields<MODE, SHADOW, 0, NF>(a, s, acc, lh, ll, cell0, c0, nf);
  }
  return bad | (nf >> 31);
}

// Fields [F0, F1) of update_cells below.
template <typename T, bool BLEND, bool SHADOW, int F0, int F1>
__device__ __forceinline__ unsigned update_fields(const StageArgs& a, int s, const Acc<T> (&acc)[NF], double lam,
                                                  size_t cell0, int c0, unsigned& nf) {
  unsigned bad = 0;
  // every load of the group first: one memory latency per group, not per field
  double uin[F1 - F0][2], u0v[BLEND ? F1 - F0 : 1][2];
#pragma unroll
  for (int f = F0; f < F1; ++f)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const size_t o = field_offset(s, f) + cell0 + (size_t)r * NP2;
      uin[f - F0][r] = a.Uin[o];
      if constexpr (BLEND) u0v[f - F0][r] = a.U0[o];
    }
#pragma unroll
  for (int f = F0; f < F1; ++f) {
    double v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const size_t o = field_offset(s, f) + cell0 + (size_t)r * NP2;
      if constexpr (BLEND) {
        double us;
        if constexpr (sizeof(T) == 4)
          us = acc[f].advance_one_fma(r, uin[f - F0][r], lam);
        else
          us = acc[f].advance(r, uin[f - F0][r], lam);
        const double u0 = u0v[f - F0][r];
        v[r] = sizeof(T) == 8 ? __dadd_rn(u0, __dmul_rn(a.beta, __dsub_rn(us, u0))) : fma(a.beta, us - u0, u0);
      } else {
        v[r] = acc[f].advance(r, uin[f - F0][r], lam);
      }
      a.Uout[o] = v[r];
      nf |= nonfinite_bit(v[r]);
      if (f == F_RHO) bad |= bad64(v[r], true);
    }
    if constexpr (SHADOW && sizeof(T) == 4)
      write_shadow(a.Sout + ((size_t)s * NF + f) * SHADOW_FIELD, c0, f64_to_f32(v[0]), f64_to_f32(v[1]));
  }
  return bad;
}

// U_out = U* (or U0 + beta (U* - U0) when BLEND) for the two owned cells of
// sub-grid s; SHADOW (mixed only) also writes the rounded cells and their
// 2x2x2 restriction (FP32 pairwise sum, the partner cells by warp shuffles).
// The loads are issued in one group (two with the blend, which reads twice as
// many) so that their latencies overlap.  Returns non-zero if a value is not
// finite or a density <= 0.
template <typename T, bool BLEND, bool SHADOW>
__device__ __forceinline__ unsigned update_cells(const StageArgs& a, int s, const Acc<T> (&acc)[NF], double lam) {
  const int c0 = owned_cell(0);
  const size_t cell0 = (size_t)((c0 >> 6) + NG) * NP2 + (((c0 >> 3) & 7) + NG) * NP + ((c0 & 7) + NG);
  unsigned nf = 0, bad = 0;
  if constexpr (BLEND) {
    bad |= update_fields<T, BLEND, SHADOW, 0, 6>(a, s, acc, lam, cell0, c0, nf);
    bad |= update_fields<T, BLEND, SHADOW, 6, NF>(a, s, acc, lam, cell0, c0, nf);
  } else {
    bad |= update_fields<T, BLEND, SHADOW, 0, NF>(a, s, acc, lam, cell0, c0, nf);
  }
  return bad | (nf >> 31);
}

// ---------------------------------------------------------------------------
// The work loop.  A stage launch (FUSED false) processes its batch with st[0].
// The one-launch RK3 step (FUSED true) processes 3 n items with st[k] for the
// stage-k ones.  An item of that step whose inputs were not complete when it
// was fetched (its halo was not gathered ahead) waits at the loop head, after
// the CTA's previous item has finished, so that a CTA never waits while it
// holds an unfinished item; every item waits only for items of lower tickets
// (the previous stage; FP64: finer sub-grids of the same stage), which running
// CTAs hold or have finished.  A finished item marks its sub-grid complete
// (done[s] = k + 1, release), except, in mixed precision, a coarse sub-grid
// with finer face neighbours: that one is marked by the CTA that brings its
// arrival count to the stage's target, which first applies the coarse-fine
// correction.
// ---------------------------------------------------------------------------

// One-launch step, warp 7: wait (bounded) until the stage-k item of s may
// start; false if the wait gave up (ERRBIT_TIMEOUT, abort raised) or found the
// launch aborted.
__device__ __forceinline__ bool wait_ready(const FusedArgs* fx, const StageArgs& a0, int s, int k, const Nbr& nb) {
  const int lane = threadIdx.x & 31;
  const int id = lane < 24 ? nb.id[lane >> 2][lane & 3] : -1;
  const int rel = lane < 24 ? nb.rel[lane >> 2] : 0;
  const long long t0 = clock64();
  while (!stage_ready(fx->done, s, k, id, rel)) {
    int stop = 0;
    if (lane == 0) {
      if (ld_volatile(a0.abort_word)) {
        stop = 1;
      } else if (clock64() - t0 > a0.wait_limit) {
        atomicOr(a0.err, ERRBIT_TIMEOUT);
        atomicExch(a0.abort_word, 1);
        stop = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    __nanosleep(200);
  }
  return true;
}

// One-launch step, thread 0, after the stage-k item of s (the CTA's writes
// ordered before it by a barrier): mark the item complete, or, for a coarse
// sub-grid with finer neighbours (mixed, correcting), count its arrival; count
// its arrival at each coarser neighbour.  Returns the number of corrections
// this item completes, their rows in corr[].
__device__ __forceinline__ int complete_item(const FusedArgs* fx, bool correct, int s, int k, const Nbr& nb,
                                             int* corr) {
  __threadfence();
  const int own = correct ? fx->cf_slot[s] : -1;
  if (own < 0) st_release(fx->done + s, k + 1);
  int nc = 0;
  if (correct) {
    for (int face = 0; face < 6; ++face) {
      if (nb.rel[face] != -1) continue;
      const int slot = fx->cf_slot[nb.id[face][0]];
      if (slot >= 0 && atomicAdd(fx->arrive + slot, 1) + 1 == (k + 1) * fx->cf_target[slot] && nc < 8)
        corr[nc++] = slot;
    }
    if (own >= 0 && atomicAdd(fx->arrive + own, 1) + 1 == (k + 1) * fx->cf_target[own] && nc < 8) corr[nc++] = own;
    if (nc) __threadfence();
  }
  return nc;
}

// One-launch step (mixed), every thread of the CTA: apply the nc corrections
// in corr[] (arguments r of the stage) and mark those sub-grids complete.  Out
// of line, and called only when there is one: its registers would crowd the
// stage's.
#ifndef HYDRO_FUSED_CORR_IPT
#define HYDRO_FUSED_CORR_IPT 1
#endif
__device__ __noinline__ void run_corrections(const RefluxArgs r, int k, int nc, const int* corr, int32_t* done) {
  __shared__ reflux::CorrSmem s_cs;
  for (int q = 0; q < nc; ++q) {
    const int row = corr[q];
    reflux::correct_coarse<float, THREADS, HYDRO_FUSED_CORR_IPT, true>(r, row, s_cs);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(done + __ldg(r.cf + (size_t)row * CF_ENTRY), k + 1);
    }
  }
}

// One item (cur) of stage K (FUSED; else st[0]'s stage).  Returns false when
// the launch must stop (a wait gave up).
template <typename T, bool FUSED, int K, bool CW>
__device__ __forceinline__ bool process_item(const Shared<T>& sh, const StageArgs* st, const FusedArgs* fx,
                                             int n_total, const Meta& cur, Meta& nxt, double dt, T gamma, T eta,
                                             unsigned& bad, unsigned long long* s_red) {
  const int tid = threadIdx.x;
  const StageArgs& a = st[K];
  const int s = cur.s;
  if constexpr (FUSED) {
    if (!cur.ready) {
      // wait (bounded) until the item's inputs are complete, then gather
      __shared__ int s_go;
      if ((tid >> 5) == THREADS / 32 - 1) {
        const bool go = wait_ready(fx, st[0], s, K, cur.nb);
        if ((tid & 31) == 0) s_go = go;
      }
      __syncthreads();
      if (!s_go) return false;
      start_item<T>(stage_src<T>(a), s, cur.nb, sh.tile, sh.halo);
    }
  }
  if constexpr (sizeof(T) == 8) {
    // FP64 path: interior of all fields, loaded synchronously
    const double* Us = a.Uin + field_offset(s, 0);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int c = tid + r * THREADS;
      const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
      const int g = (k + NG) * NP2 + (j + NG) * NP + (i + NG);
      const int t = k * SK + j * SJ + i;
#pragma unroll
      for (int f = 0; f < NF; ++f) sh.tile[f * ISZ + t] = Us[(size_t)f * NP3 + g];
    }
  }
  cp_async_wait_all();
  __syncthreads();  // interior tile and x halo in place
  if constexpr (CW && sizeof(T) == 4) cw84_interior_pressures<T>(sh, gamma, eta);
  const bool flux_only = cur.flux_only != 0;
  if (sizeof(T) == 4 && a.fb_stamp && tid == 0) a.fb_stamp[s] = flux_only ? -a.call_id : a.call_id;

  Acc<T> acc[NF];
  Pf pf;
  T amax = T(0);
  direction_pass<T, 0, FUSED, CW>(sh, st, fx, n_total, a, cur, nxt, pf, dt, acc, amax, gamma, eta);
  direction_pass<T, 1, FUSED, CW>(sh, st, fx, n_total, a, cur, nxt, pf, dt, acc, amax, gamma, eta);
  const bool exported_z =
      direction_pass<T, 2, FUSED, CW>(sh, st, fx, n_total, a, cur, nxt, pf, dt, acc, amax, gamma, eta);

  // update of the owned cells (and, mixed, the output's shadow); an item
  // that only exports its fluxes writes no state and posts no speed.  The
  // one-launch step's stages are fixed: mixed stage K runs mode K + 1, FP64
  // stage K blends for K > 0 and writes no shadow.
  if (flux_only) {
    amax = T(0);
  } else if constexpr (FUSED && sizeof(T) == 4) {
    const float lh = cur.lh, ll = cur.ll;
    if constexpr (K == 0)
      bad |= update_inc<1, true>(a, s, acc, lh, ll);
    else if constexpr (K == 1)
      bad |= update_inc<2, true>(a, s, acc, lh, ll);
    else if (a.Sout != nullptr)
      bad |= update_inc<3, true>(a, s, acc, lh, ll);
    else
      bad |= update_inc<3, false>(a, s, acc, lh, ll);
  } else if constexpr (FUSED) {
    bad |= update_cells<T, (K > 0), false>(a, s, acc, cur.lam);
  } else {
    const bool blend = a.beta != 1.0;
    const bool shadow_out = sizeof(T) == 4 && a.Sout != nullptr;
    if (sizeof(T) == 4 && a.mode != 0) {
      if constexpr (sizeof(T) == 4) {
        const float lh = cur.lh, ll = cur.ll;
        if (a.mode == 1)
          bad |= update_inc<1, true>(a, s, acc, lh, ll);
        else if (a.mode == 2)
          bad |= update_inc<2, true>(a, s, acc, lh, ll);
        else if (shadow_out)
          bad |= update_inc<3, true>(a, s, acc, lh, ll);
        else
          bad |= update_inc<3, false>(a, s, acc, lh, ll);
      }
    } else if (blend) {
      if (shadow_out)
        bad |= update_cells<T, true, true>(a, s, acc, cur.lam);
      else
        bad |= update_cells<T, true, false>(a, s, acc, cur.lam);
    } else {
      if (shadow_out)
        bad |= update_cells<T, false, true>(a, s, acc, cur.lam);
      else
        bad |= update_cells<T, false, false>(a, s, acc, cur.lam);
    }
  }

  // largest face speed of this sub-grid (non-negative values order as their bits)
  unsigned long long bits;
  if constexpr (sizeof(T) == 4) {
    unsigned b = __float_as_uint((float)amax) & 0x7fffffffu;
    b = __reduce_max_sync(0xffffffffu, b);
    bits = b;
  } else {
    bits = (unsigned long long)__double_as_longlong((double)amax) & 0x7fffffffffffffffull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, bits, o);
      bits = w > bits ? w : bits;
    }
  }
  if ((tid & 31) == 0) s_red[tid >> 5] = bits;
  __syncthreads();
  if (sizeof(T) == 8 && exported_z && tid == 0) {
    __threadfence();
    st_release(a.cf_flag + s, a.flag_base + 3);
  }
  if (tid == 0) {
    unsigned long long m = 0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) m = s_red[w] > m ? s_red[w] : m;
    double v;
    if constexpr (sizeof(T) == 4)
      v = (double)__uint_as_float((unsigned)m);
    else
      v = __longlong_as_double((long long)m);
    const unsigned long long mask = 0x7fffffffffffffffull;
    atomicMax(&a.max_speed[0], (unsigned long long)__double_as_longlong(v) & mask);
    const double vdx = sizeof(T) == 8 ? __ddiv_rn(v, cur.sdx) : v * cur.sdx;
    atomicMax(&a.max_speed[1], (unsigned long long)__double_as_longlong(vdx) & mask);
  }
  if constexpr (FUSED) {
    __shared__ int s_corr[8];
    __shared__ int s_ncorr;
    if (tid == 0) s_ncorr = complete_item(fx, sizeof(T) == 4 && a.fb, s, K, cur.nb, s_corr);
    if constexpr (sizeof(T) == 4) {
      __syncthreads();
      const int nc = s_ncorr;
      if (nc) run_corrections(fx->rf[K], K, nc, s_corr, fx->done);
    }
  }
  return true;
}

template <typename T, bool FUSED, bool CW>
__device__ __forceinline__ void stage_body(const StageArgs* __restrict__ st, const FusedArgs* __restrict__ fx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared<T> sh;
  sh.tile = reinterpret_cast<T*>(smem_raw);
  sh.halo = reinterpret_cast<T*>(smem_raw + StageSmem<T>::interior);
  sh.fsl = reinterpret_cast<T*>(smem_raw + StageSmem<T>::interior + StageSmem<T>::halo);
  sh.fsr = sh.fsl + NF * FACES_DIR;
  __shared__ Meta s_meta[2];
  __shared__ unsigned long long s_red[THREADS / 32];

  const StageArgs& a0 = st[0];
  const int tid = threadIdx.x;
  const bool warp7 = (tid >> 5) == THREADS / 32 - 1;
  const T gamma = T(a0.gamma), eta = T(a0.eta);
  const double dt = a0.dt_dev ? *a0.dt_dev : a0.dt;
  const int n_total = FUSED ? 3 * fx->n : a0.n_items;
  unsigned bad = 0;

  // prologue: the first work item, its neighbour table and x halo
  if (warp7) prefetch_meta<sizeof(T) == 8, FUSED>(st, fx, n_total, dt, s_meta[0]);
  __syncthreads();
  if (s_meta[0].s >= 0 && s_meta[0].ready) {
    start_item<T>(next_src<T, FUSED>(st, s_meta[0].stage), s_meta[0].s, s_meta[0].nb, sh.tile, sh.halo);
    if constexpr (CW) cw84_prefetch_layer4<T, 0>(st[0], s_meta[0].s, s_meta[0].nb);
  }
  int par = 0;
  for (;;) {
    const Meta& cur = s_meta[par];
    Meta& nxt = s_meta[par ^ 1];
    if (cur.item >= n_total) break;
    if (cur.s < 0) {  // bad id: skip it
      __syncthreads();
      if (warp7) prefetch_meta<sizeof(T) == 8, FUSED>(st, fx, n_total, dt, nxt);
      __syncthreads();
      if (nxt.s >= 0 && nxt.ready) {
        start_item<T>(next_src<T, FUSED>(st, nxt.stage), nxt.s, nxt.nb, sh.tile, sh.halo);
        if constexpr (CW) cw84_prefetch_layer4<T, 0>(st[0], nxt.s, nxt.nb);
      }
      par ^= 1;
      continue;
    }
    bool go;
    if constexpr (FUSED) {
      const int k = cur.stage;
      if (k == 0)
        go = process_item<T, true, 0, false>(sh, st, fx, n_total, cur, nxt, dt, gamma, eta, bad, s_red);
      else if (k == 1)
        go = process_item<T, true, 1, false>(sh, st, fx, n_total, cur, nxt, dt, gamma, eta, bad, s_red);
      else
        go = process_item<T, true, 2, false>(sh, st, fx, n_total, cur, nxt, dt, gamma, eta, bad, s_red);
    } else {
      go = process_item<T, false, 0, CW>(sh, st, fx, n_total, cur, nxt, dt, gamma, eta, bad, s_red);
    }
    if (!go) break;
    par ^= 1;
  }
  cp_async_wait_all();
  if (bad) atomicOr(a0.err, ERRBIT_NONFINITE);
}

template <typename T, bool CW>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 2 : 1) stage_kernel(const __grid_constant__ StageArgs a) {
  stage_body<T, false, CW>(&a, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 2 : 1) rk3_kernel(const __grid_constant__ FusedArgs F) {
  stage_body<T, true, false>(F.st, &F);
}

// The kernel's shared-memory limit is an attribute of the function on each
// device: set it once per device (under a lock, for callers on several threads).
template <typename T, int KIND>
cudaError_t configure_smem() {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    if constexpr (KIND == 1)
      e = cudaFuncSetAttribute(rk3_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)StageSmem<T>::total);
    else
      e = cudaFuncSetAttribute(stage_kernel<T, KIND == 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)StageSmem<T>::total);
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch(const StageArgs& a, int grid, cudaStream_t st) {
  cudaError_t e = a.cw84 ? configure_smem<T, 2>() : configure_smem<T, 0>();
  if (e != cudaSuccess) return e;
  if (a.cw84)
    stage_kernel<T, true><<<grid, THREADS, StageSmem<T>::total, st>>>(a);
  else
    stage_kernel<T, false><<<grid, THREADS, StageSmem<T>::total, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fused(const FusedArgs& f, int grid, cudaStream_t st) {
  cudaError_t e = configure_smem<T, 1>();
  if (e != cudaSuccess) return e;
  rk3_kernel<T><<<grid, THREADS, StageSmem<T>::total, st>>>(f);
  return cudaGetLastError();
}

template <typename T, int KIND>
int blocks_per_sm() {
  int n = 0;
  if (configure_smem<T, KIND>() != cudaSuccess) return 1;
  cudaError_t e;
  if constexpr (KIND == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rk3_kernel<T>, THREADS, StageSmem<T>::total);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<T, KIND == 2>, THREADS,
                                                      StageSmem<T>::total);
  if (e != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

}  // namespace

bool encode_state_map(CUtensorMap* tm, const double* U, int n) {
  EncodeTiled fn = encoder();
  if (!fn || !U || n < 1) return false;
  const cuuint64_t dims[4] = {NP, NP, NP, (cuuint64_t)n * NF};
  const cuuint64_t strides[3] = {NP * sizeof(double), NP2 * sizeof(double), NP3 * sizeof(double)};
  const cuuint32_t box[4] = {NX + 2, NX, NX, NF};  // i = 2..11 keeps the box start on a 16-byte boundary
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<double*>(U), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_stage_fp64(const StageArgs& a, int grid, cudaStream_t st) { return launch<double>(a, grid, st); }
cudaError_t launch_stage_mixed(const StageArgs& a, int grid, cudaStream_t st) { return launch<float>(a, grid, st); }
cudaError_t launch_rk3_fp64(const FusedArgs& f, int grid, cudaStream_t st) { return launch_fused<double>(f, grid, st); }
cudaError_t launch_rk3_mixed(const FusedArgs& f, int grid, cudaStream_t st) { return launch_fused<float>(f, grid, st); }
int stage_blocks_per_sm_fp64() { return blocks_per_sm<double, 0>(); }
int stage_blocks_per_sm_mixed() { return blocks_per_sm<float, 0>(); }
int rk3_blocks_per_sm_fp64() { return blocks_per_sm<double, 1>(); }
int rk3_blocks_per_sm_mixed() { return blocks_per_sm<float, 1>(); }
int cw_blocks_per_sm_fp64() { return blocks_per_sm<double, 2>(); }
int cw_blocks_per_sm_mixed() { return blocks_per_sm<float, 2>(); }

}  // namespace hydro
