// hydro_reflux.cuh -- the coarse-fine flux correction of one coarse sub-grid
// after a mixed-precision RK stage (paper Section V-B.1: compute_fluxes
// corrects the fluxes on coarse-fine boundaries), shared by the correction
// pass (hydro_reflux.cu, one CTA per coarse sub-grid) and the one-launch RK3
// step (hydro_stage.cu, run by the CTA that completes the sub-grid's stage).
//
// On a face where a sub-grid meets four finer neighbours, the coarse side used
// its own flux; the fine side lost exactly the mean of its four fluxes over
// each coarse face.  The stage kernel exports both sides' boundary fluxes; the
// correction replaces, for every coarse boundary face, its flux F by
//   F' = ((F(0,0) + F(1,0)) + (F(0,1) + F(1,1))) / 4
// (a, b the fine offsets along the face's two transverse axes), i.e. it adds
// sgn * lam * (F' - F) to the flux sum of the adjacent coarse cell (sgn = +1 on
// a low face, -1 on a high one) and carries that through the stage's output.
// Only quadrants whose fine neighbour was advanced by the same call (stamp)
// are corrected.  The faces of a cell are applied in order 0..5, so that edge
// and corner cells take their corrections in a fixed order.  F' - F is formed
// exactly as a float pair, and the correction applies to whatever the stage
// wrote (the state, or the increment pair of the RK3 increment form) and its
// shadow.
#pragma once
#include "hydro_fp.cuh"
#include "hydro_internal.cuh"

namespace hydro {
namespace reflux {

// loads of data written by other CTAs: through L2 when COHERENT (the stage
// that wrote them runs in the same launch), else read-only cached
template <bool COHERENT, typename V>
__device__ __forceinline__ V ld_in(const V* p) {
  if constexpr (COHERENT)
    return __ldcg(p);
  else
    return __ldg(p);
}
template <bool COHERENT, typename V>
__device__ __forceinline__ V ld_rw(const V* p) {
  if constexpr (COHERENT)
    return __ldcg(p);
  else
    return *p;
}

__device__ __forceinline__ size_t interior_offset(int i, int j, int k) {
  return (size_t)(k + NG) * NP2 + (j + NG) * NP + (i + NG);
}

__device__ __forceinline__ bool bad_value(double v, bool density) {
  return !(v == v) || v - v != 0.0 || (density && !(v > 0.0));
}

// The correction of one (field, cell) by one face: mean of the four fine
// fluxes over the coarse face minus the coarse flux.  Mixed handles return the
// scaled correction as a float pair (ch, cl) = sgn * lam * (F' - F), exact in
// the sum of four floats and their difference; FP64 handles return it in dh.
template <typename T>
struct FaceTerm {
  T a00, a10, a01, a11, own;
};

template <typename T, bool COHERENT>
__device__ __forceinline__ FaceTerm<T> load_term(const T* __restrict__ fb, int s, int fs, int face, int f, int t1,
                                                 int t2) {
  const int q1 = t1 >> 2, q2 = t2 >> 2;
  const T* fine = fb + ((size_t)fs * 6 + (face ^ 1)) * NF * NPEN + f * NPEN;
  const int b = (2 * (t2 - 4 * q2)) * NX + 2 * (t1 - 4 * q1);
  FaceTerm<T> t;
  t.a00 = ld_in<COHERENT>(fine + b);
  t.a10 = ld_in<COHERENT>(fine + b + 1);
  t.a01 = ld_in<COHERENT>(fine + b + NX);
  t.a11 = ld_in<COHERENT>(fine + b + NX + 1);
  t.own = ld_in<COHERENT>(fb + ((size_t)s * 6 + face) * NF * NPEN + f * NPEN + t2 * NX + t1);
  return t;
}

__device__ __forceinline__ void scaled_delta(const FaceTerm<float>& t, float lh, float ll, float& ch, float& cl) {
  float h, l, h2, l2;
  pair_add1(t.a00, 0.0f, t.a10, 0.0f, h, l);
  pair_add1(t.a01, 0.0f, t.a11, 0.0f, h2, l2);
  pair_add1(h, l, h2, l2, h, l);
  h = __fmul_rn(h, 0.25f);
  l = __fmul_rn(l, 0.25f);
  pair_add1(h, l, -t.own, 0.0f, h, l);
  pair_mul1(h, l, lh, ll, ch, cl);
}

// the face's transverse position (t1, t2) of cell (i, j, k)
__device__ __forceinline__ void face_pos(int face, int i, int j, int k, int& t1, int& t2) {
  const int d = face >> 1;
  t1 = d == 0 ? j : i;
  t2 = d == 2 ? j : k;
}

// the faces of the sub-grid that cell (i, j, k) lies on, as a bit mask
__device__ __forceinline__ unsigned cell_faces(int i, int j, int k) {
  return (i == 0 ? 1u : 0u) | (i == NX - 1 ? 2u : 0u) | (j == 0 ? 4u : 0u) | (j == NX - 1 ? 8u : 0u) |
         (k == 0 ? 16u : 0u) | (k == NX - 1 ? 32u : 0u);
}

// Shared memory of one correction.
struct CorrSmem {
  int cf[CF_ENTRY];          // id, then the fine neighbour of each face quadrant
  int ok[CF_ENTRY];          // stamp check of each of them
  double lam;                // dt * (1/dx) of the sub-grid
  unsigned char blocks[64];  // 2x2x2 blocks of the restriction next to a corrected face
};

// The correction of coarse sub-grid row `row` of r.cf, by the RT threads of a
// CTA (at least 128; every thread calls it).  Work item = (face, field,
// position) over the corrected faces; a cell on several corrected faces (edge,
// corner) is handled by the item of its lowest face, which applies the faces
// in ascending order, so the result does not depend on the thread schedule.
// The loads of up to IPT items are issued before any of them is written back.
// COHERENT: the stage that wrote the fluxes, stamps and outputs runs in the
// same launch (loads through L2).
template <typename T, int RT, int IPT, bool COHERENT>
__device__ __forceinline__ void correct_coarse(const RefluxArgs& r, int row, CorrSmem& sm) {
  const int tid = threadIdx.x;
  if (tid < CF_ENTRY) {
    const int v = __ldg(r.cf + (size_t)row * CF_ENTRY + tid);
    sm.cf[tid] = v;
    // the coarse sub-grid itself must have been advanced by the call (stamp
    // +call_id); a fine neighbour must have exported its fluxes in it (advanced,
    // or a flux-only item: -call_id)
    const int st = v >= 0 ? ld_in<COHERENT>(r.fb_stamp + v) : 0;
    sm.ok[tid] = v >= 0 && (st == r.call_id || (tid > 0 && st == -r.call_id));
  } else if (tid == 32) {
    const double dt = r.dt_dev ? *r.dt_dev : r.dt;
    sm.lam = dt * __ldg(r.inv_dx + __ldg(r.cf + (size_t)row * CF_ENTRY));  // as the mixed stage's dt * (1/dx)
  }
  if (tid >= 64 && tid < 128) sm.blocks[tid - 64] = 0;
  __syncthreads();
  if (!sm.ok[0]) return;  // this sub-grid was not advanced by this call
  const int s = sm.cf[0];
  unsigned mask = 0;  // faces with at least one advanced fine quadrant
#pragma unroll
  for (int g = 0; g < 6; ++g)
    mask |= (sm.ok[1 + 4 * g] | sm.ok[2 + 4 * g] | sm.ok[3 + 4 * g] | sm.ok[4 + 4 * g]) ? 1u << g : 0u;
  const double lam = sm.lam;
  const T* __restrict__ fb = static_cast<const T*>(r.fb);
  const float lh = (float)lam, ll = (float)(lam - (double)lh);
  const int nface = __popc(mask);
  const int n_items = nface * NF * NPEN;
  int bad = 0;
  for (int base = 0; base < n_items; base += IPT * RT) {
    FaceTerm<T> term[IPT];
    double val[IPT];
    float s0[IPT];
    int info[IPT];  // cell | field << 9 | lowest face << 13, -1 for no work
    // decode the items and issue their loads
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int e = base + u * RT + tid;
      info[u] = -1;
      if (e >= n_items) continue;
      const int rank = e / (NF * NPEN), rem = e - rank * (NF * NPEN);
      int face = __ffs(mask) - 1;
      for (int q = 0; q < rank; ++q) face = __ffs(mask & ~((2u << face) - 1u)) - 1;
      const int f = rem >> 6, p = rem & 63, t1 = p & 7, t2 = p >> 3;
      const int d = face >> 1, c = (face & 1) ? NX - 1 : 0;
      const int i = d == 0 ? c : t1, j = d == 1 ? c : (d == 0 ? t1 : t2), k = d == 2 ? c : t2;
      const unsigned cf = cell_faces(i, j, k) & mask;
      if ((int)(__ffs(cf) - 1) != face) continue;  // handled by the item of a lower face
      const int qi = 1 + face * 4 + (t1 >> 2) + 2 * (t2 >> 2);
      if (!sm.ok[qi]) {
        // this quadrant's fine neighbour was not advanced; a later face of the
        // cell may still apply (the apply loop re-checks each face)
        if ((cf & ~(1u << face)) == 0) continue;
      }
      info[u] = ((k * NX + j) * NX + i) | (f << 9) | (face << 13);
      if (sm.ok[qi]) term[u] = load_term<T, COHERENT>(fb, s, sm.cf[qi], face, f, t1, t2);
      const size_t o = ((size_t)s * NF + f) * NP3 + interior_offset(i, j, k);
      if (sizeof(T) == 4 && (r.mode == 1 || r.mode == 2)) {
        val[u] = ld_rw<COHERENT>(r.D + ((size_t)s * NF + f) * CELLS + (k * NX + j) * NX + i);  // packed increments
        s0[u] = ld_in<COHERENT>(r.S0 + ((size_t)s * NF + f) * SHADOW_FIELD + (k * NX + j) * NX + i);
      } else {
        val[u] = ld_rw<COHERENT>(r.U + o);
      }
    }
    // apply every corrected face of each item's cell in ascending order
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      if (info[u] < 0) continue;
      const int c = info[u] & 511, f = (info[u] >> 9) & 15, face0 = info[u] >> 13;
      const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
      const unsigned cf = cell_faces(i, j, k) & mask;
      double v = val[u];
      float dh = 0.0f, dl = 0.0f;
      if (sizeof(T) == 4 && (r.mode == 1 || r.mode == 2)) {
        dh = __int_as_float(__double2hiint(v));
        dl = __int_as_float(__double2loint(v));
      }
      for (unsigned rest = cf; rest; rest &= rest - 1) {
        const int face = __ffs(rest) - 1;
        int t1, t2;
        face_pos(face, i, j, k, t1, t2);
        const int qi = 1 + face * 4 + (t1 >> 2) + 2 * (t2 >> 2);
        if (!sm.ok[qi]) continue;
        const FaceTerm<T> t = face == face0 ? term[u] : load_term<T, COHERENT>(fb, s, sm.cf[qi], face, f, t1, t2);
        const int sgn = (face & 1) ? -1 : 1;
        {
          float ch, cl;
          scaled_delta(t, sgn * lh, sgn * ll, ch, cl);
          if (r.mode == 0) {
            const double w = r.beta * 1.0;
            v = fma(w, f32_to_f64(ch), fma(w, f32_to_f64(cl), v));
          } else if (r.mode == 3) {
            constexpr float th = (float)(2.0 / 3.0), tl = (float)(2.0 / 3.0 - (double)(float)(2.0 / 3.0));
            pair_mul1(ch, cl, th, tl, ch, cl);
            v = __dadd_rn(__dadd_rn(v, f32_to_f64(ch)), f32_to_f64(cl));
          } else {
            if (r.mode == 2) {
              ch = __fmul_rn(ch, 0.25f);
              cl = __fmul_rn(cl, 0.25f);
            }
            pair_add1(dh, dl, ch, cl, dh, dl);
          }
        }
      }
      const size_t o = ((size_t)s * NF + f) * NP3 + interior_offset(i, j, k);
      float x;  // the cell's new shadow value (mixed)
      if (sizeof(T) == 4 && (r.mode == 1 || r.mode == 2)) {
        r.D[((size_t)s * NF + f) * CELLS + c] = __hiloint2double(__float_as_int(dh), __float_as_int(dl));
        x = __fadd_rn(__fadd_rn(s0[u], dh), dl);  // the corrected pair may be unnormalized: both parts
        if (!(x - x == 0.0f) || (f == F_RHO && !(x > 0.0f))) bad = 1;
      } else {
        r.U[o] = v;
        bad |= bad_value(v, f == F_RHO);
        x = sizeof(T) == 4 ? f64_to_f32(v) : 0.0f;
      }
      if (sizeof(T) == 4 && r.Sout) r.Sout[((size_t)s * NF + f) * SHADOW_FIELD + c] = x;
      if (f == 0) sm.blocks[((k >> 1) * 4 + (j >> 1)) * 4 + (i >> 1)] = 1;
    }
  }
  __syncthreads();
  // refresh the restriction blocks next to corrected faces
  if constexpr (sizeof(T) == 4) {
    if (r.Sout) {
      for (int e = tid; e < NF * 64; e += RT) {
        const int f = e >> 6, cc = e & 63;
        if (!sm.blocks[cc]) continue;
        const int I = cc & 3, J = (cc >> 2) & 3, K = cc >> 4;
        const float* x = r.Sout + ((size_t)s * NF + f) * SHADOW_FIELD;
        float h[2];
#pragma unroll
        for (int dk = 0; dk < 2; ++dk) {
          const float* b = x + (2 * K + dk) * 64 + (2 * J) * 8 + 2 * I;
          // cells this thread or another wrote just before the barrier, or the stage wrote
          h[dk] = __fadd_rn(__fadd_rn(ld_rw<COHERENT>(b), ld_rw<COHERENT>(b + 1)),
                            __fadd_rn(ld_rw<COHERENT>(b + 8), ld_rw<COHERENT>(b + 9)));
        }
        r.Sout[((size_t)s * NF + f) * SHADOW_FIELD + SHADOW_COARSE + cc] = __fmul_rn(__fadd_rn(h[0], h[1]), 0.125f);
      }
    }
  }
  if (bad) atomicOr(r.err, ERRBIT_NONFINITE);
}

}  // namespace reflux
}  // namespace hydro
