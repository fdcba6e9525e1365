// hydro_reflux.cu -- coarse-fine flux correction after a mixed-precision RK
// stage (paper Section V-B.1: compute_fluxes corrects the fluxes on
// coarse-fine boundaries).  (FP64 stages correct inside the stage kernel,
// which keeps them bit-identical to a plain evaluation; for the FP32 stage a
// separate pass is cheaper: measured on the 65536-leaf octree, the in-stage
// form's export flags, waits and correction terms cost 1.6 ms per RK3 step,
// this pass 0.45 ms.)
//
// On a face where a sub-grid meets four finer neighbours, the coarse side used
// its own flux; the fine side lost exactly the mean of its four fluxes over
// each coarse face.  The stage kernel exports both sides' boundary fluxes; this
// pass replaces, for every coarse boundary face, its flux F by
//   F' = ((F(0,0) + F(1,0)) + (F(0,1) + F(1,1))) / 4
// (a, b the fine offsets along the face's two transverse axes), i.e. it adds
// sgn * lam * (F' - F) to the flux sum of the adjacent coarse cell (sgn = +1 on
// a low face, -1 on a high one) and carries that through the stage's output.
// Only quadrants whose fine neighbour was advanced by the same call (stamp)
// are corrected.  One CTA per coarse sub-grid; its faces in order 0..5 with a
// barrier in between, so that edge and corner cells take their corrections in
// a fixed order.  F' - F is formed exactly as a float pair, and the pass
// corrects whatever the stage wrote (the state, or the increment pair of the
// RK3 increment form) and its shadow.
#include "hydro_fp.cuh"
#include "hydro_internal.cuh"

namespace hydro {
namespace {


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

template <typename T>
__device__ __forceinline__ FaceTerm<T> load_term(const T* __restrict__ fb, int s, int fs, int face, int f, int t1,
                                                 int t2) {
  const int q1 = t1 >> 2, q2 = t2 >> 2;
  const T* fine = fb + ((size_t)fs * 6 + (face ^ 1)) * NF * NPEN + f * NPEN;
  const int b = (2 * (t2 - 4 * q2)) * NX + 2 * (t1 - 4 * q1);
  FaceTerm<T> t;
  t.a00 = __ldg(fine + b);
  t.a10 = __ldg(fine + b + 1);
  t.a01 = __ldg(fine + b + NX);
  t.a11 = __ldg(fine + b + NX + 1);
  t.own = __ldg(fb + ((size_t)s * 6 + face) * NF * NPEN + f * NPEN + t2 * NX + t1);
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

// One CTA per coarse sub-grid.  Work item = (face, field, position) over the
// corrected faces; a cell on several corrected faces (edge, corner) is handled
// by the item of its lowest face, which applies the faces in ascending order,
// so the result does not depend on the thread schedule.  The loads of up to
// IPT items are issued before any of them is written back.  RT threads per
// CTA (at least 128) and IPT are the launch shape, a tuning parameter.
template <typename T, int RT, int IPT>
__global__ void __launch_bounds__(RT, 1024 / RT) reflux_kernel(const RefluxArgs r) {
  __shared__ int s_cf[CF_ENTRY];      // id, then the fine neighbour of each face quadrant
  __shared__ int s_ok[CF_ENTRY];      // stamp check of each of them
  __shared__ double s_lam;            // dt / dx of the sub-grid
  __shared__ unsigned char blocks[64];  // 2x2x2 blocks of the restriction next to a corrected face
  const int tid = threadIdx.x;
  if (tid < CF_ENTRY) {
    const int v = __ldg(r.cf + (size_t)blockIdx.x * CF_ENTRY + tid);
    s_cf[tid] = v;
    // the coarse sub-grid itself must have been advanced by the call (stamp
    // +call_id); a fine neighbour must have exported its fluxes in it (advanced,
    // or a flux-only item: -call_id)
    const int st = v >= 0 ? __ldg(r.fb_stamp + v) : 0;
    s_ok[tid] = v >= 0 && (st == r.call_id || (tid > 0 && st == -r.call_id));
  } else if (tid == 32) {
    const double dt = r.dt_dev ? *r.dt_dev : r.dt;
    s_lam = dt * __ldg(r.inv_dx + __ldg(r.cf + (size_t)blockIdx.x * CF_ENTRY));  // as the mixed stage's dt * (1/dx)
  }
  if (tid >= 64 && tid < 128) blocks[tid - 64] = 0;
  __syncthreads();
  if (!s_ok[0]) return;  // this sub-grid was not advanced by this call
  const int s = s_cf[0];
  unsigned mask = 0;  // faces with at least one advanced fine quadrant
#pragma unroll
  for (int g = 0; g < 6; ++g)
    mask |= (s_ok[1 + 4 * g] | s_ok[2 + 4 * g] | s_ok[3 + 4 * g] | s_ok[4 + 4 * g]) ? 1u << g : 0u;
  const double lam = s_lam;
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
      const int fs = s_cf[1 + face * 4 + (t1 >> 2) + 2 * (t2 >> 2)];
      if (!s_ok[1 + face * 4 + (t1 >> 2) + 2 * (t2 >> 2)]) {
        // this quadrant's fine neighbour was not advanced; a later face of the
        // cell may still apply (the apply loop re-checks each face)
        if ((cf & ~(1u << face)) == 0) continue;
      }
      info[u] = ((k * NX + j) * NX + i) | (f << 9) | (face << 13);
      if (s_ok[1 + face * 4 + (t1 >> 2) + 2 * (t2 >> 2)]) term[u] = load_term(fb, s, fs, face, f, t1, t2);
      const size_t o = ((size_t)s * NF + f) * NP3 + interior_offset(i, j, k);
      if (sizeof(T) == 4 && (r.mode == 1 || r.mode == 2)) {
        val[u] = r.D[((size_t)s * NF + f) * CELLS + (k * NX + j) * NX + i];  // packed increment layout
        s0[u] = __ldg(r.S0 + ((size_t)s * NF + f) * SHADOW_FIELD + (k * NX + j) * NX + i);
      } else {
        val[u] = r.U[o];
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
        if (!s_ok[qi]) continue;
        const FaceTerm<T> t = face == face0 ? term[u] : load_term(fb, s, s_cf[qi], face, f, t1, t2);
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
      if (f == 0) blocks[((k >> 1) * 4 + (j >> 1)) * 4 + (i >> 1)] = 1;
    }
  }
  __syncthreads();
  // refresh the restriction blocks next to corrected faces
  if constexpr (sizeof(T) == 4) {
    if (r.Sout) {
      for (int e = tid; e < NF * 64; e += RT) {
        const int f = e >> 6, cc = e & 63;
        if (!blocks[cc]) continue;
        const int I = cc & 3, J = (cc >> 2) & 3, K = cc >> 4;
        const float* x = r.Sout + ((size_t)s * NF + f) * SHADOW_FIELD;
        float h[2];
#pragma unroll
        for (int dk = 0; dk < 2; ++dk) {
          const float* b = x + (2 * K + dk) * 64 + (2 * J) * 8 + 2 * I;
          h[dk] = __fadd_rn(__fadd_rn(b[0], b[1]), __fadd_rn(b[8], b[9]));
        }
        r.Sout[((size_t)s * NF + f) * SHADOW_FIELD + SHADOW_COARSE + cc] = __fmul_rn(__fadd_rn(h[0], h[1]), 0.125f);
      }
    }
  }
  if (bad) atomicOr(r.err, ERRBIT_NONFINITE);
}

}  // namespace

cudaError_t launch_reflux_mixed(const RefluxArgs& r, cudaStream_t st) {
  if (r.n_list < 1) return cudaSuccess;
  switch (r.shape) {
    case 1: reflux_kernel<float, 128, 3><<<r.n_list, 128, 0, st>>>(r); break;
    case 2: reflux_kernel<float, 256, 2><<<r.n_list, 256, 0, st>>>(r); break;
    case 3: reflux_kernel<float, 512, 3><<<r.n_list, 512, 0, st>>>(r); break;
    default: reflux_kernel<float, 256, 3><<<r.n_list, 256, 0, st>>>(r); break;
  }
  return cudaGetLastError();
}

}  // namespace hydro
