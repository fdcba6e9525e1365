// hydro_reflux.cu -- coarse-fine flux correction after an RK stage (paper
// Section V-B.1: compute_fluxes corrects the fluxes on coarse-fine boundaries).
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
// a fixed order.  FP64 handles correct U_out in FP64; mixed handles form
// F' - F exactly as a float pair and correct whatever the stage wrote (the
// state, or the increment pair of the RK3 increment form) and its shadow.
#include "hydro_fp.cuh"
#include "hydro_internal.cuh"

namespace hydro {
namespace {

constexpr int RT = 256;

__device__ __forceinline__ size_t interior_offset(int i, int j, int k) {
  return (size_t)(k + NG) * NP2 + (j + NG) * NP + (i + NG);
}

// cell (i, j, k) next to face `face` at transverse position (t1, t2)
__device__ __forceinline__ void face_cell(int face, int t1, int t2, int& i, int& j, int& k) {
  const int d = face >> 1, c = (face & 1) ? NX - 1 : 0;
  i = d == 0 ? c : t1;
  j = d == 1 ? c : (d == 0 ? t1 : t2);
  k = d == 2 ? c : t2;
}

__device__ __forceinline__ bool bad_value(double v, bool density) {
  return !(v == v) || v - v != 0.0 || (density && !(v > 0.0));
}

template <typename T>
__global__ void __launch_bounds__(RT) reflux_kernel(const RefluxArgs r) {
  const int s = r.list[blockIdx.x];
  if (r.fb_stamp[s] != r.call_id) return;  // not advanced by this call
  __shared__ unsigned char blocks[64];  // 2x2x2 blocks of the restriction next to a corrected face
  __shared__ int q_fs[6][4];             // the fine neighbour of each face quadrant, -1 if not advanced
  if (threadIdx.x < 64) blocks[threadIdx.x] = 0;
  if (threadIdx.x < 24) {
    const int face = threadIdx.x >> 2;
    int fs = -1;
    if (r.rel[s * 6 + face] == 1) {
      fs = r.nb[(size_t)s * 24 + threadIdx.x];
      if (r.fb_stamp[fs] != r.call_id) fs = -1;
    }
    q_fs[face][threadIdx.x & 3] = fs;
  }
  const double dt = r.dt_dev ? *r.dt_dev : r.dt;
  const double lam = dt * r.inv_dx[s];
  const T* fb = static_cast<const T*>(r.fb);
  int bad = 0;
  __syncthreads();
  for (int face = 0; face < 6; ++face) {
    if (r.rel[s * 6 + face] != 1) continue;
    const int sgn = (face & 1) ? -1 : 1;
    const T* own = fb + ((size_t)s * 6 + face) * NF * NPEN;
    for (int e = threadIdx.x; e < NF * NPEN; e += RT) {
      const int f = e >> 6, p = e & 63, t1 = p & 7, t2 = p >> 3;
      const int q1 = t1 >> 2, q2 = t2 >> 2;
      const int fs = q_fs[face][q1 + 2 * q2];
      if (fs < 0) continue;
      const T* fine = fb + ((size_t)fs * 6 + (face ^ 1)) * NF * NPEN + f * NPEN;
      const int b = (2 * (t2 - 4 * q2)) * NX + 2 * (t1 - 4 * q1);
      const T a00 = fine[b], a10 = fine[b + 1], a01 = fine[b + NX], a11 = fine[b + NX + 1];
      int i, j, k;
      face_cell(face, t1, t2, i, j, k);
      const int c = (k * NX + j) * NX + i;
      const size_t o = ((size_t)s * NF + f) * NP3 + interior_offset(i, j, k);
      if (f == 0) blocks[((k >> 1) * 4 + (j >> 1)) * 4 + (i >> 1)] = 1;
      float x = 0.0f;  // the cell's new shadow value (mixed)
      if constexpr (sizeof(T) == 8) {
        const double delta = (((double)a00 + (double)a10) + ((double)a01 + (double)a11)) * 0.25 - (double)own[e];
        const double v = fma(r.beta * lam * sgn, delta, r.U[o]);
        r.U[o] = v;
        bad |= bad_value(v, f == F_RHO);
      } else {
        // delta = mean - own as a float pair (the sum of four floats exactly)
        float h, l, h2, l2;
        pair_add1((float)a00, 0.0f, (float)a10, 0.0f, h, l);
        pair_add1((float)a01, 0.0f, (float)a11, 0.0f, h2, l2);
        pair_add1(h, l, h2, l2, h, l);
        h = __fmul_rn(h, 0.25f);
        l = __fmul_rn(l, 0.25f);
        pair_add1(h, l, -(float)own[e], 0.0f, h, l);
        // times lam (split as for the stage: lam = lh + ll) and the sign
        const float lh = (float)lam, ll = (float)(lam - (double)lh);
        float ch, cl;
        pair_mul1(h, l, sgn * lh, sgn * ll, ch, cl);
        if (r.mode == 0) {
          const double w = r.beta * 1.0;
          const double v = fma(w, f32_to_f64(ch), fma(w, f32_to_f64(cl), r.U[o]));
          r.U[o] = v;
          bad |= bad_value(v, f == F_RHO);
          x = f64_to_f32(v);
        } else if (r.mode == 3) {
          constexpr float th = (float)(2.0 / 3.0), tl = (float)(2.0 / 3.0 - (double)(float)(2.0 / 3.0));
          pair_mul1(ch, cl, th, tl, ch, cl);
          const double v = __dadd_rn(__dadd_rn(r.U[o], f32_to_f64(ch)), f32_to_f64(cl));
          r.U[o] = v;
          bad |= bad_value(v, f == F_RHO);
          x = f64_to_f32(v);
        } else {
          if (r.mode == 2) {
            ch = __fmul_rn(ch, 0.25f);
            cl = __fmul_rn(cl, 0.25f);
          }
          const double d = r.D[o];
          float dh = __int_as_float(__double2hiint(d)), dl = __int_as_float(__double2loint(d));
          pair_add1(dh, dl, ch, cl, dh, dl);
          r.D[o] = __hiloint2double(__float_as_int(dh), __float_as_int(dl));
          x = __fadd_rn(r.S0[((size_t)s * NF + f) * SHADOW_FIELD + c], dh);
          if (!(x - x == 0.0f) || (f == F_RHO && !(x > 0.0f))) bad = 1;
        }
        // a cell on two or three corrected faces is rewritten by each in turn
        if (r.Sout) r.Sout[((size_t)s * NF + f) * SHADOW_FIELD + c] = x;
      }
    }
    __syncthreads();
  }
  // refresh the restriction blocks next to corrected faces
  if constexpr (sizeof(T) == 4) {
    if (r.Sout) {
      for (int e = threadIdx.x; e < NF * 64; e += RT) {
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

cudaError_t launch_reflux_fp64(const RefluxArgs& r, cudaStream_t st) {
  if (r.n_list < 1) return cudaSuccess;
  reflux_kernel<double><<<r.n_list, RT, 0, st>>>(r);
  return cudaGetLastError();
}

cudaError_t launch_reflux_mixed(const RefluxArgs& r, cudaStream_t st) {
  if (r.n_list < 1) return cudaSuccess;
  reflux_kernel<float><<<r.n_list, RT, 0, st>>>(r);
  return cudaGetLastError();
}

}  // namespace hydro
