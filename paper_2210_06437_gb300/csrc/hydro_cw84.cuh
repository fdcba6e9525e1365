// hydro_cw84.cuh -- CW84 extensions of the PPM in the stage kernel (optional,
// StageArgs::cw84): shock flattening (Colella & Woodward 1984, Section 4, eqs.
// 4.1-4.5; epsilon = 0.33, omega1 = 0.75, omega2 = 10) and contact steepening
// (eqs. 1.14-1.17; eta1 = 20, eta2 = 0.05, epsilon = 0.01, K0 = 0.1).  Both are
// coefficients of the cell, applied to every conserved field before the
// parabola limiter: flattening f from the pressures p_{m-2..m+2} and
// velocities u_{m-1}, u_{m+1} along the pencil and the upstream neighbour's
// candidate, steepening eta detected on the density (and the pressure jump).
// The faces of cells -1..8 need the pressure four cells out, one layer beyond
// the halo: a fourth layer of the six fields the pressure needs is read from
// the neighbours' interiors by the halo rules (same level, coarse injection,
// fine mean or restriction, outflow); in mixed precision every such value is
// one shadow cell, copied asynchronously with the direction's halo slabs.  The
// pressures of the 512 interior cells do not depend on the direction; the
// mixed kernel forms them once per sub-grid.  The FP64 kernel evaluates every
// expression in the order and rounding of its plain statement.
//
// Included by hydro_stage.cu inside its namespace, after the tile layout and
// the PPM helpers.
#pragma once

constexpr int CW_P = 16;   // pressures of cells m = -1..14 of a pencil
constexpr int CW_U = 14;   // velocities of cells m = 0..13
constexpr int CW_C = 10;   // coefficients of cells m = 2..11
constexpr int CW_F = 6;    // fields the pressure needs: rho, sx, sy, sz, E, tau
__device__ __forceinline__ int cw_field(int k) { return k == 0 ? F_RHO : (k < 4 ? F_SX + k - 1 : (k == 4 ? F_EGAS : F_TAU)); }

// Shared storage of the extensions, one per kernel: the coefficients of the
// current direction, the interior pressures of the current sub-grid, and (mixed)
// the fourth layer of the direction whose halo is in flight.
template <typename T>
struct CwSmem {
  T coef[2 * NPEN][CW_C];  // [0, 64): flattening, [64, 128): steepening
  T pint[CELLS];           // pressure of interior cell (k * 8 + j) * 8 + i
  float l4[CW_F][2][NPEN]; // mixed: fourth-layer cells [field][side][pencil]
};

template <typename T>
__device__ __forceinline__ CwSmem<T>& cw_smem() {
  __shared__ CwSmem<T> m;
  return m;
}

// The source of field f of the fourth-layer ghost cell of sub-grid s on `side`
// of direction D at transverse position (t1, t2), in the shadow (mixed: every
// such value is one cell of it) -- the halo rules with ghost coordinate
// ga = -4 (low side) or 11 (high side).
template <int D>
__device__ __forceinline__ const float* layer4_shadow(const float* S, int s, const Nbr& nb, int side, int t1, int t2,
                                                      int f) {
  constexpr int b1 = D == 0 ? 1 : 0, b2 = D == 2 ? 1 : 2;
  const int face = 2 * D + side;
  const int ga = side ? NX + 3 : -4;
  const int n0 = nb.id[face][0], rel = nb.rel[face];
  int c[3], src_s;
  c[b1] = t1;
  c[b2] = t2;
  if (n0 < 0) {
    src_s = s;
    c[D] = side ? NX - 1 : 0;
  } else if (rel == 0) {
    src_s = n0;
    c[D] = side ? ga - NX : ga + NX;
  } else if (rel < 0) {
    src_s = n0;
    const int fa = ga >= 0 ? ga / 2 : -((1 - ga) / 2);
    c[D] = (side ? -4 : 8) + fa;
    c[b1] = 4 * ((nb.oct >> b1) & 1) + (t1 >> 1);
    c[b2] = 4 * ((nb.oct >> b2) & 1) + (t2 >> 1);
  } else {
    const int q1 = t1 >> 2, q2 = t2 >> 2;
    int r[3];
    r[D] = side ? ga - NX : ga + 4;
    r[b1] = t1 - 4 * q1;
    r[b2] = t2 - 4 * q2;
    return S + ((size_t)nb.id[face][q1 + 2 * q2] * NF + f) * SHADOW_FIELD + SHADOW_COARSE + (r[2] * 4 + r[1]) * 4 +
           r[0];
  }
  return S + ((size_t)src_s * NF + f) * SHADOW_FIELD + (c[2] * NX + c[1]) * NX + c[0];
}

// Mixed: start the asynchronous copies of direction D's fourth layer (all
// threads call it; 128 of them issue 6 four-byte copies each).
template <typename T, int D>
__device__ __forceinline__ void cw84_prefetch_layer4(const StageArgs& a, int s, const Nbr& nb) {
  if constexpr (sizeof(T) == 4) {
    if (!(a.cw84 & 1)) return;
    const int tid = threadIdx.x;
    if (tid >= 2 * NPEN) return;
    const int side = tid >> 6, p = tid & 63;
    CwSmem<T>& m = cw_smem<T>();
#pragma unroll
    for (int k = 0; k < CW_F; ++k)
      cp_async4(&m.l4[k][side][p], layer4_shadow<D>(a.Sin, s, nb, side, p & 7, p >> 3, cw_field(k)));
  }
}

// FP64: field f of the fourth-layer ghost cell, loaded (the fine mean summed
// in (k, j, i) order, as the halo rule).
template <int D>
__device__ __forceinline__ double layer4_fp64(const StageArgs& a, int s, const Nbr& nb, int side, int t1, int t2,
                                              int f) {
  constexpr int b1 = D == 0 ? 1 : 0, b2 = D == 2 ? 1 : 2;
  const int face = 2 * D + side;
  const int ga = side ? NX + 3 : -4;
  const int n0 = nb.id[face][0], rel = nb.rel[face];
  int c[3], src_s;
  c[b1] = t1;
  c[b2] = t2;
  if (n0 < 0) {
    src_s = s;
    c[D] = side ? NX - 1 : 0;
  } else if (rel == 0) {
    src_s = n0;
    c[D] = side ? ga - NX : ga + NX;
  } else if (rel < 0) {
    src_s = n0;
    const int fa = ga >= 0 ? ga / 2 : -((1 - ga) / 2);
    c[D] = (side ? -4 : 8) + fa;
    c[b1] = 4 * ((nb.oct >> b1) & 1) + (t1 >> 1);
    c[b2] = 4 * ((nb.oct >> b2) & 1) + (t2 >> 1);
  } else {
    const int q1 = t1 >> 2, q2 = t2 >> 2;
    int b[3];
    b[D] = 2 * (side ? ga - NX : ga + 4) + NG;
    b[b1] = 2 * (t1 - 4 * q1) + NG;
    b[b2] = 2 * (t2 - 4 * q2) + NG;
    const double* g = a.Uin + field_offset(nb.id[face][q1 + 2 * q2], f) + pad_offset(b[0], b[1], b[2]);
    double sum = 0.0;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int di = 0; di < 2; ++di) sum = __dadd_rn(sum, g[dk * NP2 + dj * NP + di]);
    return __dmul_rn(sum, 0.125);
  }
  return a.Uin[field_offset(src_s, f) + pad_offset(c[0] + NG, c[1] + NG, c[2] + NG)];
}

// Field f of cell m (0..13, padded pencil position) of pencil p in direction D
// from the interior tile and the current halo slabs.
template <typename T, int D>
__device__ __forceinline__ T pencil_cell(const Shared<T>& sh, int f, int p, int m) {
  if (m >= NG && m < NG + NX) return sh.tile[f * ISZ + tile_index(D, p, m - NG)];
  const int side = m >= NG + NX ? 1 : 0, l = side ? m - NG - NX : m;
  if constexpr (sizeof(T) == 4 && D == 0)
    return sh.halo[((f * 2 + side) * NPEN + p) * 4 + (side ? l : l + 1)];
  else
    return sh.halo[(f * 2 + side) * HALO + l * NPEN + p];
}

// The pressure of a cell from its conserved fields, by the face EOS
// (dual-energy switch included; FP64 in the plain statement's order and
// rounding), and its velocity along d.
template <typename T>
__device__ __forceinline__ T cell_p(const T (&U)[NF], T gamma, T eta) {
  if constexpr (sizeof(T) == 8) {
    const double rho = U[F_RHO], y = __drcp_rn(rho);
    const double sx = U[F_SX], sy = U[F_SX + 1], sz = U[F_SX + 2], E = U[F_EGAS];
    const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)), __dmul_rn(sz, sz));
    double ei = __dsub_rn(E, div_by(__dmul_rn(0.5, s2), rho, y));
    if (eta > 0.0 && ei < __dmul_rn(eta, E)) ei = pow(U[F_TAU], gamma);
    return __dmul_rn(__dsub_rn(gamma, 1.0), ei);
  } else {
    const T inv = Arith<T>::rcp(U[F_RHO]);
    const T sx = U[F_SX], sy = U[F_SX + 1], sz = U[F_SX + 2];
    T ei = U[F_EGAS] - T(0.5) * ((sx * sx + sy * sy) + sz * sz) * inv;
    if (eta > T(0) && ei < eta * U[F_EGAS]) ei = Arith<T>::pow_(U[F_TAU], gamma);
    return (gamma - T(1)) * ei;
  }
}
template <typename T>
__device__ __forceinline__ T cell_u(T s_d, T rho) {
  if constexpr (sizeof(T) == 8)
    return div_by(s_d, rho, __drcp_rn(rho));
  else
    return s_d * Arith<T>::rcp(rho);
}

// T arithmetic rounded as written for FP64, plain for FP32 (quotients by the
// hardware's approximate reciprocal, as elsewhere in the mixed stage).
template <typename T> __device__ __forceinline__ T xadd(T a, T b) {
  if constexpr (sizeof(T) == 8) return __dadd_rn(a, b); else return a + b;
}
template <typename T> __device__ __forceinline__ T xsub(T a, T b) {
  if constexpr (sizeof(T) == 8) return __dsub_rn(a, b); else return a - b;
}
template <typename T> __device__ __forceinline__ T xmul(T a, T b) {
  if constexpr (sizeof(T) == 8) return __dmul_rn(a, b); else return a * b;
}
template <typename T> __device__ __forceinline__ T xdiv(T a, T b) {  // FP32: by the approximate reciprocal
  if constexpr (sizeof(T) == 8) return __ddiv_rn(a, b); else return a * Arith<T>::rcp(b);
}

// The pressures of the sub-grid's 512 interior cells from the tile (every
// thread calls it, with the tile in place; ends with a barrier).  Mixed only:
// the FP64 kernel, at one CTA per SM, measured faster forming them in each
// direction's pass (560 against 574 ms per RK3 step on the 65536-leaf octree).
template <typename T>
__device__ void cw84_interior_pressures(const Shared<T>& sh, T gamma, T eta) {
  CwSmem<T>& m = cw_smem<T>();
  for (int c = threadIdx.x; c < CELLS; c += THREADS) {
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int t = k * SK + j * SJ + i;
    T U[NF];
#pragma unroll
    for (int q = 0; q < CW_F; ++q) U[cw_field(q)] = sh.tile[cw_field(q) * ISZ + t];
    m.pint[c] = cell_p(U, gamma, eta);
  }
  __syncthreads();
}

// The cell coefficients of direction D for the 64 pencils of the tile:
// coef[p][m - 2] (flattening) and coef[64 + p][m - 2] (steepening), m =
// 2..11.  Every thread of the CTA calls it; three passes (cell pressures and
// velocities; flattening candidates and steepening coefficients; the upstream
// maximum), scratch in the left face buffer, free before the PPM.
template <typename T, int D>
__device__ void cw84_coefficients(const Shared<T>& sh, const StageArgs& a, int s, const Nbr& nb, T gamma, T eta) {
  const int tid = threadIdx.x;
  const bool flat = (a.cw84 & 1) != 0, steep = (a.cw84 & 2) != 0;
  CwSmem<T>& cm = cw_smem<T>();
  T* P = sh.fsl;                 // [64][CW_P], P[p][m + 1] = pressure of cell m
  T* Uv = P + NPEN * CW_P;       // [64][CW_U] velocities along D
  T* FT = Uv + NPEN * CW_U;      // [64][NP] flattening candidates of cells m = 1..12
  // pressures of cells -1..14 (flattening) or 1..12 (steepening alone): the
  // interior ones from the sub-grid's table, the halo and fourth-layer ones by
  // the EOS; velocities of cells 0..13 (flattening)
  const int m_lo = flat ? -1 : 1, per = flat ? NP + 2 : 12;
  for (int e = tid; e < NPEN * per; e += THREADS) {
    const int p = e / per, m = m_lo + (e - p * per);
    T pr, u = T(0);
    if (sizeof(T) == 4 && m >= NG && m < NG + NX) {
      // mixed: the interior pressures were formed once for the sub-grid
      const int t = tile_index(D, p, m - NG);
      const int k = t / SK, j = (t - k * SK) / SJ, i = t - k * SK - j * SJ;
      pr = cm.pint[(k * NX + j) * NX + i];
      if (flat) u = cell_u(sh.tile[(F_SX + D) * ISZ + t], sh.tile[F_RHO * ISZ + t]);
    } else {
      T U[NF];
      if (m < 0 || m >= NP) {
        const int side = m < 0 ? 0 : 1;
#pragma unroll
        for (int q = 0; q < CW_F; ++q) {
          if constexpr (sizeof(T) == 4)
            U[cw_field(q)] = cm.l4[q][side][p];
          else
            U[cw_field(q)] = layer4_fp64<D>(a, s, nb, side, p & 7, p >> 3, cw_field(q));
        }
      } else {
#pragma unroll
        for (int q = 0; q < CW_F; ++q) U[cw_field(q)] = pencil_cell<T, D>(sh, cw_field(q), p, m);
      }
      pr = cell_p(U, gamma, eta);
      if (flat && m >= 0 && m < NP) u = cell_u(U[F_SX + D], U[F_RHO]);
    }
    P[p * CW_P + m + 1] = pr;
    if (m >= 0 && m < NP) Uv[p * CW_U + m] = u;
  }
  __syncthreads();
  // flattening candidates of cells 1..12 and steepening coefficients of 2..11
  for (int e = tid; e < NPEN * 22; e += THREADS) {
    const int p = e / 22, k = e - p * 22;
    const T* Pp = P + p * CW_P;
    if (k < 12) {
      const int m = 1 + k;
      T ft = T(0);
      if (flat) {
        const T* u = Uv + p * CW_U;
        const T pm1 = Pp[m], pp1 = Pp[m + 2], pm2 = Pp[m - 1], pp2 = Pp[m + 3];
        const T dp = xsub(pp1, pm1);
        const T pmin = pp1 < pm1 ? pp1 : pm1;
        if (fabs(dp) > xmul(T(0.33), pmin) && xsub(u[m - 1], u[m + 1]) > T(0)) {
          const T t = xmul(T(10), xsub(xdiv(dp, xsub(pp2, pm2)), T(0.75)));
          const T v = t > T(1) ? T(1) : t;
          ft = v > T(0) ? v : T(0);
        }
      }
      FT[p * NP + m] = ft;
    } else {
      const int m = 2 + (k - 12);
      T eta_c = T(0);
      if (steep) {
        T r[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) r[j] = pencil_cell<T, D>(sh, F_RHO, p, m - 2 + j);
        const T d2p = xsub(xadd(r[4], r[2]), xmul(T(2), r[3]));
        const T d2m = xsub(xadd(r[2], r[0]), xmul(T(2), r[1]));
        const T dr = xsub(r[3], r[1]);
        const T a1 = fabs(r[3]), a0 = fabs(r[1]);
        const T amin = a1 < a0 ? a1 : a0;
        T etat = T(0);
        if (xmul(d2p, d2m) < T(0) && xsub(fabs(dr), xmul(T(0.01), amin)) > T(0)) {
          const T rmin = r[3] < r[1] ? r[3] : r[1];
          const T pp1 = Pp[m + 2], pm1 = Pp[m];
          const T pmin = pp1 < pm1 ? pp1 : pm1;
          if (xdiv(xmul(xmul(gamma, T(0.1)), fabs(dr)), rmin) >= xdiv(fabs(xsub(pp1, pm1)), pmin))
            etat = xdiv(-xsub(d2p, d2m), xmul(T(6), dr));
        }
        const T t = xmul(T(20), xsub(etat, T(0.05)));
        const T v = t > T(1) ? T(1) : t;
        eta_c = v > T(0) ? v : T(0);
      }
      cm.coef[NPEN + p][m - 2] = eta_c;
    }
  }
  __syncthreads();
  // the flattening coefficient: the larger of the cell's candidate and its
  // upstream neighbour's (sigma = sgn(p_{m+1} - p_{m-1}), neighbour m - sigma)
  for (int e = tid; e < NPEN * CW_C; e += THREADS) {
    const int p = e / CW_C, m = 2 + (e - p * CW_C);
    T f = T(0);
    if (flat) {
      const T* Pp = P + p * CW_P;
      const T* ft = FT + p * NP;
      const T dp = xsub(Pp[m + 2], Pp[m]);
      const T fu = dp > T(0) ? ft[m - 1] : (dp < T(0) ? ft[m + 1] : ft[m]);
      f = fu > ft[m] ? fu : ft[m];
    }
    cm.coef[p][m - 2] = f;
  }
  __syncthreads();
}

// ppm_pencil with the cell coefficients fl, es of the pencil (m = 2..11):
// after the interpolant, l and r move to the steepened faces (q_{m-1} +
// dm_{m-1}/2, q_{m+1} - dm_{m+1}/2) by es, then toward q_m by fl, then the
// parabola limiter.
template <typename T>
__device__ __forceinline__ void ppm_pencil_cw(const T (&q)[NP], const T* fl, const T* es, T (&ul)[NFACE],
                                              T (&ur)[NFACE]) {
  T dm[NP];
#pragma unroll
  for (int m = 1; m <= 12; ++m) dm[m] = limited_slope2(q[m - 1], q[m], q[m + 1]);  // 2 x slope
  T face[NP];
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
    const T e = es[m - 2], f = fl[m - 2];
    if (e > T(0)) {
      const T w = xsub(T(1), e);
      l = xadd(xmul(l, w), xmul(xadd(q[m - 1], xmul(T(0.25), dm[m - 1])), e));
      r = xadd(xmul(r, w), xmul(xsub(q[m + 1], xmul(T(0.25), dm[m + 1])), e));
    }
    if (f > T(0)) {
      const T w = xsub(T(1), f);
      l = xadd(xmul(f, q[m]), xmul(w, l));
      r = xadd(xmul(f, q[m]), xmul(w, r));
    }
    parabola_limit(q[m], l, r);
    if (m <= 10) ul[m - 2] = r;
    if (m >= 3) ur[m - 3] = l;
  }
}

