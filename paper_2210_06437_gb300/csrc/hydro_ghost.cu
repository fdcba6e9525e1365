// hydro_ghost.cu -- face ghost-slab fill of all sub-grids (paper Section VI:
// the hydro boundary exchange, done here as a direct device gather from the
// neighbours' interiors, the on-device analogue of the paper's direct memory
// access between sub-grids of the same locality).
//
// One thread per (sub-grid, face, field, layer, row, column) ghost cell,
// column fastest, so the 8 cells of a row are contiguous for y/z faces.
//   same level : copy of the neighbour's interior cell;
//   coarser    : value of the coarse cell containing the ghost-cell centre;
//   finer      : mean of the 2x2x2 fine cells, summed in (k, j, i) order, * 1/8;
//   boundary   : copy of the nearest interior cell (outflow).
// Reads only interior cells and writes only ghost cells, so the result does
// not depend on the order in which threads run.
#include "hydro_internal.cuh"

namespace hydro {
namespace {

__device__ __forceinline__ size_t cell_at(int s, int f, int i, int j, int k) {
  return field_offset(s, f) + (size_t)k * NP2 + j * NP + i;
}

__global__ void ghost_kernel(const GhostArgs a) {
  const size_t total = (size_t)a.n_sub * 6 * NF * NG * NX * NX;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int c1 = (int)(g & 7);
    const int c2 = (int)((g >> 3) & 7);
    size_t rest = g >> 6;
    const int layer = (int)(rest % NG);
    rest /= NG;
    const int f = (int)(rest % NF);
    rest /= NF;
    const int face = (int)(rest % 6);
    const int s = (int)(rest / 6);
    const int ax = face >> 1, side = face & 1;
    const int b1 = ax == 0 ? 1 : 0;   // first transverse axis
    const int b2 = ax == 2 ? 1 : 2;   // second transverse axis
    const int ga = side ? NX + layer : -1 - layer;  // interior coordinate of the ghost along ax
    int dst[3];
    dst[ax] = ga + NG;
    dst[b1] = c1 + NG;
    dst[b2] = c2 + NG;
    const int32_t* nb = a.nb + ((size_t)s * 6 + face) * 4;
    const int rel = a.rel[s * 6 + face];
    double v;
    if (nb[0] < 0) {
      int src[3] = {dst[0], dst[1], dst[2]};
      src[ax] = side ? NG + NX - 1 : NG;
      v = a.U[cell_at(s, f, src[0], src[1], src[2])];
    } else if (rel == 0) {
      int src[3] = {dst[0], dst[1], dst[2]};
      src[ax] = (side ? ga - NX : ga + NX) + NG;
      v = a.U[cell_at(nb[0], f, src[0], src[1], src[2])];
    } else if (rel < 0) {
      const int oc = a.oct[s];
      const int fa = ga >= 0 ? ga / 2 : -((1 - ga) / 2);  // floor(ga / 2)
      int src[3];
      src[ax] = (side ? -4 : 8) + fa + NG;
      src[b1] = 4 * ((oc >> b1) & 1) + (c1 >> 1) + NG;
      src[b2] = 4 * ((oc >> b2) & 1) + (c2 >> 1) + NG;
      v = a.U[cell_at(nb[0], f, src[0], src[1], src[2])];
    } else {
      const int q1 = c1 >> 2, q2 = c2 >> 2;
      const int fs = nb[q1 + 2 * q2];
      int base[3];
      base[ax] = 2 * (side ? ga - NX : ga + 4) + NG;
      base[b1] = 2 * (c1 - 4 * q1) + NG;
      base[b2] = 2 * (c2 - 4 * q2) + NG;
      double sum = 0.0;
#pragma unroll
      for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
          for (int di = 0; di < 2; ++di) sum = __dadd_rn(sum, a.U[cell_at(fs, f, base[0] + di, base[1] + dj, base[2] + dk)]);
      v = __dmul_rn(sum, 0.125);
    }
    a.U[cell_at(s, f, dst[0], dst[1], dst[2])] = v;
  }
}

}  // namespace

cudaError_t launch_ghost_fill(const GhostArgs& a, int threads, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t total = (size_t)a.n_sub * 6 * NF * NG * NX * NX;
  size_t blocks = (total + threads - 1) / threads;
  const size_t cap = (size_t)sms * (2048 / threads) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ghost_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hydro

// ---------------------------------------------------------------------------
// FP32 shadow of the interior: per sub-grid field, the 512 interior cells
// RN32(U[s][f][k+3][j+3][i+3]) at (k*8 + j)*8 + i, then the 64 cells of its
// 2x2x2 restriction at 512 + (K*4 + J)*4 + I: the FP32 pairwise sum of the 8
// rounded cells (pairs in i, then in j, then in k), times 1/8.  The mixed stage reads its
// reconstruction inputs (own interior, the neighbours' boundary layers and the
// finer neighbours' restrictions) from the shadow: half the bytes of the FP64
// state, in 32-byte rows, every halo cell a plain copy.
// ---------------------------------------------------------------------------

namespace hydro {
namespace {

// FP64 -> FP32 with integer operations: round to nearest on the magnitude
// (ties away from zero); values below the FP32 normal range become signed
// zero, larger finite values infinity, NaN stays NaN.  (The same rounding as
// the stage kernel's own conversion.)
__device__ __forceinline__ float shadow_round(double x) {
  const unsigned lo = (unsigned)__double2loint(x), hi = (unsigned)__double2hiint(x);
  const unsigned mag = hi & 0x7fffffffu;
  unsigned r = __funnelshift_l(lo, hi, 3) + ((lo >> 28) & 1u) - 0xC0000000u;
  if (mag - 0x38100000u >= 0x0FE00000u) {
    r = mag < 0x38100000u ? 0u : ((mag > 0x7ff00000u || (mag == 0x7ff00000u && lo)) ? 0x7fc00000u : 0x7f800000u);
  }
  return __uint_as_float(r | (hi & 0x80000000u));
}

__global__ void __launch_bounds__(256) shadow_kernel(const double* __restrict__ U, float* __restrict__ S, int n) {
  const size_t total = (size_t)n * NF * SHADOW_FIELD;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const size_t sf = g / SHADOW_FIELD;  // s * NF + f
    const int c = (int)(g - sf * SHADOW_FIELD);
    const double* u = U + sf * NP3;
    if (c < SHADOW_COARSE) {
      const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
      S[g] = shadow_round(u[(size_t)(k + NG) * NP2 + (j + NG) * NP + (i + NG)]);
    } else {
      const int cc = c - SHADOW_COARSE;
      const int I = cc & 3, J = (cc >> 2) & 3, K = cc >> 4;
      const double* b = u + (size_t)(2 * K + NG) * NP2 + (2 * J + NG) * NP + (2 * I + NG);
      float h[2];  // pairwise: ((c000 + c001) + (c010 + c011)) + ((c100 + c101) + (c110 + c111)), c_{dk dj di}
#pragma unroll
      for (int dk = 0; dk < 2; ++dk) {
        const double* bk = b + dk * NP2;
        h[dk] = __fadd_rn(__fadd_rn(shadow_round(bk[0]), shadow_round(bk[1])),
                          __fadd_rn(shadow_round(bk[NP]), shadow_round(bk[NP + 1])));
      }
      S[g] = __fmul_rn(__fadd_rn(h[0], h[1]), 0.125f);
    }
  }
}

// The shadows a stage over a batch reads: one CTA per batch item writes the
// shadow of the item's sub-grid and of every face neighbour its halo gather
// reads (the neighbour of a same-level or coarser face, the four of a finer
// one), each value as shadow_kernel writes it; a sub-grid named by several
// items is written several times with the same values.  Ids outside [0, n)
// are skipped (the stage reports them); a flux-only flag is ignored.
__global__ void __launch_bounds__(256) shadow_ids_kernel(const double* __restrict__ U, float* __restrict__ S,
                                                         const int32_t* __restrict__ ids, int n,
                                                         const int32_t* __restrict__ nb,
                                                         const int8_t* __restrict__ rel) {
  __shared__ int list[25];
  __shared__ int count;
  int s = ids[blockIdx.x];
  if (s >= 0) s &= ~ITEM_FLUX_ONLY;
  if (s < 0 || s >= n) return;  // uniform over the block
  if (threadIdx.x == 0) {
    int c = 0;
    list[c++] = s;
    for (int face = 0; face < 6; ++face) {
      const int r = rel[s * 6 + face];
      for (int q = 0; q < (r == 1 ? 4 : 1); ++q) {
        const int x = nb[((size_t)s * 6 + face) * 4 + q];
        if (x >= 0 && x < n) list[c++] = x;
      }
    }
    count = c;
  }
  __syncthreads();
  for (int e = 0; e < count; ++e) {
    const int x = list[e];
    for (int t = threadIdx.x; t < NF * SHADOW_FIELD; t += blockDim.x) {
      const size_t g = (size_t)x * NF * SHADOW_FIELD + t;
      const size_t sf = g / SHADOW_FIELD;
      const int c = t % SHADOW_FIELD;
      const double* u = U + sf * NP3;
      if (c < SHADOW_COARSE) {
        const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
        S[g] = shadow_round(u[(size_t)(k + NG) * NP2 + (j + NG) * NP + (i + NG)]);
      } else {
        const int cc = c - SHADOW_COARSE;
        const int I = cc & 3, J = (cc >> 2) & 3, K = cc >> 4;
        const double* b = u + (size_t)(2 * K + NG) * NP2 + (2 * J + NG) * NP + (2 * I + NG);
        float h[2];
#pragma unroll
        for (int dk = 0; dk < 2; ++dk) {
          const double* bk = b + dk * NP2;
          h[dk] = __fadd_rn(__fadd_rn(shadow_round(bk[0]), shadow_round(bk[1])),
                            __fadd_rn(shadow_round(bk[NP]), shadow_round(bk[NP + 1])));
        }
        S[g] = __fmul_rn(__fadd_rn(h[0], h[1]), 0.125f);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Dual-energy reset of the entropy tracer (the paper is silent on the EOS;
// this completes the dual-energy switch of the face EOS): in every interior cell where
// the internal energy e_i = E - |s|^2 / 2 rho is positive and at least eta E
// (the complement of the face EOS test e_i < eta E), tau = e_i^(1/gamma).
// e_k and e_i are formed in FP64 (FP64 handles: as the face EOS forms them;
// mixed: 1/rho from a refined FP32 reciprocal); the power is FP64 for FP64
// handles and FP32 (powf, about 1 ulp) for mixed ones.  One CTA per
// sub-grid; with a shadow S (mixed), its tau field and tau restriction are
// rewritten exactly as the shadow kernel would write them from the new state.
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void __launch_bounds__(256) tau_resync_kernel(double* __restrict__ U, float* __restrict__ S,
                                                         double inv_gamma, double eta) {
  __shared__ float st[CELLS];  // RN32 of the new tracer (mixed shadow)
  double* u = U + (size_t)blockIdx.x * NF * NP3;
  for (int c = threadIdx.x; c < CELLS; c += blockDim.x) {
    const size_t o = (size_t)((c >> 6) + NG) * NP2 + (((c >> 3) & 7) + NG) * NP + ((c & 7) + NG);
    const double rho = u[o], sx = u[NP3 + o], sy = u[2 * NP3 + o], sz = u[3 * NP3 + o], E = u[4 * NP3 + o];
    double tau = u[(size_t)F_TAU * NP3 + o];
    double ek;
    if constexpr (MIXED) {
      // 1/rho: FP32 reciprocal, one Newton step in FP64 (relative error about
      // 2^-46), a handful of FP64 operations where a division takes a dozen
      const double r0 = (double)__frcp_rn((float)rho);
      const double r = fma(r0, fma(-rho, r0, 1.0), r0);
      ek = 0.5 * (fma(sx, sx, fma(sy, sy, sz * sz)) * r);
    } else {
      const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)), __dmul_rn(sz, sz));
      ek = __ddiv_rn(__dmul_rn(0.5, s2), rho);
    }
    const double ei = __dsub_rn(E, ek);
    if (ei > 0.0 && ei >= __dmul_rn(eta, E)) {
      if constexpr (MIXED)
        tau = (double)powf((float)ei, (float)inv_gamma);
      else
        tau = pow(ei, inv_gamma);
      u[(size_t)F_TAU * NP3 + o] = tau;
    }
    if constexpr (MIXED) st[c] = shadow_round(tau);
  }
  if (!MIXED || !S) return;  // uniform over the block
  __syncthreads();
  float* sf = S + ((size_t)blockIdx.x * NF + F_TAU) * SHADOW_FIELD;
  for (int c = threadIdx.x; c < CELLS; c += blockDim.x) sf[c] = st[c];
  if (threadIdx.x < CELLS / 8) {
    const int cc = threadIdx.x, I = cc & 3, J = (cc >> 2) & 3, K = cc >> 4;
    const float* b = st + (2 * K) * 64 + (2 * J) * 8 + 2 * I;
    float h[2];  // pairwise, as the shadow kernel: in i, then j, then k
#pragma unroll
    for (int dk = 0; dk < 2; ++dk) {
      const float* bk = b + dk * 64;
      h[dk] = __fadd_rn(__fadd_rn(bk[0], bk[1]), __fadd_rn(bk[8], bk[9]));
    }
    sf[SHADOW_COARSE + cc] = __fmul_rn(__fadd_rn(h[0], h[1]), 0.125f);
  }
}

}  // namespace

cudaError_t launch_tau_resync(double* U, float* S, int n, double gamma, double eta, bool mixed, cudaStream_t st) {
  if (n < 1 || !(eta > 0.0)) return cudaSuccess;
  if (mixed)
    tau_resync_kernel<true><<<n, 256, 0, st>>>(U, S, 1.0 / gamma, eta);
  else
    tau_resync_kernel<false><<<n, 256, 0, st>>>(U, nullptr, 1.0 / gamma, eta);
  return cudaGetLastError();
}

cudaError_t launch_shadow_ids(const double* U, float* S, const int32_t* ids, int n_items, int n, const int32_t* nb,
                              const int8_t* rel, cudaStream_t st) {
  if (n_items < 1) return cudaSuccess;
  shadow_ids_kernel<<<n_items, 256, 0, st>>>(U, S, ids, n, nb, rel);
  return cudaGetLastError();
}

cudaError_t launch_shadow(const double* U, float* S, int n, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t total = (size_t)n * NF * SHADOW_FIELD;
  size_t blocks = (total + 255) / 256;
  const size_t cap = (size_t)sms * 8 * 4;
  if (blocks > cap) blocks = cap;
  shadow_kernel<<<(unsigned)(blocks ? blocks : 1), 256, 0, st>>>(U, S, n);
  return cudaGetLastError();
}

}  // namespace hydro

// ---------------------------------------------------------------------------
// Packed interiors: P[s][f][(k*8 + j)*8 + i] = U[s][f][k+3][j+3][i+3], the
// state without its ghost cells (5.36x fewer bytes than the padded layout), for
// moving states between host and device.
// ---------------------------------------------------------------------------

namespace hydro {
namespace {

__global__ void __launch_bounds__(256) pack_kernel(const double* __restrict__ U, double* __restrict__ P, int n) {
  const size_t total = (size_t)n * NF * CELLS;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(g & (CELLS - 1));
    const size_t sf = g >> 9;
    P[g] = U[sf * NP3 + (size_t)((c >> 6) + NG) * NP2 + (((c >> 3) & 7) + NG) * NP + ((c & 7) + NG)];
  }
}

__global__ void __launch_bounds__(256) unpack_kernel(const double* __restrict__ P, double* __restrict__ U, int n) {
  const size_t total = (size_t)n * NF * CELLS;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(g & (CELLS - 1));
    const size_t sf = g >> 9;
    U[sf * NP3 + (size_t)((c >> 6) + NG) * NP2 + (((c >> 3) & 7) + NG) * NP + ((c & 7) + NG)] = P[g];
  }
}

size_t layout_blocks(int n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t total = (size_t)n * NF * CELLS;
  size_t blocks = (total + 255) / 256;
  const size_t cap = (size_t)sms * 8 * 4;
  return blocks > cap ? cap : (blocks ? blocks : 1);
}

}  // namespace

cudaError_t launch_pack(const double* U, double* P, int n, cudaStream_t st) {
  pack_kernel<<<(unsigned)layout_blocks(n), 256, 0, st>>>(U, P, n);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const double* P, double* U, int n, cudaStream_t st) {
  unpack_kernel<<<(unsigned)layout_blocks(n), 256, 0, st>>>(P, U, n);
  return cudaGetLastError();
}

}  // namespace hydro
