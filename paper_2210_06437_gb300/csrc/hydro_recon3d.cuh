// hydro_recon3d.cuh -- the launch interface of the three-dimensional
// reconstruction with Simpson face quadrature (hydro_recon3d.cu; not part of
// the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace hydro {

// One stage with the three-dimensional reconstruction and Simpson face
// quadrature (grids of one level; FP64, or mixed precision).
struct Recon3dArgs {
  const double* Uin;
  const double* U0;      // nullptr when beta == 1
  double* Uout;
  const int32_t* ids;    // [n_items] sub-grid ids
  int32_t n_items;
  int32_t n_sub;
  const double* dx;      // [n]
  const int32_t* nb;     // [n][6][4] face neighbours
  double beta;
  double dt;
  const double* dt_dev;  // when non-null, dt is read from device memory
  double gamma;
  double eta;
  int32_t form;          // 0 KNP, 1 KT
  int32_t mixed;         // 0: FP64 throughout; 1: FP32 reconstruction and fluxes, FP64 update
  double* fa;            // scratch: face averages, recon3d_scratch_doubles(n_items, 0) (FP32 uses half)
  double* fl;            // scratch: face fluxes, recon3d_scratch_doubles(n_items, 1) (FP32 uses half)
  unsigned long long* max_speed;  // [2] ordered bits of non-negative doubles
  int* err;
};

cudaError_t recon3d_prepare();  // kernel attributes of the current device (once per device; the launch calls it too)
cudaError_t launch_recon3d(const Recon3dArgs& a, cudaStream_t st);
// scratch doubles of the 3D stage for n_items items: which 0 face averages, 1 fluxes
size_t recon3d_scratch_doubles(int n_items, int which);

}  // namespace hydro
