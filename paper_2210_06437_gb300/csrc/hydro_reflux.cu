// hydro_reflux.cu -- coarse-fine flux correction after a mixed-precision RK
// stage, as a pass of its own: one CTA per coarse sub-grid (the correction
// itself is in hydro_reflux.cuh).  FP64 stages correct inside the stage
// kernel, which keeps them bit-identical to a plain evaluation; for the FP32
// stage a separate pass is cheaper: measured on the 65536-leaf octree, the
// in-stage form's export flags, waits and correction terms cost 1.6 ms per RK3
// step, this pass 0.45 ms.  (The one-launch RK3 step runs the same correction
// inside its launch, see hydro_stage.cu.)
#include "hydro_reflux.cuh"

namespace hydro {
namespace {

// RT threads per CTA and IPT items per thread: the launch shape, a tuning parameter.
template <typename T, int RT, int IPT>
__global__ void __launch_bounds__(RT, 1024 / RT) reflux_kernel(const RefluxArgs r) {
  __shared__ reflux::CorrSmem sm;
  reflux::correct_coarse<T, RT, IPT, false>(r, blockIdx.x, sm);
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
