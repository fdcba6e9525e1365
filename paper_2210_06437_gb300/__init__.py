"""GB300-native batched octree hydro step (PPM + central-upwind flux + update).

Modules: ``workloads`` (seeded synthetic inputs), ``hydro`` (binding of the C
ABI in include/hydro.h), ``build`` (in-tree nvcc build of libhydro.so),
``driver`` (lagged-CFL time stepping on the device), ``tune`` (launch-shape
autotuner).
"""
