"""GB300-native batched octree hydro step (PPM + central-upwind flux + update).

Modules: ``workloads`` (seeded synthetic inputs), ``hydro`` (binding of the C
ABI in include/hydro.h), ``build`` (in-tree nvcc build of libhydro.so),
``partition`` (Morton-range partition and proxy exchange of the sharded step),
``tune`` (launch-shape autotuner).
"""
