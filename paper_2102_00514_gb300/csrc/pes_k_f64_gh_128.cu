// Persistent smoother kernel: double, LIN_GH (Gauss-Hermite product rule), 128 threads per block.
#include "pes_launch_impl.cuh"
PES_INSTANTIATE(double, pes::LIN_GH, 128)
