// Persistent smoother kernel: float, LIN_GH (Gauss-Hermite product rule), 128 threads per block.
#include "pes_launch_impl.cuh"
PES_INSTANTIATE(float, pes::LIN_GH, 128)
