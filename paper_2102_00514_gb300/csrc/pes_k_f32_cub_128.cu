// Persistent smoother kernel: float, LIN_CUBATURE, 128 threads per block.
#include "pes_launch_impl.cuh"
PES_INSTANTIATE(float, pes::LIN_CUBATURE, 128)
