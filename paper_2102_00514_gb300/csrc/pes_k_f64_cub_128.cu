// Persistent smoother kernel: double, LIN_CUBATURE, 128 threads per block.
#include "pes_launch_impl.cuh"
PES_INSTANTIATE(double, pes::LIN_CUBATURE, 128)
