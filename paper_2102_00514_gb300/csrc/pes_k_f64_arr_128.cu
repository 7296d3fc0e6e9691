// Persistent smoother kernel: double, LIN_ARRAYS, 128 threads per block.
#include "pes_launch_impl.cuh"
PES_INSTANTIATE(double, pes::LIN_ARRAYS, 128)
