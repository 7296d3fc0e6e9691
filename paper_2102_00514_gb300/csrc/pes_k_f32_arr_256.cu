// Persistent smoother kernel: float, LIN_ARRAYS, 256 threads per block.
#include "pes_launch_impl.cuh"
PES_INSTANTIATE(float, pes::LIN_ARRAYS, 256)
