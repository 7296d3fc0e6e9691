// Persistent smoother kernel: float, LIN_IEKS, 256 threads per block.
#include "pes_launch_impl.cuh"
PES_INSTANTIATE(float, pes::LIN_IEKS, 256)
