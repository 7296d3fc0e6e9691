// Dispatch from run-time (precision, linearisation, block size) to the
// compiled configurations of the persistent kernel.
#include "pes_internal.h"

namespace pes {

template <typename T, int NT>
static cudaError_t launch_nt(const KParams<T>& p, int lin, int nb, cudaStream_t st)
{
    if (lin == LIN_ARRAYS) return launch_cfg<T, LIN_ARRAYS, NT>(p, nb, st);
    if (lin == LIN_IEKS) return launch_cfg<T, LIN_IEKS, NT>(p, nb, st);
    if (lin == LIN_GH) return launch_cfg<T, LIN_GH, NT>(p, nb, st);
    return launch_cfg<T, LIN_CUBATURE, NT>(p, nb, st);
}

template <typename T, int NT>
static int capacity_nt(int lin, int device)
{
    if (lin == LIN_ARRAYS) return capacity_cfg<T, LIN_ARRAYS, NT>(device);
    if (lin == LIN_IEKS) return capacity_cfg<T, LIN_IEKS, NT>(device);
    if (lin == LIN_GH) return capacity_cfg<T, LIN_GH, NT>(device);
    return capacity_cfg<T, LIN_CUBATURE, NT>(device);
}

cudaError_t launch_persistent(const KParams<float>& p, int lin, int nt, int nb, cudaStream_t st)
{
    if (nt == 256) return launch_nt<float, 256>(p, lin, nb, st);
    if (nt == 128) return launch_nt<float, 128>(p, lin, nb, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_persistent(const KParams<double>& p, int lin, int nt, int nb, cudaStream_t st)
{
    if (nt == 128) return launch_nt<double, 128>(p, lin, nb, st);
    return cudaErrorInvalidValue;
}

int coop_capacity(float, int lin, int nt, int device)
{
    if (nt == 256) return capacity_nt<float, 256>(lin, device);
    if (nt == 128) return capacity_nt<float, 128>(lin, device);
    return 0;
}

int coop_capacity(double, int lin, int nt, int device)
{
    if (nt == 128) return capacity_nt<double, 128>(lin, device);
    return 0;
}

bool nt_supported(float, int nt) { return nt == 128 || nt == 256; }
bool nt_supported(double, int nt) { return nt == 128; }

}  // namespace pes
