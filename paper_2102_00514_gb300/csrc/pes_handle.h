// Host-side state behind a pes_handle (shared by the library's host
// translation units; not part of the public interface).
#pragma once

#include <stdint.h>

// Launch shape chosen by pes_autotune for one (linearisation, precision):
// threads per block and the minimum steps per lane (0: the defaults).
struct pes_tune {
    int nt = 0;
    int min_steps = 0;
};

struct pes_handle {
    int device = 0;
    int num_sms = 0;
    int64_t max_states = 0;
    int32_t max_batch = 0;
    int nl_max = 0;      // lanes the workspace is sized for
    int nb_max = 0;      // blocks the workspace is sized for
    void* hand = nullptr;
    void* aggF = nullptr;
    void* aggS = nullptr;
    unsigned* bar = nullptr;
    int* status = nullptr;
    double* conv = nullptr;
    int* iters_done = nullptr;
    int* traj_iters = nullptr;   // [max_batch]: per-trajectory iterations of the last tolerance-mode run
    int traj_iters_B = 0;        // its number of trajectories (0: none recorded)
    pes_tune tune[4][2];         // [linearisation (LIN_*)][FP32, FP64]
    // device copies for pes_ieks_run_host (allocated by its first call)
    void* hy = nullptr;
    int64_t* hoff = nullptr;
    void* hm0 = nullptr;
    void* hP0 = nullptr;
    void* hx = nullptr;
    void* hP = nullptr;
    double* hsens = nullptr;
    void* sensT = nullptr;   // sensors converted to the kernel precision
    void* lanes = nullptr;   // x, P, y in the kernel's lane-major layout
    void* lin = nullptr;     // cubature linearisation handed from the fold to the re-run
    void* mix = nullptr;     // FP64 copies for PES_MIXED (allocated by its first call)
    void* refw = nullptr;    // PES_REFINED workspace (allocated by its first call)
    void* lmw = nullptr;     // per-trajectory state of pes_ieks_run_lm (allocated by its first call)
    long long* ptime = nullptr;   // phase timestamps (PES_PHASE_TIMES=1)
    int ptime_blocks = 0;
    long long timeout_ns = 2000000000LL;
    // The test of the smoother kernel's barrier timeout (PES_TEST_BARRIER_SHORT
    // at pes_create): its launches start the barrier count one arrival short,
    // so no grid barrier completes; the first gives up after timeout_ns, the
    // kernel ends and the call returns PES_ERR_TIMEOUT. false otherwise.
    bool bar_short = false;
    char err[512] = {0};
};
