// pes_ieks_run_noalloc: the iterated smoother for callers that must not
// allocate device memory.
//
// Some callers cannot create a pes_handle, because creating one allocates its
// workspace with cudaMalloc: code that runs where the process's memory plan is
// fixed after start-up (a real-time loop, a service with a pre-reserved memory
// budget), code living inside a framework that owns every device allocation
// through its own pool and forbids raw allocations, or latency-critical code
// that cannot afford an allocation that may synchronise the device. For them
// this entry point runs the same smoother with its scratch in one file-scope
// __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "pes.h"
#include "pes_handle.h"
#include "pes_internal.h"
#include "pes_trace.h"

namespace {

constexpr int64_t kMaxStates = PES_NOALLOC_MAX_STATES;
constexpr int32_t kMaxBatch = PES_NOALLOC_MAX_BATCH;
constexpr int kMaxBlocks = 8;                  // cooperative blocks one call may use
constexpr int kMaxThreads = 256;               // threads per block of any compiled configuration
// Lane-major arrays hold L * lanes >= N states: N plus one launch's lanes at most.
constexpr int64_t kLaneCap = kMaxStates + (int64_t)kMaxBlocks * kMaxThreads;

// Scratch layout, in doubles (a float run uses the first half of each region).
constexpr size_t kHand = (size_t)pes::HAND * kLaneCap;
constexpr size_t kLanes = (size_t)22 * kLaneCap;
constexpr size_t kLin = (size_t)pes::LINS * kLaneCap;
constexpr size_t kAggF = (size_t)kMaxBlocks * pes::FE;
constexpr size_t kAggS = (size_t)kMaxBlocks * pes::SE;
constexpr size_t kConv = (size_t)4 * kMaxBatch;
constexpr size_t kSens = (size_t)4 * kMaxBatch;
constexpr size_t kWords = 4;                   // barrier counter, status, iteration count (one double each)
constexpr size_t kTotal = kHand + kLanes + kLin + kAggF + kAggS + kConv + kSens + kWords;

constexpr int kMaxDevices = 64;

}  // namespace

// The scratch of every call on this device. Calls share it: their contents
// persist from one call to the next, and calls that overlap in time on the
// GPU (e.g. on two streams) race on it.
static __device__ __align__(256) double g_pes_noalloc_scratch[kTotal];

namespace {

std::mutex g_mu;
bool g_ready[kMaxDevices];
pes_handle g_handle[kMaxDevices];

// Once per device, with that device current: find the device address of the
// scratch array (host code cannot use the symbol itself as an address), carve
// it into the workspace a pes_handle describes, and clear the words that must
// start at zero.
pes_status setup(int dev)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_ready[dev]) return PES_OK;
    void* base = nullptr;
    if (cudaGetSymbolAddress(&base, g_pes_noalloc_scratch) != cudaSuccess || !base) return PES_ERR_CUDA;
    int coop = 0, sms = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
        return PES_ERR_UNSUPPORTED;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PES_ERR_CUDA;
    double* p = static_cast<double*>(base);
    pes_handle& h = g_handle[dev];
    h.device = dev;
    h.num_sms = sms;
    // the same time limit on grid-wide waits as pes_create gives a handle
    if (const char* env = getenv("PES_BARRIER_TIMEOUT_MS")) {
        const long long ms = atoll(env);
        if (ms > 0) h.timeout_ns = ms * 1000000LL;
    }
    h.max_states = kMaxStates;
    h.max_batch = kMaxBatch;
    h.nb_max = kMaxBlocks;
    h.nl_max = kMaxBlocks * kMaxThreads;
    h.hand = p;
    p += kHand;
    h.lanes = p;
    p += kLanes;
    h.lin = p;
    p += kLin;
    h.aggF = p;
    p += kAggF;
    h.aggS = p;
    p += kAggS;
    h.conv = p;
    p += kConv;
    h.sensT = p;
    p += kSens;
    h.bar = reinterpret_cast<unsigned*>(p);
    h.status = reinterpret_cast<int*>(p + 1);
    h.iters_done = reinterpret_cast<int*>(p + 2);
    if (cudaMemset(p, 0, sizeof(double) * kWords) != cudaSuccess) return PES_ERR_CUDA;
    g_ready[dev] = true;
    return PES_OK;
}

}  // namespace

extern "C" pes_status pes_ieks_run_noalloc(const pes_model* model, pes_method method, pes_precision prec,
                                           const void* y, const int64_t* offsets, int32_t B, int64_t N,
                                           const void* m0, const void* P0, const void* x_init, const void* P_init,
                                           int32_t max_iters, double tol, void* x_out, void* P_out,
                                           int32_t* iters_used, void* stream)
{
    pes::TraceRange trace_("pes_ieks_run_noalloc");
    if (N > kMaxStates || B > kMaxBatch || N < 1 || B < 1) return PES_ERR_INVALID_ARG;
    // PES_MIXED's FP64 copies and PES_REFINED's workspace would be allocated
    if (prec == PES_MIXED || prec == PES_REFINED) return PES_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PES_ERR_CUDA;
    const pes_status st = setup(dev);
    if (st != PES_OK) return st;
    int32_t used = 0;
    // iters_used != NULL makes pes_ieks_run wait for the work and report the
    // device status, so the call returns with its scratch no longer in use.
    const pes_status r = pes_ieks_run(&g_handle[dev], model, method, prec, y, offsets, B, N, m0, P0, x_init, P_init,
                                      max_iters, tol, x_out, P_out, &used, stream);
    if (r != PES_OK && r != PES_ERR_NOT_CONVERGED) {
        // a failure after some work was queued returns before that work is
        // waited for: wait here, and clear the status word, so that the call
        // still returns with the scratch idle and the next call starts clean
        cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        cudaMemset(g_handle[dev].status, 0, sizeof(int));
        cudaGetLastError();
    }
    if (iters_used) *iters_used = used;
    return r;
}
