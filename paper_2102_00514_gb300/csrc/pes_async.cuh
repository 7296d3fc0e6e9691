// Per-warp streams of per-step blocks, prefetched into shared memory by bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier).
//
// The handoff buffers are laid out [warp][step][component][32 lanes], so the
// data a warp needs at one step is one contiguous block. A stream keeps two
// shared-memory stages per warp: while the warp consumes step s from one
// stage, the copy of the next step lands in the other. One lane issues the
// copies; every lane reads its own column of the stage.
//
// Every wait is bounded: after about a second a wait gives up, sets
// ST_TIMEOUT in the status word and returns, so the kernel always ends.
#pragma once

#include "pes_model.cuh"

namespace pes {

PES_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

PES_DEV void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the asynchronous proxy.
PES_DEV void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Order earlier generic-proxy shared-memory accesses before later bulk copies.
PES_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing a transaction count on `bar`.
PES_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

PES_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

PES_DEV long long async_now_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of `bar` with the given parity to complete.
PES_DEV void mbar_wait(uint64_t* bar, uint32_t parity, int* status)
{
    if (mbar_try_wait(bar, parity)) return;
    const long long t0 = async_now_ns();
    for (unsigned polls = 0;; ++polls) {
        if (mbar_try_wait(bar, parity)) return;
        if (polls > (1u << 24) || async_now_ns() - t0 > 1000000000LL) {
            atomicOr(status, ST_TIMEOUT);
            return;
        }
    }
}

// Stream of one warp through blocks of NC * 32 scalars spaced SLOT * 32
// scalars apart (step s of the warp's slot range at base + s * SLOT * 32).
template <typename T, int NC, int SLOT>
struct WarpStream {
    static constexpr uint32_t kBytes = NC * 32 * sizeof(T);
    static_assert(kBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
    const T* base;   // global: this warp's step 0
    T* stage;        // shared: [2][NC * 32]
    uint64_t* bar;   // shared: 2 barriers
    uint32_t parity; // expected parity per stage (bit i)
    int lane;

    // `par` is the warp's barrier parity state, carried across streams that
    // reuse the same barriers.
    PES_DEV void init(const T* warp_base, T* stage_mem, uint64_t* bars, uint32_t par)
    {
        base = warp_base;
        stage = stage_mem;
        bar = bars;
        parity = par;
        lane = threadIdx.x & 31;
    }
    // Start the copy of step s into stage i (all lanes call; lane 0 issues).
    // The stage must no longer be read (a __syncwarp since its last use).
    PES_DEV void issue(int s, int i)
    {
        if (lane == 0) {
            fence_proxy_async();
            bulk_g2s(stage + i * NC * 32, base + (size_t)s * SLOT * 32, kBytes, bar + i);
        }
    }
    PES_DEV void wait(int i, int* status)
    {
        mbar_wait(bar + i, (parity >> i) & 1u, status);
        parity ^= (1u << i);
    }
    PES_DEV T get(int i, int c) const { return stage[i * NC * 32 + c * 32 + lane]; }
};

}  // namespace pes
