// Tensor-core building blocks for sm_103a: TMA tile loads, tcgen05 MMAs with
// accumulators in tensor memory (TMEM), and their completion barriers.
//
// Operand tiles are bf16, K-major, 128-byte swizzled: a tile of R rows holds
// 64 bf16 (128 B) per row in 1024-byte atoms of 8 rows, exactly what a TMA
// load with CU_TENSOR_MAP_SWIZZLE_128B and a {64, R} box writes. One MMA
// consumes K = 16 of the 64 columns; the next 16 start 32 bytes further on.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "pes_async.cuh"

namespace pes {
namespace tc {

// 2-D tiled TMA load of the box at (x, y) into shared memory, completing
// bytes on `bar`. x (the inner coordinate) must be a multiple of 8 bf16
// elements (16 bytes); y may be negative or past the end (zero fill).
PES_DEV void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 2-D tiled TMA store of the shared-memory box at (x, y) (both >= 0; rows past
// the end are not written), in the issuing thread's bulk async-group.
PES_DEV void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
                 "r"(y), "r"(smem_u32(src))
                 : "memory");
}

PES_DEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until at most N of this thread's bulk groups still read shared memory.
template <int N>
PES_DEV void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until all of this thread's bulk groups have completed.
PES_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

PES_DEV void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

PES_DEV void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait; returns false (and sets ST_TIMEOUT) when it gives up or when
// another role of the block has already given up (`*abort` != 0).
PES_DEV bool wait_or_abort(uint64_t* bar, uint32_t parity, int* status, volatile int* abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = async_now_ns();
    for (unsigned polls = 0;; ++polls) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (polls > (1u << 24) || async_now_ns() - t0 > 1000000000LL) {
            atomicOr(status, ST_TIMEOUT);
            *abort = 1;
            return false;
        }
    }
}

// ---- tensor memory -------------------------------------------------------------

// Allocate `ncols` TMEM columns (power of two >= 32); the whole warp calls.
// The TMEM address lands in *slot (shared memory).
PES_DEV void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

PES_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

PES_DEV void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
PES_DEV void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- descriptors ---------------------------------------------------------------

// Shared-memory matrix descriptor of a K-major, 128-byte-swizzled bf16 tile
// whose 8-row atoms are 1024 bytes apart, inside a swizzled region that begins
// 1024-aligned. The tile may start at any 128-byte row of that region: the
// swizzle follows the shared-memory address itself, so the base offset stays
// 0. Advancing along K inside the row adds multiples of 32 bytes.
PES_DEV uint64_t smem_desc_sw128(const void* tile)
{
    const uint64_t addr = smem_u32(tile);
    return ((addr >> 4) & 0x3FFFull)        // start address
           | (1ull << 16)                   // leading byte offset (unused for swizzled K-major)
           | ((1024ull >> 4) << 32)         // stride byte offset: next 8-row atom
           | (1ull << 46)                   // descriptor version
           | (2ull << 61);                  // 128-byte swizzle
}

// Shared-memory matrix descriptor of an MN-major, 128-byte-swizzled bf16
// operand: 64 consecutive M (or N) elements fill one 128-byte row, and
// consecutive K indices are consecutive rows, 8 rows to a 1024-byte atom
// (stride byte offset 1024 between 8-row K groups). This is what a TMA load of
// a row-major [rows][64] bf16 array with a 128-byte swizzle writes when the
// array's rows are the reduction (K) dimension. A 128-wide M spans two such
// 64-element blocks, `lbo` bytes apart (leading byte offset). As for the
// K-major form, the start may sit at any 128-byte row of a 1024-aligned
// swizzled region; the next K = 16 slice starts 2048 bytes further on.
PES_DEV uint64_t smem_desc_sw128_mn(const void* tile, uint32_t lbo)
{
    const uint64_t addr = smem_u32(tile);
    return ((addr >> 4) & 0x3FFFull)              // start address
           | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16)   // leading byte offset: next 64 M (N) elements
           | ((1024ull >> 4) << 32)               // stride byte offset: next 8 K rows
           | (1ull << 46)                         // descriptor version
           | (2ull << 61);                        // 128-byte swizzle
}

// Instruction descriptor of kind::f16: bf16 A and B (both K-major unless
// a_mn / b_mn select the MN-major form), f32 accumulator, shape M x N.
constexpr uint32_t idesc_bf16_f32(int M, int N, bool a_mn = false, bool b_mn = false)
{
    return (1u << 4)                        // D: f32
           | (1u << 7)                      // A: bf16
           | (1u << 10)                     // B: bf16
           | ((uint32_t)a_mn << 15)         // A major-ness (1: MN-major)
           | ((uint32_t)b_mn << 16)         // B major-ness
           | ((uint32_t)(N >> 3) << 17)     // N / 8
           | ((uint32_t)(M >> 4) << 24);    // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T for one K = 16 slice; issued by one thread.
PES_DEV void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// Arrive on `bar` once every MMA this thread has issued so far completes.
PES_DEV void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane (32x32b shape: the
// warp reads lanes 32 * (warp % 4) .. + 31, thread t lane + t).
PES_DEV void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive 32-bit columns of this thread's TMEM lane in one load and one
// wait (same lane layout as tmem_ld16).
PES_DEV void tmem_ld64(uint32_t taddr, float* v)
{
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, "
        "%36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, "
        "%57, %58, %59, %60, %61, %62, %63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
          "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
          "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
          "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
          "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace pes
