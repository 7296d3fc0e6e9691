// The learned initialiser (include/pes_init.h): a 1-D conv / MLP network on
// the tensor cores that maps a trajectory's measurements to the initial
// nominal trajectory of the iterated smoother (Sec. 3), with its training.
//
// Row layout. The states of B trajectories are stored as activation rows of
// 64 bf16 channels (128 bytes): state k of trajectory b sits at row
// k + 2 (b + 1), so that two zero rows separate consecutive trajectories and
// frame the batch. A kernel-5 convolution over rows then sees zeros outside
// each trajectory, which is the "same" zero padding per trajectory, and the
// 1x1 layers need no special case. The features kernel writes every row of the
// input (zeros on the gap rows), every bf16 layer writes zeros on the gap rows
// of its output (the FP32 head writes the state rows only) and the loss
// gradient's gap rows are zeroed apart; R = N + 2 (B + 1) rows in all.
//
// Every layer is one GEMM on the tensor cores (conv_tc_kernel): a tile of 128
// rows times K = taps x 64 input channels, N = 64 output channels, bf16
// operands and an FP32 accumulator in tensor memory. Per row tile one TMA load
// brings the 128 + taps - 1 rows starting taps / 2 rows earlier (rows outside
// 0..R-1 read as zero), and tap j's MMAs read them from row j on; the layer's
// weights, one 64 x 64 tile per tap, stay in shared memory for the whole
// launch. Warp 0 issues the loads, warp 1 the MMAs; two accumulators in TMEM,
// drained by two epilogue warpgroups (warps 2-5 and 6-9), let the epilogues of
// consecutive tiles run at once and overlap the MMAs of the next. An epilogue
// applies bias and ReLU (or the ReLU mask of the backward pass), stages its
// warp's 32 bf16 rows in shared memory and writes them with one TMA store. The
// backward pass through a layer is the same GEMM with the weights transposed
// and the taps reversed. The last convolution and the two head layers run as
// one launch (tail_tc_kernel), their intermediate tiles kept in shared memory. The weight gradients, a reduction over rows, are a
// GEMM on the tensor cores too (wgrad_tc_kernel), split over the CTAs and
// summed in a fixed order.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "pes.h"
#include "pes_init.h"
#include "pes_trace.h"
#include "pes_tc.cuh"

namespace {

using namespace pes;
using bf16 = __nv_bfloat16;

constexpr int C = 64;                  // channels
constexpr int G = 2;                   // zero rows around each trajectory (kernel 5 / 2)
constexpr int TM = 128;                // rows per tile (MMA M)
constexpr int NSTAGE = 8;              // activation tiles in flight per CTA
constexpr int NLAYER = 6;              // 4 conv + 2 head
// A convolution with TAPS > 1 loads one halo tile of TM + TAPS - 1 rows per row
// tile (tap j reads its rows j .. j + TM - 1); a stage is rounded up to the
// 1024-byte swizzle pattern.
constexpr int halo_rows(int taps) { return TM + taps - 1; }
constexpr int stage_bytes(int taps) { return (halo_rows(taps) * C * 2 + 1023) / 1024 * 1024; }
constexpr int kWTileBytes = C * C * 2;
constexpr int kEpiThreads = 128;      // one epilogue warpgroup (per accumulator)
constexpr int kConvThreads = 64 + 2 * kEpiThreads;
constexpr uint32_t kTmemCols = 128;    // two 64-column FP32 accumulators
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(TM, C);

constexpr int kTaps[NLAYER] = {5, 5, 5, 5, 1, 1};
constexpr int kWTile0[NLAYER] = {0, 5, 10, 15, 20, 21};   // first weight tile of each layer
constexpr int kWTiles = 22;
constexpr int kPOff[NLAYER + 1] = {0, 20544, 41088, 61632, 82176, 86336, 86661};   // packed offsets
static_assert(kPOff[NLAYER] == PES_INIT_NPARAMS, "parameter packing");
static_assert(kTaps[0] == 5 && kTaps[NLAYER - 1] == 1 && kWTile0[NLAYER - 1] + kTaps[NLAYER - 1] == kWTiles, "layer tables");
constexpr int kOutCols = 8;            // the head's FP32 output row (5 used)
constexpr int kOutWarpBytes = 32 * C * 2;                  // 32 bf16 rows of one epilogue warp
constexpr int kOutStageOffset = 1024;                       // after the barriers and the bias (1024-aligned)

enum { EPI_RELU = 0, EPI_F32 = 1, EPI_MASK = 2 };

// Weight gradients on the tensor cores (wgrad_tc_kernel, and the backward
// convolutions that fuse them): MN-major operands straight from the row-major
// activation tiles, two taps stacked along M = 128, the odd last tap paired
// with an all-ones block (its products are the bias gradient).
constexpr int kWgStages = 4;
constexpr int kWgThreads = 192;
constexpr int kOnesBytes = TM * C * 2;                    // 128 rows of bf16 1.0
constexpr int kDyBytes = TM * C * 2;
constexpr int wg_groups(int taps) { return (taps + 1) / 2; }
constexpr int wg_stage(int taps) { return stage_bytes(taps) + kDyBytes; }
constexpr uint32_t wg_tmem_cols(int taps) { return wg_groups(taps) * C <= 64 ? 64u : 256u; }
constexpr int kWgPart = 3 * C * TM;                       // floats per CTA partial ([group][o][m])
constexpr uint32_t kIdescWg = tc::idesc_bf16_f32(TM, C, true, true);

// The conv kernel's pipeline depth and tensor memory (a fused weight gradient
// doubles the stage and adds its accumulators after the two conv ones).
constexpr int conv_nstage(bool wg) { return wg ? 4 : NSTAGE; }
constexpr int conv_stage(int taps, bool wg) { return stage_bytes(taps) * (wg ? 2 : 1); }
constexpr uint32_t conv_tmem_cols(int taps, bool wg) { return !wg ? kTmemCols : (taps > 1 ? 512u : 256u); }

// The same layer tables for device code.
PES_DEV int taps_of(int l) { return l < 4 ? 5 : 1; }
PES_DEV int wtile0_of(int l) { return l < 4 ? 5 * l : 16 + l; }
PES_DEV int coreal_of(int l) { return l == 5 ? 5 : C; }
PES_DEV int poff_of(int l) { return l < 4 ? 20544 * l : (l == 4 ? 82176 : 86336); }

struct ConvParams {
    int R;                      // rows
    int ntiles;                 // ceil(R / TM)
    int w_tile0;                // first weight tile of the layer
    const float* bias;          // [64] (EPI_RELU, EPI_F32)
    const uint8_t* rowmask;     // [R]: 1 for state rows
    bf16* out;                  // [R][64] (EPI_RELU, EPI_MASK)
    float* out_f32;             // [R][8] (EPI_F32)
    const bf16* relu_src;       // [R][64] (EPI_MASK): the layer input whose ReLU is differentiated
    float* part;                // fused weight gradient: [gridDim.x][kWgPart] partials
    int co_real;                // output channels that exist (the partial rows written)
    int* status;
};

PES_DEV uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

PES_DEV float2 unpack_bf16x2(uint32_t u)
{
    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&u);
    return __bfloat1622float2(h);
}

// Bounded wait that ignores the abort flag (used while draining).
PES_DEV void drain_wait(uint64_t* bar, uint32_t parity)
{
    const long long t0 = async_now_ns();
    while (!mbar_try_wait(bar, parity))
        if (async_now_ns() - t0 > 1000000000LL) return;
}

// Programmatic dependent launch: every kernel here is launched so that it may
// start while its predecessor in the stream is still finishing. A kernel
// waits for the predecessor (and so, transitively, for everything before it)
// before it touches data that the predecessor may write or read, then lets
// its own successor launch. Since every kernel triggers only after its own
// wait, whatever was written two or more launches earlier is final when a
// kernel starts: the layers read their weights before the wait (every entry
// point runs the features kernel between a parameter update and a layer).
PES_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
PES_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// WG (with EPI_MASK): the same launch also accumulates the layer's weight
// gradient. The layer input's halo tile (tmX, the ReLU source) is loaded beside
// each gradient tile; after a tile's conv MMAs the MMA thread adds, as in
// wgrad_tc_kernel, the products of the input taps with the tile's own gradient
// rows (rows TAPS / 2 .. TAPS / 2 + TM - 1 of the gradient's halo tile) into
// accumulators after the two conv ones, and the epilogue warps write the
// CTA's partial once all tiles are done.
template <int TAPS, int EPI, bool WG = false>
__global__ void __launch_bounds__(kConvThreads, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
                   const __grid_constant__ CUtensorMap tmOut, const __grid_constant__ CUtensorMap tmX,
                   const ConvParams p)
{
    static_assert(!WG || EPI == EPI_MASK, "the weight gradient fuses into backward convolutions");
    constexpr int NS = conv_nstage(WG);
    constexpr int NG = wg_groups(TAPS);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sW = smem;                                   // TAPS weight tiles
    uint8_t* sOnes = smem + TAPS * kWTileBytes;           // WG: the all-ones block
    constexpr int kStage = conv_stage(TAPS, WG);
    uint8_t* sA = sOnes + (WG ? kOnesBytes : 0);          // NS stages: halo tile (and, WG, the input's)
    uint64_t* full = reinterpret_cast<uint64_t*>(sA + NS * kStage);
    uint64_t* empty = full + NS;
    uint64_t* wbar = empty + NS;
    uint64_t* tfull = wbar + 1;
    uint64_t* tempty = tfull + 2;
    uint64_t* done = tempty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    float* sbias = reinterpret_cast<float*>(tslot + 4);   // 16-byte aligned, 64 floats
    // bf16 outputs leave through TMA stores: per epilogue warp one 32-row
    // staging tile (4 KB, 128-byte swizzled like the tensor map)
    uint8_t* sOut = sA + NS * kStage + kOutStageOffset;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (WG) {
        uint4* o = reinterpret_cast<uint4*>(sOnes);
        for (int i = threadIdx.x; i < kOnesBytes / 16; i += kConvThreads)
            o[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
        fence_proxy_async();   // generic writes, read by the tensor cores
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(wbar, 1);
        mbar_init(tfull, 1);
        mbar_init(tfull + 1, 1);
        mbar_init(tempty, kEpiThreads);
        mbar_init(tempty + 1, kEpiThreads);
        mbar_init(done, 1);
        *abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(tslot, conv_tmem_cols(TAPS, WG));
    // The weights and biases are written only by the Adam step or the
    // publication of new parameters, at least two launches before any layer;
    // the predecessor has passed its own wait before this launch could start,
    // so they are final here and load before this launch's wait, overlapping
    // the predecessor's tail. Activations load after it.
    if (EPI != EPI_MASK && threadIdx.x >= 64 && threadIdx.x < 64 + C) sbias[threadIdx.x - 64] = p.bias[threadIdx.x - 64];
    if (threadIdx.x == 0) {
        tc::mbar_expect_tx(wbar, TAPS * kWTileBytes);
        for (int j = 0; j < TAPS; ++j) tc::tma_load_2d(sW + j * kWTileBytes, &tmW, 0, (p.w_tile0 + j) * C, wbar);
    }
    pdl_wait();
    pdl_trigger();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ---- producer (the weights are already on their way): one halo tile
        // (two, WG) per row tile
        if (lane == 0) {
            int armed[NS];
            for (int s = 0; s < NS; ++s) armed[s] = -1;
            int st = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < p.ntiles; tile += gridDim.x) {
                if (!tc::wait_or_abort(empty + st, ph ^ 1, p.status, abort_flag)) break;
                // rows before 0 or past the end arrive as zeros and count in full
                tc::mbar_expect_tx(full + st, (WG ? 2 : 1) * halo_rows(TAPS) * C * 2);
                tc::tma_load_2d(sA + st * kStage, &tmA, 0, tile * TM - TAPS / 2, full + st);
                if constexpr (WG)
                    tc::tma_load_2d(sA + st * kStage + stage_bytes(TAPS), &tmX, 0, tile * TM - TAPS / 2, full + st);
                armed[st] = (int)ph;
                if (++st == NS) {
                    st = 0;
                    ph ^= 1;
                }
            }
            if (*abort_flag) {
                // no copy of this block may still be landing when it exits
                drain_wait(wbar, 0);
                for (int s = 0; s < NS; ++s)
                    if (armed[s] >= 0) drain_wait(full + s, (uint32_t)armed[s]);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: TAPS x 4 MMAs (K = 16 each) per tile into one of two
        // accumulators (WG: then 8 x NG weight-gradient MMAs)
        if (lane == 0) {
            bool ok = tc::wait_or_abort(wbar, 0, p.status, abort_flag);
            int st = 0, acc = 0;
            uint32_t ph = 0, tph = 0;
            bool first = true;
            for (int tile = blockIdx.x; ok && tile < p.ntiles; tile += gridDim.x) {
                if (!tc::wait_or_abort(tempty + acc, ((tph >> acc) & 1u) ^ 1u, p.status, abort_flag)) break;
                tph ^= 1u << acc;
                tc::fence_after_sync();
                const uint32_t d = tbase + (uint32_t)(acc * C);
                if (!tc::wait_or_abort(full + st, ph, p.status, abort_flag)) break;
                tc::fence_after_sync();
                const uint8_t* sa = sA + st * kStage;
#pragma unroll
                for (int j = 0; j < TAPS; ++j) {
                    // tap j: the TM rows starting at row j of the halo tile
                    const uint64_t ad = tc::smem_desc_sw128(sa + j * C * 2);
                    const uint64_t bd = tc::smem_desc_sw128(sW + j * kWTileBytes);
#pragma unroll
                    for (int k = 0; k < C / 16; ++k)   // +32 bytes along K per MMA
                        tc::mma_bf16(d, ad + 2 * k, bd + 2 * k, kIdesc, (j | k) != 0);
                }
                tc::mma_commit(tfull + acc);
                acc ^= 1;
                if constexpr (WG) {
                    const uint8_t* xs = sa + stage_bytes(TAPS);
                    const uint8_t* dy = sa + (TAPS / 2) * (C * 2);   // the tile's own gradient rows
#pragma unroll
                    for (int kk = 0; kk < TM / 16; ++kk) {
                        const uint64_t bd = tc::smem_desc_sw128_mn(dy + kk * 2048, 128);
#pragma unroll
                        for (int g = 0; g < NG; ++g) {
                            const uint64_t ad =
                                g < NG - 1
                                    ? tc::smem_desc_sw128_mn(xs + 2 * g * (C * 2) + kk * 2048, C * 2)
                                    : tc::smem_desc_sw128_mn(sOnes + kk * 2048,
                                                             (uint32_t)(xs + (TAPS - 1) * (C * 2) - sOnes));
                            tc::mma_bf16(tbase + (uint32_t)(2 * C + g * C), ad, bd, kIdescWg, !(first && kk == 0));
                        }
                    }
                    first = false;
                }
                tc::mma_commit(empty + st);
                if (++st == NS) {
                    st = 0;
                    ph ^= 1;
                }
            }
            tc::mma_commit(done);
            drain_wait(done, 0);
        }
    } else {
        // ---- epilogue: two warpgroups, group g drains accumulator g (the
        // CTA's tiles alternate between them), one accumulator row per thread
        const int g = (warp - 2) >> 2;
        const int q = warp & 3;   // TMEM lane quadrant this warp may read
        const int rin = q * 32 + lane;
        uint8_t* stg = sOut + (warp - 2) * kOutWarpBytes;
        uint32_t fph = 0;
        for (int tile = blockIdx.x + g * gridDim.x; tile < p.ntiles; tile += 2 * gridDim.x) {
            // the row's mask (and, backward, its ReLU source) are read before
            // the accumulator is waited for, so their latency overlaps the MMAs
            const int r = tile * TM + rin;
            const bool live = r < p.R && p.rowmask[r];
            uint4 src[EPI == EPI_MASK ? C / 8 : 1];
            if constexpr (EPI == EPI_MASK) {
                const uint4* s = reinterpret_cast<const uint4*>(p.relu_src + (size_t)r * C);
#pragma unroll
                for (int i = 0; i < C / 8; ++i) src[i] = live ? __ldg(s + i) : make_uint4(0, 0, 0, 0);
            }
            bool ok = tc::wait_or_abort(tfull + g, fph, p.status, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) break;
            fph ^= 1u;
            tc::fence_after_sync();
            float v[C];
            tc::tmem_ld64(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * C), v);
            tc::fence_before_sync();
            tc::mbar_arrive(tempty + g);
            if constexpr (EPI == EPI_F32) {
                if (live) {
                    float4* dst = reinterpret_cast<float4*>(p.out_f32 + (size_t)r * kOutCols);
                    dst[0] = make_float4(v[0] + sbias[0], v[1] + sbias[1], v[2] + sbias[2], v[3] + sbias[3]);
                    dst[1] = make_float4(v[4] + sbias[4], v[5] + sbias[5], v[6] + sbias[6], v[7] + sbias[7]);
                }
            } else {
                if constexpr (EPI == EPI_MASK) {
#pragma unroll
                    for (int i = 0; i < C / 8; ++i) {
                        const uint32_t w[4] = {src[i].x, src[i].y, src[i].z, src[i].w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float2 f = unpack_bf16x2(w[h]);
                            if (!(f.x > 0.f)) v[8 * i + 2 * h] = 0.f;
                            if (!(f.y > 0.f)) v[8 * i + 2 * h + 1] = 0.f;
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c) v[c] = fmaxf(v[c] + sbias[c], 0.f);
                }
                // stage the warp's 32 rows (gap rows as zeros, which they stay)
                // and store them with one TMA box; the store of the group's
                // previous tile must have read the buffer out first
                if (lane == 0) tc::bulk_wait_read<0>();
                __syncwarp();
#pragma unroll
                for (int i = 0; i < C / 8; ++i) {
                    const uint4 u = live ? make_uint4(pack_bf16x2(v[8 * i], v[8 * i + 1]),
                                                      pack_bf16x2(v[8 * i + 2], v[8 * i + 3]),
                                                      pack_bf16x2(v[8 * i + 4], v[8 * i + 5]),
                                                      pack_bf16x2(v[8 * i + 6], v[8 * i + 7]))
                                         : make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4*>(stg + lane * 128 + ((i ^ (lane & 7)) << 4)) = u;
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    tc::tma_store_2d(&tmOut, 0, tile * TM + q * 32, stg);
                    tc::bulk_commit();
                }
            }
        }
        if (EPI != EPI_F32 && lane == 0) tc::bulk_wait_all();
        if constexpr (WG) {
            // the CTA's weight-gradient partial: warpgroup g writes groups g, g + 2
            const bool ok = __all_sync(0xffffffffu, tc::wait_or_abort(done, 0, p.status, abort_flag));
            if (ok) {
                tc::fence_after_sync();
                float* outp = p.part + (size_t)blockIdx.x * kWgPart;
#pragma unroll 1
                for (int gg = g; gg < NG; gg += 2) {
                    float v[C];
                    tc::tmem_ld64(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(2 * C + gg * C), v);
                    // rows of the all-ones block are all the bias gradient: row 0 is kept
                    if (gg < NG - 1 || rin >= C || rin == 0)
#pragma unroll
                        for (int o = 0; o < C; ++o)
                            if (o < p.co_real) outp[(gg * C + o) * TM + rin] = v[o];
                }
            }
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tbase, conv_tmem_cols(TAPS, WG));
}

constexpr size_t conv_smem_bytes(int taps, bool wg = false)
{
    return 1024 + (size_t)taps * kWTileBytes + (wg ? (size_t)kOnesBytes : 0) +
           (size_t)conv_nstage(wg) * conv_stage(taps, wg) + kOutStageOffset + (size_t)2 * 4 * kOutWarpBytes;
}
static_assert(conv_smem_bytes(5) <= 227 * 1024 && conv_smem_bytes(1) <= 227 * 1024, "shared memory per CTA");
static_assert(conv_smem_bytes(5, true) <= 227 * 1024 && conv_smem_bytes(1, true) <= 227 * 1024, "shared memory per CTA");
// tap j of a halo tile ends at row j + TM, inside its stage
static_assert(halo_rows(5) * C * 2 <= stage_bytes(5) && stage_bytes(1) == TM * C * 2, "halo stages");
// barriers, TMEM slot, abort flag and bias fit before the output staging
static_assert((2 * NSTAGE + 6) * 8 + 16 + C * 4 <= kOutStageOffset, "control block");

// ---- the last convolution and the head, fused -------------------------------------
//
// Layer 3 (5 taps, ReLU), layer 4 (64 -> 64, ReLU) and layer 5 (64 -> 5, FP32
// output) in one launch. Per row tile the convolution's output stays in shared
// memory as the A operand of layer 4's GEMM, and layer 4's as that of layer
// 5's (N = 16, five outputs used); both are also stored, for the backward
// pass. The MMA warp runs the three GEMMs of the CTA's tiles one tile apart
// (for its j-th tile the convolution, then layer 4 of tile j - 1, then layer 5
// of tile j - 2); epilogue warpgroup g takes tiles j = g (mod 2) through the
// three epilogues in order, so the accumulators and output tiles are double
// buffered by warpgroup.
constexpr int kTailStages = 4;
constexpr int kTailW = 7 * kWTileBytes;                 // layer 3's five taps, then W4, W5
constexpr int kTailAct = TM * C * 2;                    // one 128-row bf16 tile
constexpr int kHeadN = 16;                              // layer 5's MMA width
constexpr uint32_t kIdescHead = tc::idesc_bf16_f32(TM, kHeadN);
constexpr int kTailLayer = 3;                           // first fused layer

struct TailParams {
    int R, ntiles;
    int store_acts;             // store layers 3 and 4's outputs (the backward pass reads them)
    const float* bias;          // [3][64]: layers 3, 4, 5
    const uint8_t* rowmask;
    float* out_f32;             // [R][8]
    int* status;
};

__global__ void __launch_bounds__(kConvThreads, 1)
    tail_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
                   const __grid_constant__ CUtensorMap tmS4, const __grid_constant__ CUtensorMap tmS5,
                   const TailParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sW = smem;
    uint8_t* sA = sW + kTailW;
    uint8_t* sS4 = sA + kTailStages * stage_bytes(5);
    uint8_t* sS5 = sS4 + 2 * kTailAct;
    uint64_t* full = reinterpret_cast<uint64_t*>(sS5 + 2 * kTailAct);
    uint64_t* empty = full + kTailStages;
    uint64_t* wbar = empty + kTailStages;
    uint64_t* a0f = wbar + 1;     // [2] each
    uint64_t* a0e = a0f + 2;
    uint64_t* s4f = a0e + 2;
    uint64_t* a1f = s4f + 2;
    uint64_t* a1e = a1f + 2;
    uint64_t* s5f = a1e + 2;
    uint64_t* a2f = s5f + 2;
    uint64_t* a2e = a2f + 2;
    uint64_t* done = a2e + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    float* sbias = reinterpret_cast<float*>(tslot + 4);   // 3 x 64

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nlocal = (int)blockIdx.x < p.ntiles ? (p.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kTailStages; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);
        }
        mbar_init(wbar, 1);
        for (int g = 0; g < 2; ++g) {
            mbar_init(a0f + g, 1);
            mbar_init(a1f + g, 1);
            mbar_init(a2f + g, 1);
            mbar_init(a0e + g, kEpiThreads);
            mbar_init(a1e + g, kEpiThreads);
            mbar_init(a2e + g, kEpiThreads);
            mbar_init(s4f + g, kEpiThreads);
            mbar_init(s5f + g, kEpiThreads);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        mbar_init_fence();
        // parameters: final before this launch (see pdl_wait)
        tc::mbar_expect_tx(wbar, kTailW);
        for (int j = 0; j < 7; ++j)
            tc::tma_load_2d(sW + j * kWTileBytes, &tmW, 0, (wtile0_of(kTailLayer) + j) * C, wbar);
    }
    if (warp == 1) tc::tmem_alloc(tslot, 512);
    if (threadIdx.x >= 64 && threadIdx.x < 64 + 3 * C) sbias[threadIdx.x - 64] = p.bias[threadIdx.x - 64];
    pdl_wait();
    pdl_trigger();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            int armed[kTailStages];
            for (int i = 0; i < kTailStages; ++i) armed[i] = -1;
            int st = 0;
            uint32_t ph = 0;
            for (int j = 0; j < nlocal; ++j) {
                const int tile = blockIdx.x + j * gridDim.x;
                if (!tc::wait_or_abort(empty + st, ph ^ 1, p.status, abort_flag)) break;
                tc::mbar_expect_tx(full + st, halo_rows(5) * C * 2);
                tc::tma_load_2d(sA + st * stage_bytes(5), &tmA, 0, tile * TM - 2, full + st);
                armed[st] = (int)ph;
                if (++st == kTailStages) {
                    st = 0;
                    ph ^= 1;
                }
            }
            if (*abort_flag) {
                drain_wait(wbar, 0);
                for (int i = 0; i < kTailStages; ++i)
                    if (armed[i] >= 0) drain_wait(full + i, (uint32_t)armed[i]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = tc::wait_or_abort(wbar, 0, p.status, abort_flag);
            int st = 0;
            uint32_t ph = 0, e0 = 0, e1 = 0, e2 = 0, f4 = 0, f5 = 0;   // parity bits per buffer
            for (int j = 0; ok && j < nlocal + 2; ++j) {
                if (j < nlocal) {   // layer 3 of tile j
                    const int g = j & 1;
                    if (!(ok = tc::wait_or_abort(a0e + g, ((e0 >> g) & 1u) ^ 1u, p.status, abort_flag))) break;
                    e0 ^= 1u << g;
                    if (!(ok = tc::wait_or_abort(full + st, ph, p.status, abort_flag))) break;
                    tc::fence_after_sync();
                    const uint8_t* sa = sA + st * stage_bytes(5);
#pragma unroll
                    for (int t = 0; t < 5; ++t) {
                        const uint64_t ad = tc::smem_desc_sw128(sa + t * C * 2);
                        const uint64_t bd = tc::smem_desc_sw128(sW + t * kWTileBytes);
#pragma unroll
                        for (int k = 0; k < C / 16; ++k)
                            tc::mma_bf16(tbase + (uint32_t)(g * C), ad + 2 * k, bd + 2 * k, kIdesc, (t | k) != 0);
                    }
                    tc::mma_commit(empty + st);
                    if (++st == kTailStages) {
                        st = 0;
                        ph ^= 1;
                    }
                    tc::mma_commit(a0f + g);
                }
                if (j >= 1 && j - 1 < nlocal) {   // layer 4 of tile j - 1
                    const int g = (j - 1) & 1;
                    if (!(ok = tc::wait_or_abort(s4f + g, (f4 >> g) & 1u, p.status, abort_flag))) break;
                    f4 ^= 1u << g;
                    if (!(ok = tc::wait_or_abort(a1e + g, ((e1 >> g) & 1u) ^ 1u, p.status, abort_flag))) break;
                    e1 ^= 1u << g;
                    tc::fence_after_sync();
                    const uint64_t ad = tc::smem_desc_sw128(sS4 + g * kTailAct);
                    const uint64_t bd = tc::smem_desc_sw128(sW + 5 * kWTileBytes);
#pragma unroll
                    for (int k = 0; k < C / 16; ++k)
                        tc::mma_bf16(tbase + (uint32_t)(2 * C + g * C), ad + 2 * k, bd + 2 * k, kIdesc, k != 0);
                    tc::mma_commit(a1f + g);
                }
                if (j >= 2) {   // layer 5 of tile j - 2
                    const int g = (j - 2) & 1;
                    if (!(ok = tc::wait_or_abort(s5f + g, (f5 >> g) & 1u, p.status, abort_flag))) break;
                    f5 ^= 1u << g;
                    if (!(ok = tc::wait_or_abort(a2e + g, ((e2 >> g) & 1u) ^ 1u, p.status, abort_flag))) break;
                    e2 ^= 1u << g;
                    tc::fence_after_sync();
                    const uint64_t ad = tc::smem_desc_sw128(sS5 + g * kTailAct);
                    const uint64_t bd = tc::smem_desc_sw128(sW + 6 * kWTileBytes);
#pragma unroll
                    for (int k = 0; k < C / 16; ++k)
                        tc::mma_bf16(tbase + (uint32_t)(4 * C + g * kHeadN), ad + 2 * k, bd + 2 * k, kIdescHead, k != 0);
                    tc::mma_commit(a2f + g);
                }
            }
            tc::mma_commit(done);
            drain_wait(done, 0);
        }
    } else {
        const int g = (warp - 2) >> 2;
        const int q = warp & 3;
        const int rin = q * 32 + lane;
        uint8_t* s4 = sS4 + g * kTailAct + q * kOutWarpBytes;
        uint8_t* s5 = sS5 + g * kTailAct + q * kOutWarpBytes;
        const uint32_t trow = (uint32_t)(q * 32) << 16;
        uint32_t w0 = 0, w1 = 0, w2 = 0;
        // bias + ReLU of one 64-column row, packed into this warp's swizzled
        // 32-row slice of an output tile (gap and padding rows as zeros)
        auto emit = [&](uint8_t* slice, const float* v, const float* b, bool live) {
#pragma unroll
            for (int i = 0; i < C / 8; ++i) {
                uint4 u = make_uint4(0, 0, 0, 0);
                if (live)
                    u = make_uint4(pack_bf16x2(fmaxf(v[8 * i] + b[8 * i], 0.f), fmaxf(v[8 * i + 1] + b[8 * i + 1], 0.f)),
                                   pack_bf16x2(fmaxf(v[8 * i + 2] + b[8 * i + 2], 0.f), fmaxf(v[8 * i + 3] + b[8 * i + 3], 0.f)),
                                   pack_bf16x2(fmaxf(v[8 * i + 4] + b[8 * i + 4], 0.f), fmaxf(v[8 * i + 5] + b[8 * i + 5], 0.f)),
                                   pack_bf16x2(fmaxf(v[8 * i + 6] + b[8 * i + 6], 0.f), fmaxf(v[8 * i + 7] + b[8 * i + 7], 0.f)));
                *reinterpret_cast<uint4*>(slice + lane * 128 + ((i ^ (lane & 7)) << 4)) = u;
            }
        };
        for (int j = g; j < nlocal; j += 2) {
            const int tile = blockIdx.x + j * gridDim.x;
            const int r = tile * TM + rin;
            const bool live = r < p.R && p.rowmask[r];
            float v[C];
            // layer 3: the tile's output into s4 (and to global)
            bool ok = tc::wait_or_abort(a0f + g, w0, p.status, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) break;
            w0 ^= 1u;
            tc::fence_after_sync();
            tc::tmem_ld64(tbase + trow + (uint32_t)(g * C), v);
            tc::fence_before_sync();
            tc::mbar_arrive(a0e + g);
            if (lane == 0) tc::bulk_wait_read<0>();   // the slices' previous stores have read them
            __syncwarp();
            emit(s4, v, sbias, live);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0 && p.store_acts) {
                tc::tma_store_2d(&tmS4, 0, tile * TM + q * 32, s4);
                tc::bulk_commit();
            }
            tc::mbar_arrive(s4f + g);
            // layer 4: into s5 (and to global)
            ok = tc::wait_or_abort(a1f + g, w1, p.status, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) break;
            w1 ^= 1u;
            tc::fence_after_sync();
            tc::tmem_ld64(tbase + trow + (uint32_t)(2 * C + g * C), v);
            tc::fence_before_sync();
            tc::mbar_arrive(a1e + g);
            emit(s5, v, sbias + C, live);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0 && p.store_acts) {
                tc::tma_store_2d(&tmS5, 0, tile * TM + q * 32, s5);
                tc::bulk_commit();
            }
            tc::mbar_arrive(s5f + g);
            // layer 5: the FP32 output of the state rows
            ok = tc::wait_or_abort(a2f + g, w2, p.status, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) break;
            w2 ^= 1u;
            tc::fence_after_sync();
            float o[16];
            tc::tmem_ld16(tbase + trow + (uint32_t)(4 * C + g * kHeadN), o);
            tc::fence_before_sync();
            tc::mbar_arrive(a2e + g);
            if (live) {
                const float* b = sbias + 2 * C;
                float4* dst = reinterpret_cast<float4*>(p.out_f32 + (size_t)r * kOutCols);
                dst[0] = make_float4(o[0] + b[0], o[1] + b[1], o[2] + b[2], o[3] + b[3]);
                dst[1] = make_float4(o[4] + b[4], o[5] + b[5], o[6] + b[6], o[7] + b[7]);
            }
        }
        if (lane == 0) tc::bulk_wait_all();
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tbase, 512);
}

constexpr size_t tail_smem_bytes()
{
    return 1024 + (size_t)kTailW + (size_t)kTailStages * stage_bytes(5) + 4 * (size_t)kTailAct + 1024;
}
static_assert(tail_smem_bytes() <= 227 * 1024, "shared memory per CTA");
// barriers (4 + 4 + 1 + 16 + 1) x 8 B, TMEM slot, abort flag and 3 x 64 biases fit the last KB
static_assert((2 * kTailStages + 18) * 8 + 16 + 3 * C * 4 <= 1024, "tail control block");
static_assert(kConvThreads - 64 >= 3 * C, "the tail's bias loaders");
static_assert(kWTile0[kTailLayer] + 5 == kWTile0[4] && kWTile0[4] + 1 == kWTile0[5], "the tail's weight tiles are consecutive");

// ---- rows, features, loss, gradients, optimiser ----------------------------------

PES_DEV int traj_of_state(const int64_t* off, int B, int64_t k)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Features of every state row and the row mask.
// Trajectory owning row r (0 .. B; B is the trailing gap): the last b whose
// leading gap starts at or before r (trajectory b's rows begin at off[b] + G b).
PES_DEV int traj_of_row(const int64_t* off, int B, int64_t r)
{
    int lo = 0, hi = B;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] + (int64_t)G * mid <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Input features of every row (Sec. 5's initialiser input): a state's
// (sin y1, cos y1, sin y2, cos y2, 1, 0) or the prior row's (0, 0, 0, 0, 0, 1),
// zeros on the gap rows, and the row mask. A warp owns 32 consecutive rows, one
// lane each; it then stores them as eight 512-byte runs (four rows each), the
// first 16 bytes of a row taken from its lane by shuffles.
template <typename T>
__global__ void features_kernel(const T* y, const int64_t* off, int B, int64_t N, int64_t R, uint8_t* mask, bf16* X0)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int64_t nw = (R + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w < nw; w += wstride) {
        const int64_t r = w * 32 + lane;
        uint4 u = make_uint4(0, 0, 0, 0);
        if (r < R) {
            const int b = traj_of_row(off, B, r);
            const int64_t k = r - (int64_t)G * (b + 1);
            const bool state = b < B && r - (off[b] + (int64_t)G * b) >= G && k >= 0 && k < N;
            if (state) {
                float f[4] = {0.f, 0.f, 0.f, 0.f};
                const bool prior = k == off[b];
                if (!prior) {
                    sincosf((float)y[k], &f[0], &f[1]);
                    sincosf((float)y[N + k], &f[2], &f[3]);
                }
                u = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]),
                               pack_bf16x2(prior ? 0.f : 1.f, prior ? 1.f : 0.f), 0u);
            }
            mask[r] = state ? 1 : 0;
        }
        uint4* dst = reinterpret_cast<uint4*>(X0) + (size_t)w * 32 * (C / 8);
#pragma unroll
        for (int i = 0; i < C / 8; ++i) {
            const int src = 4 * i + (lane >> 3);   // row w * 32 + src, chunk lane & 7
            uint4 v;
            v.x = __shfl_sync(0xffffffffu, u.x, src);
            v.y = __shfl_sync(0xffffffffu, u.y, src);
            v.z = __shfl_sync(0xffffffffu, u.z, src);
            v.w = __shfl_sync(0xffffffffu, u.w, src);
            if (w * 32 + src < R) dst[32 * i + lane] = (lane & 7) == 0 ? v : make_uint4(0, 0, 0, 0);
        }
    }
}

struct Norm {
    double mu[5], sigma[5], inv_sigma[5];
    float mu_f[5], inv_sigma_f[5];
};

// The normalised target (x - mu) / sigma: in FP32 for FP32 targets (FP64 is
// a slow pipe on this GPU; the result is rounded to bf16 in the gradient), in
// FP64 for FP64 ones.
PES_DEV float norm_target(float x, const Norm& nm, int c) { return (x - nm.mu_f[c]) * nm.inv_sigma_f[c]; }
PES_DEV float norm_target(double x, const Norm& nm, int c) { return (float)((x - nm.mu[c]) * nm.inv_sigma[c]); }

// Loss terms (o - t)^2 and the output gradient dO = 2 (o - t) / (5 N) in bf16
// over all R rows (gap rows get zeros). A warp owns 32 consecutive rows, one
// lane each, and stores them as eight 512-byte runs (four rows each, the first
// 16 bytes of a row taken from its lane by shuffles), so every store is
// coalesced. Squares and block sums are FP32 (a thread holds about one row);
// each block leaves its sum in part[block] and the last block to finish adds
// the partials in block order in FP64 (so the loss does not depend on
// scheduling), writes loss_scale x the total to *loss and re-arms the ticket.
template <typename T>
__global__ void __launch_bounds__(256) loss_kernel(const float* o, const T* xt, const int64_t* off, int B, int64_t N,
                                                   int64_t R, Norm nm, float scale, double loss_scale, bf16* dO,
                                                   double* part, unsigned* ticket, double* loss)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int64_t nw = (R + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x / 32);
    float s = 0.f;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w < nw; w += wstride) {
        const int64_t r = w * 32 + lane;
        uint4 u = make_uint4(0, 0, 0, 0);
        if (r < R) {
            const int b = traj_of_row(off, B, r);
            const int64_t k = r - (int64_t)G * (b + 1);
            if (b < B && r - (off[b] + (int64_t)G * b) >= G && k >= 0 && k < N) {
                const float4 o0 = *reinterpret_cast<const float4*>(o + (size_t)r * kOutCols);
                const float o4 = o[(size_t)r * kOutCols + 4];
                const float e0 = o0.x - norm_target(xt[k], nm, 0);
                const float e1 = o0.y - norm_target(xt[(size_t)N + k], nm, 1);
                const float e2 = o0.z - norm_target(xt[(size_t)2 * N + k], nm, 2);
                const float e3 = o0.w - norm_target(xt[(size_t)3 * N + k], nm, 3);
                const float e4 = o4 - norm_target(xt[(size_t)4 * N + k], nm, 4);
                s = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, e4 * e4))));
                u = make_uint4(pack_bf16x2(scale * e0, scale * e1), pack_bf16x2(scale * e2, scale * e3),
                               pack_bf16x2(scale * e4, 0.f), 0u);
            }
        }
        uint4* dst = reinterpret_cast<uint4*>(dO) + (size_t)w * 32 * (C / 8);
#pragma unroll
        for (int i = 0; i < C / 8; ++i) {
            const int src = 4 * i + (lane >> 3);   // row w * 32 + src, chunk lane & 7
            uint4 v;
            v.x = __shfl_sync(0xffffffffu, u.x, src);
            v.y = __shfl_sync(0xffffffffu, u.y, src);
            v.z = __shfl_sync(0xffffffffu, u.z, src);
            v.w = __shfl_sync(0xffffffffu, u.w, src);
            if (w * 32 + src < R) dst[32 * i + lane] = (lane & 7) == 0 ? v : make_uint4(0, 0, 0, 0);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    __shared__ float wsum[8];
    __shared__ double red[256];
    __shared__ bool last;
    if (lane == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int v = 0; v < (int)(blockDim.x >> 5); ++v) t += (double)wsum[v];
        part[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(part + i);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int v = blockDim.x / 2; v > 0; v >>= 1) {
        if ((int)threadIdx.x < v) red[threadIdx.x] += red[threadIdx.x + v];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *loss = red[0] * loss_scale;
        *ticket = 0u;
    }
}

// Weight and bias gradients of one layer on the tensor cores:
//   dW_j[o][i] = sum_r dY[r][o] X[r + j - TAPS/2][i],  db[o] = sum_r dY[r][o],
// a GEMM whose reduction dimension is the rows. The activation arrays are
// row-major [rows][64], so a TMA tile of them is an MN-major operand with the
// rows as K, and no transpose is needed: per 128-row tile, B = the dY tile
// (N = 64 output channels) and A = two taps of the X halo tile stacked along
// M = 128 (tap pair (2g, 2g + 1): the second 64-row block of A starts one row,
// 128 bytes, after the first). The odd last tap is paired with a constant
// all-ones tile, whose products with dY are the bias gradient. Each CTA owns a
// fixed set of row tiles (split-K), accumulates them in tensor memory, and
// writes its partial [group][o][m] to `part`; wgrad_reduce_kernel sums the
// partials in a fixed order, so the gradient does not depend on scheduling.
// Warp 0 issues the TMA loads, warp 1 the MMAs, warps 2-5 write the partial.
struct WgradParams {
    int ntiles;     // ceil(R / TM)
    float* part;    // [gridDim.x][kWgPart]
    int co_real;    // output channels that exist (the partial rows written)
    int* status;
};

template <int TAPS>
__global__ void __launch_bounds__(kWgThreads, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmDY,
                    const WgradParams p)
{
    constexpr int NG = wg_groups(TAPS);
    constexpr int kStage = wg_stage(TAPS);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sOnes = smem;
    uint8_t* sStage = smem + kOnesBytes;                  // per stage: X halo tile, then dY tile
    uint64_t* full = reinterpret_cast<uint64_t*>(sStage + kWgStages * kStage);
    uint64_t* empty = full + kWgStages;
    uint64_t* done = empty + kWgStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {   // the ones tile (no swizzle matters: every element is 1)
        uint4* o = reinterpret_cast<uint4*>(sOnes);
        for (int i = threadIdx.x; i < kOnesBytes / 16; i += kWgThreads) o[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
        fence_proxy_async();   // generic writes, read by the tensor cores
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(tslot, wg_tmem_cols(TAPS));
    pdl_wait();
    pdl_trigger();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            int armed[kWgStages];
            for (int s = 0; s < kWgStages; ++s) armed[s] = -1;
            int st = 0;
            uint32_t ph = 0;
            for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
                if (!tc::wait_or_abort(empty + st, ph ^ 1, p.status, abort_flag)) break;
                uint8_t* xs = sStage + st * kStage;
                tc::mbar_expect_tx(full + st, halo_rows(TAPS) * C * 2 + kDyBytes);
                tc::tma_load_2d(xs, &tmX, 0, tile * TM - TAPS / 2, full + st);
                tc::tma_load_2d(xs + stage_bytes(TAPS), &tmDY, 0, tile * TM, full + st);
                armed[st] = (int)ph;
                if (++st == kWgStages) {
                    st = 0;
                    ph ^= 1;
                }
            }
            if (*abort_flag)
                for (int s = 0; s < kWgStages; ++s)
                    if (armed[s] >= 0) drain_wait(full + s, (uint32_t)armed[s]);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0;
            bool first = true;
            for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
                if (!tc::wait_or_abort(full + st, ph, p.status, abort_flag)) break;
                tc::fence_after_sync();
                const uint8_t* xs = sStage + st * kStage;
                const uint8_t* ds = xs + stage_bytes(TAPS);
#pragma unroll
                for (int kk = 0; kk < TM / 16; ++kk) {   // 16 rows (two 8-row K groups) per MMA
                    const uint64_t bd = tc::smem_desc_sw128_mn(ds + kk * 2048, 128);
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        // group g < NG - 1: taps 2g, 2g + 1; the last: ones, tap TAPS - 1
                        const uint64_t ad =
                            g < NG - 1
                                ? tc::smem_desc_sw128_mn(xs + 2 * g * (C * 2) + kk * 2048, C * 2)
                                : tc::smem_desc_sw128_mn(sOnes + kk * 2048,
                                                         (uint32_t)(xs + (TAPS - 1) * (C * 2) - sOnes));
                        tc::mma_bf16(tbase + (uint32_t)(g * C), ad, bd, kIdescWg, !(first && kk == 0));
                    }
                }
                first = false;
                tc::mma_commit(empty + st);
                if (++st == kWgStages) {
                    st = 0;
                    ph ^= 1;
                }
            }
            tc::mma_commit(done);
            drain_wait(done, 0);
        }
    } else {
        // the CTA's partial: TMEM lane m (quadrant warp % 4) holds row m of A
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const bool ok = __all_sync(0xffffffffu, tc::wait_or_abort(done, 0, p.status, abort_flag));
        if (ok) {
            tc::fence_after_sync();
            float* out = p.part + (size_t)blockIdx.x * kWgPart;
#pragma unroll 1
            for (int g = 0; g < NG; ++g) {
                float v[C];
                tc::tmem_ld64(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * C), v);
                // rows of the all-ones block are all the bias gradient: row 0 is kept
                if (g < NG - 1 || m >= C || m == 0)
#pragma unroll
                    for (int o = 0; o < C; ++o)
                        if (o < p.co_real) out[(g * C + o) * TM + m] = v[o];
            }
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tbase, wg_tmem_cols(TAPS));
}

constexpr size_t wgrad_smem_bytes(int taps)
{
    return 1024 + (size_t)kOnesBytes + (size_t)kWgStages * wg_stage(taps) + 256;
}
static_assert(wgrad_smem_bytes(5) <= 227 * 1024 && wgrad_smem_bytes(1) <= 227 * 1024, "shared memory per CTA");
// the last MMA of a tile reads rows up to TAPS - 1 + TM - 1 of the halo tile
static_assert(stage_bytes(5) % 1024 == 0 && kDyBytes % 1024 == 0 && kOnesBytes % 1024 == 0, "swizzle atoms");

// One Adam step of packed parameter i with gradient g, and the new value
// published where the GEMMs read it: a weight W_l[o][i][j] into forward tile
// (l, j) at [o][i] and backward tile (l, TAPS - 1 - j) at [i][o] (bf16), a bias
// into the FP32 bias row. Entries of output channels that do not exist stay
// the zeros that publish_kernel wrote.
struct AdamStep {
    float *p, *m, *v;
    bf16 *Wf, *Wb;
    float* bias;
    float lr, b1, b2, eps, c1, c2;
};

PES_DEV void adam_apply(const AdamStep& a, int i, float g)
{
    const float mi = a.b1 * a.m[i] + (1.f - a.b1) * g;
    const float vi = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
    a.m[i] = mi;
    a.v[i] = vi;
    const float pi = a.p[i] - a.lr * (mi * a.c1) / (sqrtf(vi * a.c2) + a.eps);
    a.p[i] = pi;
    int l = 0;
    while (l + 1 < NLAYER && poff_of(l + 1) <= i) ++l;
    const int taps = taps_of(l), nw = coreal_of(l) * C * taps, loc = i - poff_of(l);
    if (loc < nw) {
        const int o = loc / (C * taps), ci = (loc / taps) % C, j = loc % taps;
        const bf16 w = __float2bfloat16_rn(pi);
        a.Wf[(size_t)(wtile0_of(l) + j) * C * C + o * C + ci] = w;
        a.Wb[(size_t)(wtile0_of(l) + taps - 1 - j) * C * C + ci * C + o] = w;
    } else {
        a.bias[l * C + (loc - nw)] = pi;
    }
}

// Sum the CTAs' partials into the packed gradients of all six layers, one
// launch after the backward pass (layer l's partials at part + l x
// layer_stride), and with apply_adam take the Adam step on each parameter as
// its gradient is complete. Block b of layer l covers partial entries 128 b .. 128 b + 127;
// warp w sums the CTAs w, w + 8, ... in order and the eight sums are added in
// warp order, so the result does not depend on scheduling. Entry (g, o, m):
// m < 64 is tap 2g, input channel m; m >= 64 tap 2g + 1, channel m - 64; in the
// last group m < 64 is the ones block (row 0 kept: the bias gradient) and
// m >= 64 tap TAPS - 1.
constexpr int kRedBlocks5 = wg_groups(5) * C * TM / 128;
constexpr int kRedBlocks1 = wg_groups(1) * C * TM / 128;
constexpr int kRedBlocks = 4 * kRedBlocks5 + 2 * kRedBlocks1;

__global__ void __launch_bounds__(256) wgrad_reduce_kernel(const float* part, size_t layer_stride, int nblk,
                                                           float* grad, const AdamStep adam, int apply_adam)
{
    pdl_wait();
    pdl_trigger();
    int blk = blockIdx.x, l;
    if (blk < 4 * kRedBlocks5) {
        l = blk / kRedBlocks5;
        blk -= l * kRedBlocks5;
    } else {
        blk -= 4 * kRedBlocks5;
        l = 4 + blk / kRedBlocks1;
        blk -= (l - 4) * kRedBlocks1;
    }
    const int taps = taps_of(l), ng = (taps + 1) / 2, co_real = coreal_of(l);
    // block blk holds the partial row (group blk / 64, output channel blk % 64)
    if ((blk % C) >= co_real) return;   // absent channel: never written, not read
    const float* pl = part + (size_t)l * layer_stride;
    float* gl = grad + poff_of(l);
    __shared__ float4 red[8][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s4 = blk * 128 + lane * 4;
    // in the last group only entry 0 of the all-ones half is written (and used)
    const bool read = !(blk / C == ng - 1 && lane > 0 && lane < C / 4);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int b = w; read && b < nblk; b += 8) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(pl + (size_t)b * kWgPart + s4));
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    red[w][lane] = acc;
    __syncthreads();
    if (threadIdx.x < 128) {
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) s += reinterpret_cast<const float*>(red[v])[threadIdx.x];
        const int e = blk * 128 + threadIdx.x;
        const int g = e / (C * TM), o = (e / TM) % C, m = e % TM, half = m / C, ci = m % C;
        int dst = -1;
        if (g < ng && o < co_real) {
            if (g == ng - 1 && half == 0) {
                if (ci == 0) dst = co_real * C * taps + o;
            } else {
                const int j = g == ng - 1 ? taps - 1 : 2 * g + half;
                dst = (o * C + ci) * taps + j;
            }
        }
        if (dst >= 0) {
            gl[dst] = s;
            if (apply_adam) adam_apply(adam, poff_of(l) + dst, s);   // each parameter once
        }
    }
}

// bf16 weight tiles for the forward GEMMs (tile (l, j): [o][i] = W_l[o][i][j])
// and for the backward GEMMs (tile (l, j): [i][o] = W_l[o][i][TAPS-1-j]), and
// the FP32 biases padded to 64 channels.
__global__ void publish_kernel(const float* p, bf16* Wf, bf16* Wb, float* bias)
{
    pdl_wait();
    pdl_trigger();
    const int total = kWTiles * C * C;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total + NLAYER * C;
         idx += gridDim.x * blockDim.x) {
        if (idx >= total) {
            const int l = (idx - total) / C, o = (idx - total) % C;
            bias[l * C + o] = o < coreal_of(l) ? p[poff_of(l) + coreal_of(l) * C * taps_of(l) + o] : 0.f;
            continue;
        }
        const int tile = idx / (C * C), n = (idx / C) % C, kc = idx % C;
        int l = 0;
        while (l + 1 < NLAYER && wtile0_of(l + 1) <= tile) ++l;
        const int j = tile - wtile0_of(l), taps = taps_of(l);
        {   // forward: row n = output channel, column kc = input channel, tap j
            const int o = n, i = kc;
            Wf[idx] = __float2bfloat16_rn(o < coreal_of(l) ? p[poff_of(l) + (o * C + i) * taps + j] : 0.f);
        }
        {   // backward: row n = input channel, column kc = output channel, tap taps-1-j
            const int i = n, o = kc;
            Wb[idx] = __float2bfloat16_rn(o < coreal_of(l) ? p[poff_of(l) + (o * C + i) * taps + (taps - 1 - j)] : 0.f);
        }
    }
}

// x = mu + sigma * output, in FP32 (the output is a bf16 network's; FP64 is a
// slow pipe on this GPU) and stored in the caller's precision.
template <typename T>
__global__ void denorm_kernel(const float* o, const int64_t* off, int B, int64_t N, Norm nm, T* x)
{
    pdl_wait();
    pdl_trigger();
    float mu[5], sg[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        mu[c] = (float)nm.mu[c];
        sg[c] = (float)nm.sigma[c];
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
        const int b = traj_of_state(off, B, k);
        const float4* row = reinterpret_cast<const float4*>(o + (size_t)(k + (int64_t)G * (b + 1)) * kOutCols);
        const float4 lo = __ldg(row), hi = __ldg(row + 1);
        const float v[5] = {lo.x, lo.y, lo.z, lo.w, hi.x};
#pragma unroll
        for (int c = 0; c < 5; ++c) x[(size_t)c * N + k] = (T)fmaf(sg[c], v[c], mu[c]);
    }
}

}  // namespace

// ---- host side -------------------------------------------------------------------

struct pes_init_net {
    int device = 0, num_sms = 0;
    int64_t max_states = 0, max_rows = 0;
    int32_t max_batch = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *bias = nullptr, *wpart = nullptr;
    double *lpart = nullptr, *loss_dev = nullptr;
    unsigned* ticket = nullptr;
    bf16 *Wf = nullptr, *Wb = nullptr;
    bf16* act[NLAYER] = {};      // X0, H1..H4, Z
    bf16 *dO = nullptr, *dA = nullptr, *dB = nullptr;
    float* out = nullptr;
    uint8_t* mask = nullptr;
    int* status = nullptr;
    CUtensorMap mapWf, mapWb;
    Norm norm;
    int adam_t = 0;
    char err[256] = {0};
};

namespace {

constexpr int kLossBlocks = 1024;

pes_status net_fail(pes_init_net* n, pes_status s, const char* fmt, ...)
{
    if (n) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(n->err, sizeof(n->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define NET_CUDA(n, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return net_fail(n, PES_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of a [rows][64] bf16 array, boxes of box_rows x 64, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint32_t box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)C * 2};
    const cuuint32_t box[2] = {(cuuint32_t)C, box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launch with programmatic stream serialization (the kernels call pdl_wait
// before touching global memory).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// One layer's GEMM; WG (backward only) also accumulates the layer's weight
// gradient from relu_src (the layer input) into its partials.
template <int TAPS, int EPI, bool WG = false>
cudaError_t launch_conv(pes_init_net* n, const bf16* in, int64_t R, bool backward, int layer, bf16* out,
                        float* out_f32, const bf16* relu_src, cudaStream_t st)
{
    CUtensorMap mA, mOut, mX;
    if (!make_map(&mA, in, (uint64_t)R, halo_rows(TAPS))) return cudaErrorInvalidValue;
    // bf16 outputs: boxes of the 32 rows of one epilogue warp (the head's FP32
    // output is stored directly; its map is a placeholder)
    if (!make_map(&mOut, out ? (const void*)out : (const void*)in, (uint64_t)R, 32)) return cudaErrorInvalidValue;
    // the weight gradient's input tiles (otherwise a placeholder)
    if (!make_map(&mX, WG ? (const void*)relu_src : (const void*)in, (uint64_t)R, halo_rows(TAPS)))
        return cudaErrorInvalidValue;
    ConvParams p;
    p.R = (int)R;
    p.ntiles = (int)((R + TM - 1) / TM);
    p.w_tile0 = kWTile0[layer];
    p.bias = n->bias + layer * C;
    p.rowmask = n->mask;
    p.out = out;
    p.out_f32 = out_f32;
    p.relu_src = relu_src;
    p.part = WG ? n->wpart + (size_t)layer * kWgPart * n->num_sms : nullptr;
    p.co_real = layer == NLAYER - 1 ? 5 : C;
    p.status = n->status;
    const size_t smem = conv_smem_bytes(TAPS, WG);
    cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<TAPS, EPI, WG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(p.ntiles, n->num_sms);
    return launch_pdl(conv_tc_kernel<TAPS, EPI, WG>, grid, kConvThreads, smem, st, mA, backward ? n->mapWb : n->mapWf,
                      mOut, mX, p);
}

pes_status check_sizes(pes_init_net* n, pes_precision prec, const void* y, const int64_t* off, int32_t B, int64_t N)
{
    if (!n) return PES_ERR_INVALID_ARG;
    if (prec != PES_FP32 && prec != PES_FP64) return net_fail(n, PES_ERR_INVALID_ARG, "precision must be FP32 or FP64");
    if (!y || !off) return net_fail(n, PES_ERR_INVALID_ARG, "NULL array");
    if (B < 1 || N < B || N > n->max_states || B > n->max_batch)
        return net_fail(n, PES_ERR_INVALID_ARG, "sizes out of range (N %lld, B %d)", (long long)N, (int)B);
    return PES_OK;
}

// Rows and features of a call; returns R.
template <typename T>
pes_status prepare_rows(pes_init_net* n, const T* y, const int64_t* off, int32_t B, int64_t N, cudaStream_t st,
                        int64_t* R_out)
{
    const int64_t R = N + (int64_t)G * (B + 1);
    const int blocks = (int)std::min<int64_t>((R + 255) / 256, (int64_t)n->num_sms * 16);
    NET_CUDA(n, launch_pdl(features_kernel<T>, blocks, 256, 0, st, y, off, B, N, R, n->mask, n->act[0]));
    // Every convolution writes zeros on the gap rows of its output, and so
    // does the loss kernel on those of the loss gradient: the weight gradients
    // sum over all rows.
    *R_out = R;
    return PES_OK;
}

// Layers 3-5 in one launch (tail_tc_kernel): act[3] -> out, and act[4], act[5]
// when a backward pass follows.
cudaError_t launch_tail(pes_init_net* n, int64_t R, bool store_acts, cudaStream_t st)
{
    CUtensorMap mA, mS4, mS5;
    if (!make_map(&mA, n->act[3], (uint64_t)R, halo_rows(5)) || !make_map(&mS4, n->act[4], (uint64_t)R, 32) ||
        !make_map(&mS5, n->act[5], (uint64_t)R, 32))
        return cudaErrorInvalidValue;
    TailParams p;
    p.R = (int)R;
    p.ntiles = (int)((R + TM - 1) / TM);
    p.store_acts = store_acts ? 1 : 0;
    p.bias = n->bias + kTailLayer * C;
    p.rowmask = n->mask;
    p.out_f32 = n->out;
    p.status = n->status;
    const size_t smem = tail_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(tail_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(p.ntiles, n->num_sms);
    return launch_pdl(tail_tc_kernel, grid, kConvThreads, smem, st, mA, n->mapWf, mS4, mS5, p);
}

// The forward pass; `training` keeps every layer's activations for the
// backward pass (inference does not store the last two).
pes_status forward_layers(pes_init_net* n, int64_t R, bool training, cudaStream_t st)
{
    for (int l = 0; l < kTailLayer; ++l)
        NET_CUDA(n, (launch_conv<5, EPI_RELU>(n, n->act[l], R, false, l, n->act[l + 1], nullptr, nullptr, st)));
    NET_CUDA(n, launch_tail(n, R, training, st));
    return PES_OK;
}

// A layer's weight-gradient partials on their own (the layer without a
// backward convolution to fuse them into), into the layer's slot of n->wpart.
template <int TAPS>
pes_status layer_grad(pes_init_net* n, const bf16* dY, const bf16* X, int64_t R, int layer, cudaStream_t st)
{
    CUtensorMap mX, mDY;
    if (!make_map(&mX, X, (uint64_t)R, halo_rows(TAPS)) || !make_map(&mDY, dY, (uint64_t)R, TM))
        return net_fail(n, PES_ERR_CUDA, "tensor map of a weight-gradient operand");
    WgradParams p;
    p.ntiles = (int)((R + TM - 1) / TM);
    p.part = n->wpart + (size_t)layer * kWgPart * n->num_sms;
    p.co_real = layer == NLAYER - 1 ? 5 : C;
    p.status = n->status;
    const int nblk = std::min(p.ntiles, n->num_sms);
    const size_t smem = wgrad_smem_bytes(TAPS);
    NET_CUDA(n, cudaFuncSetAttribute(wgrad_tc_kernel<TAPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    NET_CUDA(n, launch_pdl(wgrad_tc_kernel<TAPS>, nblk, kWgThreads, smem, st, mX, mDY, p));
    return PES_OK;
}

// Backward pass from dO: every layer's packed gradient into `grad`. Each
// backward convolution also accumulates its layer's weight gradient (both read
// the same gradient tiles, and the layer input that gives the ReLU mask is the
// gradient's other operand); the first layer has no backward convolution, so
// its weight gradient runs alone. One launch then sums all partials.
pes_status backward_layers(pes_init_net* n, int64_t R, float* grad, const AdamStep* adam, cudaStream_t st)
{
    pes_status s;
    NET_CUDA(n, (launch_conv<1, EPI_MASK, true>(n, n->dO, R, true, 5, n->dA, nullptr, n->act[5], st)));
    NET_CUDA(n, (launch_conv<1, EPI_MASK, true>(n, n->dA, R, true, 4, n->dB, nullptr, n->act[4], st)));
    bf16* cur = n->dB;
    bf16* nxt = n->dA;
    for (int l = 3; l > 0; --l) {   // cur: gradient at the pre-activation of conv layer l
        NET_CUDA(n, (launch_conv<5, EPI_MASK, true>(n, cur, R, true, l, nxt, nullptr, n->act[l], st)));
        bf16* t = cur;
        cur = nxt;
        nxt = t;
    }
    if ((s = layer_grad<5>(n, cur, n->act[0], R, 0, st)) != PES_OK) return s;
    const int nblk = (int)std::min<int64_t>((R + TM - 1) / TM, n->num_sms);
    const AdamStep none{};
    NET_CUDA(n, launch_pdl(wgrad_reduce_kernel, kRedBlocks, 256, 0, st, (const float*)n->wpart,
                           (size_t)kWgPart * n->num_sms, nblk, grad, adam ? *adam : none, adam ? 1 : 0));
    return PES_OK;
}

pes_status read_status(pes_init_net* n, cudaStream_t st)
{
    int h = 0;
    NET_CUDA(n, cudaMemcpyAsync(&h, n->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NET_CUDA(n, cudaStreamSynchronize(st));
    if (h) {
        NET_CUDA(n, cudaMemsetAsync(n->status, 0, sizeof(int), st));
        return net_fail(n, PES_ERR_TIMEOUT, "a tensor-core pipeline wait ran out of time (status %d)", h);
    }
    return PES_OK;
}

template <typename T>
pes_status loss_grad_t(pes_init_net* n, const T* y, const int64_t* off, int32_t B, int64_t N, const T* xt,
                       float* grad, double* loss, const AdamStep* adam, cudaStream_t st)
{
    int64_t R = 0;
    pes_status s = prepare_rows<T>(n, y, off, B, N, st, &R);
    if (s != PES_OK) return s;
    if ((s = forward_layers(n, R, true, st)) != PES_OK) return s;
    const float scale = (float)(2.0 / (5.0 * (double)N));
    const int lblocks = (int)std::min<int64_t>((R + 255) / 256, kLossBlocks);
    NET_CUDA(n, launch_pdl(loss_kernel<T>, lblocks, 256, 0, st, (const float*)n->out, xt, off, B, N, R, n->norm, scale,
                           1.0 / (5.0 * (double)N), n->dO, n->lpart, n->ticket, n->loss_dev));
    if ((s = backward_layers(n, R, grad, adam, st)) != PES_OK) return s;
    if (loss) {
        NET_CUDA(n, cudaMemcpyAsync(loss, n->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
        return read_status(n, st);
    }
    return PES_OK;
}

pes_status publish(pes_init_net* n, cudaStream_t st)
{
    NET_CUDA(n, launch_pdl(publish_kernel, (kWTiles * C * C + NLAYER * C + 255) / 256, 256, 0, st,
                           (const float*)n->params, n->Wf, n->Wb, n->bias));
    return PES_OK;
}

}  // namespace

extern "C" {

pes_status pes_init_create(pes_init_net** out, int64_t max_states, int32_t max_batch)
{
    if (!out || max_states < 1 || max_batch < 1) return PES_ERR_INVALID_ARG;
    *out = nullptr;
    pes_init_net* n = new (std::nothrow) pes_init_net();
    if (!n) return PES_ERR_CUDA;
    auto bail = [&](pes_status s) {
        pes_init_destroy(n);
        return s;
    };
    if (cudaGetDevice(&n->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, n->device) != cudaSuccess)
        return bail(PES_ERR_CUDA);
    int major = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, n->device);
    if (major < 10 || !encode_fn()) return bail(PES_ERR_UNSUPPORTED);
    n->max_states = max_states;
    n->max_batch = max_batch;
    n->max_rows = max_states + (int64_t)G * (max_batch + 1);
    const size_t rows = (size_t)n->max_rows;
    bool ok = cudaMalloc(&n->params, sizeof(float) * PES_INIT_NPARAMS) == cudaSuccess &&
              cudaMalloc(&n->m, sizeof(float) * PES_INIT_NPARAMS) == cudaSuccess &&
              cudaMalloc(&n->v, sizeof(float) * PES_INIT_NPARAMS) == cudaSuccess &&
              cudaMalloc(&n->grad, sizeof(float) * PES_INIT_NPARAMS) == cudaSuccess &&
              cudaMalloc(&n->bias, sizeof(float) * NLAYER * C) == cudaSuccess &&
              cudaMalloc(&n->wpart, sizeof(float) * (size_t)kWgPart * NLAYER * n->num_sms) == cudaSuccess &&
              cudaMalloc(&n->lpart, sizeof(double) * kLossBlocks) == cudaSuccess &&
              cudaMalloc(&n->loss_dev, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&n->ticket, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&n->Wf, sizeof(bf16) * kWTiles * C * C) == cudaSuccess &&
              cudaMalloc(&n->Wb, sizeof(bf16) * kWTiles * C * C) == cudaSuccess &&
              cudaMalloc(&n->out, sizeof(float) * kOutCols * rows) == cudaSuccess &&
              cudaMalloc(&n->mask, rows) == cudaSuccess && cudaMalloc(&n->status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&n->dO, sizeof(bf16) * C * rows) == cudaSuccess &&
              cudaMalloc(&n->dA, sizeof(bf16) * C * rows) == cudaSuccess &&
              cudaMalloc(&n->dB, sizeof(bf16) * C * rows) == cudaSuccess;
    for (int l = 0; ok && l < NLAYER; ++l) ok = cudaMalloc(&n->act[l], sizeof(bf16) * C * rows) == cudaSuccess;
    if (!ok) return bail(PES_ERR_CUDA);
    ok = cudaMemset(n->params, 0, sizeof(float) * PES_INIT_NPARAMS) == cudaSuccess &&
         cudaMemset(n->m, 0, sizeof(float) * PES_INIT_NPARAMS) == cudaSuccess &&
         cudaMemset(n->v, 0, sizeof(float) * PES_INIT_NPARAMS) == cudaSuccess &&
         cudaMemset(n->status, 0, sizeof(int)) == cudaSuccess &&
         cudaMemset(n->ticket, 0, sizeof(unsigned)) == cudaSuccess &&
         cudaMemset(n->dO, 0, sizeof(bf16) * C * rows) == cudaSuccess;
    if (!ok) return bail(PES_ERR_CUDA);
    for (int c = 0; c < 5; ++c) {
        n->norm.mu[c] = 0.0;
        n->norm.sigma[c] = 1.0;
        n->norm.inv_sigma[c] = 1.0;
        n->norm.mu_f[c] = 0.f;
        n->norm.inv_sigma_f[c] = 1.f;
    }
    if (!make_map(&n->mapWf, n->Wf, (uint64_t)kWTiles * C, C) || !make_map(&n->mapWb, n->Wb, (uint64_t)kWTiles * C, C))
        return bail(PES_ERR_CUDA);
    if (publish(n, 0) != PES_OK || cudaDeviceSynchronize() != cudaSuccess) return bail(PES_ERR_CUDA);
    *out = n;
    return PES_OK;
}

pes_status pes_init_destroy(pes_init_net* n)
{
    if (!n) return PES_ERR_INVALID_ARG;
    void* ptrs[] = {n->params, n->m, n->v, n->grad, n->bias, n->wpart, n->lpart, n->loss_dev, n->ticket, n->Wf, n->Wb,
                    n->out, n->mask, n->status, n->dO, n->dA, n->dB};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < NLAYER; ++l)
        if (n->act[l]) cudaFree(n->act[l]);
    delete n;
    return PES_OK;
}

const char* pes_init_last_error(const pes_init_net* n) { return n ? n->err : "NULL net"; }

pes_status pes_init_set_params(pes_init_net* n, const float* params, const double* mu, const double* sigma)
{
    if (!n || !params || !mu || !sigma) return net_fail(n, PES_ERR_INVALID_ARG, "NULL argument");
    for (int c = 0; c < 5; ++c)
        if (!(sigma[c] > 0.0) || !std::isfinite(mu[c]))
            return net_fail(n, PES_ERR_INVALID_ARG, "sigma must be positive and mu finite");
    for (int c = 0; c < 5; ++c) {
        n->norm.mu[c] = mu[c];
        n->norm.sigma[c] = sigma[c];
        n->norm.inv_sigma[c] = 1.0 / sigma[c];
        n->norm.mu_f[c] = (float)mu[c];
        n->norm.inv_sigma_f[c] = (float)(1.0 / sigma[c]);
    }
    NET_CUDA(n, cudaMemcpy(n->params, params, sizeof(float) * PES_INIT_NPARAMS, cudaMemcpyHostToDevice));
    NET_CUDA(n, cudaMemset(n->m, 0, sizeof(float) * PES_INIT_NPARAMS));
    NET_CUDA(n, cudaMemset(n->v, 0, sizeof(float) * PES_INIT_NPARAMS));
    n->adam_t = 0;
    pes_status s = publish(n, 0);
    if (s != PES_OK) return s;
    NET_CUDA(n, cudaDeviceSynchronize());
    return PES_OK;
}

pes_status pes_init_get_params(pes_init_net* n, float* params)
{
    if (!n || !params) return net_fail(n, PES_ERR_INVALID_ARG, "NULL argument");
    NET_CUDA(n, cudaDeviceSynchronize());
    NET_CUDA(n, cudaMemcpy(params, n->params, sizeof(float) * PES_INIT_NPARAMS, cudaMemcpyDeviceToHost));
    return PES_OK;
}

pes_status pes_init_get_state(pes_init_net* n, float* params, double* mu, double* sigma, float* adam_m,
                              float* adam_v, int64_t* adam_t)
{
    if (!n) return net_fail(n, PES_ERR_INVALID_ARG, "NULL net");
    NET_CUDA(n, cudaDeviceSynchronize());
    const size_t bytes = sizeof(float) * PES_INIT_NPARAMS;
    if (params) NET_CUDA(n, cudaMemcpy(params, n->params, bytes, cudaMemcpyDeviceToHost));
    if (adam_m) NET_CUDA(n, cudaMemcpy(adam_m, n->m, bytes, cudaMemcpyDeviceToHost));
    if (adam_v) NET_CUDA(n, cudaMemcpy(adam_v, n->v, bytes, cudaMemcpyDeviceToHost));
    for (int c = 0; c < 5; ++c) {
        if (mu) mu[c] = n->norm.mu[c];
        if (sigma) sigma[c] = n->norm.sigma[c];
    }
    if (adam_t) *adam_t = n->adam_t;
    return PES_OK;
}

pes_status pes_init_set_state(pes_init_net* n, const float* params, const double* mu, const double* sigma,
                              const float* adam_m, const float* adam_v, int64_t adam_t)
{
    if (!n || !params || !mu || !sigma || !adam_m || !adam_v) return net_fail(n, PES_ERR_INVALID_ARG, "NULL argument");
    if (adam_t < 0 || adam_t > INT32_MAX) return net_fail(n, PES_ERR_INVALID_ARG, "adam_t out of range");
    for (int i = 0; i < PES_INIT_NPARAMS; ++i)
        if (!std::isfinite(adam_m[i]) || !std::isfinite(adam_v[i]) || !(adam_v[i] >= 0.f))
            return net_fail(n, PES_ERR_INVALID_ARG, "Adam moments must be finite, the second ones non-negative");
    pes_status s = pes_init_set_params(n, params, mu, sigma);
    if (s != PES_OK) return s;
    const size_t bytes = sizeof(float) * PES_INIT_NPARAMS;
    NET_CUDA(n, cudaMemcpy(n->m, adam_m, bytes, cudaMemcpyHostToDevice));
    NET_CUDA(n, cudaMemcpy(n->v, adam_v, bytes, cudaMemcpyHostToDevice));
    n->adam_t = (int)adam_t;
    return PES_OK;
}

pes_status pes_init_forward(pes_init_net* n, pes_precision prec, const void* y, const int64_t* offsets, int32_t B,
                            int64_t N, void* x_init, void* stream)
{
    pes::TraceRange trace_("pes_init_forward");
    pes_status s = check_sizes(n, prec, y, offsets, B, N);
    if (s != PES_OK) return s;
    if (!x_init) return net_fail(n, PES_ERR_INVALID_ARG, "NULL x_init");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t R = 0;
    s = prec == PES_FP64 ? prepare_rows<double>(n, (const double*)y, offsets, B, N, st, &R)
                         : prepare_rows<float>(n, (const float*)y, offsets, B, N, st, &R);
    if (s != PES_OK) return s;
    if ((s = forward_layers(n, R, false, st)) != PES_OK) return s;
    const int blocks = (int)std::min<int64_t>((N + 255) / 256, (int64_t)n->num_sms * 16);
    if (prec == PES_FP64)
        NET_CUDA(n, launch_pdl(denorm_kernel<double>, blocks, 256, 0, st, (const float*)n->out, offsets, B, N, n->norm,
                               (double*)x_init));
    else
        NET_CUDA(n, launch_pdl(denorm_kernel<float>, blocks, 256, 0, st, (const float*)n->out, offsets, B, N, n->norm,
                               (float*)x_init));
    return PES_OK;
}

pes_status pes_init_loss_grad(pes_init_net* n, pes_precision prec, const void* y, const int64_t* offsets, int32_t B,
                              int64_t N, const void* x_target, float* grad, double* loss, void* stream)
{
    pes::TraceRange trace_("pes_init_loss_grad");
    pes_status s = check_sizes(n, prec, y, offsets, B, N);
    if (s != PES_OK) return s;
    if (!x_target || !grad) return net_fail(n, PES_ERR_INVALID_ARG, "NULL x_target or grad");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return prec == PES_FP64
               ? loss_grad_t<double>(n, (const double*)y, offsets, B, N, (const double*)x_target, grad, loss, nullptr, st)
               : loss_grad_t<float>(n, (const float*)y, offsets, B, N, (const float*)x_target, grad, loss, nullptr, st);
}

pes_status pes_init_train_step(pes_init_net* n, pes_precision prec, const void* y, const int64_t* offsets,
                               int32_t B, int64_t N, const void* x_target, float lr, double* loss, void* stream)
{
    pes::TraceRange trace_("pes_init_train_step");
    pes_status s = check_sizes(n, prec, y, offsets, B, N);
    if (s != PES_OK) return s;
    if (!(lr > 0.f)) return net_fail(n, PES_ERR_INVALID_ARG, "lr must be positive");
    if (!x_target) return net_fail(n, PES_ERR_INVALID_ARG, "NULL x_target");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the Adam step runs in the gradient reduction, each parameter as soon as
    // its gradient is summed
    const double b1 = 0.9, b2 = 0.999;
    const int t = n->adam_t + 1;
    AdamStep a;
    a.p = n->params;
    a.m = n->m;
    a.v = n->v;
    a.Wf = n->Wf;
    a.Wb = n->Wb;
    a.bias = n->bias;
    a.lr = lr;
    a.b1 = (float)b1;
    a.b2 = (float)b2;
    a.eps = 1e-8f;
    a.c1 = (float)(1.0 / (1.0 - std::pow(b1, t)));
    a.c2 = (float)(1.0 / (1.0 - std::pow(b2, t)));
    s = prec == PES_FP64
            ? loss_grad_t<double>(n, (const double*)y, offsets, B, N, (const double*)x_target, n->grad, loss, &a, st)
            : loss_grad_t<float>(n, (const float*)y, offsets, B, N, (const float*)x_target, n->grad, loss, &a, st);
    if (s != PES_OK) return s;
    n->adam_t = t;
    return PES_OK;
}

}  // extern "C"
