// apply_tcgen05.cu -- aggregated k-qubit gate apply on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), 3xFP16 split precision, k = 4, 5 and 6.
//
// Same real-embedded GEMM as apply_tc.cu (W^T = V^T . R^T with R = [[Re M, -Im M],
// [Im M, Re M]]), as tcgen05.mma steps of M = 128 (groups) x N = 2^(k+1) (output reals) x
// K = 16.  A tile is 128 consecutive groups: 2^(k+7) amplitudes whose addresses differ only in
// the tile's free bits, the k targets and the 7 lowest other bits.  Those always include bits
// 0..6, so a tile is at most 2^k runs of >= 128 contiguous amplitudes, moved by the bulk-copy
// (TMA) engine into shared memory in address order.  Where bit 7 is not a target the runs are
// only 1 KiB, and the kernel takes 256-group tiles (two M = 128 sub-tiles, row bit 7 = sub-tile)
// so that every copy moves 2 KiB (measured: 1 KiB copies cap the kernel at ~74% of the 2 KiB
// rate).  6-qubit blocks keep 128-group tiles in a 2-stage ring beside 64 KiB of R^T; they run on
// k_apply_tc6a below, which keeps their A operand in tensor memory so that a stage is free as soon
// as it has been read (the pipeline described next is that of k = 4 and 5).
//
// One persistent CTA per SM, warp-specialised, tiles pipelined through a ring of S shared-memory
// stages (one tile each, 128 x 2^k complex64):
//  * warp 8 loads tile i into stage i % S with cp.async.bulk (a run per lane), completing on an
//    mbarrier by byte count, as soon as the stage's previous tile has been drained;
//  * converter warps 0-7: thread = (row, half of the members).  It reads its half-row (staging
//    index = row bits | member bits in address order: no bank conflicts while no target is
//    below bit 4; with one such target each row XORs its member index by one of its own row
//    bits, which restores that), the two halves combine their maxima, and the row is scaled by a power of two
//    (largest component < 2^14, so FP16 stays normal), split hi = fp16(a), lo = fp16(a - hi)
//    and written in place as the MMA's A operand (K-major core matrices: 8 rows x 16 bytes;
//    128 B between the two K halves of a 16-wide slice, 256 B between 8-row groups);
//  * warp 9 (one thread) issues the MMAs: hi*hi chained through one TMEM accumulator, the
//    corrections hi*lo + lo*hi through a second (their rounding is 2^-11 smaller), and commits
//    them to the stage's mbarrier;
//  * drainer warps 10-17 read both accumulators (tcgen05.ld 32x32b: warp w sees TMEM lanes
//    32 (w % 4) ..), add them and undo the row's scale.  With a deep stage ring the amplitudes
//    go back into the stage and the lanes of warp 10 store its runs with bulk copies; with the
//    3-stage ring of 64 KiB tiles, or a target below bit 4, they are stored from registers (16
//    consecutive rows cover 64-128 contiguous bytes), which frees the stage as soon as TMEM is
//    read.  Blocks with two or more targets below bit 4 are left to the other kernels.
// K (input reals) is interleaved, column 2m + p is part p (Re, Im) of member m, so a row's
// 16-byte chunk is four consecutive members; N likewise.  R^T (hi, lo; FP16, core-matrix layout)
// is built on the host and staged in shared memory once per CTA.  Two TMEM accumulator sets let
// tile i + 1 be multiplied while tile i is drained.
//
// BF16x3 (SIM_BF16X3) is the same pipeline with BF16 pieces (8 significant bits each instead of
// FP16's 11): hi = bf16(a), lo = bf16(a - hi), the same three products, the operand format bits
// of the instruction descriptor set to BF16.  The row scale is kept (a power of two, exact).
//
// Every wait is bounded in time (%globaltimer): a timeout records the failure in an error word
// and a shared abort flag that ends every role's loop; the CTA then waits for its bulk copies in
// flight and frees its tensor memory before returning.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "internal.h"

namespace sycsim {
namespace {

#ifndef SYCSIM_TC6_ATMEM
#define SYCSIM_TC6_ATMEM 1  // 6-qubit blocks: A operand in tensor memory (k_apply_tc6a)
#endif

#ifndef SYCSIM_TC5_RUN_LOG2_MAX
#define SYCSIM_TC5_RUN_LOG2_MAX 8  // 2 KiB copies: measured fastest (1 KiB: -26%, 4 KiB: -9%)
#endif

constexpr int kRows = 128;                     // groups per tile = MMA M
constexpr unsigned long long kWaitNs = 4000000000ull;  // 4 s: far above any legitimate wait
constexpr int kConv = 256;                     // converter threads: warps 0-7
constexpr int kLoadWarp = 8;
constexpr int kMmaWarp = 9;
constexpr int kDrain = 256;                    // drainer threads: warps 10-17
constexpr int kThreadsTc5 = kConv + 64 + kDrain;

struct Tc5Geom {
    float2 *psi;
    uint64_t n_tiles;        // 2^(nbits - k - 7) / R2
    int tpos[kMaxK];         // target bit positions, ascending
    int run_log2;            // L: a tile is 2^(k+7+log2 R2-L) runs of 2^L contiguous amplitudes
    int nlow;                // targets below bit 4 (they are member bits 0 .. nlow-1)
    uint64_t off_run[64];    // address offset of run c (c's bits deposited on the free bits >= L)
    uint32_t midx[64];       // staging index of member m in row 0 (row r: midx[m] | ridx(r))
    uint32_t ridx[8];        // staging-index bit of row bit j (bit 7: sub-tile)
    uint64_t roff[8];        // address offset of row bit j
    uint64_t moff[64];       // address offset of member m
    const uint32_t *bmat;    // R^T hi then lo, FP16 core-matrix layout, as 32-bit words
    int *err;                // set to 1 if a wait timed out
    double *red;             // if set: this CTA's (sum p, sum p^2) of the results at red[2 blockIdx.x]
};

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The drainers' fused reduction: each thread's FP64 sums of p = |psi_i|^2 and p^2 over the results
// it stored (FP32 within a tile), combined in a fixed order into the CTA's pair (deterministic).
// Called by all 256 drainer threads (dtid 0..255) after their last tile.
__device__ __forceinline__ void drain_partials(double r1, double r2, int dtid, double (*part)[2], double *out)
{
    r1 = warp_sum_d(r1);
    r2 = warp_sum_d(r2);
    if ((dtid & 31) == 0) {
        part[dtid >> 5][0] = r1;
        part[dtid >> 5][1] = r2;
    }
    asm volatile("bar.sync 2, 256;\n" ::: "memory");
    if (dtid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += part[w][0];
            b += part[w][1];
        }
        out[2 * blockIdx.x] = a;
        out[2 * blockIdx.x + 1] = b;
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    // K-major, no swizzle: LBO = 128 B (between K halves), SBO = 256 B (between 8-row groups),
    // descriptor version 1
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint64_t insert_zero_bits_g(uint64_t x, const int *pos, int cnt)
{
#pragma unroll
    for (int i = 0; i < kMaxK; ++i) {
        if (i >= cnt) break;
        const int p = pos[i];
        const uint64_t lo = x & ((1ull << p) - 1);
        x = ((x >> p) << (p + 1)) | lo;
    }
    return x;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t mbar_try(uint32_t bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return done;
}

// Wait for the phase of the given parity, the thread suspended in between polls; gives up after
// kWaitNs or once another role has aborted.
__device__ __forceinline__ bool mbar_wait_abort(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity, 0)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity, 20000)) return true;
        if (*abort_flag || global_ns() - t0 > kWaitNs) return false;
    }
}

// Wait for work this thread issued itself (copies, MMAs) to land, even after an abort.
__device__ __forceinline__ void mbar_wait_own(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    while (!mbar_try(bar, parity, 20000) && global_ns() - t0 <= kWaitNs) {
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Named barrier over n threads that also ANDs a predicate across them.
__device__ __forceinline__ bool bar_and(int id, int n, bool p)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.and.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// A tile is R2 sub-tiles of 128 groups (row bit 7 = sub-tile), one MMA M = 128 each.
__device__ __forceinline__ void bulk_store(void *dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}

// Shared memory: S stages of one tile each (raw amplitudes, then A hi | A lo of each sub-tile in
// place, then the results), then B hi | B lo (KS slices of N x 16 FP16 each).
template <int K, int R2>
struct Tc5Layout {
    static constexpr int D = 1 << K;
    static constexpr int KS = 2 * D / 16;         // K slices of 16 reals
    static constexpr int N = 2 * D;               // output reals
    static constexpr int A_SLICE = kRows * 32;    // bytes
    static constexpr int B_SLICE = N * 32;
    static constexpr int A_BYTES = KS * A_SLICE;  // one of hi, lo, one sub-tile
    static constexpr int B_BYTES = KS * B_SLICE;
    static constexpr int SUB = kRows * D * 8;     // one sub-tile = 2 * A_BYTES
    static constexpr int STAGE = R2 * SUB;
    // stages: K <= 5 within 200 KiB (at most 8); K = 6 (64 KiB tiles, 64 KiB of B hi/lo) fits 2
    static constexpr int S = K == 6 ? 2 : ((200 * 1024) / STAGE < 8 ? (200 * 1024) / STAGE : 8);
    static constexpr int SMEM = S * STAGE + 2 * B_BYTES;
    static constexpr int TMEM_SUB = 2 * N;        // main + corrections of one sub-tile
    static constexpr int TMEM_SET = R2 * TMEM_SUB;
    static constexpr int TMEM_COLS = 2 * TMEM_SET;  // two sets
    static_assert(SUB == 2 * A_BYTES, "A hi/lo fill a sub-tile");
    static_assert(S >= (K == 6 ? 2 : 3), "stage ring too short");
    static_assert(K < 6 || R2 == 1, "6-qubit blocks: one 128-group sub-tile (tensor memory)");
    // results leave through the stage with bulk stores when the ring is deep enough to hold a
    // stage until its store has read it; the 3-stage ring (64 KiB tiles) stores from registers so
    // that a stage is free as soon as its accumulators are read (measured: +20% there, -8% at 6+)
    static constexpr bool BULK_STORE = S >= 6;
    static_assert(TMEM_COLS <= 512, "tensor memory");
};

__device__ __forceinline__ void swap_u32(uint32_t &a, uint32_t &b)
{
    const uint32_t t = a;
    a = b;
    b = t;
}

__device__ __forceinline__ uint32_t cm_off(int row, int k) { return (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 + (k & 7) * 2; }

// Per tile i (local index; stage s = i % S, stage phase (i / S) & 1; TMEM set i % 2, set phase
// (i / 2) & 1):
//   loader: wait drained[s] of tile i - S, load the runs into stage s (loaded[s] counts bytes);
//   converters: wait loaded[s], read the rows, combine the halves' maxima (barrier), write A and
//     the row scales in place, arrive full[s];
//   MMA thread: wait full[s] and tmem_free of tile i - 2, multiply, commit to mma_done[s];
//   drainers: wait mma_done[s] and full[s], take the row scales and the tile base into registers;
//     storing from registers, arrive drained[s] right then (the MMAs have read the stage), read
//     TMEM, arrive tmem_free and store; with bulk stores, read TMEM, arrive tmem_free, write the
//     results into stage s, barrier, and warp 10 stores the runs and, once the store of tile
//     i - 1 has read its stage, arrives drained for it.
// A stage is reloaded only after every drainer has passed its waits for it and taken what it
// needs, and a TMEM set reused only after its read, so no barrier can run a phase ahead of a
// waiter that still has to see the previous phase.
template <int K, int R2, bool LOWT, bool BF>
__global__ void __launch_bounds__(kThreadsTc5, 1) k_apply_tcgen05(Tc5Geom g)
{
    using L = Tc5Layout<K, R2>;
    constexpr bool BULK = L::BULK_STORE && !LOWT;  // results back through the stage
    constexpr int D = L::D, KS = L::KS, N = L::N, S = L::S, H = D / 2;  // H members per thread
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *bHi = sm + S * L::STAGE, *bLo = bHi + L::B_BYTES;
    __shared__ __align__(8) uint64_t loaded[S], full[S], mma_done[S], drained[S], tmem_free[2];
    __shared__ float row_inv[S][R2][kRows];
    __shared__ float amax_part[R2][2][kRows];
    __shared__ double red_part[8][2];
    __shared__ uint64_t tile_base[S];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n_runs = (R2 << (K + 7)) >> g.run_log2;
    const uint32_t run_bytes = 8u << g.run_log2;

    {
        const uint32_t *src = g.bmat;
        uint32_t *dst = reinterpret_cast<uint32_t *>(bHi);
        for (int i = tid; i < (2 * L::B_BYTES) / 4; i += blockDim.x) dst[i] = src[i];
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // B is read by the MMA unit
    }
    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&loaded[st])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&full[st])), "r"(kConv) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mma_done[st])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&drained[st])),
                         "r"(BULK ? 1 : kDrain)
                         : "memory");
        }
        for (int st = 0; st < 2; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&tmem_free[st])), "r"(kDrain)
                         : "memory");
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "n"(L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    volatile int *ab = &abort_flag;
    auto give_up = [&]() {
        *ab = 1;
        atomicExch(g.err, 1);
    };

    if (warp < kLoadWarp) {
        // ---------------- converters ----------------
        const int row = tid & (kRows - 1), half = tid >> 7;
        uint32_t rx = 0;
#pragma unroll
        for (int j = 0; j < 7; ++j)
            if ((row >> j) & 1) rx |= g.ridx[j];
        // With targets below bit 4 (member bits 0 .. nlow-1; the launcher takes nlow <= 1) the
        // rows of one member do not cover 16 bank pairs; register j of this thread then holds
        // member (H half + j) ^ mu, with mu taken from the row bits that do not reach address
        // bits 0..3, so that the 16 rows of a half-warp read 16 distinct bank pairs.
        uint32_t mu = 0, mux = 0;
        if constexpr (LOWT) {
            mu = (row >> (4 - g.nlow)) & ((1u << g.nlow) - 1);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((mu >> q) & 1) mux ^= g.midx[1 << q];
        }
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
            const int st = i % S;
            const bool ok = mbar_wait_abort(smem_u32(&loaded[st]), (i / S) & 1, ab);
            if (!bar_and(1, kConv, ok)) {
                give_up();
                break;
            }
            uint8_t *stage = sm + st * L::STAGE;
            float2 x[R2][H];
#pragma unroll
            for (int u = 0; u < R2; ++u) {
                const uint32_t rxu = u ? rx | g.ridx[7] : rx;
                float amax = 0.f;
#pragma unroll
                for (int m = 0; m < H; ++m) {
                    x[u][m] = *reinterpret_cast<const float2 *>(stage + 8 * ((g.midx[H * half + m] ^ mux) | rxu));
                    amax = fmaxf(amax, fmaxf(fabsf(x[u][m].x), fabsf(x[u][m].y)));
                }
                amax_part[u][half][row] = amax;
            }
            bar_sync(1, kConv);  // every row read before A overwrites the stage; both halves' maxima
#pragma unroll
            for (int u = 0; u < R2; ++u) {
                const float amax = fmaxf(amax_part[u][0][row], amax_part[u][1][row]);
                int e = 0;
                frexpf(amax, &e);
                const int sh = amax > 0.f ? max(-100, min(100, 14 - e)) : 0;
                const float sc = ldexpf(1.f, sh);
                if (half == 0) row_inv[st][u][row] = ldexpf(1.f, -sh);
                uint8_t *aHi = stage + u * L::SUB, *aLo = aHi + L::A_BYTES;
#pragma unroll
                for (int cc = 0; cc < H / 4; ++cc) {
                    const int c = (half * (H / 4) + cc) ^ (int)(mu >> 2);  // 4-member chunk of the row
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float re = x[u][4 * cc + j].x * sc, im = x[u][4 * cc + j].y * sc;
                        if constexpr (BF) {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
                            const float2 hf = __bfloat1622float2(h);
                            const __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
                            hi[j] = *reinterpret_cast<const uint32_t *>(&h);
                            lo[j] = *reinterpret_cast<const uint32_t *>(&l);
                        } else {
                            const __half2 h = __floats2half2_rn(re, im);
                            const float2 hf = __half22float2(h);
                            const __half2 l = __floats2half2_rn(re - hf.x, im - hf.y);
                            hi[j] = *reinterpret_cast<const uint32_t *>(&h);
                            lo[j] = *reinterpret_cast<const uint32_t *>(&l);
                        }
                    }
                    if constexpr (LOWT) {  // position p of the chunk takes register p ^ (mu & 3)
                        if (mu & 1) {
                            swap_u32(hi[0], hi[1]), swap_u32(hi[2], hi[3]);
                            swap_u32(lo[0], lo[1]), swap_u32(lo[2], lo[3]);
                        }
                        if (mu & 2) {
                            swap_u32(hi[0], hi[2]), swap_u32(hi[1], hi[3]);
                            swap_u32(lo[0], lo[2]), swap_u32(lo[1], lo[3]);
                        }
                    }
                    const uint32_t off = (c >> 1) * L::A_SLICE + cm_off(row, 8 * (c & 1));
                    *reinterpret_cast<uint4 *>(aHi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(aLo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(smem_u32(&full[st]));
        }
    } else if (warp == kLoadWarp) {
        // ---------------- bulk loads (one run per lane) ----------------
        const int lane = tid & 31;
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
            const int st = i % S;
            const bool ok = i < (uint32_t)S || mbar_wait_abort(smem_u32(&drained[st]), (i / S - 1) & 1, ab);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) give_up();
                break;
            }
            const uint64_t base = insert_zero_bits_g(tile * (kRows * R2), g.tpos, K);
            const uint32_t bar = smem_u32(&loaded[st]);
            if (lane == 0) {
                tile_base[st] = base;
                mbar_expect_tx(bar, L::STAGE);  // before any of the copies can complete
            }
            __syncwarp();
            const uint32_t dst = smem_u32(sm + st * L::STAGE);
            for (int c = lane; c < n_runs; c += 32) bulk_load(dst + c * run_bytes, g.psi + base + g.off_run[c], run_bytes, bar);
        }
        // no load may still be writing the stages when the CTA leaves (matters after an abort)
        if (lane == 0)
            for (uint32_t j = i > (uint32_t)S ? i - S : 0; j < i; ++j) mbar_wait_own(smem_u32(&loaded[j % S]), (j / S) & 1);
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if ((tid & 31) == 0) {
            // F32 accumulate; A and B FP16 (format 0) or BF16 (format 1, bits 7 and 10); K-major
            const uint32_t idesc = (1u << 4) | (BF ? (1u << 7) | (1u << 10) : 0u) | ((uint32_t)(N >> 3) << 17) |
                                   ((uint32_t)(kRows >> 4) << 24);
            uint32_t i = 0;
            for (uint64_t tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
                const int st = i % S;
                if (!mbar_wait_abort(smem_u32(&full[st]), (i / S) & 1, ab) ||
                    (i >= 2 && !mbar_wait_abort(smem_u32(&tmem_free[i & 1]), (i / 2 - 1) & 1, ab))) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
                for (int u = 0; u < R2; ++u) {
                    const uint8_t *aHi = sm + st * L::STAGE + u * L::SUB, *aLo = aHi + L::A_BYTES;
                    const uint32_t acc = tmem + (i & 1) * L::TMEM_SET + u * L::TMEM_SUB;
#pragma unroll
                    for (int s = 0; s < KS; ++s)
                        umma_f16(acc, umma_desc(smem_u32(aHi + s * L::A_SLICE)),
                                 umma_desc(smem_u32(bHi + s * L::B_SLICE)), idesc, s > 0);
#pragma unroll
                    for (int s = 0; s < KS; ++s) {
                        umma_f16(acc + N, umma_desc(smem_u32(aHi + s * L::A_SLICE)),
                                 umma_desc(smem_u32(bLo + s * L::B_SLICE)), idesc, s > 0);
                        umma_f16(acc + N, umma_desc(smem_u32(aLo + s * L::A_SLICE)),
                                 umma_desc(smem_u32(bHi + s * L::B_SLICE)), idesc, 1);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&mma_done[st]))
                             : "memory");
            }
            // the tensor memory is freed only after the last MMA issued has completed
            if (i > 0) mbar_wait_own(smem_u32(&mma_done[(i - 1) % S]), ((i - 1) / S) & 1);
        }
    } else {
        // ---------------- drainers ----------------
        const int q = warp & 3;                        // TMEM lane quarter this warp may read
        const int half = (warp - kMmaWarp - 1) >> 2;   // warps 10-13: members 0..H-1; 14-17: H..D-1
        const int row = 32 * q + (tid & 31);
        const bool store_warp = warp == kMmaWarp + 1;  // bulk stores: its lanes store a run each
        const int lane = tid & 31;
        uint32_t rx = 0;  // staging index of this row
        uint64_t ro = 0;  // address offset of this row within the tile (16 consecutive rows: 128 B)
#pragma unroll
        for (int j = 0; j < 7; ++j)
            if ((row >> j) & 1) {
                rx |= g.ridx[j];
                ro += g.roff[j];
            }
        double r1 = 0.0, r2 = 0.0;  // fused reduction (g.red)
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
            const int st = i % S;
            const bool ok = mbar_wait_abort(smem_u32(&mma_done[st]), (i / S) & 1, ab) &&
                            mbar_wait_abort(smem_u32(&full[st]), (i / S) & 1, ab);
            if (!bar_and(2, kDrain, ok)) {  // uniform: tcgen05.ld below needs whole warps
                give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint8_t *stage = sm + st * L::STAGE;
            float2 *const dst = g.psi + tile_base[st] + ro;
            float inv[R2];
#pragma unroll
            for (int u = 0; u < R2; ++u) inv[u] = row_inv[st][u][row];
            // storing from registers, the stage is dead once the MMAs have read it (mma_done): with
            // its row scales and base in registers, release it now so the next tile's copies start
            // while this one is drained
            if constexpr (!BULK) mbar_arrive(smem_u32(&drained[st]));
            if constexpr (K == 6) {
                // 64 output reals per thread: read, add, unscale and store 16 columns at a time
                // (registers), releasing the tensor memory and the stage after the last read
                const uint32_t lane_base = tmem + (i & 1) * L::TMEM_SET + ((uint32_t)(32 * q) << 16) + half * (N / 2);
#pragma unroll
                for (int c0 = 0; c0 < N / 2; c0 += 16) {
                    float a[16], b[16];
                    tmem_ld16(lane_base + c0, a);
                    tmem_ld16(lane_base + N + c0, b);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    if (c0 == N / 2 - 16) {
                        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                        mbar_arrive(smem_u32(&tmem_free[i & 1]));
                    }
                    float t1 = 0.f, t2 = 0.f;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float2 v =
                            make_float2((a[2 * j] + b[2 * j]) * inv[0], (a[2 * j + 1] + b[2 * j + 1]) * inv[0]);
                        const float p = fmaf(v.x, v.x, v.y * v.y);
                        t1 += p;
                        t2 = fmaf(p, p, t2);
                        __stcs(dst + g.moff[H * half + c0 / 2 + j], v);
                    }
                    r1 += t1;
                    r2 += t2;
                }
                continue;
            }
#pragma unroll
            for (int u = 0; u < R2; ++u) {
                const uint32_t lane_base =
                    tmem + (i & 1) * L::TMEM_SET + u * L::TMEM_SUB + ((uint32_t)(32 * q) << 16) + half * (N / 2);
                float a[N / 2], b[N / 2];
#pragma unroll
                for (int c0 = 0; c0 < N / 2; c0 += 16) {
                    tmem_ld16(lane_base + c0, *reinterpret_cast<float(*)[16]>(a + c0));
                    tmem_ld16(lane_base + N + c0, *reinterpret_cast<float(*)[16]>(b + c0));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (u == R2 - 1) {  // TMEM set read: release it
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    mbar_arrive(smem_u32(&tmem_free[i & 1]));
                }
                float2 o[H];
                float t1 = 0.f, t2 = 0.f;
#pragma unroll
                for (int j = 0; j < H; ++j) {
                    o[j] = make_float2((a[2 * j] + b[2 * j]) * inv[u], (a[2 * j + 1] + b[2 * j + 1]) * inv[u]);
                    const float p = fmaf(o[j].x, o[j].x, o[j].y * o[j].y);
                    t1 += p;
                    t2 = fmaf(p, p, t2);
                }
                r1 += t1;
                r2 += t2;
                if constexpr (BULK) {
                    const uint32_t rxu = u ? rx | g.ridx[7] : rx;
#pragma unroll
                    for (int j = 0; j < H; ++j)
                        *reinterpret_cast<float2 *>(stage + 8 * (g.midx[H * half + j] | rxu)) = o[j];
                } else {
                    float2 *const du = u ? dst + g.roff[7] : dst;
#pragma unroll
                    for (int j = 0; j < H; ++j) __stcs(du + g.moff[H * half + j], o[j]);
                }
            }
            if constexpr (BULK) {
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the bulk store reads it
                bar_sync(2, kDrain);  // the whole tile is back in the stage
                if (store_warp) {
                    float2 *const tb = g.psi + tile_base[st];
                    const uint32_t src = smem_u32(stage);
                    for (int c = lane; c < n_runs; c += 32) bulk_store(tb + g.off_run[c], src + c * run_bytes, run_bytes);
                    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
                    if (i > 0) {
                        asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");  // tile i - 1 read out
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&drained[(i - 1) % S]));
                    }
                }
            }
        }
        if (BULK && store_warp) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
        if (g.red) drain_partials(r1, r2, tid - (kConv + 64), red_part, g.red);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(L::TMEM_COLS));
}

// ---- 6-qubit blocks with the A operand in tensor memory ----------------------------------------
// A 6-qubit tile (128 groups x 64 members) fills a 64 KiB stage, and R^T hi/lo take another 64 KiB,
// so only two stages fit; writing the A operand back into the stage keeps each stage busy from its
// load through the conversion and the MMAs.  Here the converters put A (hi, lo) into tensor memory
// instead (tcgen05.st; one row per TMEM lane, column c = member c as a packed (re, im) pair, the
// K order of R^T), and release the stage as soon as they have read it: the next tile's copies start
// while this one is still being multiplied.  Tensor memory: A buffers for two tiles (hi 64 | lo 64
// columns each) at columns 0-255, one accumulator set (main 128 | corrections 128) at 256-511.
// Per tile i (stage i % 2, A buffer i % 2, scale slot i % 4):
//   loader: wait stage_free of tile i - 2, load the runs (loaded counts bytes);
//   converters: wait mma_done of tile i - 2 (A buffer free) and loaded, read the rows, combine the
//     halves' maxima, arrive stage_free, write the row scales (arrive scales), split hi / lo into
//     the A buffer, arrive a_full;
//   MMA thread: wait a_full and tmem_free of tile i - 1, issue, commit to mma_done;
//   drainers: wait mma_done and scales, read the accumulators 16 columns at a time, arrive tmem_free
//     after the last read, store from registers.
// Every barrier's next phase needs the waiter's own progress first (e.g. the converters of tile
// i + 4 rewrite scale slot i % 4 only after the MMAs of tile i + 2, which wait for the drain of
// tile i + 1), so no parity wait can miss a phase.
constexpr int kTc6Stage = kRows * 64 * 8;        // 64 KiB of raw amplitudes
constexpr int kTc6Stages = 2;
constexpr int kTc6BBytes = 8 * (128 * 32);       // R^T hi (or lo): 8 K-slices of 128 x 16 FP16
constexpr int kTc6Smem = kTc6Stages * kTc6Stage + 2 * kTc6BBytes;

__device__ __forceinline__ void umma_f16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc,
                                            uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st16(uint32_t ta, const uint32_t *r)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
            ta),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

template <bool BF>
__device__ __forceinline__ void split_pair(float re, float im, uint32_t &hi, uint32_t &lo)
{
    if constexpr (BF) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __half2 h = __floats2half2_rn(re, im);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(re - hf.x, im - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

template <bool LOWT, bool BF>
__global__ void __launch_bounds__(kThreadsTc5, 1) k_apply_tc6a(Tc5Geom g)
{
    constexpr int D = 64, KS = 8, N = 128, S = kTc6Stages, H = D / 2;  // H members per thread
    constexpr int B_SLICE = N * 32;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *bHi = sm + S * kTc6Stage, *bLo = bHi + kTc6BBytes;
    __shared__ __align__(8) uint64_t loaded[S], stage_free[S], a_full[2], mma_done[2], tmem_free, scales[4];
    __shared__ float row_inv[4][kRows];
    __shared__ float amax_part[2][kRows];
    __shared__ double red_part[8][2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n_runs = (1 << (6 + 7)) >> g.run_log2;
    const uint32_t run_bytes = 8u << g.run_log2;

    {
        const uint32_t *src = g.bmat;
        uint32_t *dst = reinterpret_cast<uint32_t *>(bHi);
        for (int i = tid; i < (2 * kTc6BBytes) / 4; i += blockDim.x) dst[i] = src[i];
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // B is read by the MMA unit
    }
    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&loaded[st])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&stage_free[st])), "r"(kConv)
                         : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&a_full[b])), "r"(kConv) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mma_done[b])) : "memory");
        }
        for (int j = 0; j < 4; ++j)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&scales[j])), "r"(kConv) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&tmem_free)), "r"(kDrain) : "memory");
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    volatile int *ab = &abort_flag;
    auto give_up = [&]() {
        *ab = 1;
        atomicExch(g.err, 1);
    };

    if (warp < kLoadWarp) {
        // ---------------- converters: stage -> registers -> A (hi, lo) in tensor memory ----------------
        const int row = tid & (kRows - 1), half = tid >> 7;
        uint32_t rx = 0;
#pragma unroll
        for (int j = 0; j < 7; ++j)
            if ((row >> j) & 1) rx |= g.ridx[j];
        // one target below bit 4 (member bit 0): register m holds member (H half + m) ^ mu for
        // conflict-free stage reads; the pairs are swapped back before the columns are written
        uint32_t mu = 0, mux = 0;
        if constexpr (LOWT) {
            mu = (row >> 3) & 1u;
            if (mu) mux = g.midx[1];
        }
        const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lanes
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
            const int st = i % S, b = i & 1, j = i & 3;
            const bool ok = (i < 2 || mbar_wait_abort(smem_u32(&mma_done[b]), ((i - 2) >> 1) & 1, ab)) &&
                            mbar_wait_abort(smem_u32(&loaded[st]), (i / S) & 1, ab);
            if (!bar_and(1, kConv, ok)) {
                give_up();
                break;
            }
            // two passes over this thread's half-row: the maximum first, then 16 members at a
            // time converted straight from the stage (a register budget of 96 per thread: 18 warps
            // share four 16,384-register sub-partitions, five warps on two of them)
            const uint8_t *stage = sm + st * kTc6Stage;
            float amax = 0.f;
#pragma unroll
            for (int m = 0; m < H; ++m) {
                const float2 v = *reinterpret_cast<const float2 *>(stage + 8 * ((g.midx[H * half + m] ^ mux) | rx));
                amax = fmaxf(amax, fmaxf(fabsf(v.x), fabsf(v.y)));
            }
            amax_part[half][row] = amax;
            bar_sync(1, kConv);  // both halves' maxima
            amax = fmaxf(amax_part[0][row], amax_part[1][row]);
            int e = 0;
            frexpf(amax, &e);
            const int sh = amax > 0.f ? max(-100, min(100, 14 - e)) : 0;
            const float sc = ldexpf(1.f, sh);
            if (half == 0) row_inv[j][row] = ldexpf(1.f, -sh);
            mbar_arrive(smem_u32(&scales[j]));
            const uint32_t ta = tmem + lane_off + (uint32_t)(b * 128 + half * H);
#pragma unroll
            for (int c = 0; c < H / 16; ++c) {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    const float2 v =
                        *reinterpret_cast<const float2 *>(stage + 8 * ((g.midx[H * half + 16 * c + m] ^ mux) | rx));
                    split_pair<BF>(v.x * sc, v.y * sc, hi[m], lo[m]);
                }
                if constexpr (LOWT) {
                    if (mu) {
#pragma unroll
                        for (int m = 0; m < 16; m += 2) {
                            swap_u32(hi[m], hi[m + 1]);
                            swap_u32(lo[m], lo[m + 1]);
                        }
                    }
                }
                tmem_st16(ta + 16 * c, hi);
                tmem_st16(ta + 64 + 16 * c, lo);
            }
            mbar_arrive(smem_u32(&stage_free[st]));  // the stage has been read for the last time
            asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(smem_u32(&a_full[b]));
        }
    } else if (warp == kLoadWarp) {
        // ---------------- bulk loads (one run per lane) ----------------
        const int lane = tid & 31;
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
            const int st = i % S;
            const bool ok = i < (uint32_t)S || mbar_wait_abort(smem_u32(&stage_free[st]), (i / S - 1) & 1, ab);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) give_up();
                break;
            }
            const uint64_t base = insert_zero_bits_g(tile * kRows, g.tpos, 6);
            const uint32_t bar = smem_u32(&loaded[st]);
            if (lane == 0) mbar_expect_tx(bar, kTc6Stage);  // before any of the copies can complete
            __syncwarp();
            const uint32_t dst = smem_u32(sm + st * kTc6Stage);
            for (int c = lane; c < n_runs; c += 32) bulk_load(dst + c * run_bytes, g.psi + base + g.off_run[c], run_bytes, bar);
        }
        if (lane == 0)
            for (uint32_t j = i > (uint32_t)S ? i - S : 0; j < i; ++j) mbar_wait_own(smem_u32(&loaded[j % S]), (j / S) & 1);
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer: A from tensor memory, B (R^T) from shared memory ----------------
        if ((tid & 31) == 0) {
            const uint32_t idesc = (1u << 4) | (BF ? (1u << 7) | (1u << 10) : 0u) | ((uint32_t)(N >> 3) << 17) |
                                   ((uint32_t)(kRows >> 4) << 24);
            const uint32_t acc = tmem + 256;  // main at 256, corrections at 256 + N
            uint32_t i = 0;
            for (uint64_t tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
                const int b = i & 1;
                if (!mbar_wait_abort(smem_u32(&a_full[b]), (i >> 1) & 1, ab) ||
                    (i >= 1 && !mbar_wait_abort(smem_u32(&tmem_free), (i - 1) & 1, ab))) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t aHi = tmem + b * 128, aLo = aHi + 64;  // 8 columns per K-slice of 16
#pragma unroll
                for (int s = 0; s < KS; ++s)
                    umma_f16_ta(acc, aHi + 8 * s, umma_desc(smem_u32(bHi + s * B_SLICE)), idesc, s > 0);
#pragma unroll
                for (int s = 0; s < KS; ++s) {
                    umma_f16_ta(acc + N, aHi + 8 * s, umma_desc(smem_u32(bLo + s * B_SLICE)), idesc, s > 0);
                    umma_f16_ta(acc + N, aLo + 8 * s, umma_desc(smem_u32(bHi + s * B_SLICE)), idesc, 1);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&mma_done[b]))
                             : "memory");
            }
            if (i > 0) mbar_wait_own(smem_u32(&mma_done[(i - 1) & 1]), ((i - 1) >> 1) & 1);
        }
    } else {
        // ---------------- drainers: accumulators -> registers -> global ----------------
        const int q = warp & 3;                        // TMEM lane quarter this warp may read
        const int half = (warp - kMmaWarp - 1) >> 2;   // warps 10-13: members 0..H-1; 14-17: H..D-1
        const int row = 32 * q + (tid & 31);
        uint64_t ro = 0;  // address offset of this row within the tile
#pragma unroll
        for (int j = 0; j < 7; ++j)
            if ((row >> j) & 1) ro += g.roff[j];
        double r1 = 0.0, r2 = 0.0;  // fused reduction (g.red)
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
            const int b = i & 1, j = i & 3;
            const bool ok = mbar_wait_abort(smem_u32(&mma_done[b]), (i >> 1) & 1, ab) &&
                            mbar_wait_abort(smem_u32(&scales[j]), (i >> 2) & 1, ab);
            if (!bar_and(2, kDrain, ok)) {  // uniform: tcgen05.ld below needs whole warps
                give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            float2 *const dst = g.psi + insert_zero_bits_g(tile * kRows, g.tpos, 6) + ro;
            const float inv = row_inv[j][row];
            const uint32_t lane_base = tmem + 256 + ((uint32_t)(32 * q) << 16) + half * (N / 2);
            float t1 = 0.f, t2 = 0.f;
#pragma unroll
            for (int c0 = 0; c0 < N / 2; c0 += 16) {
                float a[16], c[16];
                tmem_ld16(lane_base + c0, a);
                tmem_ld16(lane_base + N + c0, c);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (c0 == N / 2 - 16) {
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    mbar_arrive(smem_u32(&tmem_free));
                }
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const float2 v = make_float2((a[2 * m] + c[2 * m]) * inv, (a[2 * m + 1] + c[2 * m + 1]) * inv);
                    const float p = fmaf(v.x, v.x, v.y * v.y);
                    t1 += p;
                    t2 = fmaf(p, p, t2);
                    __stcs(dst + g.moff[H * half + c0 / 2 + m], v);
                }
            }
            r1 += t1;
            r2 += t2;
        }
        if (g.red) drain_partials(r1, r2, tid - (kConv + 64), red_part, g.red);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
}

uint16_t half_bits(float f)
{
    const __half h = __float2half_rn(f);
    uint16_t u;
    std::memcpy(&u, &h, 2);
    return u;
}

float half_value(uint16_t u)
{
    __half h;
    std::memcpy(&h, &u, 2);
    return __half2float(h);
}

uint16_t bf16_bits(float f)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    uint16_t u;
    std::memcpy(&u, &h, 2);
    return u;
}

float bf16_value(uint16_t u)
{
    __nv_bfloat16 h;
    std::memcpy(&h, &u, 2);
    return __bfloat162float(h);
}

// Host: R^T = B[n][k] (n = 2o + po output real, k = 2i + pi input real), split hi/lo in FP16 (or
// BF16), written in the K-major core-matrix layout, KS slices of N x 16.
template <int K, bool BF>
void build_b(const float2 *mat, uint16_t *out)
{
    using L = Tc5Layout<K, 1>;
    constexpr int D = L::D, N = L::N;
    uint16_t *hi = out, *lo = out + L::B_BYTES / 2;
    for (int n = 0; n < N; n++)
        for (int k = 0; k < 2 * D; k++) {
            const int o = n >> 1, po = n & 1, i = k >> 1, pi = k & 1;
            const float2 m = mat[o * D + i];
            const float v = po == 0 ? (pi == 0 ? m.x : -m.y) : (pi == 0 ? m.y : m.x);
            const uint16_t h = BF ? bf16_bits(v) : half_bits(v);
            const uint16_t l = BF ? bf16_bits(v - bf16_value(h)) : half_bits(v - half_value(h));
            const int s = k >> 4, kk = k & 15;
            const size_t off = ((size_t)s * L::B_SLICE + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) / 2;
            hi[off] = h;
            lo[off] = l;
        }
}

// The tile's free address bits F (ascending): the targets and the `rows` lowest other bits.  The
// staging index of an amplitude is its address bits on F, packed: bit i = address bit F[i].
// Returns the length L of F's prefix 0, 1, .., L-1 (the contiguous run), or -1.
template <int K>
int tile_geometry(int nbits, const int *tpos, int rows, Tc5Geom &g)
{
    int is_target[64] = {0}, target_index[64];
    for (int q = 0; q < K; q++) {
        is_target[tpos[q]] = 1;
        target_index[tpos[q]] = q;
    }
    int free_bits[kMaxK + 8], n_free = 0, rank = 0;
    for (int b = 0; b < nbits && n_free < K + rows; b++) {
        if (is_target[b]) {
            free_bits[n_free++] = b;
        } else if (rank < rows) {
            g.roff[rank] = 1ull << b;
            g.ridx[rank++] = 1u << n_free;
            free_bits[n_free++] = b;
        }
    }
    if (n_free != K + rows) return -1;
    int run_log2 = 0;
    while (run_log2 < n_free && free_bits[run_log2] == run_log2) run_log2++;
    const int full_run = run_log2;
    run_log2 = std::min(run_log2, SYCSIM_TC5_RUN_LOG2_MAX);  // longer runs go as several copies
    g.run_log2 = run_log2;
    for (int m = 0; m < (1 << K); m++) {
        g.moff[m] = 0;
        for (int q = 0; q < K; q++)
            if ((m >> q) & 1) g.moff[m] += 1ull << tpos[q];
        uint32_t mi = 0;
        for (int i = 0; i < n_free; i++)
            if (is_target[free_bits[i]] && ((m >> target_index[free_bits[i]]) & 1)) mi |= 1u << i;
        g.midx[m] = mi;
    }
    for (int c = 0; c < (1 << (n_free - run_log2)); c++) {
        uint64_t o = 0;
        for (int i = run_log2; i < n_free; i++)
            if ((c >> (i - run_log2)) & 1) o += 1ull << free_bits[i];
        g.off_run[c] = o;
    }
    return full_run;
}

template <int K, int R2, bool LOWT, bool BF>
int launch_tc5_kr(const Tc5Geom &g, int nbits, cudaStream_t st, int *grid_out)
{
    using L = Tc5Layout<K, R2>;
    auto kern = k_apply_tcgen05<K, R2, LOWT, BF>;
    // one CTA per SM: the stage ring takes most of the SM's shared memory, which also keeps the
    // resident CTAs' tensor memory within the SM's 512 columns (initialised once, thread-safe)
    static std::atomic<uint64_t> smem_done{0};
    if (!smem_opt_in(kern, L::SMEM, smem_done)) return -1;
    static const LaunchCfg cfg = [&] {
        LaunchCfg c;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return c;
        if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return c;
        c.ok = true;
        return c;
    }();
    if (!cfg.ok) return -1;
    Tc5Geom gg = g;
    gg.n_tiles = 1ull << (nbits - K - 7 - (R2 == 2));
    const uint64_t grid = std::min<uint64_t>(gg.n_tiles, (uint64_t)cfg.sms);
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, kThreadsTc5, L::SMEM, st>>>(gg);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <bool LOWT, bool BF>
int launch_tc6a(const Tc5Geom &g, int nbits, cudaStream_t st, int *grid_out)
{
    auto kern = k_apply_tc6a<LOWT, BF>;
    static std::atomic<uint64_t> smem_done{0};
    if (!smem_opt_in(kern, kTc6Smem, smem_done)) return -1;
    static const LaunchCfg cfg = [&] {
        LaunchCfg c;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return c;
        if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return c;
        c.ok = true;
        return c;
    }();
    if (!cfg.ok) return -1;
    Tc5Geom gg = g;
    gg.n_tiles = 1ull << (nbits - 6 - 7);
    const uint64_t grid = std::min<uint64_t>(gg.n_tiles, (uint64_t)cfg.sms);
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, kThreadsTc5, kTc6Smem, st>>>(gg);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Geometry of the block and launch, B (hi, lo) already in device memory at d_b.
template <int K, bool BF>
int launch_tc5_staged(sim_t *h, float2 *psi, int nbits, const int *tpos, const uint32_t *d_b, cudaStream_t st,
                      double *red = nullptr, int *grid_out = nullptr)
{
    Tc5Geom g{};
    g.psi = psi;
    g.red = red;
    for (int i = 0; i < K; i++) g.tpos[i] = tpos[i];  // ascending
    g.bmat = d_b;
    g.err = h->d_errflag;
    g.nlow = 0;
    while (g.nlow < K && tpos[g.nlow] < 4) g.nlow++;
    if (g.nlow > (K >= 5 ? 1 : 0)) return -2;  // not eligible (see tcgen05_eligible)
    if constexpr (K == 6) {  // 128-group tiles only: two 256-column accumulator sets fill the TMEM
        if (tile_geometry<K>(nbits, tpos, 7, g) < 0) return -1;
#if SYCSIM_TC6_ATMEM
        if (g.nlow > 0) return launch_tc6a<true, BF>(g, nbits, st, grid_out);
        return launch_tc6a<false, BF>(g, nbits, st, grid_out);
#else
        if (g.nlow > 0) return launch_tc5_kr<K, 1, true, BF>(g, nbits, st, grid_out);
        return launch_tc5_kr<K, 1, false, BF>(g, nbits, st, grid_out);
#endif
    } else {
        // 128-group tiles when their runs reach 2 KiB (bit 7 is a target, or a target lies below
        // it); otherwise 256-group tiles, whose 8th row bit is bit 7, so that every bulk copy
        // moves at least 2 KiB.  A target below bit 4 always lengthens the run: those blocks take
        // 128 groups.
        const int run = tile_geometry<K>(nbits, tpos, 7, g);
        if (run < 0) return -1;
        if (g.nlow > 0) {
            if constexpr (K == 5) return launch_tc5_kr<K, 1, true, BF>(g, nbits, st, grid_out);
            return -2;
        }
        if (run >= 8 || nbits < K + 8) return launch_tc5_kr<K, 1, false, BF>(g, nbits, st, grid_out);
        if (tile_geometry<K>(nbits, tpos, 8, g) < 8) return -1;
        return launch_tc5_kr<K, 2, false, BF>(g, nbits, st, grid_out);
    }
}

template <int K, bool BF>
int launch_tc5_k(sim_t *h, float2 *psi, int nbits, const int *tpos, const float2 *mat, cudaStream_t st,
                 uint32_t *h_frag, uint32_t *d_frag, cudaEvent_t ev)
{
    using L = Tc5Layout<K, 1>;
    build_b<K, BF>(mat, reinterpret_cast<uint16_t *>(h_frag));
    if (cudaMemcpyAsync(d_frag, h_frag, 2 * L::B_BYTES, cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
    const int rc = launch_tc5_staged<K, BF>(h, psi, nbits, tpos, d_frag, st);
    // the staging slot is free again once this kernel, which reads it, has run (on any stream)
    if (cudaEventRecord(ev, st) != cudaSuccess) return -1;
    return rc;
}

}  // namespace

// At least one 128-group tile, and at most one target below bit 4 (k = 5) or none (k = 4).
// Measured on 2^30 amplitudes: with one such target the per-row member XOR keeps the row reads
// conflict-free and the register stores sector-efficient (16 rows cover 64-128 contiguous
// bytes), as fast as the high-target case for k = 5 (k = 4: 3.27 ms, the mma.sync kernel
// 2.60 ms); with two or more the stores scatter (each row's members fill the low address bits,
// so the lanes of a store instruction hit 2^t lines: up to one L2 request per lane), and
// routing them through the stage instead costs more instructions (register permutations) than
// it saves.  Those blocks run on the mma.sync 3xFP16 kernel.
bool tcgen05_eligible(int nbits, int k, const int *tpos)
{
    if (k < 4 || k > 6 || nbits < k + 7) return false;
    int low = 0;
    for (int q = 0; q < k; q++) low += tpos[q] < 4;
    return low <= (k >= 5 ? 1 : 0);
}

size_t tcgen05_staged_bytes(int k)
{
    switch (k) {
    case 4: return 2 * Tc5Layout<4, 1>::B_BYTES;
    case 5: return 2 * Tc5Layout<5, 1>::B_BYTES;
    case 6: return 2 * Tc5Layout<6, 1>::B_BYTES;
    default: return 0;
    }
}

void tcgen05_build_staged(int k, const float2 *mat, bool bf16, void *h_out)
{
    uint16_t *o = static_cast<uint16_t *>(h_out);
    if (k == 4) bf16 ? build_b<4, true>(mat, o) : build_b<4, false>(mat, o);
    if (k == 5) bf16 ? build_b<5, true>(mat, o) : build_b<5, false>(mat, o);
    if (k == 6) bf16 ? build_b<6, true>(mat, o) : build_b<6, false>(mat, o);
}

int tcgen05_launch_staged(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, bool bf16,
                          const void *d_staged, cudaStream_t st, double *red, int *grid_out)
{
    const uint32_t *d_b = static_cast<const uint32_t *>(d_staged);
    switch (k) {
    case 4: return bf16 ? launch_tc5_staged<4, true>(h, psi, nbits, tpos, d_b, st, red, grid_out)
                        : launch_tc5_staged<4, false>(h, psi, nbits, tpos, d_b, st, red, grid_out);
    case 5: return bf16 ? launch_tc5_staged<5, true>(h, psi, nbits, tpos, d_b, st, red, grid_out)
                        : launch_tc5_staged<5, false>(h, psi, nbits, tpos, d_b, st, red, grid_out);
    case 6: return bf16 ? launch_tc5_staged<6, true>(h, psi, nbits, tpos, d_b, st, red, grid_out)
                        : launch_tc5_staged<6, false>(h, psi, nbits, tpos, d_b, st, red, grid_out);
    default: return -1;
    }
}

int launch_apply_tcgen05(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat, bool bf16,
                         cudaStream_t st)
{
    const int slot = h->frag_next;
    h->frag_next = (slot + 1) % sim_s::kFragSlots;
    if (cudaEventSynchronize(h->frag_ev[slot]) != cudaSuccess) return -1;
    uint32_t *hf = h->h_frag + sim_s::kFragWords * slot;
    uint32_t *df = h->d_frag + sim_s::kFragWords * slot;
    cudaEvent_t ev = h->frag_ev[slot];
    switch (k) {
    case 4: return bf16 ? launch_tc5_k<4, true>(h, psi, nbits, tpos, mat, st, hf, df, ev)
                        : launch_tc5_k<4, false>(h, psi, nbits, tpos, mat, st, hf, df, ev);
    case 5: return bf16 ? launch_tc5_k<5, true>(h, psi, nbits, tpos, mat, st, hf, df, ev)
                        : launch_tc5_k<5, false>(h, psi, nbits, tpos, mat, st, hf, df, ev);
    case 6: return bf16 ? launch_tc5_k<6, true>(h, psi, nbits, tpos, mat, st, hf, df, ev)
                        : launch_tc5_k<6, false>(h, psi, nbits, tpos, mat, st, hf, df, ev);
    default: return -1;
    }
}

}  // namespace sycsim
