// apply_tcgen05.cu -- aggregated k-qubit gate apply on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), 3xFP16 split precision, k = 4 and 5.
//
// Same real-embedded GEMM as apply_tc.cu (W^T = V^T . R^T with R = [[Re M, -Im M],
// [Im M, Re M]]), as one tcgen05.mma M = 128 (groups) x N = 2^(k+1) (output reals) x K = 16
// per step:
//  * thread t of the 128-thread CTA owns row t = one group: it loads the group's 2^k
//    amplitudes, scales them by a power of two (largest component < 2^14, so FP16 keeps them
//    normal), splits hi = fp16(a), lo = fp16(a - hi) and writes both to shared memory in the
//    K-major core-matrix layout (8 rows x 16 bytes per core matrix; 128 B between the two K
//    halves of a 16-wide slice, 256 B between 8-row groups);
//  * K (input reals) is interleaved: column 2m + p is part p (Re, Im) of member m, so a row's
//    16-byte chunk is four consecutive members; N likewise, so a row of the result is the
//    group's outputs (Re, Im) in member order;
//  * one thread issues the MMAs: the main products hi*hi chained through one TMEM accumulator,
//    the corrections hi*lo + lo*hi through a second (their truncation bias is 2^-11 smaller),
//    then commits them to an mbarrier;
//  * while they run, every thread issues the loads of its next tile;
//  * the epilogue reads both accumulators (tcgen05.ld 32x32b: warp w sees TMEM lanes
//    32w..32w+31), adds them in FP32, removes the row's scale and stores the amplitudes.
// R^T (hi, lo; FP16, the same core-matrix layout) is built on the host and staged in shared
// memory once per CTA.  The wait on the mbarrier is bounded; on timeout the kernel records the
// failure in an error word, stops, and still frees its tensor memory.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "internal.h"

namespace sycsim {
namespace {

constexpr int kRows = 128;           // groups per tile = MMA M
constexpr long kWaitLimit = 1L << 26;  // mbarrier polls before giving up (far above any MMA)

struct Tc5Geom {
    float2 *psi;
    uint64_t n_tiles;        // 2^(nbits - k - 7)
    int tpos[kMaxK];
    uint64_t moff[32];
    const uint32_t *bmat;    // R^T hi then lo, FP16 core-matrix layout, as 32-bit words
    int *err;                // set to 1 if an MMA wait timed out
};

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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    for (long it = 0; it < kWaitLimit && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
    return done != 0;
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

// Shared memory: A hi | A lo (KS slices of 4 KiB each) | B hi | B lo (KS slices of N*32 B each).
template <int K>
struct Tc5Layout {
    static constexpr int D = 1 << K;
    static constexpr int KS = 2 * D / 16;       // K slices of 16 reals
    static constexpr int N = 2 * D;             // output reals
    static constexpr int A_SLICE = kRows * 32;  // bytes
    static constexpr int B_SLICE = N * 32;
    static constexpr int A_BYTES = KS * A_SLICE;
    static constexpr int B_BYTES = KS * B_SLICE;
    static constexpr int SMEM = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int TMEM_COLS = 2 * N;     // main + corrections
};

__device__ __forceinline__ uint32_t cm_off(int row, int k) { return (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 + (k & 7) * 2; }

template <int K>
__global__ void __launch_bounds__(kRows) k_apply_tcgen05(Tc5Geom g)
{
    using L = Tc5Layout<K>;
    constexpr int D = L::D, KS = L::KS, N = L::N;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *aHi = sm, *aLo = sm + L::A_BYTES;
    uint8_t *bHi = sm + 2 * L::A_BYTES, *bLo = bHi + L::B_BYTES;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;

    {
        const uint32_t *src = g.bmat;
        uint32_t *dst = reinterpret_cast<uint32_t *>(bHi);
        for (int i = tid; i < (2 * L::B_BYTES) / 4; i += kRows) dst[i] = src[i];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)) : "memory");
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
    const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

    uint64_t tile = blockIdx.x;
    float2 x[D];
    auto load = [&](uint64_t t) {
        const float2 *p = g.psi + insert_zero_bits_g(t * kRows + tid, g.tpos, K);
#pragma unroll
        for (int m = 0; m < D; ++m) x[m] = __ldcs(p + g.moff[m]);
    };
    if (tile < g.n_tiles) load(tile);
    uint32_t parity = 0;
    bool ok = true;
    for (; tile < g.n_tiles && ok; tile += gridDim.x, parity ^= 1) {
        // scale, split and stage this row
        float amax = 0.f;
#pragma unroll
        for (int m = 0; m < D; ++m) amax = fmaxf(amax, fmaxf(fabsf(x[m].x), fabsf(x[m].y)));
        int e = 0;
        frexpf(amax, &e);
        const int sh = amax > 0.f ? max(-100, min(100, 14 - e)) : 0;
        const float sc = ldexpf(1.f, sh), inv = ldexpf(1.f, -sh);
#pragma unroll
        for (int c = 0; c < D / 4; ++c) {  // 16-byte chunk c = members 4c..4c+3 = K columns 8c..8c+7
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float re = x[4 * c + j].x * sc, im = x[4 * c + j].y * sc;
                const __half2 h = __floats2half2_rn(re, im);
                const float2 hf = __half22float2(h);
                const __half2 l = __floats2half2_rn(re - hf.x, im - hf.y);
                hi[j] = *reinterpret_cast<const uint32_t *>(&h);
                lo[j] = *reinterpret_cast<const uint32_t *>(&l);
            }
            const uint32_t off = (c >> 1) * L::A_SLICE + cm_off(tid, 8 * (c & 1));
            *reinterpret_cast<uint4 *>(aHi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(aLo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < KS; ++s)
                umma_f16(tmem, umma_desc(smem_u32(aHi + s * L::A_SLICE)), umma_desc(smem_u32(bHi + s * L::B_SLICE)),
                         idesc, s > 0);
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                umma_f16(tmem + N, umma_desc(smem_u32(aHi + s * L::A_SLICE)),
                         umma_desc(smem_u32(bLo + s * L::B_SLICE)), idesc, s > 0);
                umma_f16(tmem + N, umma_desc(smem_u32(aLo + s * L::A_SLICE)),
                         umma_desc(smem_u32(bHi + s * L::B_SLICE)), idesc, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&mbar))
                         : "memory");
        }
        // this tile's addresses, then the next tile's loads while the MMAs run
        float2 *const dst = g.psi + insert_zero_bits_g(tile * kRows + tid, g.tpos, K);
        const uint64_t next = tile + gridDim.x;
        if (next < g.n_tiles) load(next);
        ok = __syncthreads_and(mbar_wait(smem_u32(&mbar), parity));  // one decision for the CTA
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) {
            if (tid == 0) atomicExch(g.err, 1);
            break;
        }
        const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            float a[16], b[16];
            tmem_ld16(lane_base + c0, a);
            tmem_ld16(lane_base + N + c0, b);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j)
                __stcs(dst + g.moff[c0 / 2 + j],
                       make_float2((a[2 * j] + b[2 * j]) * inv, (a[2 * j + 1] + b[2 * j + 1]) * inv));
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();  // TMEM read and A staging consumed before the next tile reuses them
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(L::TMEM_COLS));
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

// Host: R^T = B[n][k] (n = 2o + po output real, k = 2i + pi input real), split hi/lo in FP16,
// written in the K-major core-matrix layout, KS slices of N x 16.
template <int K>
void build_b(const float2 *mat, uint16_t *out)
{
    using L = Tc5Layout<K>;
    constexpr int D = L::D, N = L::N;
    uint16_t *hi = out, *lo = out + L::B_BYTES / 2;
    for (int n = 0; n < N; n++)
        for (int k = 0; k < 2 * D; k++) {
            const int o = n >> 1, po = n & 1, i = k >> 1, pi = k & 1;
            const float2 m = mat[o * D + i];
            const float v = po == 0 ? (pi == 0 ? m.x : -m.y) : (pi == 0 ? m.y : m.x);
            const uint16_t h = half_bits(v);
            const uint16_t l = half_bits(v - half_value(h));
            const int s = k >> 4, kk = k & 15;
            const size_t off = ((size_t)s * L::B_SLICE + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) / 2;
            hi[off] = h;
            lo[off] = l;
        }
}

template <int K>
int launch_tc5_k(sim_t *h, float2 *psi, int nbits, const int *tpos, const float2 *mat, cudaStream_t st,
                 uint32_t *h_frag, uint32_t *d_frag, cudaEvent_t ev)
{
    using L = Tc5Layout<K>;
    build_b<K>(mat, reinterpret_cast<uint16_t *>(h_frag));
    if (cudaMemcpyAsync(d_frag, h_frag, 2 * L::B_BYTES, cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
    if (cudaEventRecord(ev, st) != cudaSuccess) return -1;
    Tc5Geom g{};
    g.psi = psi;
    g.n_tiles = 1ull << (nbits - K - 7);
    for (int i = 0; i < K; i++) g.tpos[i] = tpos[i];
    for (int j = 0; j < L::D; j++) {
        uint64_t o = 0;
        for (int b = 0; b < K; b++)
            if ((j >> b) & 1) o += 1ull << tpos[b];
        g.moff[j] = o;
    }
    g.bmat = d_frag;
    g.err = h->d_errflag;
    auto kern = k_apply_tcgen05<K>;
    static int occ = 0, sms = 0;
    static size_t smem = 0;
    if (!occ) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return -1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int smem_sm = 0, regs_sm = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        // resident CTAs x TMEM columns must stay within the SM's 512 columns (an allocation
        // beyond that would wait for a CTA that never leaves): size the shared-memory request so
        // that at most 512 / TMEM_COLS CTAs fit on an SM
        const int max_ctas = 512 / L::TMEM_COLS;
        smem = std::max<size_t>(L::SMEM, (size_t)smem_sm / (max_ctas + 1) + 1024);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess) return -1;
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return -1;
        const int regs = ((fa.numRegs + 7) / 8) * 8;  // allocation granularity
        const int by_regs = regs_sm / (regs * kRows);
        const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
        occ = std::max(1, std::min({by_regs, by_smem, max_ctas}));
    }
    const uint64_t grid = std::min<uint64_t>(g.n_tiles, (uint64_t)sms * occ);
    kern<<<(unsigned)grid, kRows, smem, st>>>(g);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

bool tcgen05_eligible(int nbits, int k) { return (k == 4 || k == 5) && nbits >= k + 7; }

int launch_apply_tcgen05(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat,
                         cudaStream_t st)
{
    const int slot = h->frag_next;
    h->frag_next = (slot + 1) % sim_s::kFragSlots;
    if (cudaEventSynchronize(h->frag_ev[slot]) != cudaSuccess) return -1;
    uint32_t *hf = h->h_frag + sim_s::kFragWords * slot;
    uint32_t *df = h->d_frag + sim_s::kFragWords * slot;
    cudaEvent_t ev = h->frag_ev[slot];
    switch (k) {
    case 4: return launch_tc5_k<4>(h, psi, nbits, tpos, mat, st, hf, df, ev);
    case 5: return launch_tc5_k<5>(h, psi, nbits, tpos, mat, st, hf, df, ev);
    default: return -1;
    }
}

}  // namespace sycsim
