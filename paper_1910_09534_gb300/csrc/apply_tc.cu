// apply_tc.cu -- aggregated k-qubit gate apply on tensor cores (k = 4..6).
//
// The block y = M x (M complex 2^k x 2^k) is written over the reals: with x as 2^(k+1) reals,
// R = [[Re M, -Im M], [Im M, Re M]] (interleaved), and for a tile of 16 groups
//     W^T (16 x 2^(k+1)) = V^T (16 x 2^(k+1)) . R^T,
// one warp-level mma.sync m16n8k8 (TF32 in, FP32 accumulate) per 8x8 piece of R^T.
//
// Orderings are chosen so that every thread moves whole complex amplitudes:
//  * K (input reals) in steps of 8 = 4 members: column c < 4 is Re of member 4s + c, column
//    c >= 4 is Im of member 4s + c - 4.  A thread's A fragment (rows g, g+8; columns t, t+4)
//    is then the two complex values member 4s + t of groups g and g + 8: one 8-byte load each.
//  * N (output reals) in tiles of 8 = 4 members: columns 2t, 2t+1 are Re, Im of member 4n + t,
//    so a thread's accumulator pairs are whole output amplitudes: one 8-byte store each.
// The B fragments (R^T, permuted as above, split hi/lo for the 3xTF32 mode) are arranged
// fragment-major on the host and staged once per CTA in shared memory.
//
// Accumulation: chaining many MMAs through one FP32 accumulator was measured to shrink the
// state's norm systematically (the tensor cores' internal accumulation is not round-to-nearest):
// -4e-7 per k = 5 pass.  So each k-step's main product starts from a zero accumulator and is
// added with round-to-nearest FP32 adds, and the small hi*lo + lo*hi corrections (2^-11 of
// the main term) are chained in a second accumulator.  Outputs are produced in chunks of at
// most 4 n-tiles to bound the accumulator registers.
//
// Modes: TF32 (one MMA per piece; TF32 keeps 10 mantissa bits, so ~1e-3 relative error per
// pass) and 3xTF32 (a = a_hi + a_lo with both parts TF32; hi*hi + hi*lo + lo*hi recovers
// ~FP32 accuracy); see also 3xFP16 below.  Used for k >= 5.  A tile's 16 groups are 16
// consecutive group indices; with every target >= bit 4 each member load is a 64-byte run
// per 8 groups, with low targets the runs interleave members instead.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace sycsim {
namespace {

struct MmaGeom {
    float2 *psi;
    uint64_t n_mtiles;      // tiles of 16 groups: 2^(nbits - k - 4)
    int tpos[kMaxK];        // ascending target bits
    uint64_t moff[64];      // offset of member j
    const uint32_t *bfrag;  // [split][kstep][ntile][lane][2] TF32 bit patterns
};

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint64_t insert_zero_bits_t(uint64_t x, const int *pos, int cnt)
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

// Tuning constants (overridable at build time): CTAs per SM each width is compiled for, and
// the n-tiles per output chunk.
#ifndef SYCSIM_MMA_MINB5
#define SYCSIM_MMA_MINB5 3
#endif
#ifndef SYCSIM_MMA_NC
#define SYCSIM_MMA_NC 2
#endif
constexpr int mma_min_blocks(int k) { return k <= 4 ? 2 : (k == 5 ? SYCSIM_MMA_MINB5 : 1); }

template <int K, bool kSplit>
__global__ void __launch_bounds__(256, mma_min_blocks(K)) k_apply_mma(MmaGeom g)
{
    constexpr int D = 1 << K;
    constexpr int KS = D / 4;  // k-steps (4 input members each)
    constexpr int NT = D / 4;  // n-tiles (4 output members each)
    constexpr int NC = NT < SYCSIM_MMA_NC ? NT : SYCSIM_MMA_NC;  // n-tiles per output chunk
    constexpr int NSPLIT = kSplit ? 2 : 1;
    constexpr int FRAG_WORDS = KS * NT * 64;
    extern __shared__ uint32_t sb[];
    for (int i = threadIdx.x; i < NSPLIT * FRAG_WORDS; i += blockDim.x) sb[i] = g.bfrag[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, gid = lane >> 2, t = lane & 3;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t mt = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; mt < g.n_mtiles;
         mt += nw) {
        const uint64_t grp = mt * 16 + gid;
        float2 *p0 = g.psi + insert_zero_bits_t(grp, g.tpos, K);
        float2 *p1 = g.psi + insert_zero_bits_t(grp + 8, g.tpos, K);
        float2 x0[KS], x1[KS];
#pragma unroll
        for (int s = 0; s < KS; ++s) {
            x0[s] = __ldcs(p0 + g.moff[4 * s + t]);
            x1[s] = __ldcs(p1 + g.moff[4 * s + t]);
        }
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += NC) {
            float acc[NC][4], cor[NC][4];
#pragma unroll
            for (int n = 0; n < NC; ++n)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[n][i] = cor[n][i] = 0.f;
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                const float av[4] = {x0[s].x, x1[s].x, x0[s].y, x1[s].y};
                uint32_t ahi[4], alo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ahi[i] = to_tf32(av[i]);
                    if constexpr (kSplit) alo[i] = to_tf32(av[i] - __uint_as_float(ahi[i]));
                }
#pragma unroll
                for (int n = 0; n < NC; ++n) {
                    const int nt = c0 + n;
                    const uint2 bh = *reinterpret_cast<const uint2 *>(sb + ((s * NT + nt) * 32 + lane) * 2);
                    float part[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_tf32(part, ahi, bh.x, bh.y);
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[n][i] += part[i];
                    if constexpr (kSplit) {
                        const uint2 bl = *reinterpret_cast<const uint2 *>(
                            sb + FRAG_WORDS + ((s * NT + nt) * 32 + lane) * 2);
                        mma_tf32(cor[n], ahi, bl.x, bl.y);
                        mma_tf32(cor[n], alo, bh.x, bh.y);
                    }
                }
            }
#pragma unroll
            for (int n = 0; n < NC; ++n) {
                const int nt = c0 + n;
                __stcs(p0 + g.moff[4 * nt + t], make_float2(acc[n][0] + cor[n][0], acc[n][1] + cor[n][1]));
                __stcs(p1 + g.moff[4 * nt + t], make_float2(acc[n][2] + cor[n][2], acc[n][3] + cor[n][3]));
            }
        }
    }
}

// ---- 3xFP16: the same GEMM with m16n8k16 FP16 MMAs (twice the TF32 rate on this GPU) ----
// K steps of 16 reals = 8 members: columns 2t, 2t+1 are (Re, Im) of member 8s + t, columns
// 2t+8, 2t+9 of member 8s + 4 + t, so each A register is one packed half2 amplitude.  The
// state is scaled per warp tile by a power of two so that its largest component sits near
// 2^14 (FP16 keeps it normal), split as hi = fp16(a), lo = fp16(a - hi); the products
// hi*hi + hi*lo + lo*hi are accumulated in FP32 and the scale is removed exactly.
__device__ __forceinline__ void mma_f16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void split_half2(float re, float im, uint32_t &hi, uint32_t &lo)
{
    const __half2 h = __floats2half2_rn(re, im);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(re - hf.x, im - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

template <int K>
__global__ void __launch_bounds__(256, mma_min_blocks(K)) k_apply_mma_f16x3(MmaGeom g)
{
    constexpr int D = 1 << K;
    constexpr int KS = D / 8;  // k-steps (8 input members each)
    constexpr int NT = D / 4;  // n-tiles (4 output members each)
    constexpr int NC = NT < SYCSIM_MMA_NC ? NT : SYCSIM_MMA_NC;
    constexpr int FRAG_WORDS = KS * NT * 64;
    extern __shared__ uint32_t sb[];
    for (int i = threadIdx.x; i < 2 * FRAG_WORDS; i += blockDim.x) sb[i] = g.bfrag[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, gid = lane >> 2, t = lane & 3;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t mt = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; mt < g.n_mtiles;
         mt += nw) {
        const uint64_t grp = mt * 16 + gid;
        float2 *p0 = g.psi + insert_zero_bits_t(grp, g.tpos, K);
        float2 *p1 = g.psi + insert_zero_bits_t(grp + 8, g.tpos, K);
        float2 x0[2 * KS], x1[2 * KS];  // members 8s + t (even index) and 8s + 4 + t (odd index)
#pragma unroll
        for (int s = 0; s < KS; ++s) {
            x0[2 * s] = __ldcs(p0 + g.moff[8 * s + t]);
            x0[2 * s + 1] = __ldcs(p0 + g.moff[8 * s + 4 + t]);
            x1[2 * s] = __ldcs(p1 + g.moff[8 * s + t]);
            x1[2 * s + 1] = __ldcs(p1 + g.moff[8 * s + 4 + t]);
        }
        float amax = 0.f;
#pragma unroll
        for (int i = 0; i < 2 * KS; ++i)
            amax = fmaxf(amax, fmaxf(fmaxf(fabsf(x0[i].x), fabsf(x0[i].y)), fmaxf(fabsf(x1[i].x), fabsf(x1[i].y))));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        int e = 0;
        frexpf(amax, &e);                       // amax < 2^e
        const int sh = amax > 0.f ? max(-100, min(100, 14 - e)) : 0;  // largest component < 2^14
        const float sc = ldexpf(1.f, sh), inv = ldexpf(1.f, -sh);
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += NC) {
            float acc[NC][4], cor[NC][4];
#pragma unroll
            for (int n = 0; n < NC; ++n)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[n][i] = cor[n][i] = 0.f;
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                uint32_t ahi[4], alo[4];
                split_half2(x0[2 * s].x * sc, x0[2 * s].y * sc, ahi[0], alo[0]);
                split_half2(x1[2 * s].x * sc, x1[2 * s].y * sc, ahi[1], alo[1]);
                split_half2(x0[2 * s + 1].x * sc, x0[2 * s + 1].y * sc, ahi[2], alo[2]);
                split_half2(x1[2 * s + 1].x * sc, x1[2 * s + 1].y * sc, ahi[3], alo[3]);
#pragma unroll
                for (int n = 0; n < NC; ++n) {
                    const int nt = c0 + n;
                    const uint2 bh = *reinterpret_cast<const uint2 *>(sb + ((s * NT + nt) * 32 + lane) * 2);
                    const uint2 bl =
                        *reinterpret_cast<const uint2 *>(sb + FRAG_WORDS + ((s * NT + nt) * 32 + lane) * 2);
                    float part[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_f16(part, ahi, bh.x, bh.y);
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[n][i] += part[i];
                    mma_f16(cor[n], ahi, bl.x, bl.y);
                    mma_f16(cor[n], alo, bh.x, bh.y);
                }
            }
#pragma unroll
            for (int n = 0; n < NC; ++n) {
                const int nt = c0 + n;
                __stcs(p0 + g.moff[4 * nt + t],
                       make_float2((acc[n][0] + cor[n][0]) * inv, (acc[n][1] + cor[n][1]) * inv));
                __stcs(p1 + g.moff[4 * nt + t],
                       make_float2((acc[n][2] + cor[n][2]) * inv, (acc[n][3] + cor[n][3]) * inv));
            }
        }
    }
}

uint32_t pack_half2(float lo, float hi)
{
    const __half a = __float2half_rn(lo), b = __float2half_rn(hi);
    uint16_t ua, ub;
    std::memcpy(&ua, &a, 2);
    std::memcpy(&ub, &b, 2);
    return (uint32_t)ua | ((uint32_t)ub << 16);
}

template <int K>
constexpr size_t f16x3_bytes() { return sizeof(uint32_t) * 2 * ((1 << K) / 8) * ((1 << K) / 4) * 64; }

// Host: the B fragments (hi, lo) of one block, as the kernel reads them.
template <int K>
void build_f16x3(const float2 *mat, uint32_t *h_frag)
{
    constexpr int D = 1 << K, KS = D / 8, NT = D / 4;
    constexpr int FRAG_WORDS = KS * NT * 64;
    // B fragment (k rows 2t, 2t+1 | 2t+8, 2t+9; n column gid) as half2 (Re-input, Im-input)
    // of input member 8s + t (b0) and 8s + 4 + t (b1) for output member 4n + gid/2.
    for (int s = 0; s < KS; s++)
        for (int n = 0; n < NT; n++)
            for (int lane = 0; lane < 32; lane++) {
                const int gid = lane >> 2, t = lane & 3;
                const int o = 4 * n + (gid >> 1);
                const bool out_im = gid & 1;
                const size_t idx = ((size_t)(s * NT + n) * 32 + lane) * 2;
                for (int j = 0; j < 2; j++) {
                    const float2 m = mat[o * D + 8 * s + 4 * j + t];
                    const float re_in = out_im ? m.y : m.x;   // coefficient of Re x
                    const float im_in = out_im ? m.x : -m.y;  // coefficient of Im x
                    const uint32_t hi = pack_half2(re_in, im_in);
                    __half hr, hm;
                    const uint16_t lo16 = (uint16_t)(hi & 0xffffu), hi16 = (uint16_t)(hi >> 16);
                    std::memcpy(&hr, &lo16, 2);
                    std::memcpy(&hm, &hi16, 2);
                    h_frag[idx + j] = hi;
                    h_frag[FRAG_WORDS + idx + j] =
                        pack_half2(re_in - __half2float(hr), im_in - __half2float(hm));
                }
            }
}

// Launch with the fragments already in device memory.
template <int K>
int launch_f16x3_staged(float2 *psi, int nbits, const int *tpos, const uint32_t *d_frag, cudaStream_t st)
{
    constexpr int D = 1 << K;
    constexpr size_t bytes = f16x3_bytes<K>();
    MmaGeom g{};
    g.psi = psi;
    g.n_mtiles = 1ull << (nbits - K - 4);
    for (int i = 0; i < K; i++) g.tpos[i] = tpos[i];
    for (int j = 0; j < D; j++) {
        uint64_t o = 0;
        for (int b = 0; b < K; b++)
            if ((j >> b) & 1) o += 1ull << tpos[b];
        g.moff[j] = o;
    }
    g.bfrag = d_frag;
    auto kern = k_apply_mma_f16x3<K>;
    static std::atomic<uint64_t> smem_done{0};
    if (bytes > 48 * 1024 && !smem_opt_in(kern, (int)bytes, smem_done)) return -1;
    static const LaunchCfg cfg = [&] {  // once per instantiation, thread-safe
        LaunchCfg c;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return c;
        if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return c;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ, kern, 256, bytes) != cudaSuccess || c.occ < 1)
            c.occ = 1;
        c.ok = true;
        return c;
    }();
    if (!cfg.ok) return -1;
    const uint64_t need = (g.n_mtiles + 7) / 8;
    const uint64_t grid = std::min<uint64_t>(need, (uint64_t)cfg.sms * cfg.occ);
    kern<<<(unsigned)grid, 256, bytes, st>>>(g);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int K>
int launch_f16x3_k(float2 *psi, int nbits, const int *tpos, const float2 *mat, cudaStream_t st,
                   uint32_t *h_frag, uint32_t *d_frag, cudaEvent_t ev)
{
    build_f16x3<K>(mat, h_frag);
    if (cudaMemcpyAsync(d_frag, h_frag, f16x3_bytes<K>(), cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
    const int rc = launch_f16x3_staged<K>(psi, nbits, tpos, d_frag, st);
    // the staging slot is free again once this kernel, which reads it, has run (on any stream)
    if (cudaEventRecord(ev, st) != cudaSuccess) return -1;
    return rc;
}

// Round an FP32 value to TF32 (nearest, ties away from zero, as cvt.rna), host side.
uint32_t host_tf32(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u & 0xffffe000u;  // inf/nan: truncate
    u += 0x1000u;                                                   // half of the dropped 13 bits
    return u & 0xffffe000u;
}

float tf32_value(uint32_t u)
{
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

template <int K, bool kSplit>
constexpr size_t mma_bytes() { return sizeof(uint32_t) * (kSplit ? 2 : 1) * ((1 << K) / 4) * ((1 << K) / 4) * 64; }

// Host: the B fragments (TF32; with the split, hi then lo) of one block.
template <int K, bool kSplit>
void build_mma(const float2 *mat, uint32_t *h_frag)
{
    constexpr int D = 1 << K, KS = D / 4, NT = D / 4;
    constexpr int FRAG_WORDS = KS * NT * 64;
    // B[k][n] = R^T, permuted: k = (step s, column c): member 4s + (c & 3), Re for c < 4, Im for
    // c >= 4; n = (tile m, column c'): member 4m + c'/2, Re for even c', Im for odd c'.
    for (int s = 0; s < KS; s++)
        for (int n = 0; n < NT; n++)
            for (int lane = 0; lane < 32; lane++) {
                const int gid = lane >> 2, t = lane & 3;
                const int i = 4 * s + t;            // input member (b0: Re part, b1: Im part)
                const int o = 4 * n + (gid >> 1);   // output member
                const bool out_im = gid & 1;
                const float2 m = mat[o * D + i];
                const float b0 = out_im ? m.y : m.x;   // Re x -> (Re y: Mr, Im y: Mi)
                const float b1 = out_im ? m.x : -m.y;  // Im x -> (Re y: -Mi, Im y: Mr)
                const size_t idx = ((size_t)(s * NT + n) * 32 + lane) * 2;
                const uint32_t h0 = host_tf32(b0), h1 = host_tf32(b1);
                h_frag[idx] = h0;
                h_frag[idx + 1] = h1;
                if (kSplit) {
                    h_frag[FRAG_WORDS + idx] = host_tf32(b0 - tf32_value(h0));
                    h_frag[FRAG_WORDS + idx + 1] = host_tf32(b1 - tf32_value(h1));
                }
            }
}

template <int K, bool kSplit>
int launch_mma_staged(float2 *psi, int nbits, const int *tpos, const uint32_t *d_frag, cudaStream_t st)
{
    constexpr int D = 1 << K;
    constexpr size_t bytes = mma_bytes<K, kSplit>();
    MmaGeom g{};
    g.psi = psi;
    g.n_mtiles = 1ull << (nbits - K - 4);
    for (int i = 0; i < K; i++) g.tpos[i] = tpos[i];
    for (int j = 0; j < D; j++) {
        uint64_t o = 0;
        for (int b = 0; b < K; b++)
            if ((j >> b) & 1) o += 1ull << tpos[b];
        g.moff[j] = o;
    }
    g.bfrag = d_frag;
    auto kern = k_apply_mma<K, kSplit>;
    static std::atomic<uint64_t> smem_done{0};
    if (bytes > 48 * 1024 && !smem_opt_in(kern, (int)bytes, smem_done)) return -1;
    static const LaunchCfg cfg = [&] {  // once per instantiation, thread-safe
        LaunchCfg c;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return c;
        if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return c;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ, kern, 256, bytes) != cudaSuccess || c.occ < 1)
            c.occ = 1;
        c.ok = true;
        return c;
    }();
    if (!cfg.ok) return -1;
    const uint64_t need = (g.n_mtiles + 7) / 8;
    const uint64_t grid = std::min<uint64_t>(need, (uint64_t)cfg.sms * cfg.occ);
    kern<<<(unsigned)grid, 256, bytes, st>>>(g);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int K, bool kSplit>
int launch_mma_k(float2 *psi, int nbits, const int *tpos, const float2 *mat, cudaStream_t st,
                 uint32_t *h_frag, uint32_t *d_frag, cudaEvent_t ev)
{
    build_mma<K, kSplit>(mat, h_frag);
    if (cudaMemcpyAsync(d_frag, h_frag, mma_bytes<K, kSplit>(), cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
    const int rc = launch_mma_staged<K, kSplit>(psi, nbits, tpos, d_frag, st);
    // the staging slot is free again once this kernel, which reads it, has run (on any stream)
    if (cudaEventRecord(ev, st) != cudaSuccess) return -1;
    return rc;
}

}  // namespace

// Measured on GB300 (n = 30): for k = 4 the CUDA-core FP32 kernel is faster than every
// tensor-core mode (2.8 ms vs >= 3.6 ms per pass), for k >= 5 the tensor cores win (3xFP16 k = 5:
// 3.3 ms vs 7.0 ms).  Any target set works: groups map to amplitude offsets by bit insertion.
bool tc_eligible(int nbits, int k, const int *) { return k >= 5 && k <= 6 && nbits >= k + 4; }

// In SIM_FP16X3_TMEM mode the blocks the tcgen05 kernel leaves (targets in the low bits) come
// here for k = 4 too: measured on 2^30 amplitudes, targets {0,1,2,3}: 2.73 ms (CUDA-core FP32
// 4.27 ms), {0,2,6,8}: 2.59 ms (3.57), {1,6,7,12}: 2.60 ms (3.24).
bool tc_eligible_low4(int nbits, int k) { return k == 4 && nbits >= k + 4; }

size_t tc_staged_bytes(int k, int precision)
{
    const bool f16 = f16x3_mode(precision), split = precision == SIM_TF32X3;
    switch (k) {
    case 4: return f16 ? f16x3_bytes<4>() : (split ? mma_bytes<4, true>() : mma_bytes<4, false>());
    case 5: return f16 ? f16x3_bytes<5>() : (split ? mma_bytes<5, true>() : mma_bytes<5, false>());
    case 6: return f16 ? f16x3_bytes<6>() : (split ? mma_bytes<6, true>() : mma_bytes<6, false>());
    default: return 0;
    }
}

void tc_build_staged(int k, const float2 *mat, int precision, void *h_out)
{
    uint32_t *o = static_cast<uint32_t *>(h_out);
    const bool f16 = f16x3_mode(precision), split = precision == SIM_TF32X3;
    switch (k) {
    case 4: f16 ? build_f16x3<4>(mat, o) : (split ? build_mma<4, true>(mat, o) : build_mma<4, false>(mat, o)); break;
    case 5: f16 ? build_f16x3<5>(mat, o) : (split ? build_mma<5, true>(mat, o) : build_mma<5, false>(mat, o)); break;
    case 6: f16 ? build_f16x3<6>(mat, o) : (split ? build_mma<6, true>(mat, o) : build_mma<6, false>(mat, o)); break;
    default: break;
    }
}

int tc_launch_staged(float2 *psi, int nbits, int k, const int *tpos, int precision, const void *d_staged,
                     cudaStream_t st)
{
    const uint32_t *d = static_cast<const uint32_t *>(d_staged);
    const bool f16 = f16x3_mode(precision), split = precision == SIM_TF32X3;
    switch (k) {
    case 4: return f16 ? launch_f16x3_staged<4>(psi, nbits, tpos, d, st)
                       : (split ? launch_mma_staged<4, true>(psi, nbits, tpos, d, st)
                                : launch_mma_staged<4, false>(psi, nbits, tpos, d, st));
    case 5: return f16 ? launch_f16x3_staged<5>(psi, nbits, tpos, d, st)
                       : (split ? launch_mma_staged<5, true>(psi, nbits, tpos, d, st)
                                : launch_mma_staged<5, false>(psi, nbits, tpos, d, st));
    case 6: return f16 ? launch_f16x3_staged<6>(psi, nbits, tpos, d, st)
                       : (split ? launch_mma_staged<6, true>(psi, nbits, tpos, d, st)
                                : launch_mma_staged<6, false>(psi, nbits, tpos, d, st));
    default: return -1;
    }
}

int launch_apply_tc(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat,
                    int precision, cudaStream_t st)
{
    const int slot = h->frag_next;
    h->frag_next = (slot + 1) % sim_s::kFragSlots;
    if (cudaEventSynchronize(h->frag_ev[slot]) != cudaSuccess) return -1;  // host staging free
    uint32_t *hf = h->h_frag + sim_s::kFragWords * slot;
    uint32_t *df = h->d_frag + sim_s::kFragWords * slot;
    cudaEvent_t ev = h->frag_ev[slot];
    if (f16x3_mode(precision)) {
        switch (k) {
        case 4: return launch_f16x3_k<4>(psi, nbits, tpos, mat, st, hf, df, ev);
        case 5: return launch_f16x3_k<5>(psi, nbits, tpos, mat, st, hf, df, ev);
        case 6: return launch_f16x3_k<6>(psi, nbits, tpos, mat, st, hf, df, ev);
        default: return -1;
        }
    }
    const bool split = precision == SIM_TF32X3;
    switch (k) {
    case 4: return split ? launch_mma_k<4, true>(psi, nbits, tpos, mat, st, hf, df, ev)
                         : launch_mma_k<4, false>(psi, nbits, tpos, mat, st, hf, df, ev);
    case 5: return split ? launch_mma_k<5, true>(psi, nbits, tpos, mat, st, hf, df, ev)
                         : launch_mma_k<5, false>(psi, nbits, tpos, mat, st, hf, df, ev);
    case 6: return split ? launch_mma_k<6, true>(psi, nbits, tpos, mat, st, hf, df, ev)
                         : launch_mma_k<6, false>(psi, nbits, tpos, mat, st, hf, df, ev);
    default: return -1;
    }
}

}  // namespace sycsim
