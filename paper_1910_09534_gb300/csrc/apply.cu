// apply.cu -- aggregated k-qubit gate apply on CUDA cores, FP32 (Sect. 5: gates are
// aggregated into k-qubit kernels, each a 2^k x 2^k unitary applied to the state).
//
// For targets t_0 < ... < t_{k-1} (physical bits), a "group" is the 2^k amplitudes that
// share every non-target bit; member j of a group sits at base + sum_b bit_b(j) 2^{t_b}.
// Each group is replaced by M times itself.  One pass reads and writes every amplitude
// once: 16 bytes per amplitude of HBM traffic, 8 * 2^k - 2 real flops per amplitude.
//
// Three kernels:
//  * reg (default for k <= 5, n >= k + 5) -- see the comment above k_apply_reg: persistent
//    warps, register-resident groups, warp-shuffle exchange for targets below bit 5.
//  * direct -- every target >= 5: thread = group; the 32 threads of a warp take 32
//    consecutive groups, so each member load/store is one contiguous 256-byte run.
//    Amplitudes go straight to registers; no shared memory.  Used for k <= 3.
//  * tiled -- small states and k = 6: a CTA stages a tile of 2^(F+k) amplitudes (2^h rows of
//    2^m contiguous amplitudes, the rows indexed by the h targets >= m) through shared
//    memory with coalesced loads, each of its 2^F threads applies M to one group, and
//    the tile is written back.  An XOR swizzle maps the low target bits onto free bits
//    so that shared-memory accesses stay conflict-free for any target set.
//
// The matrix (FP32, complex64) is a kernel parameter for k <= 5: the FMAs read it
// straight from the constant bank.  k = 6 (32 KiB) exceeds the parameter space and is
// read from device memory into shared memory once per CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "internal.h"

namespace sycsim {
namespace {

template <int K>
struct MatP {
    float2 m[(1 << K) * (1 << K)];
};

struct MatPtr {
    const float2 *p;
};

struct DirectGeom {
    float2 *psi;
    uint64_t n_groups;
    int tpos[kMaxK];     // ascending physical target bits
    uint64_t moff[64];   // offset of member j
};

struct TiledGeom {
    float2 *psi;
    int F;               // log2(threads per CTA) = log2(groups per tile)
    int m;               // log2(row length) = F + nlow
    int nlow, nhigh;     // targets below / at-or-above m
    int ltpos[kMaxK];    // low target bits (ascending, < m)
    int hpos[kMaxK];     // high target bits (ascending, >= m)
    int nsw;             // swizzle pairs: bit sw_src[i] of a tile position is XORed into bit sw_dst[i]
    int sw_src[4], sw_dst[4];
    uint32_t soff[64];   // tile-local offset of member j
    uint64_t rowoff[64]; // global offset of tile row r
};

__device__ __forceinline__ uint64_t insert_zero_bits(uint64_t x, const int *pos, int cnt)
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

// 8-byte asynchronous global -> shared copy (no register staging) and its completion wait.
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Opaque copies: stop the compiler from keeping load-phase addresses alive through the
// compute phase (it would otherwise reuse them for the stores and spill).
__device__ __forceinline__ float2 *opaque(float2 *p)
{
    float2 *q;
    asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p));
    return q;
}

__device__ __forceinline__ uint32_t opaque_tid()
{
    uint32_t t;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
    return t;
}

__device__ __forceinline__ uint32_t swizzle(uint32_t p, const TiledGeom &g)
{
    uint32_t x = p;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (i < g.nsw) x ^= ((p >> g.sw_src[i]) & 1u) << g.sw_dst[i];
    return x;
}

// y = M x for one group; rows are produced RB at a time (RB independent FMA chains per
// real/imag part) and handed to `st(row, value)`.
template <int K, bool kUnrollRows, typename MatAt, typename Store>
__device__ __forceinline__ void apply_group(const float2 (&x)[1 << K], MatAt M, Store st)
{
    constexpr int D = 1 << K;
    constexpr int RB = D >= 4 ? 4 : D;
#pragma unroll(kUnrollRows ? D / RB : 1)
    for (int r0 = 0; r0 < D; r0 += RB) {
        float yr[RB], yi[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) yr[b] = yi[b] = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                const float2 mm = M(r0 + b, c);
                yr[b] = fmaf(mm.x, x[c].x, yr[b]);
                yr[b] = fmaf(mm.y, -x[c].y, yr[b]);
                yi[b] = fmaf(mm.x, x[c].y, yi[b]);
                yi[b] = fmaf(mm.y, x[c].x, yi[b]);
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) st(r0 + b, make_float2(yr[b], yi[b]));
    }
}

// Copy a 2^K x 2^K matrix from global memory to shared memory (all threads).
template <int K>
__device__ __forceinline__ void stage_matrix(float2 *sm, const float2 *gm)
{
    constexpr int N = (1 << K) * (1 << K);
    for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = gm[i];
    __syncthreads();
}

// Occupancy targets (CTAs per SM) that bound the register count of each width.
constexpr int direct_min_blocks(int k) { return k <= 3 ? 4 : (k <= 5 ? 2 : 1); }
constexpr int tiled_threads(int k) { return k <= 4 ? 256 : (k == 5 ? 128 : 64); }
constexpr int tiled_min_blocks(int k) { return k <= 3 ? 4 : (k <= 5 ? 2 : 4); }

template <int K, typename MatSrc>
__global__ void __launch_bounds__(256, direct_min_blocks(K)) k_apply_direct(DirectGeom g, MatSrc M)
{
    constexpr int D = 1 << K;
    constexpr bool kSmemMat = std::is_same<MatSrc, MatPtr>::value;
    extern __shared__ float2 smem[];
    if constexpr (kSmemMat) stage_matrix<K>(smem, M.p);
    const uint64_t gi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= g.n_groups) return;
    float2 *p = g.psi + insert_zero_bits(gi, g.tpos, K);
    float2 x[D];
#pragma unroll
    for (int j = 0; j < D; ++j) x[j] = __ldcs(p + g.moff[j]);
    float2 *const q = opaque(p);
    auto st = [&](int r, float2 y) { __stcs(q + g.moff[r], y); };
    if constexpr (kSmemMat)
        apply_group<K, false>(x, [&](int r, int c) { return smem[r * D + c]; }, st);
    else
        apply_group<K, true>(x, [&](int r, int c) { return M.m[r * D + c]; }, st);
}

template <int K, typename MatSrc>
__global__ void __launch_bounds__(tiled_threads(K), tiled_min_blocks(K)) k_apply_tiled(TiledGeom g, MatSrc M)
{
    constexpr int D = 1 << K;
    constexpr bool kSmemMat = std::is_same<MatSrc, MatPtr>::value;
    extern __shared__ float2 smem[];
    float2 *tile = smem;
    float2 *msm = smem + ((size_t)D << g.F);
    if constexpr (kSmemMat) stage_matrix<K>(msm, M.p);

    const uint32_t tid = threadIdx.x;
    const int F = g.F;
    const uint32_t lowmask = (1u << g.nlow) - 1;
    const uint64_t base = insert_zero_bits((uint64_t)blockIdx.x << g.m, g.hpos, g.nhigh);
    float2 *gp = g.psi + base;

    // load: linear tile position p = tid + c 2^F; row r = c >> nlow, column ((c & lowmask) << F) | tid
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const uint32_t p = tid + ((uint32_t)c << F);
        const uint32_t col = ((c & lowmask) << F) | tid;
        cp_async8(&tile[swizzle(p, g)], gp + g.rowoff[c >> g.nlow] + col);
    }
    cp_async_wait_all();
    __syncthreads();

    // compute: thread tid owns group tid
    const uint32_t bg = (uint32_t)insert_zero_bits(tid, g.ltpos, g.nlow);
    const uint32_t sb = swizzle(bg, g);
    float2 x[D];
#pragma unroll
    for (int j = 0; j < D; ++j) x[j] = tile[sb ^ g.soff[j]];
    auto st = [&](int r, float2 y) { tile[sb ^ g.soff[r]] = y; };
    if constexpr (kSmemMat)
        apply_group<K, false>(x, [&](int r, int c) { return msm[r * D + c]; }, st);
    else
        apply_group<K, true>(x, [&](int r, int c) { return M.m[r * D + c]; }, st);
    __syncthreads();

    // store
    const uint32_t tid2 = opaque_tid();
    float2 *const gq = opaque(gp);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const uint32_t p = tid2 + ((uint32_t)c << F);
        const uint32_t col = ((c & lowmask) << F) | tid2;
        __stcs(gq + g.rowoff[c >> g.nlow] + col, tile[swizzle(p, g)]);
    }
}

// Threads per CTA (log2) of the tiled kernel for width k.
int tiled_F(int k) { return k <= 4 ? 8 : (k == 5 ? 7 : 6); }
static_assert(tiled_threads(4) == 256 && tiled_threads(5) == 128 && tiled_threads(6) == 64, "F");

template <typename Kern>
cudaError_t ensure_smem(Kern kern, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int K, typename MatSrc>
int launch_k(float2 *psi, int nbits, const int *tpos, const MatSrc &M, cudaStream_t st)
{
    constexpr int D = 1 << K;
    constexpr bool kSmemMat = std::is_same<MatSrc, MatPtr>::value;
    const size_t mat_bytes = kSmemMat ? sizeof(float2) * D * D : 0;
    const bool direct = tpos[0] >= 5 && nbits - K >= 8;
    if (direct) {
        DirectGeom g{};
        g.psi = psi;
        g.n_groups = 1ull << (nbits - K);
        for (int i = 0; i < K; i++) g.tpos[i] = tpos[i];
        for (int j = 0; j < D; j++) {
            uint64_t o = 0;
            for (int b = 0; b < K; b++)
                if ((j >> b) & 1) o += 1ull << tpos[b];
            g.moff[j] = o;
        }
        const uint64_t blocks = (g.n_groups + 255) / 256;
        auto kern = k_apply_direct<K, MatSrc>;
        if (ensure_smem(kern, mat_bytes) != cudaSuccess) return -1;
        kern<<<(unsigned)blocks, 256, mat_bytes, st>>>(g, M);
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }

    TiledGeom g{};
    g.psi = psi;
    g.F = std::min(tiled_F(K), nbits - K);
    int m = g.F;
    for (;;) {  // m = F + #(targets below m)
        int below = 0;
        for (int i = 0; i < K; i++) below += tpos[i] < m;
        if (g.F + below == m) break;
        m = g.F + below;
    }
    g.m = m;
    g.nlow = g.nhigh = 0;
    for (int i = 0; i < K; i++) {
        if (tpos[i] < m)
            g.ltpos[g.nlow++] = tpos[i];
        else
            g.hpos[g.nhigh++] = tpos[i];
    }
    // swizzle: the free (non-target) tile bits f0 < f1 < ... ; the first four of them at or
    // above bit 4 are XORed into the target bits below 4, in order.
    {
        int dsts[4], nd = 0, srcs[4], ns = 0;
        for (int i = 0; i < g.nlow; i++)
            if (g.ltpos[i] < 4) dsts[nd++] = g.ltpos[i];
        int free_seen = 0;
        for (int b = 0; b < m && free_seen < 4; b++) {
            bool is_t = false;
            for (int i = 0; i < g.nlow; i++) is_t |= g.ltpos[i] == b;
            if (is_t) continue;
            if (b >= 4 && ns < nd) srcs[ns++] = b;
            free_seen++;
        }
        g.nsw = std::min(nd, ns);
        for (int i = 0; i < g.nsw; i++) {
            g.sw_src[i] = srcs[i];
            g.sw_dst[i] = dsts[i];
        }
    }
    for (int j = 0; j < D; j++) {
        uint32_t o = 0;
        for (int b = 0; b < g.nlow; b++)
            if ((j >> b) & 1) o |= 1u << g.ltpos[b];
        o |= (uint32_t)(j >> g.nlow) << m;
        g.soff[j] = o;
    }
    for (int r = 0; r < (1 << g.nhigh); r++) {
        uint64_t o = 0;
        for (int b = 0; b < g.nhigh; b++)
            if ((r >> b) & 1) o += 1ull << g.hpos[b];
        g.rowoff[r] = o;
    }
    const uint64_t tiles = 1ull << (nbits - g.F - K);
    const size_t smem = (sizeof(float2) << (g.F + K)) + mat_bytes;
    auto kern = k_apply_tiled<K, MatSrc>;
    if (ensure_smem(kern, smem) != cudaSuccess) return -1;
    kern<<<(unsigned)tiles, 1u << g.F, smem, st>>>(g, M);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------------------
// Register-resident apply for k <= 5 (the default path when n >= k + 5).
//
// A warp owns a "warp tile": 32 lanes (index bits 0..4) x 2^k registers.  Register bit
// j < J (J = number of targets below bit 5) first stands for a free index bit E_j >= 5,
// register bits j >= J for the high targets.  Loads and stores are therefore 256-byte runs
// per register.  Each low target t_j (a lane bit) is then exchanged with register bit j by
// warp shuffles, after which every lane holds one complete group in registers and applies M
// with the matrix read from the constant bank; the same exchanges undo the transpose before
// the stores.  Warps are persistent.  (Double-buffering the next tile in registers was
// measured slower than simply running more CTAs per SM, so it is off by default.)
// ---------------------------------------------------------------------------------------
struct RegGeom {
    float2 *psi;
    uint64_t n_wtiles;  // 2^(n - 5 - k)
    int J;              // targets below bit 5
    int lt[5];          // their bit positions (lane bits), ascending
    int nfix;           // index bits >= 5 owned by registers (high targets + E), ascending
    int fix[kMaxK];
    uint64_t xoff[32];  // offset of register x (pre-exchange meaning)
};

template <int K>
__device__ __forceinline__ void lane_reg_exchange(float2 (&v)[1 << K], const RegGeom &g, int lane)
{
#pragma unroll
    for (int b = 0; b < (K < 5 ? K : 5); ++b) {
        if (b < g.J) {
            const int t = g.lt[b];
            const bool s = (lane >> t) & 1;
#pragma unroll
            for (int x = 0; x < (1 << K); ++x) {
                if (x & (1 << b)) continue;
                const int x1 = x | (1 << b);
                const float2 send = s ? v[x] : v[x1];
                float2 r;
                r.x = __shfl_xor_sync(0xffffffffu, send.x, 1 << t);
                r.y = __shfl_xor_sync(0xffffffffu, send.y, 1 << t);
                v[x] = s ? r : v[x];
                v[x1] = s ? v[x1] : r;
            }
        }
    }
}

// Tuning constants (overridable at build time): widest k that double-buffers the next tile
// in registers, and the CTAs per SM each width is compiled for.
#ifndef SYCSIM_REG_PREFETCH_KMAX
#define SYCSIM_REG_PREFETCH_KMAX 0
#endif
#ifndef SYCSIM_REG_MINB_K3
#define SYCSIM_REG_MINB_K3 4
#endif
#ifndef SYCSIM_REG_MINB_K4
#define SYCSIM_REG_MINB_K4 3
#endif
#ifndef SYCSIM_REG_MINB_K5
#define SYCSIM_REG_MINB_K5 1
#endif
constexpr bool reg_prefetch(int k) { return k <= SYCSIM_REG_PREFETCH_KMAX; }
constexpr int reg_min_blocks(int k, bool low)
{
    return k <= 2 ? 4
                  : (k == 3 ? SYCSIM_REG_MINB_K3
                            : (k == 4 ? SYCSIM_REG_MINB_K4 : (low ? SYCSIM_REG_MINB_K5 : 2)));
}

template <int K, bool kLow>
__global__ void __launch_bounds__(256, reg_min_blocks(K, kLow)) k_apply_reg(RegGeom g, MatP<K> M)
{
    constexpr int D = 1 << K;
    constexpr bool kPrefetch = reg_prefetch(K);
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= g.n_wtiles) return;
    auto tile_ptr = [&](uint64_t wt) {
        return g.psi + insert_zero_bits(wt << 5, g.fix, g.nfix) + lane;
    };
    auto MatAt = [&](int r, int c) { return M.m[r * D + c]; };
    float2 x[D];
    {
        const float2 *p = tile_ptr(w);
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = __ldcs(p + g.xoff[j]);
    }
    for (; w < g.n_wtiles; w += nw) {
        const uint64_t wn = w + nw;
        float2 xn[D];
        if constexpr (kPrefetch) {
            if (wn < g.n_wtiles) {
                const float2 *pn = tile_ptr(wn);
#pragma unroll
                for (int j = 0; j < D; ++j) xn[j] = __ldcs(pn + g.xoff[j]);
            }
        }
        float2 *const q = opaque(tile_ptr(w));
        if constexpr (kLow) {
            lane_reg_exchange<K>(x, g, lane);
            float2 y[D];
            apply_group<K, true>(x, MatAt, [&](int r, float2 v) { y[r] = v; });
            lane_reg_exchange<K>(y, g, lane);
#pragma unroll
            for (int j = 0; j < D; ++j) __stcs(q + g.xoff[j], y[j]);
        } else {
            apply_group<K, true>(x, MatAt, [&](int r, float2 v) { __stcs(q + g.xoff[r], v); });
        }
        if constexpr (kPrefetch) {
#pragma unroll
            for (int j = 0; j < D; ++j) x[j] = xn[j];
        } else if (wn < g.n_wtiles) {
            const float2 *pn = tile_ptr(wn);
#pragma unroll
            for (int j = 0; j < D; ++j) x[j] = __ldcs(pn + g.xoff[j]);
        }
    }
}

template <int K, bool kLow>
int launch_reg_kernel(const RegGeom &g, const MatP<K> &M, cudaStream_t st)
{
    auto kern = k_apply_reg<K, kLow>;
    // resident CTAs per SM for this instantiation (function-local static: initialised once,
    // thread-safe)
    static const LaunchCfg cfg = [&] {
        LaunchCfg c;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return c;
        if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return c;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ, kern, 256, 0) != cudaSuccess || c.occ < 1)
            c.occ = 1;
        c.ok = true;
        return c;
    }();
    if (!cfg.ok) return -1;
    const uint64_t need = (g.n_wtiles + 7) / 8;  // 8 warps per CTA
    const uint64_t grid = std::min<uint64_t>(need, (uint64_t)cfg.sms * cfg.occ);
    kern<<<(unsigned)grid, 256, 0, st>>>(g, M);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int K>
int launch_reg(float2 *psi, int nbits, const int *tpos, const MatP<K> &M, cudaStream_t st)
{
    RegGeom g{};
    g.psi = psi;
    g.n_wtiles = 1ull << (nbits - 5 - K);
    g.J = 0;
    int high[kMaxK], nh = 0;
    for (int i = 0; i < K; i++) {
        if (tpos[i] < 5)
            g.lt[g.J++] = tpos[i];
        else
            high[nh++] = tpos[i];
    }
    int extra[5], ne = 0;  // the J lowest free bits >= 5
    for (int b = 5; ne < g.J && b < nbits; b++) {
        bool used = false;
        for (int i = 0; i < nh; i++) used |= high[i] == b;
        if (!used) extra[ne++] = b;
    }
    if (ne < g.J) return -1;
    g.nfix = 0;
    for (int i = 0; i < ne; i++) g.fix[g.nfix++] = extra[i];
    for (int i = 0; i < nh; i++) g.fix[g.nfix++] = high[i];
    std::sort(g.fix, g.fix + g.nfix);
    for (int x = 0; x < (1 << K); x++) {
        uint64_t o = 0;
        for (int b = 0; b < g.J; b++)
            if ((x >> b) & 1) o += 1ull << extra[b];
        for (int i = 0; i < nh; i++)
            if ((x >> (g.J + i)) & 1) o += 1ull << high[i];
        g.xoff[x] = o;
    }
    return g.J ? launch_reg_kernel<K, true>(g, M, st) : launch_reg_kernel<K, false>(g, M, st);
}

template <int K>
int launch_param(float2 *psi, int nbits, const int *tpos, const float2 *mat, cudaStream_t st)
{
    MatP<K> M;
    std::memcpy(M.m, mat, sizeof(M.m));
    // Measured on GB300 at n = 30: for k <= 3 with every target >= 5 the one-group-per-thread
    // kernel streams at ~7.0 TB/s, ~10% above the persistent register kernel; everywhere
    // else (k = 4, or any target below bit 5) the register kernel is faster.
    const bool all_high = tpos[0] >= 5;
    if (K <= 3 && all_high && nbits - K >= 8) return launch_k<K, MatP<K>>(psi, nbits, tpos, M, st);
    if (nbits >= K + 5) return launch_reg<K>(psi, nbits, tpos, M, st);
    return launch_k<K, MatP<K>>(psi, nbits, tpos, M, st);
}

}  // namespace

int launch_apply_fp32(sim_t *, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat,
                      const float2 *mat6_dev, cudaStream_t st)
{
    switch (k) {
    case 1: return launch_param<1>(psi, nbits, tpos, mat, st);
    case 2: return launch_param<2>(psi, nbits, tpos, mat, st);
    case 3: return launch_param<3>(psi, nbits, tpos, mat, st);
    case 4: return launch_param<4>(psi, nbits, tpos, mat, st);
    case 5: return launch_param<5>(psi, nbits, tpos, mat, st);
    case 6: return launch_k<6, MatPtr>(psi, nbits, tpos, MatPtr{mat6_dev}, st);
    default: return -1;
    }
}

// Validate targets, map them to physical bits through phys_of (a qubit whose entry is < 0 or
// >= nlocal is not local), sort, and reorder + round the FP64 matrix to FP32 in sorted-bit
// order.  Returns SIM_OK or an error code (message set on h).
int prepare_block_map(sim_t *h, int k, const int *targets, const double *matrix, const int *phys_of,
                      int nlocal, int *tpos, float2 *mat, int nq)
{
    if (nq < 0) nq = h->n;
    if (k < 1 || k > kMaxK) return fail(h, SIM_E_INVAL, "apply: k=%d outside 1..%d", k, kMaxK);
    if (!targets || !matrix) return fail(h, SIM_E_INVAL, "apply: NULL targets or matrix");
    if (k > nlocal)
        return fail(h, SIM_E_NONLOCAL, "apply: k=%d exceeds the %d local qubits", k, nlocal);
    int phys[kMaxK], order[kMaxK];
    for (int j = 0; j < k; j++) {
        const int q = targets[j];
        if (q < 0 || q >= nq) return fail(h, SIM_E_INVAL, "apply: target %d outside 0..%d", q, nq - 1);
        for (int i = 0; i < j; i++)
            if (targets[i] == q) return fail(h, SIM_E_INVAL, "apply: duplicate target %d", q);
        phys[j] = phys_of[q];
        if (phys[j] < 0 || phys[j] >= nlocal)
            return fail(h, SIM_E_NONLOCAL, "apply: qubit %d is sliced (not among the %d local bits)", q,
                        nlocal);
        order[j] = j;
    }
    std::sort(order, order + k, [&](int a, int b) { return phys[a] < phys[b]; });
    for (int i = 0; i < k; i++) tpos[i] = phys[order[i]];
    const int D = 1 << k;
    int map[64];
    for (int x = 0; x < D; x++) {
        int y = 0;
        for (int i = 0; i < k; i++)
            if ((x >> i) & 1) y |= 1 << order[i];
        map[x] = y;
    }
    for (int r = 0; r < D; r++)
        for (int c = 0; c < D; c++) {
            const double *e = matrix + 2 * ((size_t)map[r] * D + map[c]);
            mat[r * D + c] = make_float2((float)e[0], (float)e[1]);
        }
    return SIM_OK;
}

int prepare_block(sim_t *h, int k, const int *targets, const double *matrix, int *tpos, float2 *mat)
{
    return prepare_block_map(h, k, targets, matrix, h->bit_of, h->n - h->s, tpos, mat);
}

// Which kernel family takes a block: the one place that decides it.
BlockPath block_path(int nbits, int k, const int *tpos, int precision)
{
    if (tmem_mode(precision) && tcgen05_eligible(nbits, k, tpos)) return BlockPath::Tcgen05;
    if (precision != SIM_FP32 && (tc_eligible(nbits, k, tpos) || (tmem_mode(precision) && tc_eligible_low4(nbits, k))))
        return BlockPath::MmaSync;
    return BlockPath::CudaCore;
}

bool staging_slot_free(sim_t *h, int nbits, int k, const int *tpos, int precision)
{
    // an event never recorded counts as complete
    if (block_path(nbits, k, tpos, precision) != BlockPath::CudaCore)
        return cudaEventQuery(h->frag_ev[h->frag_next]) != cudaErrorNotReady;
    if (k == 6) return cudaEventQuery(h->mat6_ev[h->mat6_next]) != cudaErrorNotReady;
    return true;
}

// Operands of a block staged once in device memory (CUDA graphs): tensor-core B fragments, or
// the matrix of a 6-qubit block on CUDA cores; nothing for narrower CUDA-core blocks, whose
// matrix travels as kernel parameters.
size_t block_staged_bytes(int nbits, int k, const int *tpos, int precision)
{
    switch (block_path(nbits, k, tpos, precision)) {
    case BlockPath::Tcgen05: return tcgen05_staged_bytes(k);
    case BlockPath::MmaSync: return tc_staged_bytes(k, precision);
    default: return k == 6 ? sizeof(float2) * 4096 : 0;
    }
}

void block_build_staged(int nbits, int k, const int *tpos, const float2 *mat, int precision, void *h_out)
{
    switch (block_path(nbits, k, tpos, precision)) {
    case BlockPath::Tcgen05: tcgen05_build_staged(k, mat, precision == SIM_BF16X3, h_out); break;
    case BlockPath::MmaSync: tc_build_staged(k, mat, precision, h_out); break;
    default:
        if (k == 6) std::memcpy(h_out, mat, sizeof(float2) * 4096);
        break;
    }
}

int launch_block_staged(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat,
                        int precision, const void *d_staged, cudaStream_t st, double *red, int *red_grid)
{
    int rc;
    if (red_grid) *red_grid = 0;
    switch (block_path(nbits, k, tpos, precision)) {
    case BlockPath::Tcgen05:
        rc = tcgen05_launch_staged(h, psi, nbits, k, tpos, precision == SIM_BF16X3, d_staged, st, red, red_grid);
        break;
    case BlockPath::MmaSync: rc = tc_launch_staged(psi, nbits, k, tpos, precision, d_staged, st); break;
    default:
        rc = launch_apply_fp32(h, psi, nbits, k, tpos, mat, k == 6 ? static_cast<const float2 *>(d_staged) : nullptr,
                               st);
        break;
    }
    if (rc != 0)
        return fail(h, SIM_E_CUDA, "apply (staged): launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return SIM_OK;
}

// Enqueue one prepared block on a buffer of 2^nbits amplitudes, on stream st.
int enqueue_block_on(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat,
                     int precision, cudaStream_t st)
{
    const BlockPath path = block_path(nbits, k, tpos, precision);
    if (path == BlockPath::Tcgen05) {
        const int ps = prof_begin(h, SIM_PROF_APPLY, 16.0 * std::ldexp(1.0, nbits), st);
        const int rc = launch_apply_tcgen05(h, psi, nbits, k, tpos, mat, precision == SIM_BF16X3, st);
        prof_end(h, ps, st);
        if (rc != 0)
            return fail(h, SIM_E_CUDA, "apply (tcgen05): launch failed: %s",
                        cudaGetErrorString(cudaGetLastError()));
        return SIM_OK;
    }
    if (path == BlockPath::MmaSync) {
        const int ps = prof_begin(h, SIM_PROF_APPLY, 16.0 * std::ldexp(1.0, nbits), st);
        const int rc = launch_apply_tc(h, psi, nbits, k, tpos, mat, precision, st);
        prof_end(h, ps, st);
        if (rc != 0)
            return fail(h, SIM_E_CUDA, "apply (tensor cores): launch failed: %s",
                        cudaGetErrorString(cudaGetLastError()));
        return SIM_OK;
    }
    const float2 *mat6 = nullptr;
    int slot6 = -1;
    if (k == 6) {
        const int slot = slot6 = h->mat6_next;
        h->mat6_next = (slot + 1) % sim_s::kMat6Slots;
        SIM_CUDA_TRY(h, cudaEventSynchronize(h->mat6_ev[slot]));  // host staging slot free
        std::memcpy(h->h_mat6 + 4096 * slot, mat, sizeof(float2) * 4096);
        float2 *dst = h->d_mat6 + 4096 * slot;
        SIM_CUDA_TRY(h, cudaMemcpyAsync(dst, h->h_mat6 + 4096 * slot, sizeof(float2) * 4096,
                                        cudaMemcpyHostToDevice, st));
        mat6 = dst;
    }
    const int ps = prof_begin(h, SIM_PROF_APPLY, 16.0 * std::ldexp(1.0, nbits), st);
    const int rc = launch_apply_fp32(h, psi, nbits, k, tpos, mat, mat6, st);
    prof_end(h, ps, st);
    // the matrix slot is free again once this kernel, which reads it, has run (on any stream)
    if (slot6 >= 0) SIM_CUDA_TRY(h, cudaEventRecord(h->mat6_ev[slot6], st));
    if (rc != 0)
        return fail(h, SIM_E_CUDA, "apply: kernel launch failed: %s",
                    cudaGetErrorString(cudaGetLastError()));
    return SIM_OK;
}

int enqueue_block(sim_t *h, int k, const int *tpos, const float2 *mat, int precision)
{
    return enqueue_block_on(h, h->d_state, h->n, k, tpos, mat, precision, h->stream);
}

bool precision_ok(int precision) { return precision >= SIM_FP32 && precision <= SIM_BF16X3; }

}  // namespace sycsim

using namespace sycsim;

extern "C" int sim_apply_fused(sim_t *h, int k, const int *targets, const double *matrix,
                               int precision)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_apply_fused: NULL handle");
    state_written(h);
    if (h->store != SIM_STORE_DEVICE)
        return fail(h, SIM_E_UNSUPPORTED, "sim_apply_fused: host-store state: use sim_run_phase");
    if (!precision_ok(precision))
        return fail(h, SIM_E_INVAL, "sim_apply_fused: precision %d", precision);
    int tpos[kMaxK];
    static thread_local float2 mat[4096];
    int rc = prepare_block(h, k, targets, matrix, tpos, mat);
    if (rc != SIM_OK) return rc;
    SIM_DEVICE_SCOPE(h, h->device);
    return enqueue_block(h, k, tpos, mat, precision);
}
