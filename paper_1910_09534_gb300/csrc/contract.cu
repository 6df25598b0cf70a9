// contract.cu -- the contraction that eliminates the entanglement indices (Appendix: the sum
// over every pair (a', a) of tensor 1 times tensor 2), as one complex GEMM.
//
// With both tensors in their canonical layouts (side qubits at the low bits, the 2c
// entanglement bits above, in the same order in both), tensor 1 is a matrix T1[e][x] and tensor
// 2 a matrix T2[e][y] (x, y contiguous), and
//     psi[P(x, y)] = sum_e T1[e][x] T2[e][y],   e < 4^c,
// where P places x's bits on the side-0 qubits and y's on the side-1 qubits in the output
// handle's current physical layout.
// Two kernels compute it:
//  * k_contract_fp32 (CUDA cores): 64 x 64 output tiles, 4 x 4 per thread, FP32 products and
//    sums, operands staged through shared memory 16 entanglement values at a time;
//  * k_contract_tcgen05 (5th-generation tensor cores): 128 x 128 output tiles as two real GEMMs
//    of M = 128 (x) x N = 256 (Re y | Im y) x K = 16 (entanglement values) per step,
//    X = [Re T1] . [Re T2 | Im T2] and Y = [Im T1] . [Re T2 | Im T2] in tensor memory, so that
//    Re psi = X_re - Y_im and Im psi = X_im + Y_re.  3xFP16: each tensor is scaled by one power
//    of two (largest component below 2^14, so FP16 stays normal) and split hi = fp16(v),
//    lo = fp16(v - hi); a step issues hi.hi + hi.lo + lo.hi into each accumulator.  A first pass
//    writes both tensors as FP16 operand images in the MMA's shared-memory layout (K-major core
//    matrices: 8 rows x 16 bytes), so a k-step of one tile is two contiguous 16 KiB blocks that
//    the bulk-copy engine moves unchanged.  One persistent CTA per SM: warp 0 loads k-steps into
//    a ring of 6 stages (mbarrier byte counts), one thread of warp 1 issues the MMAs and commits
//    each stage back, warps 2-9 read the accumulators once a tile is done, combine, unscale
//    and store (a warp's lanes are 32 consecutive x: 256-byte rows).  Tiles are visited in
//    groups of 8 y-tiles so the CTAs running together share operand blocks in L2.  Every wait
//    is bounded in time (%globaltimer); a timeout sets the handle's error word and ends every
//    role, and the CTA waits for its own copies and MMAs before releasing tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

using namespace sycsim;

namespace {

constexpr int kFx = 64, kFy = 64, kFk = 16;  // FP32 kernel: tile x, tile y, entanglement chunk

// Where psi lands: bit i of x (side-0 qubit i, increasing qubit order) adds xbit[i] to the
// physical index, bit j of y adds ybit[j] (powers of two from the output handle's layout).
struct CtOut {
    uint64_t xbit[kMaxQubits];
    uint64_t ybit[kMaxQubits];
};

__device__ __forceinline__ uint64_t ct_dep(uint64_t v, const uint64_t *bit, int nb)
{
    uint64_t o = 0;
    for (int i = 0; i < nb; ++i)
        if ((v >> i) & 1) o += bit[i];
    return o;
}

// t1 (t2): 2^n1 (2^n2) columns of each entanglement row, rows ld1 (ld2) amplitudes apart.
__global__ void __launch_bounds__(256) k_contract_fp32(const float2 *__restrict__ t1, const float2 *__restrict__ t2,
                                                       float2 *__restrict__ psi, int n1, int n2, uint64_t n_e,
                                                       uint64_t ld1, uint64_t ld2, const __grid_constant__ CtOut o)
{
    __shared__ __align__(16) float2 sa[kFk][kFx];
    __shared__ __align__(16) float2 sb[kFk][kFy];
    __shared__ uint64_t xoff[kFx], yoff[kFy];
    const uint64_t X = 1ull << n1, Y = 1ull << n2;
    const uint64_t tiles_x = (X + kFx - 1) / kFx;
    const uint64_t x0 = (blockIdx.x % tiles_x) * kFx, y0 = (blockIdx.x / tiles_x) * kFy;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < kFx)
        xoff[tid] = ct_dep(x0 + tid, o.xbit, n1);
    else if (tid < kFx + kFy)
        yoff[tid - kFx] = ct_dep(y0 + tid - kFx, o.ybit, n2);
    float2 acc[4][4];  // [y][x]
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = make_float2(0.f, 0.f);
    for (uint64_t e0 = 0; e0 < n_e; e0 += kFk) {
#pragma unroll
        for (int r = 0; r < (kFk * kFx) / 256; ++r) {
            const int idx = tid + 256 * r, k = idx / kFx, c = idx % kFx;
            const uint64_t e = e0 + k;
            sa[k][c] = (e < n_e && x0 + c < X) ? t1[x0 + c + e * ld1] : make_float2(0.f, 0.f);
            sb[k][c] = (e < n_e && y0 + c < Y) ? t2[y0 + c + e * ld2] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kFk; ++k) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sa[k][4 * tx + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sb[k][4 * ty + j];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    acc[j][i].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[j][i].x));
                    acc[j][i].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[j][i].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint64_t y = y0 + 4 * ty + j;
        if (y >= Y) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t x = x0 + 4 * tx + i;
            if (x < X) psi[xoff[4 * tx + i] + yoff[4 * ty + j]] = acc[j][i];
        }
    }
}

int launch_contract_fp32(const float2 *t1, const float2 *t2, float2 *psi, int n1, int n2, int e_bits, uint64_t ld1,
                         uint64_t ld2, const CtOut &o, cudaStream_t st)
{
    const uint64_t X = 1ull << n1, Y = 1ull << n2;
    const uint64_t blocks = ((X + kFx - 1) / kFx) * ((Y + kFy - 1) / kFy);
    if (blocks > 0x7fffffffull) return -1;
    k_contract_fp32<<<(unsigned)blocks, 256, 0, st>>>(t1, t2, psi, n1, n2, 1ull << e_bits, ld1, ld2, o);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------------------------
// tcgen05 contraction
// ---------------------------------------------------------------------------------------------

constexpr int kCtStages = 6;
constexpr int kCtStage = 32768;     // one k-step of one tile: A 4 x 4 KiB + B 2 x 8 KiB
constexpr int kCtSlab = 16384;      // bytes of one operand's k-step block
constexpr int kCtEpi = 256;         // epilogue threads: warps 2-9
constexpr int kCtThreads = 64 + kCtEpi;
constexpr int kCtGroupY = 8;        // y tiles per raster group
constexpr unsigned long long kCtWaitNs = 4000000000ull;  // 4 s: far above any legitimate wait

struct CtArgs {
    const uint8_t *aimg;  // tensor 1 as the A operand: [x tile][k-step] blocks of 16 KiB
    const uint8_t *bimg;  // tensor 2 as the B operand: [y tile][k-step] blocks of 16 KiB
    float2 *psi;
    int n1, n2;           // psi's physical index: CtOut offsets of x (n1 bits) plus of y (n2 bits)
    uint32_t ks;          // k-steps (16 entanglement values each) per tile
    uint32_t tiles_x, tiles_y;
    const float *amax;    // largest |component| of tensor 1, tensor 2
    int *err;
    int bf16;             // operand images in BF16 (SIM_BF16X3) instead of FP16
};

__device__ __forceinline__ uint32_t ct_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t ct_desc(uint32_t saddr)
{
    // K-major, no swizzle: LBO = 128 B (between the two 8-wide K halves), SBO = 256 B (between
    // 8-row groups), descriptor version 1
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ void ct_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void ct_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void ct_ld16(uint32_t ta, float (&v)[16])
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

__device__ __forceinline__ uint64_t ct_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool ct_try(uint32_t bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}

// Wait for the phase of the given parity; gives up after kCtWaitNs or once another role aborted.
__device__ __forceinline__ bool ct_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (ct_try(bar, parity, 0)) return true;
    const uint64_t t0 = ct_ns();
    for (;;) {
        if (ct_try(bar, parity, 20000)) return true;
        if (*abort_flag || ct_ns() - t0 > kCtWaitNs) return false;
    }
}

// Wait for work this thread issued itself, even after an abort (bounded).
__device__ __forceinline__ void ct_wait_own(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = ct_ns();
    while (!ct_try(bar, parity, 20000) && ct_ns() - t0 <= kCtWaitNs) {
    }
}

__device__ __forceinline__ void ct_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool ct_bar_and(int id, int n, bool p)
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

__device__ __forceinline__ void ct_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void ct_bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Power-of-two scale exponent: the largest component lands in [2^13, 2^14).
__device__ __forceinline__ int ct_shift(float amax)
{
    int e = 0;
    frexpf(amax, &e);
    return amax > 0.f ? max(-100, min(100, 14 - e)) : 0;
}

__device__ __forceinline__ void ct_tile(uint64_t i, uint32_t tiles_x, uint32_t tiles_y, uint32_t &tx, uint32_t &ty)
{
    const uint64_t per_group = (uint64_t)tiles_x * kCtGroupY;
    const uint32_t gy0 = (uint32_t)(i / per_group) * kCtGroupY;
    const uint32_t r = (uint32_t)(i % per_group);
    const uint32_t gh = min((uint32_t)kCtGroupY, tiles_y - gy0);
    ty = gy0 + r % gh;
    tx = r / gh;
}

// Largest |Re|, |Im| of n amplitudes into *out (a float's bits; non-negative floats order as
// unsigned integers).  *out must be 0 before the launch.
// The tensor is read as pairs of amplitudes (16 bytes), four pairs in flight per thread.
__global__ void __launch_bounds__(256) k_absmax(const float4 *__restrict__ t, uint64_t n4, unsigned *out)
{
    float m = 0.f;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        float4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = t[i + j * stride];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v[j].x), fabsf(v[j].y)), fmaxf(fabsf(v[j].z), fabsf(v[j].w))));
    }
    for (; i < n4; i += stride) {
        const float4 v = t[i];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// hi / lo pieces of v as FP16 (or BF16, SIM_BF16X3) bit patterns
template <bool BF>
__device__ __forceinline__ void ct_split(float v, uint16_t &h, uint16_t &l)
{
    if constexpr (BF) {
        const __nv_bfloat16 a = __float2bfloat16_rn(v);
        const __nv_bfloat16 b = __float2bfloat16_rn(v - __bfloat162float(a));
        h = __bfloat16_as_ushort(a);
        l = __bfloat16_as_ushort(b);
    } else {
        const __half a = __float2half_rn(v);
        const __half b = __float2half_rn(v - __half2float(a));
        h = __half_as_ushort(a);
        l = __half_as_ushort(b);
    }
}

// Operand image of one tensor T[e][c] (c < 2^nside contiguous, e < n_e; e >= n_e reads as 0).
// Thread = (tile, k-step, row r < 128, K half kh): 8 entanglement values of column c = 128 tile + r.
// role 0 (A, tensor 1): slabs Re hi | Re lo | Im hi | Im lo, 128 rows x 16 each (4 KiB).
// role 1 (B, tensor 2): slabs hi | lo, 256 rows x 16 each (8 KiB): row r = Re, row 128 + r = Im.
template <bool BF>
__global__ void __launch_bounds__(256) k_contract_image(const float2 *__restrict__ t, int nside, uint64_t n_e,
                                                        uint32_t ks, const float *amax, uint8_t *img, int role)
{
    const uint64_t C = 1ull << nside;
    const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (gid >= (C / 128) * ks * 256) return;
    const int r = (int)(gid & 127), kh = (int)((gid >> 7) & 1);
    const uint64_t ts = gid >> 8;  // tile * ks + k-step
    const uint64_t tile = ts / ks, step = ts % ks;
    const float sc = ldexpf(1.f, ct_shift(*amax));
    __align__(16) uint16_t rh[8], rl[8], ih[8], il[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint64_t e = 16 * step + 8 * kh + j;
        const float2 v = e < n_e ? t[e * C + tile * 128 + r] : make_float2(0.f, 0.f);
        ct_split<BF>(v.x * sc, rh[j], rl[j]);
        ct_split<BF>(v.y * sc, ih[j], il[j]);
    }
    uint8_t *base = img + ts * kCtSlab;
    const uint32_t off = (r >> 3) * 256 + kh * 128 + (r & 7) * 16;
    if (role == 0) {
        *reinterpret_cast<uint4 *>(base + off) = *reinterpret_cast<const uint4 *>(rh);
        *reinterpret_cast<uint4 *>(base + 4096 + off) = *reinterpret_cast<const uint4 *>(rl);
        *reinterpret_cast<uint4 *>(base + 8192 + off) = *reinterpret_cast<const uint4 *>(ih);
        *reinterpret_cast<uint4 *>(base + 12288 + off) = *reinterpret_cast<const uint4 *>(il);
    } else {  // rows 128 + r sit 16 row groups (4 KiB) further
        *reinterpret_cast<uint4 *>(base + off) = *reinterpret_cast<const uint4 *>(rh);
        *reinterpret_cast<uint4 *>(base + 4096 + off) = *reinterpret_cast<const uint4 *>(ih);
        *reinterpret_cast<uint4 *>(base + 8192 + off) = *reinterpret_cast<const uint4 *>(rl);
        *reinterpret_cast<uint4 *>(base + 12288 + off) = *reinterpret_cast<const uint4 *>(il);
    }
}

// Per tile (local count tl) and k-step (running count it, stage it % 6, stage phase (it / 6) & 1):
//   loader: wait empty[stage] of k-step it - 6, copy the A and B blocks, full[stage] counts bytes;
//   MMA thread: before a tile's first step wait acc_empty of tile tl - 1; wait full[stage], issue
//     the 6 MMAs, commit to empty[stage]; after the last step commit to acc_full;
//   epilogue: wait acc_full (phase tl), read, store, arrive acc_empty.
__global__ void __launch_bounds__(kCtThreads, 1) k_contract_tcgen05(CtArgs g, const __grid_constant__ CtOut o)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t full[kCtStages], empty[kCtStages], acc_full, acc_empty;
    __shared__ uint64_t xoff[128], yoff[128];  // offsets of x, y within a tile (bits 0-6)
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint64_t n_tiles = (uint64_t)g.tiles_x * g.tiles_y;
    if (tid == 0) {
        for (int st = 0; st < kCtStages; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ct_smem(&full[st])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ct_smem(&empty[st])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ct_smem(&acc_full)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(ct_smem(&acc_empty)), "r"(kCtEpi) : "memory");
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(ct_smem(&tmem_base)));
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

    if (warp == 0) {
        // ---------------- bulk loads: lanes 0-3 the A block, 4-7 the B block (4 KiB each) ----------------
        uint32_t it = 0;
        bool stop = false;
        for (uint64_t tile = blockIdx.x; tile < n_tiles && !stop; tile += gridDim.x) {
            uint32_t tx, ty;
            ct_tile(tile, g.tiles_x, g.tiles_y, tx, ty);
            const uint8_t *a = g.aimg + (uint64_t)tx * g.ks * kCtSlab;
            const uint8_t *b = g.bimg + (uint64_t)ty * g.ks * kCtSlab;
            for (uint32_t s = 0; s < g.ks; ++s, ++it) {
                const int st = it % kCtStages;
                const bool ok = it < (uint32_t)kCtStages || ct_wait(ct_smem(&empty[st]), (it / kCtStages - 1) & 1, ab);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) give_up();
                    stop = true;
                    break;
                }
                const uint32_t bar = ct_smem(&full[st]);
                if (lane == 0) ct_expect_tx(bar, kCtStage);
                __syncwarp();
                const uint32_t dst = ct_smem(sm + st * kCtStage);
                if (lane < 4)
                    ct_bulk_load(dst + lane * 4096, a + (uint64_t)s * kCtSlab + lane * 4096, 4096, bar);
                else if (lane < 8)
                    ct_bulk_load(dst + kCtSlab + (lane - 4) * 4096, b + (uint64_t)s * kCtSlab + (lane - 4) * 4096,
                                 4096, bar);
            }
        }
        // no copy may still be writing the stages when the CTA leaves (matters after an abort)
        if (lane == 0)
            for (uint32_t j = it > (uint32_t)kCtStages ? it - kCtStages : 0; j < it; ++j)
                ct_wait_own(ct_smem(&full[j % kCtStages]), (j / kCtStages) & 1);
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            // F32 accumulate, A/B FP16 or BF16 (format bits 7 and 10), N = 256, M = 128
            const uint32_t idesc = (1u << 4) | (g.bf16 ? (1u << 7) | (1u << 10) : 0u) | ((uint32_t)(256 >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
            uint32_t it = 0, tl = 0;
            bool stop = false;
            for (uint64_t tile = blockIdx.x; tile < n_tiles && !stop; tile += gridDim.x, ++tl) {
                if (tl > 0 && !ct_wait(ct_smem(&acc_empty), (tl - 1) & 1, ab)) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                for (uint32_t s = 0; s < g.ks; ++s, ++it) {
                    const int st = it % kCtStages;
                    if (!ct_wait(ct_smem(&full[st]), (it / kCtStages) & 1, ab)) {
                        give_up();
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t base = ct_smem(sm + st * kCtStage);
                    const uint64_t rh = ct_desc(base), rl = ct_desc(base + 4096), ih = ct_desc(base + 8192),
                                   il = ct_desc(base + 12288), bh = ct_desc(base + kCtSlab),
                                   bl = ct_desc(base + kCtSlab + 8192);
                    const uint32_t acc = s > 0;
                    ct_mma(tmem, rh, bh, idesc, acc);
                    ct_mma(tmem, rh, bl, idesc, 1);
                    ct_mma(tmem, rl, bh, idesc, 1);
                    ct_mma(tmem + 256, ih, bh, idesc, acc);
                    ct_mma(tmem + 256, ih, bl, idesc, 1);
                    ct_mma(tmem + 256, il, bh, idesc, 1);
                    ct_commit(ct_smem(&empty[st]));
                }
                if (!stop) ct_commit(ct_smem(&acc_full));
            }
            // tensor memory is released only after the last MMA issued has completed
            if (it > 0) ct_wait_own(ct_smem(&empty[(it - 1) % kCtStages]), ((it - 1) / kCtStages) & 1);
        }
    } else {
        // ---------------- epilogue ----------------
        const int q = warp & 3;                 // TMEM lane quarter this warp may read
        const int half = (warp - 2) >> 2;       // warps 2-5: y 0..63 of the tile, 6-9: y 64..127
        const int row = 32 * q + lane;          // x within the tile
        const float inv = ldexpf(1.f, -(ct_shift(g.amax[0]) + ct_shift(g.amax[1])));
        const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
        {
            const int e = tid - 64;
            if (e < 128)
                xoff[e] = ct_dep(e, o.xbit, 7);
            else
                yoff[e - 128] = ct_dep(e - 128, o.ybit, 7);
            ct_bar_and(1, kCtEpi, true);  // tables written before any store reads them
        }
        uint32_t tl = 0;
        for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++tl) {
            const bool ok = ct_wait(ct_smem(&acc_full), tl & 1, ab);
            if (!ct_bar_and(1, kCtEpi, ok)) {  // uniform: tcgen05.ld below needs whole warps
                give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint32_t tx, ty;
            ct_tile(tile, g.tiles_x, g.tiles_y, tx, ty);
            float2 *dst = g.psi + ct_dep((uint64_t)tx << 7, o.xbit, g.n1) + ct_dep((uint64_t)ty << 7, o.ybit, g.n2) +
                          xoff[row];
#pragma unroll 1
            for (int c = 0; c < 64; c += 16) {
                const int y0 = half * 64 + c;
                float xr[16], xi[16], yr[16], yi[16];
                ct_ld16(tq + y0, xr);
                ct_ld16(tq + 128 + y0, xi);
                ct_ld16(tq + 256 + y0, yr);
                ct_ld16(tq + 384 + y0, yi);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    __stcs(dst + yoff[y0 + j], make_float2((xr[j] - yi[j]) * inv, (xi[j] + yr[j]) * inv));
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            ct_arrive(ct_smem(&acc_empty));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
}

// Images, then the GEMM, all on st.  The scratch (images + maxima) belongs to the output handle
// and is kept between calls: allocating it per call from the stream-ordered pool re-mapped it
// every time the pool trimmed at a synchronisation, on the host's critical path.
size_t tcgen05_scratch_bytes(int n1, int n2, int e_bits)
{
    const uint64_t ks = ((1ull << e_bits) + 15) / 16;
    return (size_t)((1ull << n1) / 128) * ks * kCtSlab + (size_t)((1ull << n2) / 128) * ks * kCtSlab + 256;
}

const LaunchCfg &ct_cfg()
{
    static const LaunchCfg cfg = [] {
        LaunchCfg c;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return c;
        if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return c;
        c.ok = true;
        return c;
    }();
    return cfg;
}

// Scales and operand images of both (whole) tensors, on st, into the scratch (the output
// handle's own, grown as needed, unless own_scratch is given).
int prepare_tcgen05(sim_t *h, const float2 *t1, const float2 *t2, int n1, int n2, int e_bits, bool bf16,
                    cudaStream_t st, uint8_t *own_scratch, const uint8_t **aimg, const uint8_t **bimg,
                    const float **amax_out)
{
    const LaunchCfg &cfg = ct_cfg();
    if (!cfg.ok) return -1;
    const uint64_t n_e = 1ull << e_bits;
    const uint32_t ks = (uint32_t)((n_e + 15) / 16);
    const uint64_t X = 1ull << n1, Y = 1ull << n2;
    const size_t a_bytes = (size_t)(X / 128) * ks * kCtSlab, b_bytes = (size_t)(Y / 128) * ks * kCtSlab;
    const size_t need = a_bytes + b_bytes + 256;
    if (!own_scratch && h->contract_bytes < need) {  // grow: cudaFree waits for kernels still reading it
        if (h->d_contract) cudaFree(h->d_contract);
        h->d_contract = nullptr;
        h->contract_bytes = 0;
        if (cudaMalloc(reinterpret_cast<void **>(&h->d_contract), need) != cudaSuccess) return -1;
        h->contract_bytes = need;
    }
    uint8_t *scratch = own_scratch ? own_scratch : h->d_contract;
    float *amax = reinterpret_cast<float *>(scratch + a_bytes + b_bytes);
    if (cudaMemsetAsync(amax, 0, 2 * sizeof(float), st) != cudaSuccess) return -1;
    // X, Y >= 128: whole pairs of amplitudes; tensor states start 256-byte aligned
    const uint64_t n4a = X * n_e / 2, n4b = Y * n_e / 2;
    const unsigned blocks = (unsigned)std::min<uint64_t>(8ull * cfg.sms, (n4a + 255) / 256);
    k_absmax<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4 *>(t1), n4a, reinterpret_cast<unsigned *>(amax));
    const unsigned blocks2 = (unsigned)std::min<uint64_t>(8ull * cfg.sms, (n4b + 255) / 256);
    k_absmax<<<blocks2, 256, 0, st>>>(reinterpret_cast<const float4 *>(t2), n4b, reinterpret_cast<unsigned *>(amax + 1));
    auto image = bf16 ? k_contract_image<true> : k_contract_image<false>;
    image<<<(unsigned)((X / 128) * ks), 256, 0, st>>>(t1, n1, n_e, ks, amax, scratch, 0);
    image<<<(unsigned)((Y / 128) * ks), 256, 0, st>>>(t2, n2, n_e, ks, amax + 1, scratch + a_bytes, 1);
    h->launches += 4;
    *aimg = scratch;
    *bimg = scratch + a_bytes;
    *amax_out = amax;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The GEMM for x tiles [x0t, x0t + 2^n1 / 128) and y tiles [y0t, y0t + 2^n2 / 128) of the images.
int launch_gemm_tcgen05(sim_t *h, const uint8_t *aimg, const uint8_t *bimg, const float *amax, uint64_t n_e,
                        uint64_t x0t, uint64_t y0t, float2 *psi, int n1, int n2, const CtOut &o, bool bf16,
                        cudaStream_t st)
{
    static std::atomic<uint64_t> smem_done{0};
    if (!smem_opt_in(k_contract_tcgen05, kCtStages * kCtStage, smem_done)) return -1;
    const LaunchCfg &cfg = ct_cfg();
    if (!cfg.ok) return -1;
    const uint64_t X = 1ull << n1, Y = 1ull << n2;
    const uint32_t ks = (uint32_t)((n_e + 15) / 16);
    CtArgs g{};
    g.aimg = aimg + x0t * ks * kCtSlab;
    g.bimg = bimg + y0t * ks * kCtSlab;
    g.psi = psi;
    g.n1 = n1;
    g.n2 = n2;
    g.ks = ks;
    g.tiles_x = (uint32_t)(X / 128);
    g.tiles_y = (uint32_t)(Y / 128);
    g.amax = amax;
    g.err = h->d_errflag;
    g.bf16 = bf16 ? 1 : 0;
    const uint64_t grid = std::min<uint64_t>((uint64_t)g.tiles_x * g.tiles_y, (uint64_t)cfg.sms);
    const int ps = prof_begin(h, SIM_PROF_CONTRACT, 8.0 * (double)X * (double)Y * (double)n_e, st);
    k_contract_tcgen05<<<(unsigned)grid, kCtThreads, kCtStages * kCtStage, st>>>(g, o);
    prof_end(h, ps, st);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

namespace sycsim {

// Where each wire of tensor t must sit for a contraction into out: the side's qubits at bits
// 0 .. n_side-1 in the order of their physical bits in out (so a warp's 32 consecutive x, or the
// y of one thread, land on the lowest physical bits the side holds), the entanglement pairs above
// in pair order.  bit_of_wire[w] = the physical bit of wire w; side_qubit[i] = the qubit at bit i.
void contract_layout(const sim_split_s *s, const int *out_bit_of, int t, int *bit_of_wire, int *side_qubit)
{
    const int ns = s->n_side[t];
    int order[kMaxQubits], q_of[kMaxQubits];  // canonical position p < ns -> qubit
    int c = 0;
    for (int q = 0; q < s->n; ++q)
        if (s->side[q] == t) q_of[c++] = q;
    for (int p = 0; p < ns; ++p) order[p] = p;
    std::sort(order, order + ns, [&](int a, int b) { return out_bit_of[q_of[a]] < out_bit_of[q_of[b]]; });
    for (int i = 0; i < ns; ++i) {
        bit_of_wire[s->wire_at[t][order[i]]] = i;
        if (side_qubit) side_qubit[i] = q_of[order[i]];
    }
    for (int p = ns; p < (int)s->wire_at[t].size(); ++p) bit_of_wire[s->wire_at[t][p]] = p;
}

bool contract_ready(const sim_split_s *s, const int *out_bit_of, int t, const int *tensor_bit_of, int top)
{
    const int ns = s->n_side[t], nw = (int)s->wire_at[t].size();
    int canon[kMaxQubits];
    contract_layout(s, out_bit_of, t, canon, nullptr);
    for (int p = ns; p < nw; ++p)
        if (tensor_bit_of[s->wire_at[t][p]] != p) return false;
    const int low = t == 0 ? std::min(5, ns - top) : 0;
    for (int p = 0; p < ns; ++p) {
        const int w = s->wire_at[t][p], b = tensor_bit_of[w];
        if (b < 0 || b >= ns || (b < low) != (canon[w] < low)) return false;
        if ((b >= ns - top || canon[w] >= ns - top) && b != canon[w]) return false;
    }
    return true;  // side wires on distinct bits: a handle's layout is a permutation
}

size_t contraction_scratch_bytes(const sim_split_s *s)
{
    return tcgen05_scratch_bytes(s->n_side[0], s->n_side[1], 2 * s->n_pairs);
}

int contract_job_prepare(sim_t *h, const sim_split_s *s, const float2 *t1, const float2 *t2,
                         const int *const *tensor_bit_of, const int *out_bit_of, int precision, const int *top,
                         uint8_t *scratch, cudaStream_t st, ContractJob *job)
{
    ContractJob &j = *job;
    j = ContractJob{};
    j.e_bits = 2 * s->n_pairs;
    j.t[0] = t1;
    j.t[1] = t2;
    int side_qubit[2][kMaxQubits], lay[kMaxQubits];
    for (int t = 0; t < 2; ++t) {
        j.n_side[t] = s->n_side[t];
        j.n_free[t] = s->n_side[t] - (top ? top[t] : 0);
        contract_layout(s, out_bit_of, t, lay, side_qubit[t]);
        if (tensor_bit_of && tensor_bit_of[t]) {  // the side qubit on each of the tensor's bits
            int q_of[kMaxQubits], c = 0;
            for (int q = 0; q < s->n; ++q)
                if (s->side[q] == t) q_of[c++] = q;
            for (int p = 0; p < s->n_side[t]; ++p) side_qubit[t][tensor_bit_of[t][s->wire_at[t][p]]] = q_of[p];
        }
    }
    for (int i = 0; i < j.n_free[0]; ++i) j.xbit[i] = 1ull << out_bit_of[side_qubit[0][i]];
    for (int i = 0; i < j.n_free[1]; ++i) j.ybit[i] = 1ull << out_bit_of[side_qubit[1][i]];
    j.tensor_cores = precision != SIM_FP32 && j.n_free[0] >= 7 && j.n_free[1] >= 7;
    j.bf16 = precision == SIM_BF16X3;
    j.ks = (uint32_t)(((1ull << j.e_bits) + 15) / 16);
    if (!j.tensor_cores) return 0;
    return prepare_tcgen05(h, t1, t2, j.n_side[0], j.n_side[1], j.e_bits, j.bf16, st, scratch, &j.img[0], &j.img[1],
                           &j.amax);
}

int contract_job_launch(sim_t *h, const ContractJob &j, float2 *psi, uint64_t fix0, uint64_t fix1, cudaStream_t st)
{
    CtOut o{};
    std::copy(j.xbit, j.xbit + j.n_free[0], o.xbit);
    std::copy(j.ybit, j.ybit + j.n_free[1], o.ybit);
    const uint64_t x0 = fix0 << j.n_free[0], y0 = fix1 << j.n_free[1];  // first column of each side's range
    if (j.tensor_cores)
        return launch_gemm_tcgen05(h, j.img[0], j.img[1], j.amax, 1ull << j.e_bits, x0 / 128, y0 / 128, psi,
                                   j.n_free[0], j.n_free[1], o, j.bf16, st);
    const int ps = prof_begin(h, SIM_PROF_CONTRACT, 8.0 * std::ldexp(1.0, j.n_free[0] + j.n_free[1] + j.e_bits), st);
    const int rc = launch_contract_fp32(j.t[0] + x0, j.t[1] + y0, psi, j.n_free[0], j.n_free[1], j.e_bits,
                                        1ull << j.n_side[0], 1ull << j.n_side[1], o, st);
    prof_end(h, ps, st);
    return rc;
}

int enqueue_contraction(sim_t *h, const sim_split_s *s, const float2 *t1, const float2 *t2, float2 *psi,
                        const int *out_bit_of, int precision, uint8_t *scratch, cudaStream_t st,
                        const int *const *tensor_bit_of)
{
    ContractJob j;
    const int rc = contract_job_prepare(h, s, t1, t2, tensor_bit_of, out_bit_of, precision, nullptr, scratch, st, &j);
    return rc != 0 ? rc : contract_job_launch(h, j, psi, 0, 0, st);
}

}  // namespace sycsim

extern "C" int sim_contract(sim_t *out, sim_t *t1, sim_t *t2, const sim_split_t *s, int precision)
{
    if (!out || !t1 || !t2 || !s) return fail(out, SIM_E_INVAL, "sim_contract: NULL argument");
    state_written(out);
    if (out == t1 || out == t2 || t1 == t2) return fail(out, SIM_E_INVAL, "sim_contract: handles must be distinct");
    if (precision != SIM_FP32 && precision != SIM_FP16X3 && precision != SIM_FP16X3_TMEM && precision != SIM_BF16X3)
        return fail(out, SIM_E_INVAL,
                    "sim_contract: precision %d is not SIM_FP32, SIM_FP16X3, SIM_FP16X3_TMEM or SIM_BF16X3", precision);
    const int n1 = s->n_side[0], n2 = s->n_side[1], e_bits = 2 * s->n_pairs;
    // out may be sliced: a resident state is one buffer, written whole in its layout
    for (sim_t *h : {out, t1, t2})
        if (h->store != SIM_STORE_DEVICE || (h != out && h->s != 0) || !h->d_state)
            return fail(out, SIM_E_INVAL, "sim_contract: every handle must be device-resident, the tensors not sliced");
    if (t1->device != out->device || t2->device != out->device)
        return fail(out, SIM_E_INVAL, "sim_contract: handles on different devices");
    if (out->n != s->n || t1->n != n1 + e_bits || t2->n != n2 + e_bits)
        return fail(out, SIM_E_INVAL, "sim_contract: qubit counts (%d, %d, %d) do not fit the split (%d, %d, %d)",
                    out->n, t1->n, t2->n, s->n, n1 + e_bits, n2 + e_bits);
    SIM_DEVICE_SCOPE(out, out->device);

    // each tensor into a layout the contraction into out can read (contract_ready), else into
    // contract_layout's
    sim_t *tens[2] = {t1, t2};
    for (int t = 0; t < 2; ++t) {
        sim_t *h = tens[t];
        int perm[kMaxQubits];
        contract_layout(s, out->bit_of, t, perm, nullptr);
        if (!contract_ready(s, out->bit_of, t, h->bit_of)) {
            const int rc = sim_permute(h, perm);
            if (rc != SIM_OK) return fail(out, rc, "sim_contract: permuting tensor %d: %s", t + 1, h->err.c_str());
        }
    }
    cudaEvent_t ev[3] = {};
    for (auto &e : ev) SIM_CUDA_TRY(out, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    auto destroy = [&]() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    };
    if (cudaEventRecord(ev[0], t1->stream) != cudaSuccess || cudaEventRecord(ev[1], t2->stream) != cudaSuccess ||
        cudaStreamWaitEvent(out->stream, ev[0], 0) != cudaSuccess ||
        cudaStreamWaitEvent(out->stream, ev[1], 0) != cudaSuccess) {
        destroy();
        return fail(out, SIM_E_CUDA, "sim_contract: stream ordering failed");
    }
    // psi goes straight into out's current layout
    const int *tbits[2] = {t1->bit_of, t2->bit_of};
    const int rc = enqueue_contraction(out, s, t1->d_state, t2->d_state, out->d_state, out->bit_of, precision,
                                       nullptr, out->stream, tbits);
    if (rc != 0) {
        destroy();
        return fail(out, SIM_E_CUDA, "sim_contract: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (cudaEventRecord(ev[2], out->stream) != cudaSuccess || cudaStreamWaitEvent(t1->stream, ev[2], 0) != cudaSuccess ||
        cudaStreamWaitEvent(t2->stream, ev[2], 0) != cudaSuccess) {
        destroy();
        return fail(out, SIM_E_CUDA, "sim_contract: stream ordering failed");
    }
    destroy();
    return SIM_OK;
}
