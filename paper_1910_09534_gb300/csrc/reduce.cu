// reduce.cu -- reductions over p_i = |psi_i|^2 (norm, 2^n sum p^2, XEB), logical-order
// gather/scatter for readout, and basis-state initialisation.
//
// The reduction reads 8 bytes per amplitude once (HBM-bound).  Each thread sums 16
// amplitudes in FP32 and then accumulates those partial sums in FP64, so FP64 work is
// 1/16 of the amplitude count (GB300's FP64 rate is far below its FP32 rate); CTA partials
// are combined by one warp in a fixed order, so the result is deterministic.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace sycsim {
namespace {

constexpr int kReduceThreads = 256;
constexpr int kReduceUnroll = 8;  // float4 loads (2 amplitudes each) per FP32 partial

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce_partials(const float4 *psi4, uint64_t n4,
                                                                    double *partials)
{
    double s1 = 0.0, s2 = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kReduceThreads * kReduceUnroll;
    for (uint64_t b = (uint64_t)blockIdx.x * kReduceThreads * kReduceUnroll + threadIdx.x; b < n4;
         b += stride) {
        float a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int u = 0; u < kReduceUnroll; ++u) {
            const uint64_t i = b + (uint64_t)u * kReduceThreads;
            if (i < n4) {
                const float4 v = __ldcs(psi4 + i);
                const float p0 = fmaf(v.x, v.x, v.y * v.y);
                const float p1 = fmaf(v.z, v.z, v.w * v.w);
                a1 += p0 + p1;
                a2 = fmaf(p0, p0, fmaf(p1, p1, a2));
            }
        }
        s1 += (double)a1;
        s2 += (double)a2;
    }
    __shared__ double w1[kReduceThreads / 32], w2[kReduceThreads / 32];
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        w1[warp] = s1;
        w2[warp] = s2;
    }
    __syncthreads();
    if (warp == 0) {
        s1 = lane < kReduceThreads / 32 ? w1[lane] : 0.0;
        s2 = lane < kReduceThreads / 32 ? w2[lane] : 0.0;
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if (lane == 0) {
            partials[2 * blockIdx.x] = s1;
            partials[2 * blockIdx.x + 1] = s2;
        }
    }
}

__global__ void k_reduce_final(const double *partials, int nblocks, double *out)
{
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 32) {
        s1 += partials[2 * i];
        s2 += partials[2 * i + 1];
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (threadIdx.x == 0) {
        out[0] = s1;
        out[1] = s2;
    }
}

// r[4..6] = {sum p, scale * sum p^2, scale * sum p^2 - 1} from r[0..1] = (sum p, sum p^2)
__global__ void k_result3(double *r, double scale)
{
    const double s2 = r[1] * scale;
    r[4] = r[0];
    r[5] = s2;
    r[6] = s2 - 1.0;
}

struct BitMap {
    int bit_of[kMaxQubits];
};

__global__ void k_gather_logical(float2 *psi, float2 *dst, uint64_t first, uint64_t count, int n,
                                 BitMap m, int scatter)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = first + j;
        uint64_t p = 0;
        for (int q = 0; q < n; ++q) p |= ((i >> q) & 1ull) << m.bit_of[q];
        if (scatter)
            psi[p] = dst[j];
        else
            dst[j] = psi[p];
    }
}

// Entries first .. first + count - 1 (logical indices through m, or physical ones with the
// identity map) whose physical index p lies in [lo, hi), between base[p - lo] and buf[j]: gathered
// into buf, or scattered from it; the others are left alone (buf[j] for them is not written).
__global__ void k_gather_region(float2 *base, uint64_t lo, uint64_t hi, float2 *buf, uint64_t first,
                                uint64_t count, int n, BitMap m, int scatter)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = first + j;
        uint64_t p = 0;
        for (int q = 0; q < n; ++q) p |= ((i >> q) & 1ull) << m.bit_of[q];
        if (p < lo || p >= hi) continue;
        if (scatter)
            base[p - lo] = buf[j];
        else
            buf[j] = base[p - lo];
    }
}

__global__ void k_set_basis(float2 *psi, uint64_t phys) { psi[phys] = make_float2(1.f, 0.f); }

// Final step of the allocation-free reduction: sum p, scale * sum p^2, and that minus 1.
__global__ void k_reduce_final3(const double *partials, int nblocks, double scale, double *out)
{
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 32) {
        s1 += partials[2 * i];
        s2 += partials[2 * i + 1];
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (threadIdx.x == 0) {
        out[0] = s1;
        out[1] = s2 * scale;
        out[2] = s2 * scale - 1.0;
    }
}

constexpr int kNoAllocPartials = 2 * kReduceBlocks;
constexpr uint64_t kNoAllocMaxAmps = 1ull << kMaxQubits;
constexpr int kNoAllocMaxDevices = 64;

std::mutex g_noalloc_mu;
double *g_noalloc_addr[kNoAllocMaxDevices] = {};

}  // namespace
}  // namespace sycsim

// Scratch of sim_reduce_noalloc: one (sum p, sum p^2) pair per CTA of the reduction grid,
// 2 * 608 doubles = 9.5 KiB.  A file-scope device array: every GPU that loads this library
// holds it until the process exits, and no call allocates it.
static __device__ __align__(256) double g_noalloc_partials[sycsim::kNoAllocPartials];

namespace sycsim {

int launch_reduce(sim_t *, const float2 *psi, uint64_t amps, double *d_partials, double *d_result,
                  cudaStream_t st)
{
    const uint64_t n4 = amps / 2;  // amps >= 2 (n >= 1)
    k_reduce_partials<<<kReduceBlocks, kReduceThreads, 0, st>>>((const float4 *)psi, n4, d_partials);
    k_reduce_final<<<1, 32, 0, st>>>(d_partials, kReduceBlocks, d_result);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_reduce_final(const double *partials, int nblocks, double *d_result, cudaStream_t st)
{
    k_reduce_final<<<1, 32, 0, st>>>(partials, nblocks, d_result);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_result3(double *d_result, double scale, cudaStream_t st)
{
    k_result3<<<1, 1, 0, st>>>(d_result, scale);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_gather_region(float2 *base, uint64_t lo, uint64_t hi, float2 *buf, uint64_t first, uint64_t count, int n,
                         const int *bit_of, int scatter, cudaStream_t st)
{
    BitMap m{};
    for (int q = 0; q < n; q++) m.bit_of[q] = bit_of ? bit_of[q] : q;
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks == 0) return 0;
    k_gather_region<<<(unsigned)blocks, 256, 0, st>>>(base, lo, hi, buf, first, count, n, m, scatter);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_gather_logical(const float2 *psi, float2 *dst, uint64_t first, uint64_t count, int n,
                          const int *bit_of, int scatter, cudaStream_t st)
{
    BitMap m{};
    for (int q = 0; q < n; q++) m.bit_of[q] = bit_of[q];
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_gather_logical<<<(unsigned)blocks, 256, 0, st>>>((float2 *)psi, dst, first, count, n, m, scatter);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace sycsim

using namespace sycsim;

// Same reduction as sim_reduce, for callers that hand in their own device buffers and cannot
// allocate.  The scratch is g_noalloc_partials; host code only ever sees a host-side stand-in
// for that name, so its device address is looked up once per device (with that device
// current) and passed to the kernels.
extern "C" int sim_reduce_noalloc(const void *d_state, uint64_t n_amps, double *d_out, void *stream)
{
    if (!d_state || !d_out) return fail(nullptr, SIM_E_INVAL, "sim_reduce_noalloc: NULL buffer");
    if (((uintptr_t)d_state & 15) != 0)
        return fail(nullptr, SIM_E_INVAL, "sim_reduce_noalloc: state must be 16-byte aligned");
    if (((uintptr_t)d_out & 7) != 0)
        return fail(nullptr, SIM_E_INVAL, "sim_reduce_noalloc: d_out must be 8-byte aligned");
    if (n_amps < 2 || (n_amps & 1))
        return fail(nullptr, SIM_E_INVAL, "sim_reduce_noalloc: n_amps=%llu must be even and >= 2",
                    (unsigned long long)n_amps);
    if (n_amps > kNoAllocMaxAmps)
        return fail(nullptr, SIM_E_INVAL,
                    "sim_reduce_noalloc: n_amps=%llu exceeds the maximum 2^%d amplitudes",
                    (unsigned long long)n_amps, kMaxQubits);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail(nullptr, SIM_E_CUDA, "sim_reduce_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(nullptr, SIM_E_INVAL, "sim_reduce_noalloc: device %d outside 0..%d", dev,
                    kNoAllocMaxDevices - 1);
    double *partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p)
                return fail(nullptr, SIM_E_CUDA, "sim_reduce_noalloc: cudaGetSymbolAddress: %s",
                            cudaGetErrorString(e));
            g_noalloc_addr[dev] = (double *)p;
        }
        partials = g_noalloc_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_reduce_partials<<<kReduceBlocks, kReduceThreads, 0, st>>>((const float4 *)d_state, n_amps / 2,
                                                                partials);
    k_reduce_final3<<<1, 32, 0, st>>>(partials, kReduceBlocks, (double)n_amps, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(nullptr, SIM_E_CUDA, "sim_reduce_noalloc: launch: %s", cudaGetErrorString(e));
    return SIM_OK;
}

namespace sycsim {

int launch_set_basis(float2 *psi, uint64_t amps, uint64_t phys, cudaStream_t st)
{
    if (phys >= amps) return -1;
    k_set_basis<<<1, 1, 0, st>>>(psi, phys);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace sycsim
