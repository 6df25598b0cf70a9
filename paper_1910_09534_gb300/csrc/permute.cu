// permute.cu -- in-place qubit-bit permutation of the state (Sect. 4: between phases the
// layout is reorganised so that a different set of qubits is local; on one GPU this is a
// permutation of the amplitude-index bits).  Pure data movement: bit-exact.
//
// A bit permutation pi is written as sigma2 o sigma1 with both sigmas involutions (products
// of disjoint bit transpositions): a cycle c_0 -> c_1 -> ... -> c_{L-1} is the reflection
// x -> 1 - x (mod L) after the reflection x -> -x (mod L).  Each involution is one pass:
//  * transpositions between two bits >= LB swap whole tiles (tile tau <-> tile sigma(tau));
//  * transpositions with one bit < LB make the other bit a "row" bit of the tile;
//  * transpositions inside [0, LB) act within the tile.
// A CTA loads a tile pair (2^(LB+q) amplitudes each, rows of 2^LB contiguous amplitudes) with
// 16-byte loads, permutes it in shared memory and writes it back with coalesced 16-byte stores.  Tiles that
// nothing moves are skipped, so a single high-bit swap touches half of the state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

// Measured on 2^30 amplitudes: 16-byte accesses 13-17 % faster than 8-byte on every pattern;
// minimum tiles of 2^11-2^12 amplitudes help tiles that permute in place a little and tile pairs
// much less (persistent CTAs looping over tile pairs were slower still).
#ifndef SYCSIM_PERM_TILE
#define SYCSIM_PERM_TILE 10  // minimum tile: 2^SYCSIM_PERM_TILE amplitudes
#endif
#ifndef SYCSIM_PERM_BULK
#define SYCSIM_PERM_BULK 1  // in-place tiles through bulk copies (k_permute_tile_bulk)
#endif
#ifndef SYCSIM_PERM_TILE_SAME
#define SYCSIM_PERM_TILE_SAME 12  // the same when no tile pairs swap (measured best of 10..13)
#endif

namespace sycsim {
namespace {

constexpr int kMaxRow = 6;

struct PermGeom {
    float2 *psi;
    int LB, q;                    // low-block bits, row bits
    int rowpos[kMaxRow];          // global bit of row bit i (ascending)
    int sig[16];                  // in-tile involution on local bits 0..LB+q-1
    int nhh, hh_a[20], hh_b[20];  // high-high transpositions
    int trivial_in;               // sig is the identity
    uint32_t fsw[1 << kMaxRow];   // row r -> XOR applied to its low index (bank spreading)
    uint64_t rowoff[1 << kMaxRow];
    // the in-tile maps are XOR-linear in the local index p: their values on each single bit
    uint64_t lin_off[16];   // global offset of p (row offset + low index)
    uint32_t lin_sidx[16];  // shared-memory slot of p (row-XOR swizzle)
    uint32_t lin_src[16];   // shared-memory slot of the amplitude that lands at p (swizzle o sig)
    // bulk in-place path: local bit of thread-index bit j (bits 0-4: the lanes of a warp, chosen so
    // that p and sig(p) both spread over the shared-memory banks), then the iteration bits
    int8_t tbit[8], ibit[16];
};

__device__ __forceinline__ uint64_t insert_zero_bits_p(uint64_t x, const int *pos, int cnt)
{
    for (int i = 0; i < cnt; ++i) {
        const int p = pos[i];
        const uint64_t lo = x & ((1ull << p) - 1);
        x = ((x >> p) << (p + 1)) | lo;
    }
    return x;
}

__global__ void __launch_bounds__(256) k_permute_pass(PermGeom g)
{
    extern __shared__ float2 sm[];
    const uint64_t baseA = insert_zero_bits_p((uint64_t)blockIdx.x << g.LB, g.rowpos, g.q);
    uint64_t baseB = baseA;
    for (int i = 0; i < g.nhh; ++i) {
        const uint64_t ba = (baseA >> g.hh_a[i]) & 1, bb = (baseA >> g.hh_b[i]) & 1;
        if (ba != bb) baseB ^= (1ull << g.hh_a[i]) | (1ull << g.hh_b[i]);
    }
    if (baseB < baseA) return;  // the partner CTA moves this pair
    const bool same = baseA == baseB;
    if (same && g.trivial_in) return;  // nothing in this tile moves

    // Thread t handles the amplitude pairs p = 2t + j * 2 * blockDim: the part of each map that
    // depends on 2t is computed once, the part that depends on j is uniform across the warp.
    const int nloc = g.LB + g.q, T = 1 << nloc;
    const uint32_t step = 2 * blockDim.x, p0 = 2 * threadIdx.x;
    int sbits = 0;
    while ((1u << sbits) < step) ++sbits;
    uint64_t off0 = 0;
    uint32_t ld0 = 0, st0 = 0;
    for (int x = 1; x < sbits && x < nloc; ++x)
        if ((p0 >> x) & 1) {
            off0 += g.lin_off[x];
            ld0 ^= g.lin_sidx[x];
            st0 ^= g.lin_src[x];
        }
    const uint32_t ld1 = g.lin_sidx[0], st1 = g.lin_src[0];  // the odd amplitude of the pair
    for (uint32_t hi = 0; p0 + hi < (uint32_t)T; hi += step) {
        uint64_t offj = 0;
        uint32_t ldj = 0;
        for (int x = sbits; x < nloc; ++x)
            if ((hi >> x) & 1) {
                offj += g.lin_off[x];
                ldj ^= g.lin_sidx[x];
            }
        const uint64_t off = off0 + offj;
        const uint32_t l = ld0 ^ ldj;
        const float4 a = __ldcs(reinterpret_cast<const float4 *>(g.psi + baseA + off));
        sm[l] = make_float2(a.x, a.y);
        sm[l ^ ld1] = make_float2(a.z, a.w);
        if (!same) {
            const float4 b = __ldcs(reinterpret_cast<const float4 *>(g.psi + baseB + off));
            sm[T + l] = make_float2(b.x, b.y);
            sm[T + (l ^ ld1)] = make_float2(b.z, b.w);
        }
    }
    __syncthreads();
    for (uint32_t hi = 0; p0 + hi < (uint32_t)T; hi += step) {
        uint64_t offj = 0;
        uint32_t stj = 0;
        for (int x = sbits; x < nloc; ++x)
            if ((hi >> x) & 1) {
                offj += g.lin_off[x];
                stj ^= g.lin_src[x];
            }
        const uint64_t off = off0 + offj;
        const uint32_t s0 = st0 ^ stj, s1 = s0 ^ st1;
        const float2 x = sm[s0], y = sm[s1];
        if (same) {
            __stcs(reinterpret_cast<float4 *>(g.psi + baseA + off), make_float4(x.x, x.y, y.x, y.y));
        } else {
            const float2 u = sm[T + s0], v = sm[T + s1];
            __stcs(reinterpret_cast<float4 *>(g.psi + baseB + off), make_float4(x.x, x.y, y.x, y.y));
            __stcs(reinterpret_cast<float4 *>(g.psi + baseA + off), make_float4(u.x, u.y, v.x, v.y));
        }
    }
}

// The global side done by the bulk-copy engine: one copy per row of 2^LB contiguous amplitudes
// into shared memory (completion counted in bytes on an mbarrier) -- the tile, and for a tile
// pair (high-high transpositions) its partner's rows too --, the threads swap the pairs
// (p, sig(p)) the in-tile involution exchanges in each tile, and one bulk store per row writes
// the tile back, or, for a pair, each tile to its partner's rows.  sig is XOR-linear in
// the local index p: sig(p) = sig(p_thread) ^ sig(p_iter), the second from a per-CTA table.
// The only wait (the copies' mbarrier) is bounded by %globaltimer: on a timeout the CTA records
// the failure, writes nothing back and waits (again bounded) for its copies before leaving.
__device__ __forceinline__ uint64_t perm_now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(256) k_permute_tile_bulk(PermGeom g, int *err)
{
    extern __shared__ __align__(128) float2 tile[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t p_it[64], sig_it[64];  // the iteration part of p, and its image under sig
    __shared__ int ok;
    const int nloc = g.LB + g.q, T = 1 << nloc;
    const uint32_t row_bytes = 8u << g.LB;
    const uint64_t base = insert_zero_bits_p((uint64_t)blockIdx.x << g.LB, g.rowpos, g.q);
    uint64_t baseB = base;
    for (int i = 0; i < g.nhh; ++i) {
        const uint64_t ba = (base >> g.hh_a[i]) & 1, bb = (base >> g.hh_b[i]) & 1;
        if (ba != bb) baseB ^= (1ull << g.hh_a[i]) | (1ull << g.hh_b[i]);
    }
    if (baseB < base) return;  // the partner CTA moves this pair
    const bool same = baseB == base;
    if (same && g.trivial_in) return;  // nothing in this tile moves
    const int ntile = same ? 1 : 2;
    const uint32_t sbar = (uint32_t)__cvta_generic_to_shared(&bar);
    const uint32_t stile = (uint32_t)__cvta_generic_to_shared(tile);
    auto sig_of = [&](uint32_t p) {
        uint32_t r = 0;
        for (int x = 0; x < nloc; ++x)
            if ((p >> x) & 1) r |= 1u << g.sig[x];
        return r;
    };
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sbar),
                     "r"((uint32_t)(ntile * T) * 8u)
                     : "memory");
        for (int t = 0; t < ntile; ++t)
            for (int r = 0; r < (1 << g.q); ++r)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                        stile + (uint32_t)t * T * 8u + r * row_bytes),
                    "l"(g.psi + (t ? baseB : base) + g.rowoff[r]), "r"(row_bytes), "r"(sbar)
                    : "memory");
    }
    for (int it = threadIdx.x; it < (T >> 8); it += blockDim.x) {
        uint32_t p = 0;
        for (int j = 0; j < nloc - 8; ++j)
            if ((it >> j) & 1) p |= 1u << g.ibit[j];
        p_it[it] = p;
        sig_it[it] = sig_of(p);
    }
    if (threadIdx.x == 0) {
        const uint64_t t0 = perm_now_ns();
        uint32_t done = 0;
        while (!done) {
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, 20000;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(done)
                : "r"(sbar)
                : "memory");
            if (!done && perm_now_ns() - t0 > 4000000000ull) break;
        }
        ok = done;
        if (!done && err) atomicExch(err, 1);
    }
    __syncthreads();
    if (ok) {
        uint32_t p_t = 0;  // blockDim = 256: p = (thread bits deposited) | (iteration bits deposited)
        for (int j = 0; j < 8; ++j)
            if ((threadIdx.x >> j) & 1) p_t |= 1u << g.tbit[j];
        const uint32_t s_t = sig_of(p_t);
        for (int t = 0; t < ntile && !g.trivial_in; ++t) {
            float2 *tt = tile + t * T;
            for (int it = 0; it < (T >> 8); ++it) {
                const uint32_t p = p_t | p_it[it], q = s_t ^ sig_it[it];
                if (p < q) {
                    const float2 a = tt[p], c = tt[q];
                    tt[p] = c;
                    tt[q] = a;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the bulk stores read the tile
        __syncthreads();
        if (threadIdx.x == 0) {  // a pair's tiles go to each other's rows
            for (int t = 0; t < ntile; ++t)
                for (int r = 0; r < (1 << g.q); ++r)
                    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(
                                     g.psi + ((t == 0) == same ? base : baseB) + g.rowoff[r]),
                                 "r"(stile + (uint32_t)t * T * 8u + r * row_bytes), "r"(row_bytes)
                                 : "memory");
            asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");  // the tile is read out
        }
    } else if (threadIdx.x == 0) {  // no copy may still be writing the tile when the CTA leaves
        const uint64_t t0 = perm_now_ns();
        uint32_t done = 0;
        while (!done && perm_now_ns() - t0 <= 4000000000ull)
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, 20000;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(done)
                : "r"(sbar)
                : "memory");
    }
}

// One involution pass; inv[b] = partner of bit b (inv[b] == b: fixed).
// Geometry of one involution pass for tiles of at least 2^min_tile amplitudes.
int build_geom(float2 *psi, int nbits, const int *inv, int min_tile, PermGeom &g)
{
    // low block: smallest LB >= min(5, nbits) with LB + q >= min(min_tile, nbits)
    int LB = std::min(5, nbits), q = 0;
    for (;; LB++) {
        q = 0;
        for (int b = 0; b < LB; b++)
            if (inv[b] >= LB) q++;
        if (LB + q >= std::min(min_tile, nbits) || LB == nbits) break;
    }
    if (q > kMaxRow) return -2;

    g = PermGeom{};
    g.psi = psi;
    g.LB = LB;
    g.q = q;
    std::vector<std::pair<int, int>> rows;  // (global high bit, low partner)
    for (int b = 0; b < LB; b++)
        if (inv[b] >= LB) rows.push_back({inv[b], b});
    std::sort(rows.begin(), rows.end());
    for (int i = 0; i < q; i++) g.rowpos[i] = rows[i].first;
    for (int x = 0; x < 16; x++) g.sig[x] = x;
    g.trivial_in = 1;
    for (int b = 0; b < LB; b++) {
        if (inv[b] == b) continue;
        g.trivial_in = 0;
        if (inv[b] < LB) {
            g.sig[b] = inv[b];
        } else {
            int i = 0;
            while (rows[i].first != inv[b]) i++;
            g.sig[b] = LB + i;
            g.sig[LB + i] = b;
        }
    }
    g.nhh = 0;
    for (int b = LB; b < nbits; b++)
        if (inv[b] > b) {
            bool row = false;
            for (int i = 0; i < q; i++) row |= g.rowpos[i] == b || g.rowpos[i] == inv[b];
            if (!row) {
                g.hh_a[g.nhh] = b;
                g.hh_b[g.nhh] = inv[b];
                g.nhh++;
            }
        }
    for (int r = 0; r < (1 << q); r++) {
        uint64_t o = 0;
        uint32_t f = 0;
        for (int i = 0; i < q; i++)
            if ((r >> i) & 1) {
                o += 1ull << g.rowpos[i];
                f ^= 1u << rows[i].second;  // row bit i lands on bank bit of its low partner
            }
        g.rowoff[r] = o;
        g.fsw[r] = f & ((1u << LB) - 1);
    }
    // values of the XOR-linear in-tile maps on each single local bit
    const int nloc = LB + q;
    auto sidx_h = [&](uint32_t p) {
        const uint32_t r = p >> LB;
        return (r << LB) | ((p & ((1u << LB) - 1)) ^ g.fsw[r]);
    };
    for (int x = 0; x < nloc; x++) {
        const uint32_t p = 1u << x;
        g.lin_off[x] = x < LB ? (uint64_t)p : g.rowoff[p >> LB];
        g.lin_sidx[x] = sidx_h(p);
        g.lin_src[x] = sidx_h(1u << g.sig[x]);  // the amplitude landing at p came from slot sig(p)
    }
    return 0;
}

// Bits of the local index the 32 lanes of a warp run over in k_permute_tile_bulk: a warp reads
// and writes both p and sig(p); with 8-byte elements the bank pair is bits 0-3 of the index, so a
// set of lane bits costs max(2, 32 >> |bits in 0-3|) wavefronts for p, the same for sig(p).  The
// cheapest 5-subset of the bits 0-4 and their images under sig is taken (ties: the lowest), then
// three more bits for the warps and the rest for the iterations, ascending.
void choose_lane_bits(PermGeom &g)
{
    const int nloc = g.LB + g.q;
    int cand[16], nc = 0;
    bool in[16] = {};
    for (int x = 0; x < 5 && x < nloc; x++) {
        for (int y : {x, g.sig[x]})
            if (!in[y]) in[y] = true, cand[nc++] = y;
    }
    std::sort(cand, cand + nc);
    auto wf = [](int low) { return std::max(2, 32 >> low); };
    int best_cost = 1 << 30;
    uint32_t best = 0;
    for (uint32_t m = 0; m < (1u << nc); m++) {
        if (__builtin_popcount(m) != 5) continue;
        int lp = 0, ls = 0;
        for (int i = 0; i < nc; i++)
            if ((m >> i) & 1) {
                lp += cand[i] < 4;
                ls += g.sig[cand[i]] < 4;
            }
        const int cost = wf(lp) + wf(ls);
        if (cost < best_cost) best_cost = cost, best = m;
    }
    bool used[16] = {};
    int j = 0;
    for (int i = 0; i < nc; i++)
        if ((best >> i) & 1) g.tbit[j++] = (int8_t)cand[i], used[cand[i]] = true;
    for (int x = 0; x < nloc && j < 8; x++)
        if (!used[x]) g.tbit[j++] = (int8_t)x, used[x] = true;
    int k = 0;
    for (int x = 0; x < nloc; x++)
        if (!used[x]) g.ibit[k++] = (int8_t)x;
}

int launch_involution(float2 *psi, int nbits, const int *inv, cudaStream_t st, int *err)
{
    bool any = false;
    for (int b = 0; b < nbits; b++) any |= inv[b] != b;
    if (!any) return 0;
    PermGeom g;
    const int rc = build_geom(psi, nbits, inv, SYCSIM_PERM_TILE, g);
    if (rc != 0) return rc;
    // tiles that only permute in place (no tile pairs) gain from more work per CTA
    if (g.nhh == 0 && SYCSIM_PERM_TILE_SAME > SYCSIM_PERM_TILE) {
        PermGeom big;
        if (build_geom(psi, nbits, inv, SYCSIM_PERM_TILE_SAME, big) == 0) g = big;
    }
    const int LB = g.LB, q = g.q;
    const uint64_t tiles = 1ull << (nbits - LB - q);
    if (SYCSIM_PERM_BULK && LB >= 5 && LB + q >= 8 && LB + q <= 14 && ((uintptr_t)psi & 15) == 0 &&
        (g.nhh == 0 ? 1 : 2) * (sizeof(float2) << (LB + q)) <= 128 * 1024) {
        const size_t tsm = (g.nhh == 0 ? 1 : 2) * (sizeof(float2) << (LB + q));
        if (tsm > 48 * 1024 &&
            cudaFuncSetAttribute(k_permute_tile_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm) !=
                cudaSuccess)
            return -1;
        choose_lane_bits(g);
        k_permute_tile_bulk<<<(unsigned)tiles, 256, tsm, st>>>(g, err);
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    const size_t smem = (g.nhh ? 2 : 1) * sizeof(float2) << (LB + q);  // a tile pair, or one tile
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_permute_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return -1;
    const int threads = std::min(256, 1 << (LB + q));
    k_permute_pass<<<(unsigned)tiles, threads, smem, st>>>(g);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

// Amplitudes an involution moves: those whose bits differ across at least one transposition.
static double moved_fraction(int nbits, const int *inv)
{
    int pairs = 0;
    for (int b = 0; b < nbits; b++) pairs += inv[b] > b;
    return 1.0 - std::ldexp(1.0, -pairs);
}

int launch_permute(sim_t *h, float2 *psi, int nbits, const int *perm, cudaStream_t st)
{
    // split pi into cycles; sigma1 = reflection x -> -x, sigma2 = reflection x -> 1 - x
    int s1[kMaxQubits], s2[kMaxQubits];
    bool seen[kMaxQubits] = {};
    for (int b = 0; b < nbits; b++) s1[b] = s2[b] = b;
    for (int b = 0; b < nbits; b++) {
        if (seen[b]) continue;
        std::vector<int> cyc;
        for (int x = b; !seen[x]; x = perm[x]) {
            seen[x] = true;
            cyc.push_back(x);
        }
        const int L = (int)cyc.size();
        for (int x = 0; x < L; x++) {
            s1[cyc[x]] = cyc[(L - x) % L];
            s2[cyc[x]] = cyc[(L + 1 - x) % L];
        }
    }
    const double amps = std::ldexp(1.0, nbits);
    int rc = 0;
    for (const int *inv : {s1, s2}) {
        const double frac = moved_fraction(nbits, inv);
        if (frac == 0.0) continue;
        const int ps = h ? prof_begin(h, SIM_PROF_PERMUTE, 16.0 * amps * frac, st) : -1;
        rc = launch_involution(psi, nbits, inv, st, h ? h->d_errflag : nullptr);
        if (h) prof_end(h, ps, st);
        if (rc != 0) return rc;
    }
    return 0;
}

}  // namespace sycsim

using namespace sycsim;

extern "C" int sim_permute(sim_t *h, const int *perm)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_permute: NULL handle");
    state_written(h);
    if (!perm) return fail(h, SIM_E_INVAL, "sim_permute: NULL perm");
    if (h->store != SIM_STORE_DEVICE)
        return fail(h, SIM_E_UNSUPPORTED, "sim_permute: the host store's layout is fixed by its sliced sets");
    bool used[kMaxQubits] = {};
    for (int q = 0; q < h->n; q++) {
        if (perm[q] < 0 || perm[q] >= h->n || used[perm[q]])
            return fail(h, SIM_E_INVAL, "sim_permute: perm is not a bijection on 0..%d", h->n - 1);
        used[perm[q]] = true;
    }
    // physical permutation: old bit bit_of[q] -> new bit perm[q]
    int phys[kMaxQubits];
    for (int q = 0; q < h->n; q++) phys[h->bit_of[q]] = perm[q];
    SIM_DEVICE_SCOPE(h, h->device);
    int rc = launch_permute(h, h->d_state, h->n, phys, h->stream);
    if (rc != 0)
        return fail(h, SIM_E_CUDA, "sim_permute: launch failed (%d): %s", rc,
                    cudaGetErrorString(cudaGetLastError()));
    for (int q = 0; q < h->n; q++) {
        h->bit_of[q] = perm[q];
        h->qubit_at[perm[q]] = q;
    }
    return SIM_OK;
}

extern "C" int sim_set_layout(sim_t *h, const int *perm)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_set_layout: NULL handle");
    state_written(h);
    if (!perm) return fail(h, SIM_E_INVAL, "sim_set_layout: NULL perm");
    bool used[kMaxQubits] = {};
    for (int q = 0; q < h->n; q++) {
        if (perm[q] < 0 || perm[q] >= h->n || used[perm[q]])
            return fail(h, SIM_E_INVAL, "sim_set_layout: perm is not a bijection on 0..%d", h->n - 1);
        used[perm[q]] = true;
    }
    if (h->store == SIM_STORE_HOST) {
        if (!host_store_relabel(h, perm))
            return fail(h, SIM_E_INVAL, "sim_set_layout: a host store keeps sets A and B on their bits");
        return SIM_OK;
    }
    for (int q = 0; q < h->n; q++) {
        h->bit_of[q] = perm[q];
        h->qubit_at[perm[q]] = q;
    }
    return SIM_OK;
}
