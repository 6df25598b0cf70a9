// store.cu -- secondary storage (Sect. 4): the state in pinned host memory, organised so that
// the "logical files" indexed by the sliced qubits are contiguous, streamed through device
// slots one slice at a time.  For states larger than the host's memory the store can keep its
// top regions (one per value of set A) in device memory instead: a hybrid store whose slice
// copies mix host->device and device->device moves.
//
// Layout of the host store (bit 0 first): the qubits in neither sliced set, ascending; then
// set B in the given order; then set A in the given order.  A file is one run of
// 2^(n - 2s) amplitudes with fixed values of A and B.  With set A sliced, slice v is the
// 2^s files with A = v -- one contiguous run -- and its device layout is [rest | B].  With set
// B sliced, slice w gathers the 2^s files with B = w (one copy per file) into [rest | A].
// Every file is read and written whole, once per phase (Sect. 4).
//
// Pipelining: slices rotate through `slots` device buffers.  Host->device copies run on
// st_in, device->host copies on st_out, the fused blocks on the handle's stream; events order
// each slot's copy-in -> compute -> copy-out and stop a copy-in from overwriting a slot before
// the previous slice has left it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

#include "internal.h"

namespace sycsim {

namespace {

// Split [0, n) over the host's cores.
template <typename F>
void parallel_for(uint64_t n, F f)
{
    const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < (1u << 20) || nt == 1) {
        f(0, n);
        return;
    }
    std::vector<std::thread> th;
    const uint64_t chunk = (n + nt - 1) / nt;
    for (unsigned t = 0; t < nt; t++) {
        const uint64_t a = t * chunk, b = std::min(n, a + chunk);
        if (a < b) th.emplace_back([=] { f(a, b); });
    }
    for (auto &x : th) x.join();
}

int s_of(const sim_t *h) { return h->s; }

// Region v of the store (the amplitudes with set A = v): pinned host memory, or device memory
// for the top regions of a hybrid store.  Copies use cudaMemcpyDefault, so both kinds move
// through the same calls.
float2 *region(const sim_t *h, uint64_t v)
{
    const uint64_t slice = 1ull << (h->n - h->s);
    return v < h->host_regions ? h->h_store + v * slice : h->d_store + (v - h->host_regions) * slice;
}

}  // namespace

int host_store_create(sim_t *h, const sim_opts &o)
{
    const int n = h->n, s = h->s;
    if (s < 1 || s > 8 || 2 * s >= n)
        return fail(nullptr, SIM_E_INVAL, "sim_create(host store): need 1 <= slice_bits <= 8 and "
                                          "2*slice_bits < n (got n=%d, slice_bits=%d)", n, s);
    bool used[kMaxQubits] = {};
    for (int w = 0; w < 2; w++)
        for (int i = 0; i < s; i++) {
            const int q = w ? o.set_b[i] : o.set_a[i];
            if (q < 0 || q >= n || used[q])
                return fail(nullptr, SIM_E_INVAL,
                            "sim_create(host store): sets A and B must be %d distinct qubits each, "
                            "disjoint, within 0..%d", s, n - 1);
            used[q] = true;
            h->set[w][i] = q;
        }
    // host layout: rest ascending, then B, then A
    int b = 0;
    for (int q = 0; q < n; q++)
        if (!used[q]) h->bit_of[q] = b++;
    for (int i = 0; i < s; i++) h->bit_of[h->set[1][i]] = n - 2 * s + i;
    for (int i = 0; i < s; i++) h->bit_of[h->set[0][i]] = n - s + i;
    for (int q = 0; q < n; q++) h->qubit_at[h->bit_of[q]] = q;
    // slot layouts: phase with set A sliced -> [rest | B]; with set B sliced -> [rest | A]
    for (int w = 0; w < 2; w++) {
        for (int q = 0; q < n; q++) h->slice_phys[w][q] = used[q] ? -1 : h->bit_of[q];
        for (int i = 0; i < s; i++) h->slice_phys[w][h->set[1 - w][i]] = n - 2 * s + i;
    }
    h->nslots = o.slots ? o.slots : 3;
    if (h->nslots < 2 || h->nslots > sim_s::kMaxSlots)
        return fail(nullptr, SIM_E_INVAL, "sim_create(host store): slots=%d outside 2..%d", h->nslots,
                    sim_s::kMaxSlots);
    const uint64_t slice = 1ull << (n - s), nreg = 1ull << s;
    if (o.store_device_regions < 0 || (uint64_t)o.store_device_regions > nreg)
        return fail(nullptr, SIM_E_INVAL, "sim_create(host store): store_device_regions=%d outside 0..%llu",
                    o.store_device_regions, (unsigned long long)nreg);
    h->host_regions = nreg - (uint64_t)o.store_device_regions;
    cudaError_t e = cudaSuccess;
    if (h->host_regions) {
        e = cudaHostAlloc(&h->h_store, sizeof(float2) * slice * h->host_regions, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            h->h_store = nullptr;
            return fail(nullptr, SIM_E_NOMEM_HOST, "sim_create(host store): pinning %llu bytes: %s",
                        (unsigned long long)(sizeof(float2) * slice * h->host_regions), cudaGetErrorString(e));
        }
    }
    if (o.store_device_regions) {
        e = cudaMalloc(&h->d_store, sizeof(float2) * slice * (uint64_t)o.store_device_regions);
        if (e != cudaSuccess) {
            h->d_store = nullptr;
            return fail(nullptr, SIM_E_NOMEM_DEV, "sim_create(host store): %d device regions: %s",
                        o.store_device_regions, cudaGetErrorString(e));
        }
    }
    for (int i = 0; i < h->nslots; i++) {
        e = cudaMalloc(&h->d_slot[i], sizeof(float2) * slice);
        if (e != cudaSuccess)
            return fail(nullptr, SIM_E_NOMEM_DEV, "sim_create(host store): slot %d: %s", i,
                        cudaGetErrorString(e));
    }
    if ((e = cudaStreamCreateWithFlags(&h->st_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->st_out, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(nullptr, SIM_E_CUDA, "sim_create(host store): streams: %s", cudaGetErrorString(e));
    for (int i = 0; i < h->nslots; i++)
        for (cudaEvent_t *ev : {&h->ev_in[i], &h->ev_done[i], &h->ev_out[i]}) {
            if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
                return fail(nullptr, SIM_E_CUDA, "sim_create(host store): events: %s",
                            cudaGetErrorString(e));
            cudaEventRecord(*ev, h->stream);
        }
    if ((e = cudaEventCreateWithFlags(&h->ev_inplace, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_ops, cudaEventDisableTiming)) != cudaSuccess)
        return fail(nullptr, SIM_E_CUDA, "sim_create(host store): events: %s", cudaGetErrorString(e));
    cudaEventRecord(h->ev_inplace, h->stream);
    e = cudaHostAlloc(&h->h_partials, sizeof(double) * 2 * ((size_t)1 << s), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        h->h_partials = nullptr;
        return fail(nullptr, SIM_E_NOMEM_HOST, "sim_create(host store): %s", cudaGetErrorString(e));
    }
    return SIM_OK;
}

void store_fill_layout(const sim_t *h, int set, int *lay)
{
    const int n = h->n, s = h->s;
    for (int q = 0; q < n; q++) lay[q] = h->bit_of[q];
    for (int i = 0; i < s; i++) {
        lay[h->set[1 - set][i]] = n - 2 * s + i;  // where the slot keeps the other set
        lay[h->set[set][i]] = n - s + i;          // the sliced set on top: its value picks the slice
    }
}

bool host_store_relabel(sim_t *h, const int *perm)
{
    const int n = h->n, s = h->s;
    bool sliced[kMaxQubits] = {};
    for (int w = 0; w < 2; w++)
        for (int i = 0; i < s; i++) {
            sliced[h->set[w][i]] = true;
            if (perm[h->set[w][i]] != h->bit_of[h->set[w][i]]) return false;
        }
    for (int q = 0; q < n; q++) {
        h->bit_of[q] = perm[q];
        h->qubit_at[perm[q]] = q;
        if (!sliced[q]) h->slice_phys[0][q] = h->slice_phys[1][q] = perm[q];  // slots: [others | B or A]
    }
    return true;
}

void host_store_release(sim_t *h)
{
    if (h->st_in) cudaStreamSynchronize(h->st_in);
    if (h->st_out) cudaStreamSynchronize(h->st_out);
    for (int i = 0; i < sim_s::kMaxSlots; i++) {
        if (h->d_slot[i]) cudaFree(h->d_slot[i]);
        for (cudaEvent_t ev : {h->ev_in[i], h->ev_done[i], h->ev_out[i]})
            if (ev) cudaEventDestroy(ev);
    }
    if (h->ev_inplace) cudaEventDestroy(h->ev_inplace);
    if (h->ev_ops) {
        cudaEventSynchronize(h->ev_ops);
        cudaEventDestroy(h->ev_ops);
    }
    if (h->h_ops) cudaFreeHost(h->h_ops);
    if (h->st_in) cudaStreamDestroy(h->st_in);
    if (h->st_out) cudaStreamDestroy(h->st_out);
    if (h->h_store) cudaFreeHost(h->h_store);
    if (h->d_store) cudaFree(h->d_store);
    if (h->h_partials) cudaFreeHost(h->h_partials);
}

// Enqueue the copy of slice `value` of sliced set `set` between the host store and device slot.
static int enqueue_slice_copy(sim_t *h, int set, uint64_t value, int dir, int slot)
{
    const int n = h->n, s = s_of(h);
    const uint64_t slice = 1ull << (n - s), file = 1ull << (n - 2 * s);
    float2 *dev = h->d_slot[slot];
    if (dir == SIM_H2D) {
        // the slot must be free: its previous compute and copy-out are done
        SIM_CUDA_TRY(h, cudaStreamWaitEvent(h->st_in, h->ev_done[slot], 0));
        SIM_CUDA_TRY(h, cudaStreamWaitEvent(h->st_in, h->ev_out[slot], 0));
        // and the files it reads must be written: a copy-out of the other set touched some of
        // them (every slice of one set meets every slice of the other), a copy-out of the same
        // slice all of them.  Copy-ins are ordered on one stream, so waiting on each slot's
        // latest copy-out also covers that slot's earlier ones.
        for (int i = 0; i < h->nslots; i++)
            if (h->out_set[i] >= 0 && (h->out_set[i] != set || h->out_val[i] == value))
                SIM_CUDA_TRY(h, cudaStreamWaitEvent(h->st_in, h->ev_out[i], 0));
        // and no device region it reads may still be computed on in place (by an earlier phase)
        SIM_CUDA_TRY(h, cudaStreamWaitEvent(h->st_in, h->ev_inplace, 0));
        if (set == 0) {
            SIM_CUDA_TRY(h, cudaMemcpyAsync(dev, region(h, value), sizeof(float2) * slice, cudaMemcpyDefault,
                                            h->st_in));
        } else {
            for (uint64_t v = 0; v < (1ull << s); v++)
                SIM_CUDA_TRY(h, cudaMemcpyAsync(dev + v * file, region(h, v) + value * file, sizeof(float2) * file,
                                                cudaMemcpyDefault, h->st_in));
        }
        SIM_CUDA_TRY(h, cudaEventRecord(h->ev_in[slot], h->st_in));
        SIM_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_in[slot], 0));
    } else {
        SIM_CUDA_TRY(h, cudaEventRecord(h->ev_done[slot], h->stream));
        SIM_CUDA_TRY(h, cudaStreamWaitEvent(h->st_out, h->ev_done[slot], 0));
        if (set == 0) {
            SIM_CUDA_TRY(h, cudaMemcpyAsync(region(h, value), dev, sizeof(float2) * slice, cudaMemcpyDefault,
                                            h->st_out));
        } else {
            for (uint64_t v = 0; v < (1ull << s); v++)
                SIM_CUDA_TRY(h, cudaMemcpyAsync(region(h, v) + value * file, dev + v * file, sizeof(float2) * file,
                                                cudaMemcpyDefault, h->st_out));
        }
        SIM_CUDA_TRY(h, cudaEventRecord(h->ev_out[slot], h->st_out));
        h->out_set[slot] = set;
        h->out_val[slot] = value;
    }
    return SIM_OK;
}

static int host_sync_all(sim_t *h)
{
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->st_in));
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->st_out));
    return SIM_OK;
}

int host_reset(sim_t *h, uint64_t basis)
{
    int rc = host_sync_all(h);
    if (rc != SIM_OK) return rc;
    const uint64_t slice = 1ull << (h->n - h->s), nreg = 1ull << h->s;
    if (h->host_regions) {
        float2 *st = h->h_store;
        parallel_for(slice * h->host_regions,
                     [st](uint64_t a, uint64_t b) { std::memset(st + a, 0, sizeof(float2) * (b - a)); });
    }
    if (h->d_store) SIM_CUDA_TRY(h, cudaMemset(h->d_store, 0, sizeof(float2) * slice * (nreg - h->host_regions)));
    const uint64_t p = logical_to_physical(h, basis);
    const float2 one = make_float2(1.f, 0.f);
    SIM_CUDA_TRY(h, cudaMemcpy(region(h, p / slice) + p % slice, &one, sizeof(float2), cudaMemcpyDefault));
    return SIM_OK;
}

// Entries first .. first + count - 1 of a host store (logical or physical order): physical indices
// below host_lim are in the pinned host regions and are read or written there in place; the rest,
// a hybrid store's device regions, go through the device in chunks (k_gather_region), so no host
// copy of a whole region is ever made.  for_chunk(c0, cnt, buf) is called per chunk with buf
// holding (read) or to be filled with (write) the chunk's device-region entries.
template <typename HostPart>
int host_store_access(sim_t *h, uint64_t first, uint64_t count, int physical, bool write, HostPart host_part)
{
    const uint64_t host_lim = h->host_regions << (h->n - h->s);
    if (!h->d_store) {  // every region on the host
        parallel_for(count, [&](uint64_t a, uint64_t b) { host_part(a, b, 0, nullptr); });
        return SIM_OK;
    }
    const uint64_t C = std::min<uint64_t>(count, 1ull << 24);
    float2 *d_buf = nullptr;
    if (C && cudaMalloc(reinterpret_cast<void **>(&d_buf), sizeof(float2) * C) != cudaSuccess)
        return fail(h, SIM_E_NOMEM_DEV, "host store access: staging buffer");
    std::vector<float2> buf(C);
    const int *bits = physical ? nullptr : h->bit_of;
    const uint64_t hi = 1ull << h->n;
    int rc = SIM_OK;
    for (uint64_t c0 = 0; c0 < count && rc == SIM_OK; c0 += C) {
        const uint64_t cnt = std::min(C, count - c0);
        if (write) {  // the host regions' entries in place, the rest scattered from the chunk
            parallel_for(cnt, [&](uint64_t a, uint64_t b) { host_part(c0 + a, c0 + b, c0, buf.data()); });
            if (cudaMemcpy(d_buf, buf.data(), sizeof(float2) * cnt, cudaMemcpyHostToDevice) != cudaSuccess ||
                launch_gather_region(h->d_store, host_lim, hi, d_buf, first + c0, cnt, h->n, bits, 1, h->stream) != 0 ||
                cudaStreamSynchronize(h->stream) != cudaSuccess)
                rc = fail(h, SIM_E_CUDA, "host store access: %s", cudaGetErrorString(cudaGetLastError()));
        } else {
            if (launch_gather_region(h->d_store, host_lim, hi, d_buf, first + c0, cnt, h->n, bits, 0, h->stream) != 0 ||
                cudaMemcpyAsync(buf.data(), d_buf, sizeof(float2) * cnt, cudaMemcpyDeviceToHost, h->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(h->stream) != cudaSuccess)
                rc = fail(h, SIM_E_CUDA, "host store access: %s", cudaGetErrorString(cudaGetLastError()));
            else
                parallel_for(cnt, [&](uint64_t a, uint64_t b) { host_part(c0 + a, c0 + b, c0, buf.data()); });
        }
    }
    if (d_buf) cudaFree(d_buf);
    return rc;
}

int host_amplitudes(sim_t *h, uint64_t first, uint64_t count, void *out, int dtype, int physical)
{
    int rc = host_sync_all(h);
    if (rc != SIM_OK) return rc;
    const uint64_t host_lim = h->host_regions << (h->n - h->s);
    const float2 *hs = h->h_store;
    // entries j in [a, b): from the host regions, or from the chunk (starting at entry c0)
    return host_store_access(h, first, count, physical, false, [&](uint64_t a, uint64_t b, uint64_t c0, const float2 *buf) {
        for (uint64_t j = a; j < b; j++) {
            const uint64_t p = physical ? first + j : logical_to_physical(h, first + j);
            const float2 v = p < host_lim ? hs[p] : buf[j - c0];
            if (dtype == SIM_C64) {
                static_cast<float2 *>(out)[j] = v;
            } else {
                static_cast<double *>(out)[2 * j] = v.x;
                static_cast<double *>(out)[2 * j + 1] = v.y;
            }
        }
    });
}

int host_load(sim_t *h, uint64_t first, uint64_t count, const void *src, int physical)
{
    int rc = host_sync_all(h);
    if (rc != SIM_OK) return rc;
    const uint64_t host_lim = h->host_regions << (h->n - h->s);
    float2 *hs = h->h_store;
    const float2 *in = static_cast<const float2 *>(src);
    // entries j in [a, b): into the host regions, or into the chunk for the device scatter
    return host_store_access(h, first, count, physical, true, [&](uint64_t a, uint64_t b, uint64_t c0, float2 *buf) {
        for (uint64_t j = a; j < b; j++) {
            const uint64_t p = physical ? first + j : logical_to_physical(h, first + j);
            if (p < host_lim)
                hs[p] = in[j];
            else
                buf[j - c0] = in[j];
        }
    });
}

int host_reduce(sim_t *h, double *s1, double *s2)
{
    const int s = s_of(h);
    const uint64_t nsl = 1ull << s, slice = 1ull << (h->n - s);
    for (uint64_t v = 0; v < nsl; v++) {
        const int slot = (int)(v % h->nslots);
        int rc = enqueue_slice_copy(h, 0, v, SIM_H2D, slot);
        if (rc != SIM_OK) return rc;
        const int ps = prof_begin(h, SIM_PROF_REDUCE, 8.0 * (double)slice, h->stream);
        h->launches++;
        rc = launch_reduce(h, h->d_slot[slot], slice, h->d_partials, h->d_result, h->stream);
        prof_end(h, ps, h->stream);
        if (rc != 0) return fail(h, SIM_E_CUDA, "sim_reduce: launch failed");
        SIM_CUDA_TRY(h, cudaMemcpyAsync(h->h_partials + 2 * v, h->d_result, sizeof(double) * 2,
                                        cudaMemcpyDeviceToHost, h->stream));
        SIM_CUDA_TRY(h, cudaEventRecord(h->ev_done[slot], h->stream));
    }
    int rc = host_sync_all(h);
    if (rc != SIM_OK) return rc;
    double a = 0.0, b = 0.0;
    for (uint64_t v = 0; v < nsl; v++) {
        a += h->h_partials[2 * v];
        b += h->h_partials[2 * v + 1];
    }
    *s1 = a;
    *s2 = b;
    return SIM_OK;
}

// ---- checkpoint / resume ----

namespace {

struct StateFileHeader {
    char magic[8];  // "SYCSTATE"
    uint32_t version;
    int32_t n, s, store;
    int32_t set_a[8], set_b[8];
    int32_t bit_of[kMaxQubits];
    uint64_t amps;
    uint64_t reserved[4];
};

constexpr uint32_t kStateFileVersion = 1;
constexpr size_t kCkptChunk = 64ull << 20;  // bytes through the pinned buffer at a time

// The state as runs of device or host memory in physical order.
std::vector<std::pair<float2 *, uint64_t>> state_runs(sim_t *h)
{
    std::vector<std::pair<float2 *, uint64_t>> runs;
    if (h->store != SIM_STORE_HOST) {
        runs.push_back({h->d_state, h->amps});
        return runs;
    }
    const uint64_t slice = 1ull << (h->n - h->s);
    for (uint64_t v = 0; v < (1ull << h->s); v++) runs.push_back({region(h, v), slice});
    return runs;
}

struct PinnedChunk {
    char *p = nullptr;
    ~PinnedChunk()
    {
        if (p) cudaFreeHost(p);
    }
};

int sync_state(sim_t *h)
{
    if (h->store == SIM_STORE_HOST) return host_sync_all(h);
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SIM_OK;
}

}  // namespace

}  // namespace sycsim

using namespace sycsim;

extern "C" int sim_state_save(sim_t *h, const char *path)
{
    if (!h || !path) return fail(h, SIM_E_INVAL, "sim_state_save: NULL argument");
    SIM_DEVICE_SCOPE(h, h->device);
    int rc = sync_state(h);
    if (rc != SIM_OK) return rc;
    StateFileHeader hd{};
    std::memcpy(hd.magic, "SYCSTATE", 8);
    hd.version = kStateFileVersion;
    hd.n = h->n;
    hd.s = h->s;
    hd.store = h->store;
    for (int i = 0; i < 8; i++) {
        hd.set_a[i] = h->set[0][i];
        hd.set_b[i] = h->set[1][i];
    }
    for (int q = 0; q < h->n; q++) hd.bit_of[q] = h->bit_of[q];
    hd.amps = h->amps;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(h, SIM_E_IO, "sim_state_save: cannot open %s for writing", path);
    PinnedChunk buf;
    if (cudaHostAlloc(reinterpret_cast<void **>(&buf.p), kCkptChunk, cudaHostAllocDefault) != cudaSuccess) {
        buf.p = nullptr;
        std::fclose(f);
        return fail(h, SIM_E_NOMEM_HOST, "sim_state_save: staging buffer");
    }
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
    for (auto &run : state_runs(h)) {
        const char *src = reinterpret_cast<const char *>(run.first);
        cudaPointerAttributes at{};
        const bool on_device = cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        for (uint64_t off = 0, total = run.second * sizeof(float2); ok && off < total; off += kCkptChunk) {
            const size_t len = (size_t)std::min<uint64_t>(kCkptChunk, total - off);
            const char *from = src + off;
            if (on_device) {
                if (cudaMemcpy(buf.p, from, len, cudaMemcpyDeviceToHost) != cudaSuccess) {
                    std::fclose(f);
                    return fail(h, SIM_E_CUDA, "sim_state_save: %s", cudaGetErrorString(cudaGetLastError()));
                }
                from = buf.p;
            }
            ok = std::fwrite(from, 1, len, f) == len;
        }
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SIM_OK : fail(h, SIM_E_IO, "sim_state_save: writing %s failed", path);
}

extern "C" int sim_state_load(sim_t *h, const char *path)
{
    if (!h || !path) return fail(h, SIM_E_INVAL, "sim_state_load: NULL argument");
    state_written(h);
    SIM_DEVICE_SCOPE(h, h->device);
    int rc = sync_state(h);
    if (rc != SIM_OK) return rc;
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(h, SIM_E_IO, "sim_state_load: cannot open %s", path);
    StateFileHeader hd{};
    if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, "SYCSTATE", 8) != 0 ||
        hd.version != kStateFileVersion) {
        std::fclose(f);
        return fail(h, SIM_E_INVAL, "sim_state_load: %s is not a state file", path);
    }
    if (hd.n != h->n || hd.s != h->s || hd.amps != h->amps) {
        std::fclose(f);
        return fail(h, SIM_E_INVAL, "sim_state_load: the file holds n=%d, slice_bits=%d; the handle n=%d, slice_bits=%d",
                    hd.n, hd.s, h->n, h->s);
    }
    bool perm_ok = true;
    std::vector<char> seen(h->n, 0);
    for (int q = 0; q < h->n; q++) {
        const int b = hd.bit_of[q];
        perm_ok &= b >= 0 && b < h->n && !seen[b];
        if (b >= 0 && b < h->n) seen[b] = 1;
    }
    if (!perm_ok) {
        std::fclose(f);
        return fail(h, SIM_E_INVAL, "sim_state_load: corrupt layout in %s", path);
    }
    if (h->store == SIM_STORE_HOST) {  // the same sliced sets in the same places; the others may differ
        for (int w = 0; w < 2; w++)
            for (int i = 0; i < h->s; i++)
                if (hd.bit_of[h->set[w][i]] != h->bit_of[h->set[w][i]]) {
                    std::fclose(f);
                    return fail(h, SIM_E_INVAL,
                                "sim_state_load: the host store's layout (its sliced sets) differs from the file's");
                }
    }
    PinnedChunk buf;
    if (cudaHostAlloc(reinterpret_cast<void **>(&buf.p), kCkptChunk, cudaHostAllocDefault) != cudaSuccess) {
        buf.p = nullptr;
        std::fclose(f);
        return fail(h, SIM_E_NOMEM_HOST, "sim_state_load: staging buffer");
    }
    bool ok = true;
    for (auto &run : state_runs(h)) {
        char *dst = reinterpret_cast<char *>(run.first);
        cudaPointerAttributes at{};
        const bool on_device = cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        for (uint64_t off = 0, total = run.second * sizeof(float2); ok && off < total; off += kCkptChunk) {
            const size_t len = (size_t)std::min<uint64_t>(kCkptChunk, total - off);
            char *to = on_device ? buf.p : dst + off;
            ok = std::fread(to, 1, len, f) == len;
            if (ok && on_device && cudaMemcpy(dst + off, buf.p, len, cudaMemcpyHostToDevice) != cudaSuccess) {
                std::fclose(f);
                return fail(h, SIM_E_CUDA, "sim_state_load: %s", cudaGetErrorString(cudaGetLastError()));
            }
        }
    }
    std::fclose(f);
    if (!ok) return fail(h, SIM_E_IO, "sim_state_load: %s is truncated", path);
    if (h->store != SIM_STORE_HOST) {  // the state takes the file's layout
        for (int q = 0; q < h->n; q++) {
            h->bit_of[q] = hd.bit_of[q];
            h->qubit_at[hd.bit_of[q]] = q;
        }
    } else {
        int perm[kMaxQubits];
        std::copy(hd.bit_of, hd.bit_of + h->n, perm);
        host_store_relabel(h, perm);  // sets checked above
    }
    return SIM_OK;
}

using namespace sycsim;

extern "C" {

int sim_stream_slice(sim_t *h, int set, uint64_t value, int dir, int slot)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_stream_slice: NULL handle");
    state_written(h);
    if (h->store != SIM_STORE_HOST)
        return fail(h, SIM_E_UNSUPPORTED, "sim_stream_slice: handle has no host store");
    if (set < 0 || set > 1 || (dir != SIM_H2D && dir != SIM_D2H) || slot < 0 || slot >= h->nslots ||
        value >= (1ull << h->s))
        return fail(h, SIM_E_INVAL, "sim_stream_slice: set=%d value=%llu dir=%d slot=%d out of range",
                    set, (unsigned long long)value, dir, slot);
    SIM_DEVICE_SCOPE(h, h->device);
    return enqueue_slice_copy(h, set, value, dir, slot);
}

int sim_slot_ptr(const sim_t *h, int slot, void **dptr)
{
    if (!h || !dptr) return fail(nullptr, SIM_E_INVAL, "sim_slot_ptr: NULL argument");
    if (h->store != SIM_STORE_HOST || slot < 0 || slot >= h->nslots)
        return fail(nullptr, SIM_E_INVAL, "sim_slot_ptr: no slot %d", slot);
    *dptr = h->d_slot[slot];
    return SIM_OK;
}

int sim_slot_read(sim_t *h, int slot, uint64_t first, uint64_t count, void *out)
{
    if (!h || !out) return fail(nullptr, SIM_E_INVAL, "sim_slot_read: NULL argument");
    if (h->store != SIM_STORE_HOST || slot < 0 || slot >= h->nslots)
        return fail(h, SIM_E_INVAL, "sim_slot_read: no slot %d", slot);
    const uint64_t slice = 1ull << (h->n - h->s);
    if (first > slice || count > slice - first)
        return fail(h, SIM_E_INVAL, "sim_slot_read: range outside the slot");
    SIM_DEVICE_SCOPE(h, h->device);
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->st_in));
    SIM_CUDA_TRY(h, cudaMemcpyAsync(out, h->d_slot[slot] + first, sizeof(float2) * count,
                                    cudaMemcpyDeviceToHost, h->stream));
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SIM_OK;
}

int sim_run_phase(sim_t *h, int set, const sim_plan_t *p)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_run_phase: NULL handle");
    state_written(h);
    if (!p || p->n != h->n) return fail(h, SIM_E_INVAL, "sim_run_phase: plan missing or for another n");
    if (set < 0 || set > 1) return fail(h, SIM_E_INVAL, "sim_run_phase: set must be 0 (A) or 1 (B)");
    SIM_DEVICE_SCOPE(h, h->device);
    if (h->store != SIM_STORE_HOST) {
        // resident state: the phase's blocks apply to the whole state
        return sim_apply_plan(h, p);
    }
    return run_phase(h, set, p, nullptr);
}

}  // extern "C"

namespace sycsim {

// One phase over a host store: every slice of the sliced set goes through a device slot (or is
// computed in place, for a hybrid store's device regions with set A sliced), gets the plan's
// blocks (p may be NULL when fill is given) and is written back.  fill, when given, makes each
// slice instead of copying it in: (*fill)(dst, v) enqueues slice v of the sliced set into dst on
// the handle's stream, in the slot's layout, and the store is written without being read.
int run_phase(sim_t *h, int set, const sim_plan_t *p, const std::function<int(float2 *, uint64_t)> *fill)
{
    const int nl = h->n - h->s;
    struct Prepared {
        int k;
        int tpos[kMaxK];
        std::vector<float2> mat;
        size_t bytes = 0, off = 0;  // staged operands
    };
    std::vector<Prepared> blocks(p ? p->blocks.size() : 0);
    size_t staged_total = 0;
    for (size_t i = 0; i < blocks.size(); i++) {
        const PlanBlock &b = p->blocks[i];
        Prepared &pb = blocks[i];
        pb.k = (int)b.qubits.size();
        pb.mat.resize((size_t)1 << (2 * pb.k));
        int rc = prepare_block_map(h, pb.k, b.qubits.data(), b.mat.data(), h->slice_phys[set], nl,
                                   pb.tpos, pb.mat.data());
        if (rc != SIM_OK) return rc;
        pb.bytes = block_staged_bytes(nl, pb.k, pb.tpos, p->precision);
        pb.off = staged_total;
        staged_total += (pb.bytes + 255) & ~size_t(255);
    }
    // Every slice gets the same blocks: their tensor-core operands (and 6-qubit matrices) are
    // uploaded once for the phase, not once per block and slice -- such small copies would queue
    // behind the slice transfers on the copy engines and hold back every kernel.
    char *d_staged = nullptr;
    auto release = [&](int rc) {  // the staged operands go once the phase's last kernel is queued
        if (d_staged) cudaFreeAsync(d_staged, h->stream);
        return rc;
    };
    if (staged_total) {
        // pinned source, reused once its previous upload is done (no wait on the device's work)
        SIM_CUDA_TRY(h, cudaEventSynchronize(h->ev_ops));
        if (staged_total > h->h_ops_bytes) {
            if (h->h_ops) cudaFreeHost(h->h_ops);
            h->h_ops = nullptr;
            h->h_ops_bytes = 0;
            if (cudaHostAlloc(reinterpret_cast<void **>(&h->h_ops), 2 * staged_total, cudaHostAllocDefault) != cudaSuccess) {
                h->h_ops = nullptr;
                return fail(h, SIM_E_NOMEM_HOST, "sim_run_phase: staging buffer");
            }
            h->h_ops_bytes = 2 * staged_total;
        }
        for (const Prepared &pb : blocks)
            if (pb.bytes) block_build_staged(nl, pb.k, pb.tpos, pb.mat.data(), p->precision, h->h_ops + pb.off);
        if (cudaMallocAsync(reinterpret_cast<void **>(&d_staged), staged_total, h->stream) != cudaSuccess) {
            d_staged = nullptr;
            return fail(h, SIM_E_NOMEM_DEV, "sim_run_phase: staged operands");
        }
        cudaError_t e = cudaMemcpyAsync(d_staged, h->h_ops, staged_total, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_ops, h->stream);
        if (e != cudaSuccess)  // give the staging allocation back (stream-ordered) before failing
            return release(fail(h, SIM_E_CUDA, "sim_run_phase: operand upload: %s", cudaGetErrorString(e)));
    }
    auto apply_blocks = [&](float2 *psi) {
        for (const Prepared &pb : blocks) {
            const int ps = prof_begin(h, SIM_PROF_APPLY, 16.0 * std::ldexp(1.0, nl), h->stream);
            const int rc = launch_block_staged(h, psi, nl, pb.k, pb.tpos, pb.mat.data(), p->precision,
                                               d_staged + pb.off, h->stream);
            prof_end(h, ps, h->stream);
            if (rc != SIM_OK) return rc;
        }
        return (int)SIM_OK;
    };
    const uint64_t nsl = 1ull << h->s;
    // With set A sliced, a slice is one region of the store, laid out [rest | B] like a slot: the
    // regions in device memory are computed in place (no copies), interleaved with the host
    // slices so that host-link copies overlap that compute.  With set B sliced every slice
    // gathers a file from every region and goes through a slot.
    const bool inplace = set == 0 && h->host_regions < nsl;
    std::vector<uint64_t> order;
    if (fill) {
        // the slices are written without being read: every copy-in queued so far (earlier phases
        // reading the regions) must be done before the first write
        for (int i = 0; i < h->nslots; i++)
            if (cudaStreamWaitEvent(h->stream, h->ev_in[i], 0) != cudaSuccess)
                return release(fail(h, SIM_E_CUDA, "run_phase: event wait"));
    }
    if (inplace) {
        // the previous phase's copy-outs may have written into the device regions
        for (int i = 0; i < h->nslots; i++)
            if (cudaStreamWaitEvent(h->stream, h->ev_out[i], 0) != cudaSuccess) return release(fail(h, SIM_E_CUDA, "sim_run_phase: event wait"));
        for (uint64_t i = 0; i < nsl; i++) {
            if (h->host_regions + i < nsl) order.push_back(h->host_regions + i);  // a device region
            if (i < h->host_regions) order.push_back(i);
        }
    } else {
        for (uint64_t v = 0; v < nsl; v++) order.push_back(v);
    }
    int next_slot = 0;
    for (const uint64_t v : order) {
        if (inplace && v >= h->host_regions) {
            int rc = fill ? (*fill)(region(h, v), v) : (int)SIM_OK;
            if (rc == SIM_OK) rc = apply_blocks(region(h, v));
            if (rc != SIM_OK) return release(rc);
            continue;
        }
        const int slot = next_slot;
        next_slot = (next_slot + 1) % h->nslots;
        int rc;
        if (fill) {  // the slot's previous slice must have left it
            if (cudaStreamWaitEvent(h->stream, h->ev_out[slot], 0) != cudaSuccess)
                return release(fail(h, SIM_E_CUDA, "run_phase: event wait"));
            rc = (*fill)(h->d_slot[slot], v);
        } else {
            rc = enqueue_slice_copy(h, set, v, SIM_H2D, slot);
        }
        if (rc != SIM_OK) return release(rc);
        if ((rc = apply_blocks(h->d_slot[slot])) != SIM_OK) return release(rc);
        rc = enqueue_slice_copy(h, set, v, SIM_D2H, slot);
        if (rc != SIM_OK) return release(rc);
    }
    release(SIM_OK);
    // copy-ins from now on (the next phase reads every region) follow the in-place computes; this
    // phase's own copy-ins read host regions only and did not wait for them
    if (inplace) SIM_CUDA_TRY(h, cudaEventRecord(h->ev_inplace, h->stream));
    // later work on the handle's stream (and sim_sync) follows the last copy-out
    for (int i = 0; i < h->nslots; i++) SIM_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_out[i], 0));
    return SIM_OK;
}

}  // namespace sycsim

extern "C" int sim_contract_phase(sim_t *out, sim_t *t1, sim_t *t2, const sim_split_t *s, int precision, int set,
                                  const sim_plan_t *p)
{
    if (!out || !t1 || !t2 || !s) return fail(out, SIM_E_INVAL, "sim_contract_phase: NULL argument");
    if (out->store != SIM_STORE_HOST) {  // a resident state: the contraction, then the blocks
        if (set < 0 || set > 1) return fail(out, SIM_E_INVAL, "sim_contract_phase: set must be 0 (A) or 1 (B)");
        int rc = sim_contract(out, t1, t2, s, precision);
        if (rc == SIM_OK && p) rc = sim_apply_plan(out, p);
        return rc;
    }
    state_written(out);
    if (out == t1 || out == t2 || t1 == t2)
        return fail(out, SIM_E_INVAL, "sim_contract_phase: handles must be distinct");
    if (precision != SIM_FP32 && precision != SIM_FP16X3 && precision != SIM_FP16X3_TMEM && precision != SIM_BF16X3)
        return fail(out, SIM_E_INVAL, "sim_contract_phase: precision %d is not SIM_FP32, SIM_FP16X3, "
                                      "SIM_FP16X3_TMEM or SIM_BF16X3", precision);
    if (set < 0 || set > 1) return fail(out, SIM_E_INVAL, "sim_contract_phase: set must be 0 (A) or 1 (B)");
    if (p && p->n != out->n) return fail(out, SIM_E_INVAL, "sim_contract_phase: plan for another n");
    if (p)
        for (const PlanBlock &b : p->blocks)
            for (int q : b.qubits)
                if (out->slice_phys[set][q] < 0)
                    return fail(out, SIM_E_NONLOCAL, "sim_contract_phase: the plan acts on qubit %d of the sliced set", q);
    const int n1 = s->n_side[0], n2 = s->n_side[1], e_bits = 2 * s->n_pairs;
    for (sim_t *h : {t1, t2})
        if (h->store != SIM_STORE_DEVICE || h->s != 0 || !h->d_state)
            return fail(out, SIM_E_INVAL, "sim_contract_phase: the tensors must be device-resident and not sliced");
    if (t1->device != out->device || t2->device != out->device)
        return fail(out, SIM_E_INVAL, "sim_contract_phase: handles on different devices");
    if (out->n != s->n || t1->n != n1 + e_bits || t2->n != n2 + e_bits)
        return fail(out, SIM_E_INVAL, "sim_contract_phase: qubit counts (%d, %d, %d) do not fit the split (%d, %d, %d)",
                    out->n, t1->n, t2->n, s->n, n1 + e_bits, n2 + e_bits);
    SIM_DEVICE_SCOPE(out, out->device);
    // the sliced set selects the slice: the slice is written in store_fill_layout's layout, where
    // that set sits highest, so contract_layout puts its qubits on each tensor's top side bits; bit
    // i of a slice's value is the set's i-th qubit, bit r of a side's fixed value its r-th qubit of
    // the set
    int olay[kMaxQubits];
    store_fill_layout(out, set, olay);
    int top[2] = {0, 0}, side_of[8] = {}, rank_of[8] = {};
    for (int i = 0; i < out->s; i++) {
        side_of[i] = s->side[out->set[set][i]];
        rank_of[i] = top[side_of[i]]++;
    }
    sim_t *tens[2] = {t1, t2};
    for (int t = 0; t < 2; ++t) {
        sim_t *h = tens[t];
        if (!contract_ready(s, olay, t, h->bit_of, top[t])) {
            int perm[kMaxQubits];
            contract_layout(s, olay, t, perm, nullptr);
            const int rc = sim_permute(h, perm);
            if (rc != SIM_OK)
                return fail(out, rc, "sim_contract_phase: permuting tensor %d: %s", t + 1, h->err.c_str());
        }
    }
    cudaEvent_t ev[3] = {};
    for (auto &e : ev) SIM_CUDA_TRY(out, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    auto finish = [&](int rc) {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        return rc;
    };
    if (cudaEventRecord(ev[0], t1->stream) != cudaSuccess || cudaEventRecord(ev[1], t2->stream) != cudaSuccess ||
        cudaStreamWaitEvent(out->stream, ev[0], 0) != cudaSuccess ||
        cudaStreamWaitEvent(out->stream, ev[1], 0) != cudaSuccess)
        return finish(fail(out, SIM_E_CUDA, "sim_contract_phase: stream ordering failed"));
    const int *tbits[2] = {t1->bit_of, t2->bit_of};
    ContractJob job;
    if (contract_job_prepare(out, s, t1->d_state, t2->d_state, tbits, olay, precision, top, nullptr, out->stream,
                             &job) != 0)
        return finish(fail(out, SIM_E_CUDA, "sim_contract_phase: operand images: %s",
                           cudaGetErrorString(cudaGetLastError())));
    const std::function<int(float2 *, uint64_t)> fill = [&](float2 *dst, uint64_t v) {
        uint64_t fix[2] = {0, 0};
        for (int i = 0; i < out->s; i++) fix[side_of[i]] |= ((v >> i) & 1ull) << rank_of[i];
        if (contract_job_launch(out, job, dst, fix[0], fix[1], out->stream) != 0)
            return fail(out, SIM_E_CUDA, "sim_contract_phase: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return (int)SIM_OK;
    };
    const int rc = run_phase(out, set, p, &fill);
    // the tensors stay untouched until the last slice has been contracted
    if (cudaEventRecord(ev[2], out->stream) != cudaSuccess || cudaStreamWaitEvent(t1->stream, ev[2], 0) != cudaSuccess ||
        cudaStreamWaitEvent(t2->stream, ev[2], 0) != cudaSuccess)
        return finish(rc != SIM_OK ? rc : fail(out, SIM_E_CUDA, "sim_contract_phase: stream ordering failed"));
    return finish(rc);
}
