// serve.cu -- continuous-batching server for many circuits on one GPU (no counterpart in the
// paper, which simulates one circuit; it reuses the paper's per-circuit path: aggregation,
// Sect. 5, and the fused-block apply).
//
// Requests arrive through srv_submit from any thread.  The caller's thread validates the gate
// list, plans it (aggregation) and rounds the block matrices, so planning runs in parallel
// with the GPU.  One scheduler thread then:
//  * admits requests in arrival order while their device footprint (8 * 2^n bytes plus
//    scratch) fits the HBM budget; a request that does not fit may be overtaken by smaller
//    ones at most kMaxBypass times, after which admission waits for it (no starvation);
//  * runs small circuits (n <= small_n) through a device-side queue served by a persistent
//    worker kernel (k_packed_worker): one CTA runs one whole circuit -- reset, every block, the
//    reduction -- with the block matrix in shared memory; circuits are uploaded in units, published
//    to the queue, claimed by idle CTAs of a worker already running (or of a new one when the
//    running workers have fewer CTAs than jobs waiting), and a worker leaves after 200 us without
//    new work, so small circuits that arrive while others run start without a new launch;
//  * runs larger circuits on one of several slot streams with stream-ordered allocation, so
//    circuits of different sizes overlap on the device; their blocks are enqueued a few at a
//    time, as far as the slot's matrix-staging ring has free slots, so the scheduler never
//    waits on device progress;
//  * detects completion by polling events, frees memory and budget, and wakes waiters.
// Results (norm, 2^n sum p^2, XEB; optionally all amplitudes into the caller's buffer) and
// latencies (submit -> completion seen) are recorded; srv_stats reports p50/p99 and circuits/s.
// The same circuit always takes the same path and the same plan, so its result does not depend
// on what else is being served.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace sycsim {
namespace {

using Clock = std::chrono::steady_clock;

struct PackedBlock {
    int k;
    int tpos[kMaxK];
    uint32_t mat_off;  // float2 offset of the block's matrix in the batch's matrix table
};

struct PackedJob {
    float2 *psi;
    const PackedBlock *blocks;
    const float2 *mats;
    double *out;  // [sum p, sum p^2]
    int n, nblocks;
};

constexpr int kPackThreads = 256;
constexpr int kPackMaxK = 5;

__device__ __forceinline__ uint64_t insert_zero_bits_s(uint64_t x, const int *pos, int cnt)
{
    for (int i = 0; i < cnt; ++i) {
        const int p = pos[i];
        const uint64_t lo = x & ((1ull << p) - 1);
        x = ((x >> p) << (p + 1)) | lo;
    }
    return x;
}

template <int K>
__device__ __forceinline__ void cta_block(float2 *psi, int n, const int *tpos, const float2 *M,
                                          const uint32_t *moff)
{
    constexpr int D = 1 << K;
    const uint64_t ngroups = 1ull << (n - K);
    for (uint64_t gi = threadIdx.x; gi < ngroups; gi += blockDim.x) {
        float2 *p = psi + insert_zero_bits_s(gi, tpos, K);
        float2 x[D];
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = p[moff[j]];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float yr = 0.f, yi = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float2 m = M[r * D + c];
                yr = fmaf(m.x, x[c].x, yr);
                yr = fmaf(m.y, -x[c].y, yr);
                yi = fmaf(m.x, x[c].y, yi);
                yi = fmaf(m.y, x[c].x, yi);
            }
            p[moff[r]] = make_float2(yr, yi);
        }
    }
}

struct PackShared {
    float2 M[32 * 32];
    uint32_t moff[32];
    int tpos[kMaxK];
    double red[2][kPackThreads / 32];
};

// One whole small circuit on one CTA: reset to |0...0>, every block with its matrix in shared
// memory, then (sum p, sum p^2) into out[0..1].
__device__ void run_circuit_cta(const PackedJob &J, PackShared &sh, double *out)
{
    float2 *M = sh.M;
    uint32_t *moff = sh.moff;
    int *tpos = sh.tpos;
    const uint64_t amps = 1ull << J.n;
    for (uint64_t i = threadIdx.x; i < amps; i += blockDim.x) J.psi[i] = make_float2(0.f, 0.f);
    __syncthreads();
    if (threadIdx.x == 0) J.psi[0] = make_float2(1.f, 0.f);
    for (int b = 0; b < J.nblocks; ++b) {
        const PackedBlock B = J.blocks[b];
        const int D = 1 << B.k;
        __syncthreads();  // previous block done with M, psi and tpos
        for (int i = threadIdx.x; i < D * D; i += blockDim.x) M[i] = J.mats[B.mat_off + i];
        if (threadIdx.x < D) {
            uint32_t o = 0;
            for (int q = 0; q < B.k; ++q)
                if ((threadIdx.x >> q) & 1) o += 1u << B.tpos[q];
            moff[threadIdx.x] = o;
        }
        if (threadIdx.x < kMaxK) tpos[threadIdx.x] = B.tpos[threadIdx.x];
        __syncthreads();
        switch (B.k) {
        case 1: cta_block<1>(J.psi, J.n, tpos, M, moff); break;
        case 2: cta_block<2>(J.psi, J.n, tpos, M, moff); break;
        case 3: cta_block<3>(J.psi, J.n, tpos, M, moff); break;
        case 4: cta_block<4>(J.psi, J.n, tpos, M, moff); break;
        default: cta_block<5>(J.psi, J.n, tpos, M, moff); break;
        }
    }
    __syncthreads();
    double s1 = 0.0, s2 = 0.0;
    for (uint64_t i = threadIdx.x; i < amps; i += blockDim.x) {
        const float2 v = J.psi[i];
        const double p = (double)v.x * v.x + (double)v.y * v.y;
        s1 += p;
        s2 += p * p;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh.red[0][warp] = s1;
        sh.red[1][warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < kPackThreads / 32; ++w) {
            a += sh.red[0][w];
            c += sh.red[1][w];
        }
        out[0] = a;
        out[1] = c;
    }
}

// The packed jobs' queue, shared by the host and the worker kernel: entries in mapped pinned host
// memory (the host writes a descriptor, the device its results and done flag), a published count
// the host raises after writing descriptors, and a claim counter in device memory.
struct QSlot {
    PackedJob job;
    double res[2];
    uint32_t done;
    uint32_t pad;
};
constexpr uint32_t kQueueCap = 4096;
constexpr uint64_t kWorkerIdleNs = 200000;  // a worker CTA leaves after 200 us without a new job

__device__ __forceinline__ uint64_t pack_now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Persistent worker: each CTA claims the next published job (compare-and-swap on the claim
// counter, so no claimed index is ever abandoned), runs it, publishes its results and done flag,
// and looks for the next one; it leaves once no job has been published for kWorkerIdleNs.  Jobs
// published while the kernel runs are picked up without a new launch.  The only wait is on the
// host's published count, bounded by the idle time.
__global__ void __launch_bounds__(kPackThreads) k_packed_worker(const uint32_t *published, QSlot *ring, uint32_t *head)
{
    __shared__ PackShared sh;
    __shared__ PackedJob J;
    __shared__ uint32_t job;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t got = 0xffffffffu;
            const uint64_t t0 = pack_now_ns();
            for (;;) {
                const uint32_t p = ld_acquire_sys(published);
                const uint32_t h = atomicAdd(head, 0u);
                if (h < p) {
                    if (atomicCAS(head, h, h + 1) == h) {
                        got = h;
                        break;
                    }
                    continue;
                }
                if (pack_now_ns() - t0 > kWorkerIdleNs) break;
                __nanosleep(1000);
            }
            job = got;
            if (got != 0xffffffffu) J = ring[got % kQueueCap].job;
        }
        __syncthreads();
        if (job == 0xffffffffu) break;
        QSlot *slot = ring + job % kQueueCap;
        run_circuit_cta(J, sh, slot->res);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence_system();  // results visible to the host before the flag
            asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(&slot->done), "r"(1u) : "memory");
        }
        __syncthreads();  // job and J are rewritten by the next claim
    }
}

struct Prepared {
    int k;
    int tpos[kMaxK];
    std::vector<float2> mat;
};

// A circuit submitted more than once (not packed, up to kGraphMaxQubits, no contraction front):
// a handle holding its state in the layout the server chose for it and its plan captured once as a
// CUDA graph (sim_graph_create); each repeat replays the graph there, one at a time.  The same
// kernels, layout, reduction and readout as the stream path, so the results are bit-identical.
struct GraphEntry {
    sim_t *h = nullptr;
    sim_plan_t *plan = nullptr;
    sim_graph_t *g = nullptr;
    std::vector<int> back;  // physical bit -> logical qubit for the readout (empty: identity)
    uint64_t bytes = 0;     // device memory held (reserved from the budget)
    bool busy = false;
};

struct Req {
    uint64_t ticket = 0;
    int n = 0;
    int precision = SIM_FP32;
    bool packed = false;
    void *out_amps = nullptr;
    std::vector<Prepared> blocks;
    std::vector<int> back;  // unpacked: the permutation from the chosen layout back to the identity
    uint64_t bytes = 0;     // admission footprint
    // contraction deferral (unpacked): blocks[0 .. nt[0]) run on tensor 1, the next nt[1] on
    // tensor 2, then the contraction writes the state (layout out_bit_of) and the rest follow
    std::shared_ptr<sim_split_s> split;
    int nt[2] = {0, 0}, nw[2] = {0, 0};
    std::vector<int> out_bit_of;
    std::vector<int> t_lay[2];  // each tensor's layout (front_tensor_layout)
    float2 *d_t[2] = {nullptr, nullptr};
    uint8_t *d_scratch = nullptr;
    bool contracted = false;
    Clock::time_point t_submit, t_done;
    int status = 1;  // 1 pending, 0 ok, < 0 error
    double norm = 0.0, s2 = 0.0;
    int bypassed = 0;
    std::shared_ptr<GraphEntry> graph;  // repeated circuit: replay this entry's graph
    // in flight (unpacked)
    int slot = -1;
    float2 *d_state = nullptr;
    size_t next_block = 0;   // blocks enqueued so far
    bool launched = false;   // everything enqueued and ev recorded
    cudaEvent_t ev = nullptr;
    double *h_res = nullptr;  // pinned pair
};

// A unit of small circuits on their way through the worker queue: uploaded together (states and
// tables in one stream-ordered allocation), published to the queue once the upload is done, their
// amplitudes copied out once every job's done flag is set, retired after that copy.
struct Batch {
    enum State { Free, Uploading, Running, CopyingOut };
    std::vector<std::shared_ptr<Req>> jobs;
    std::vector<double> res;        // (sum p, sum p^2) per job, taken from the queue
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;       // upload done, then copy-out done
    void *d_mem = nullptr;          // states + tables, one stream-ordered allocation
    char *h_stage = nullptr;        // pinned copy source of the tables
    size_t stage_bytes = 0;
    uint64_t first = 0;             // queue index of the first job
    State state = Free;
};

constexpr int kMaxBypass = 64;
constexpr int kFrontMinQubits = 26;      // smaller states: the passes a front saves are too short
constexpr double kFrontMinShare = 0.3;   // a front with fewer of the gates is not worth a contraction
constexpr int kFp32FrontPairs = 2;       // FP32 fronts: their contraction (CUDA cores) grows 4x a pair
constexpr double kFp32FrontMinShare = 0.1;
constexpr int kSrvPlanSearch = 1;  // requests are planned on the submitting thread: the greedy
                                   // schedule (a beam search adds milliseconds a circuit)
constexpr int kResultRing = 1 << 16;
constexpr int kGraphMaxQubits = 24;  // graph entries hold their own state: 8 * 2^24 bytes at most
constexpr int kGraphMaxEntries = 8;
constexpr int kLargeQubits = 27;  // "large" for srv_opts.max_large

}  // namespace
}  // namespace sycsim

using namespace sycsim;

struct srv_s {
    srv_opts o{};
    uint64_t budget = 0, used = 0;
    int max_large = 0;  // most large circuits at once (0: no limit)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
    uint64_t next_ticket = 1;
    std::vector<sim_t *> slots;
    std::vector<std::shared_ptr<Req>> slot_req;
    std::vector<Batch> batches;
    // repeated circuits (CUDA graphs): gate-list hash -> entry; hashes seen once
    std::mutex graph_mu;
    std::unordered_map<uint64_t, std::shared_ptr<GraphEntry>> graphs;
    std::unordered_map<uint64_t, int> seen;
    std::vector<std::shared_ptr<Req>> graph_inflight;
    // the packed jobs' queue (see k_packed_worker): ring entries in mapped pinned memory, the
    // published count beside them, the claim counter in device memory, up to two workers in flight
    QSlot *ring = nullptr, *d_ring = nullptr;
    uint32_t *ctl = nullptr, *d_ctl = nullptr;  // ctl[0]: published count
    uint32_t *d_head = nullptr;
    uint64_t next_index = 0, published = 0, retired = 0;
    cudaStream_t wst[2] = {nullptr, nullptr};
    cudaEvent_t wev[2] = {nullptr, nullptr};
    int wctas[2] = {0, 0};  // CTAs of a worker still running (0: none)
    int sms = 0;
    double *h_results = nullptr;  // pinned ring of result pairs for unpacked requests
    std::thread worker;
    bool stop = false;
    std::string err;
    // autotuned choices for circuits above small_n (srv_autotune): (n, gates-per-qubit bucket) ->
    // block width and whether the contraction-deferral front runs
    struct Tune {
        int kmax = 0, front = 0;
        double ms = 0.0;
    };
    std::map<std::pair<int, int>, Tune> tune;
    std::mutex tune_mu;
    // stats
    uint64_t submitted = 0, completed = 0, rejected = 0, graph_replays = 0;
    std::vector<double> lat_ms;
    Clock::time_point t_first, t_last;
    bool any_done = false;
};

namespace {

int srv_fail(srv_t *s, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s)
        s->err = buf;
    else
        set_thread_error("%s", buf);
    return code;
}

// kmax by size: launch-bound small and mid-size states gain from fewer, wider blocks;
// HBM-bound large states from the width whose pass stays HBM-bound on CUDA cores (4) or on the
// tensor cores: 6 with tcgen05 (its 6-qubit pass costs 1.05-1.15 times a 5-qubit one and saves a
// quarter of the passes on 30-qubit circuits, once the layout keeps low targets out of them), 5
// with the mma.sync arithmetic.
// Depth class of a circuit for the autotuner's cache: gates per qubit, which for these circuits
// is about 1.4 cycles + 1 (8-12 cycles: < 18, 12-16: < 24, deeper: the rest).
int depth_bucket(int n_qubits, int n_gates)
{
    const int r = n_gates / std::max(n_qubits, 1);
    return r < 18 ? 0 : (r < 24 ? 1 : 2);
}

int auto_kmax(int n, bool packed, int precision)
{
    if (packed) return 5;
    if (tmem_mode(precision)) return 6;
    if (precision != SIM_FP32) return 5;
    return n <= 24 ? 5 : 4;
}

void finish(srv_t *s, const std::shared_ptr<Req> &r, int status, double a, double b)
{
    r->status = status;
    r->norm = a;
    r->s2 = b;
    r->t_done = Clock::now();
    s->used -= r->bytes;
    s->completed++;
    const double ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    s->lat_ms.push_back(ms);
    if (!s->any_done || r->t_done > s->t_last) s->t_last = r->t_done;
    s->any_done = true;
}

// Start one unpacked request on slot i (scheduler thread, lock held): state and |0...0>.
int start_unpacked(srv_t *s, int i, const std::shared_ptr<Req> &r)
{
    sim_t *h = s->slots[i];
    cudaStream_t st = h->stream;
    const uint64_t amps = 1ull << r->n;
    r->slot = i;
    r->next_block = 0;
    r->launched = false;
    s->slot_req[i] = r;
    r->contracted = false;
    if (cudaMallocAsync(&r->d_state, sizeof(float2) * amps, st) != cudaSuccess) {
        r->d_state = nullptr;
        return SIM_E_NOMEM_DEV;
    }
    if (r->split) {  // the two tensors from |0...0>; the contraction will write every amplitude
        for (int t = 0; t < 2; ++t) {
            const uint64_t ta = 1ull << r->nw[t];
            if (cudaMallocAsync(&r->d_t[t], sizeof(float2) * ta, st) != cudaSuccess) {
                r->d_t[t] = nullptr;
                return SIM_E_NOMEM_DEV;
            }
            if (cudaMemsetAsync(r->d_t[t], 0, sizeof(float2) * ta, st) != cudaSuccess) return SIM_E_CUDA;
            if (launch_set_basis(r->d_t[t], ta, 0, st) != 0) return SIM_E_CUDA;
        }
        if (cudaMallocAsync(reinterpret_cast<void **>(&r->d_scratch), contraction_scratch_bytes(r->split.get()), st) !=
            cudaSuccess) {
            r->d_scratch = nullptr;
            return SIM_E_NOMEM_DEV;
        }
        return SIM_OK;
    }
    if (cudaMemsetAsync(r->d_state, 0, sizeof(float2) * amps, st) != cudaSuccess) return SIM_E_CUDA;
    if (launch_set_basis(r->d_state, amps, 0, st) != 0) return SIM_E_CUDA;
    return SIM_OK;
}

// Enqueue as many of the request's blocks as go without waiting for a matrix-staging slot (the
// slot of a tensor-core block is free once the kernel that last read it has run), then, after
// the last block, the reduction, the copies out and the completion event.  Never blocks the
// scheduler on device progress.  *progressed is set if anything was enqueued.
int advance_unpacked(srv_t *s, const std::shared_ptr<Req> &r, bool *progressed)
{
    sim_t *h = s->slots[r->slot];
    cudaStream_t st = h->stream;
    const uint64_t amps = 1ull << r->n;
    const size_t tensor_blocks = (size_t)r->nt[0] + r->nt[1];
    auto contract = [&]() {  // after both tensors' blocks: the state from the two tensors
        const int *tbits[2] = {r->t_lay[0].data(), r->t_lay[1].data()};
        if (enqueue_contraction(h, r->split.get(), r->d_t[0], r->d_t[1], r->d_state, r->out_bit_of.data(),
                                r->precision, r->d_scratch, st, tbits) != 0)
            return SIM_E_CUDA;
        // each pointer is dropped before its status is checked: after a failed free, the abort
        // path must not free it again
        bool freed = true;
        for (auto &p : r->d_t) {
            freed &= cudaFreeAsync(p, st) == cudaSuccess;
            p = nullptr;
        }
        freed &= cudaFreeAsync(r->d_scratch, st) == cudaSuccess;
        r->d_scratch = nullptr;
        if (!freed) return SIM_E_CUDA;
        r->contracted = true;
        *progressed = true;
        return SIM_OK;
    };
    while (r->next_block < r->blocks.size()) {
        if (r->split && !r->contracted && r->next_block == tensor_blocks) {
            const int rc = contract();
            if (rc != SIM_OK) return rc;
        }
        const Prepared &b = r->blocks[r->next_block];
        const int t = r->next_block < (size_t)r->nt[0] ? 0 : (r->next_block < tensor_blocks ? 1 : -1);
        float2 *buf = t < 0 || !r->split ? r->d_state : r->d_t[t];
        const int nbits = t < 0 || !r->split ? r->n : r->nw[t];
        if (!staging_slot_free(h, nbits, b.k, b.tpos, r->precision)) return SIM_OK;
        const int rc = enqueue_block_on(h, buf, nbits, b.k, b.tpos, b.mat.data(), r->precision, st);
        if (rc != SIM_OK) return rc;
        r->next_block++;
        *progressed = true;
    }
    if (r->split && !r->contracted) {
        const int rc = contract();
        if (rc != SIM_OK) return rc;
    }
    if (launch_reduce(h, r->d_state, amps, h->d_partials, h->d_result, st) != 0) return SIM_E_CUDA;
    if (cudaMemcpyAsync(r->h_res, h->d_result, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SIM_E_CUDA;
    if (r->out_amps && !r->back.empty() && launch_permute(h, r->d_state, r->n, r->back.data(), st) != 0)
        return SIM_E_CUDA;  // amplitudes leave in logical order
    if (r->out_amps &&
        cudaMemcpyAsync(r->out_amps, r->d_state, sizeof(float2) * amps, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SIM_E_CUDA;
    const cudaError_t fe = cudaFreeAsync(r->d_state, st);
    r->d_state = nullptr;  // not freed twice by the abort path
    if (fe != cudaSuccess) return SIM_E_CUDA;
    if (cudaEventRecord(r->ev, st) != cudaSuccess) return SIM_E_CUDA;
    r->launched = true;
    *progressed = true;
    return SIM_OK;
}

// A request on slot i failed before its completion event was recorded: release what it holds.
void abort_unpacked(srv_t *s, int i, int rc)
{
    auto r = s->slot_req[i];
    cudaStream_t st = s->slots[i]->stream;
    if (r->d_state) cudaFreeAsync(r->d_state, st);
    r->d_state = nullptr;
    for (auto &p : r->d_t)
        if (p) cudaFreeAsync(p, st), p = nullptr;
    if (r->d_scratch) cudaFreeAsync(r->d_scratch, st);
    r->d_scratch = nullptr;
    s->slot_req[i].reset();
    finish(s, r, rc, 0.0, 0.0);
    s->cv_done.notify_all();
}

// Upload one unit of small requests (scheduler thread, lock held): tables and states in one
// stream-ordered allocation, the tables copied from pinned staging, the queue descriptors written
// (published later, once the upload is done: the worker may then run them at once).
int upload_packed(srv_t *s, Batch &B)
{
    size_t nblk = 0, nmat = 0, state_amps = 0;
    for (auto &r : B.jobs) {
        nblk += r->blocks.size();
        for (auto &b : r->blocks) nmat += b.mat.size();
        state_amps += 1ull << r->n;
    }
    const size_t nj = B.jobs.size();
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t off_blk = 0, off_mat = align(off_blk + nblk * sizeof(PackedBlock));
    const size_t off_state = align(off_mat + nmat * sizeof(float2));
    const size_t table_bytes = off_state;
    const size_t total = off_state + state_amps * sizeof(float2);
    if (B.stage_bytes < table_bytes) {
        if (B.h_stage) cudaFreeHost(B.h_stage);
        B.h_stage = nullptr;
        B.stage_bytes = 0;  // a failed allocation leaves no buffer behind
        if (cudaHostAlloc(&B.h_stage, table_bytes * 2, cudaHostAllocDefault) != cudaSuccess) {
            B.h_stage = nullptr;
            return SIM_E_NOMEM_HOST;
        }
        B.stage_bytes = table_bytes * 2;
    }
    if (cudaMallocAsync(&B.d_mem, total, B.st) != cudaSuccess) {
        B.d_mem = nullptr;
        return SIM_E_NOMEM_DEV;
    }
    struct ReleaseOnError {  // an early return below gives the allocation back (stream-ordered)
        Batch &b;
        bool armed = true;
        ~ReleaseOnError()
        {
            if (armed && b.d_mem) cudaFreeAsync(b.d_mem, b.st);
            if (armed) b.d_mem = nullptr;
        }
    } release_on_error{B};
    char *d = (char *)B.d_mem;
    PackedBlock *hb = (PackedBlock *)(B.h_stage + off_blk);
    float2 *hm = (float2 *)(B.h_stage + off_mat);
    size_t bi = 0, mi = 0, si = 0;
    B.first = s->next_index;
    for (size_t j = 0; j < nj; j++) {
        auto &r = B.jobs[j];
        QSlot &q = s->ring[(B.first + j) % kQueueCap];
        q.job.psi = (float2 *)(d + off_state) + si;
        q.job.blocks = (const PackedBlock *)(d + off_blk) + bi;
        q.job.mats = (const float2 *)(d + off_mat);
        q.job.out = nullptr;
        q.job.n = r->n;
        q.job.nblocks = (int)r->blocks.size();
        q.res[0] = q.res[1] = 0.0;
        q.done = 0;
        for (auto &b : r->blocks) {
            PackedBlock &pb = hb[bi++];
            pb.k = b.k;
            for (int t = 0; t < kMaxK; t++) pb.tpos[t] = t < b.k ? b.tpos[t] : 0;
            pb.mat_off = (uint32_t)mi;
            std::memcpy(hm + mi, b.mat.data(), b.mat.size() * sizeof(float2));
            mi += b.mat.size();
        }
        si += 1ull << r->n;
    }
    if (cudaMemcpyAsync(d, B.h_stage, table_bytes, cudaMemcpyHostToDevice, B.st) != cudaSuccess) return SIM_E_CUDA;
    if (cudaEventRecord(B.ev, B.st) != cudaSuccess) return SIM_E_CUDA;
    s->next_index += nj;
    B.res.assign(2 * nj, 0.0);
    B.state = Batch::Uploading;
    release_on_error.armed = false;
    return SIM_OK;
}

// After its jobs are done: each requested amplitude vector copied out, the allocation freed, the
// event recorded (scheduler thread, lock held).
int copy_out_packed(Batch &B)
{
    size_t si = 0;
    const char *d = (const char *)B.d_mem;
    size_t nblk = 0, nmat = 0;
    for (auto &r : B.jobs) {
        nblk += r->blocks.size();
        for (auto &b : r->blocks) nmat += b.mat.size();
    }
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t off_state = align(align(nblk * sizeof(PackedBlock)) + nmat * sizeof(float2));
    int rc = SIM_OK;
    for (auto &r : B.jobs) {
        if (r->out_amps && rc == SIM_OK &&
            cudaMemcpyAsync(r->out_amps, (const float2 *)(d + off_state) + si, sizeof(float2) << r->n,
                            cudaMemcpyDeviceToHost, B.st) != cudaSuccess)
            rc = SIM_E_CUDA;
        si += 1ull << r->n;
    }
    if (cudaFreeAsync(B.d_mem, B.st) != cudaSuccess) rc = SIM_E_CUDA;
    B.d_mem = nullptr;
    if (cudaEventRecord(B.ev, B.st) != cudaSuccess) rc = SIM_E_CUDA;
    B.state = Batch::CopyingOut;
    return rc;
}

// Jobs published and not yet seen done; launch a worker when they outnumber the CTAs of the
// workers still running (scheduler thread, lock held).
void manage_workers(srv_t *s, uint64_t not_done, bool *progressed)
{
    int running = 0;
    for (int w = 0; w < 2; w++) {
        if (s->wctas[w] && cudaEventQuery(s->wev[w]) != cudaErrorNotReady) s->wctas[w] = 0;
        running += s->wctas[w];
    }
    if (not_done <= (uint64_t)running) return;
    for (int w = 0; w < 2; w++)
        if (!s->wctas[w]) {
            const int ctas = (int)std::min<uint64_t>(not_done - running, (uint64_t)(2 * s->sms));
            k_packed_worker<<<ctas, kPackThreads, 0, s->wst[w]>>>(s->d_ctl, s->d_ring, s->d_head);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(s->wev[w], s->wst[w]) != cudaSuccess) return;
            s->wctas[w] = ctas;
            *progressed = true;
            return;
        }
}

// Replay a repeated circuit's graph on its entry's handle (scheduler thread, lock held): reset,
// the plan's blocks, the reduction and the readout, all enqueued on the entry's stream.
int start_graph(srv_t *s, const std::shared_ptr<Req> &r)
{
    GraphEntry &E = *r->graph;
    sim_t *h = E.h;
    cudaStream_t st = h->stream;
    if (sim_reset(h, 0) != SIM_OK || sim_graph_launch(h, E.g) != SIM_OK) return SIM_E_CUDA;
    if (launch_reduce(h, h->d_state, h->amps, h->d_partials, h->d_result, st) != 0) return SIM_E_CUDA;
    if (cudaMemcpyAsync(r->h_res, h->d_result, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SIM_E_CUDA;
    if (r->out_amps && !E.back.empty() && launch_permute(h, h->d_state, r->n, E.back.data(), st) != 0)
        return SIM_E_CUDA;  // amplitudes leave in logical order (the next replay resets the state)
    if (r->out_amps &&
        cudaMemcpyAsync(r->out_amps, h->d_state, sizeof(float2) << r->n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SIM_E_CUDA;
    if (cudaEventRecord(r->ev, st) != cudaSuccess) return SIM_E_CUDA;
    (void)s;
    return SIM_OK;
}

void scheduler(srv_t *s)
{
    cudaSetDevice(s->o.device);
    std::vector<std::shared_ptr<Req>> pack_pending;
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progressed = false;
        // completions: graph replays
        for (auto it = s->graph_inflight.begin(); it != s->graph_inflight.end();) {
            auto r = *it;
            const cudaError_t e = cudaEventQuery(r->ev);
            if (e == cudaErrorNotReady) {
                ++it;
                continue;
            }
            finish(s, r, e == cudaSuccess ? SIM_OK : SIM_E_CUDA, r->h_res[0], r->h_res[1]);
            r->graph->busy = false;
            it = s->graph_inflight.erase(it);
            progressed = true;
        }
        // completions: unpacked slots
        for (size_t i = 0; i < s->slots.size(); i++) {
            auto &r = s->slot_req[i];
            if (!r || !r->launched) continue;
            const cudaError_t e = cudaEventQuery(r->ev);
            if (e == cudaErrorNotReady) continue;
            finish(s, r, e == cudaSuccess ? SIM_OK : SIM_E_CUDA, r->h_res[0], r->h_res[1]);
            r.reset();
            progressed = true;
        }
        // packed units: publish uploaded jobs to the worker queue, collect the done ones, retire
        // them once their amplitudes are out
        // Units publish in queue order: the published count makes every index below it visible to
        // the workers, so a unit whose upload finished before an earlier unit's waits for it (its
        // jobs would otherwise expose the earlier unit's, whose tables and memory may not be on the
        // device yet).  A failed upload (the device context is then unusable) fails its unit's
        // jobs and stops the count there.
        for (bool moved = true; moved;) {
            moved = false;
            for (auto &B : s->batches) {
                if (B.state != Batch::Uploading || B.first != s->published) continue;
                const cudaError_t e = cudaEventQuery(B.ev);
                if (e == cudaErrorNotReady) break;
                if (e != cudaSuccess) {
                    // the context is unusable after a failed upload: fail the unit's jobs; its
                    // indices stay unpublished and no later unit can be published either
                    cudaStreamSynchronize(B.st);
                    for (auto &r : B.jobs) finish(s, r, SIM_E_CUDA, 0.0, 0.0);
                    B.jobs.clear();
                    B.state = Batch::Free;
                    progressed = true;
                    break;
                }
                s->published += B.jobs.size();  // descriptors were written before the upload
                std::atomic_thread_fence(std::memory_order_release);
                __atomic_store_n(s->ctl, (uint32_t)s->published, __ATOMIC_RELEASE);
                B.state = Batch::Running;
                progressed = moved = true;
            }
        }
        uint64_t not_done = 0;
        for (auto &B : s->batches) {
            const size_t nj = B.jobs.size();
            if (B.state == Batch::Running) {
                size_t done = 0;
                for (size_t j = 0; j < nj; j++)
                    done += __atomic_load_n(&s->ring[(B.first + j) % kQueueCap].done, __ATOMIC_ACQUIRE) != 0;
                if (done < nj) {
                    not_done += nj - done;
                    continue;
                }
                for (size_t j = 0; j < nj; j++) {
                    const QSlot &q = s->ring[(B.first + j) % kQueueCap];
                    B.res[2 * j] = q.res[0];
                    B.res[2 * j + 1] = q.res[1];
                }
                const int rc = copy_out_packed(B);
                if (rc != SIM_OK) {  // the queued copies drain before the waiters learn of it
                    cudaStreamSynchronize(B.st);
                    for (auto &r : B.jobs) finish(s, r, rc, 0.0, 0.0);
                    s->retired += nj;
                    B.jobs.clear();
                    B.state = Batch::Free;
                }
                progressed = true;
            }
            if (B.state == Batch::CopyingOut) {
                const cudaError_t e = cudaEventQuery(B.ev);
                if (e == cudaErrorNotReady) continue;
                for (size_t j = 0; j < nj; j++)
                    finish(s, B.jobs[j], e == cudaSuccess ? SIM_OK : SIM_E_CUDA, B.res[2 * j], B.res[2 * j + 1]);
                s->retired += nj;
                B.jobs.clear();
                B.state = Batch::Free;
                progressed = true;
            }
        }
        manage_workers(s, not_done, &progressed);
        if (progressed) s->cv_done.notify_all();
        if (s->stop && s->queue.empty()) {
            bool idle = pack_pending.empty();
            for (auto &r : s->slot_req) idle &= !r;
            for (auto &B : s->batches) idle &= B.state == Batch::Free;
            idle &= s->graph_inflight.empty();
            if (idle) break;
        }
        // admission, in arrival order; a request that does not fit may be overtaken by later ones
        // at most kMaxBypass times, then admission waits for it
        std::shared_ptr<Req> first_blocked;
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            if (first_blocked && first_blocked->bypassed >= kMaxBypass) break;
            auto r = *it;
            bool admitted = false;
            if (r->graph) {  // its memory is the entry's: it waits only for the entry's previous replay
                if (!r->graph->busy) {
                    r->graph->busy = true;
                    const int rc = start_graph(s, r);
                    if (rc != SIM_OK) {
                        r->graph->busy = false;
                        finish(s, r, rc, 0.0, 0.0);
                    } else {
                        s->graph_inflight.push_back(r);
                        s->graph_replays++;
                    }
                    admitted = true;
                }
            } else if (s->used + r->bytes <= s->budget) {
                // a large circuit waits while max_large of them run (it may still be overtaken)
                bool large_full = false;
                if (r->n >= kLargeQubits && s->max_large > 0) {
                    int running = 0;
                    for (auto &q : s->slot_req) running += q && q->n >= kLargeQubits;
                    large_full = running >= s->max_large;
                }
                if (large_full) {
                    // not admitted now
                } else if (r->packed) {
                    s->used += r->bytes;
                    pack_pending.push_back(r);
                    admitted = true;
                } else {
                    for (size_t i = 0; i < s->slots.size(); i++)
                        if (!s->slot_req[i]) {
                            s->used += r->bytes;
                            const int rc = start_unpacked(s, (int)i, r);
                            if (rc != SIM_OK) abort_unpacked(s, (int)i, rc);
                            admitted = true;
                            break;
                        }
                }
            }
            if (admitted) {
                if (first_blocked) first_blocked->bypassed++;
                it = s->queue.erase(it);
                progressed = true;
                continue;
            }
            if (!first_blocked) first_blocked = r;
            ++it;
        }
        // stream-path requests: enqueue what the staging rings allow
        for (size_t i = 0; i < s->slots.size(); i++) {
            auto r = s->slot_req[i];
            if (!r || r->launched) continue;
            const int rc = advance_unpacked(s, r, &progressed);
            if (rc != SIM_OK) {
                abort_unpacked(s, (int)i, rc);
                progressed = true;
            }
        }
        // packed upload: whenever a unit is free and the queue has room (a ring entry is reused only
        // once its job has been retired)
        if (!pack_pending.empty())
            for (auto &B : s->batches)
                if (B.state == Batch::Free) {
                    // ring entries from the oldest unit still holding some up to next_index are in use
                    uint64_t oldest = s->next_index;
                    for (auto &U : s->batches)
                        if (U.state != Batch::Free) oldest = std::min(oldest, U.first);
                    const uint64_t room = kQueueCap - (s->next_index - oldest);
                    const size_t take = std::min<size_t>({pack_pending.size(), (size_t)s->o.max_pack, (size_t)room});
                    if (take == 0) break;
                    B.jobs.assign(pack_pending.begin(), pack_pending.begin() + take);
                    pack_pending.erase(pack_pending.begin(), pack_pending.begin() + take);
                    const int rc = upload_packed(s, B);
                    if (rc != SIM_OK) {
                        // a copy from the pinned staging buffer may already be queued: let it drain
                        // before the staging is reused or any waiter is told its request failed
                        cudaStreamSynchronize(B.st);
                        for (auto &r : B.jobs) finish(s, r, rc, 0.0, 0.0);
                        B.jobs.clear();
                        B.state = Batch::Free;
                        s->cv_done.notify_all();
                    }
                    progressed = true;
                    break;
                }
        if (!progressed) s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
}

void srv_release(srv_t *s)
{
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    DeviceScope dev_scope(s->o.device);
    for (int w = 0; w < 2; w++) {  // workers leave within their idle time once nothing is published
        if (s->wst[w]) cudaStreamSynchronize(s->wst[w]);
        if (s->wev[w]) cudaEventDestroy(s->wev[w]);
        if (s->wst[w]) cudaStreamDestroy(s->wst[w]);
    }
    for (auto &B : s->batches) {
        if (B.st) cudaStreamSynchronize(B.st);
        if (B.ev) cudaEventDestroy(B.ev);
        if (B.st) cudaStreamDestroy(B.st);
        if (B.h_stage) cudaFreeHost(B.h_stage);
    }
    if (s->ring) cudaFreeHost(s->ring);
    if (s->ctl) cudaFreeHost(s->ctl);
    if (s->d_head) cudaFree(s->d_head);
    for (auto &kv : s->reqs)
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    for (auto &kv : s->graphs) {
        GraphEntry &E = *kv.second;
        if (E.g) sim_graph_destroy(E.g);
        if (E.plan) sim_plan_destroy(E.plan);
        if (E.h) sim_destroy(E.h);
    }
    for (auto *h : s->slots) sim_destroy(h);
    if (s->h_results) cudaFreeHost(s->h_results);
    delete s;
}

}  // namespace

extern "C" {

int srv_create(const srv_opts *opts, srv_t **out)
{
    if (!out) return srv_fail(nullptr, SIM_E_INVAL, "srv_create: out is NULL");
    *out = nullptr;
    auto *s = new srv_s();
    if (opts) s->o = *opts;
    if (s->o.slots <= 0) s->o.slots = 6;
    if (s->o.small_n <= 0) s->o.small_n = 20;
    if (s->o.max_pack <= 0) s->o.max_pack = 1024;
    // measured on 2000-circuit Poisson streams: FP32 p99 548 ms with 1 against 591 unlimited (573
    // one at a time); 3xFP16 p50 / p99 15.9 / 190 ms with 2, 17.5 / 206 unlimited, 13.7 / 237 with 1
    s->max_large = s->o.max_large > 0 ? s->o.max_large : (s->o.max_large < 0 ? 0 : (s->o.precision == SIM_FP32 ? 1 : 2));
    if (s->o.slots > 32 || s->o.small_n > 24 || s->o.max_pack > 65536 ||
        !precision_ok(s->o.precision)) {
        delete s;
        return srv_fail(nullptr, SIM_E_INVAL, "srv_create: slots <= 32, small_n <= 24, max_pack <= 65536");
    }
    DeviceScope dev_scope(s->o.device);
    if (dev_scope.err != cudaSuccess) {
        const int device = s->o.device;
        delete s;
        return srv_fail(nullptr, SIM_E_CUDA, "srv_create: device %d unavailable", device);
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->budget = s->o.hbm_budget ? s->o.hbm_budget : (uint64_t)(0.8 * (double)free_b);
    // keep freed stream-ordered memory in the pool instead of returning it to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->o.device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    for (int i = 0; i < s->o.slots; i++) {
        sim_opts so{};
        so.device = s->o.device;
        sim_t *h = nullptr;
        const int rc = sim_create(1, 0, &so, &h);
        if (rc != SIM_OK) {
            srv_release(s);
            return srv_fail(nullptr, rc, "srv_create: slot %d: %s", i, sim_last_error(nullptr));
        }
        s->slots.push_back(h);
    }
    s->slot_req.resize(s->slots.size());
    s->batches.resize(4);
    for (auto &B : s->batches) {
        if (cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming) != cudaSuccess) {
            srv_release(s);
            return srv_fail(nullptr, SIM_E_CUDA, "srv_create: stream setup failed");
        }
    }
    // the packed jobs' queue: ring and published count in mapped pinned memory, claim counter on
    // the device; two worker streams
    bool qok = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->o.device) == cudaSuccess &&
               cudaHostAlloc(reinterpret_cast<void **>(&s->ring), sizeof(QSlot) * kQueueCap, cudaHostAllocMapped) ==
                   cudaSuccess &&
               cudaHostAlloc(reinterpret_cast<void **>(&s->ctl), 128, cudaHostAllocMapped) == cudaSuccess &&
               cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->d_ring), s->ring, 0) == cudaSuccess &&
               cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->d_ctl), s->ctl, 0) == cudaSuccess &&
               cudaMalloc(reinterpret_cast<void **>(&s->d_head), sizeof(uint32_t)) == cudaSuccess &&
               cudaMemset(s->d_head, 0, sizeof(uint32_t)) == cudaSuccess;
    for (int w = 0; w < 2 && qok; w++)
        qok = cudaStreamCreateWithFlags(&s->wst[w], cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->wev[w], cudaEventDisableTiming) == cudaSuccess;
    if (!qok) {
        srv_release(s);
        return srv_fail(nullptr, SIM_E_CUDA, "srv_create: packed-job queue setup failed");
    }
    std::memset(s->ring, 0, sizeof(QSlot) * kQueueCap);
    std::memset(s->ctl, 0, 128);
    if (cudaHostAlloc(&s->h_results, sizeof(double) * 2 * kResultRing, cudaHostAllocDefault) != cudaSuccess) {
        s->h_results = nullptr;
        srv_release(s);
        return srv_fail(nullptr, SIM_E_NOMEM_HOST, "srv_create: pinned results");
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return SIM_OK;
}

int srv_destroy(srv_t *s)
{
    if (!s) return srv_fail(nullptr, SIM_E_INVAL, "srv_destroy: NULL");
    srv_release(s);
    return SIM_OK;
}

const char *srv_last_error(const srv_t *s) { return s ? s->err.c_str() : thread_error(); }

static int make_graph_entry(srv_t *s, uint64_t key, int n, int n_gates, const sim_gate *gates,
                            const sim_plan_opts &po);
static int enqueue_request(srv_t *s, const std::shared_ptr<Req> &r, uint64_t *ticket);

// Contraction deferral per arithmetic: the tensor-core modes contract on tcgen05 (o.front_pairs
// bridging gates, 5 by default); FP32 contracts on CUDA cores, whose cost grows 4x per bridging
// gate while an FP32 pass it saves costs 2.8-4.3 ms per 2^30 amplitudes, so at most 2 bridging
// gates and a lower share of the circuit (measured on 28-30 qubits: 13-22 % less time); the other
// modes run no front.  0: none.
static int front_pairs_for(const srv_t *s, int precision)
{
    if (s->o.front_pairs < 0) return 0;
    if (tmem_mode(precision)) return s->o.front_pairs ? s->o.front_pairs : 5;
    if (precision == SIM_FP32) return s->o.front_pairs ? std::min(s->o.front_pairs, kFp32FrontPairs) : kFp32FrontPairs;
    return 0;
}

static double front_min_share(int precision) { return precision == SIM_FP32 ? kFp32FrontMinShare : kFrontMinShare; }

int srv_submit(srv_t *s, int n_qubits, int n_gates, const sim_gate *gates, void *out_amps, uint64_t *ticket)
{
    if (!s || !ticket) return srv_fail(s, SIM_E_INVAL, "srv_submit: NULL argument");
    *ticket = 0;
    auto r = std::make_shared<Req>();
    r->t_submit = Clock::now();  // latency counts from the call: planning below is part of it
    r->n = n_qubits;
    r->packed = n_qubits <= s->o.small_n;
    r->precision = r->packed ? SIM_FP32 : s->o.precision;
    r->out_amps = out_amps;
    r->bytes = (sizeof(float2) << n_qubits) + (1u << 16);
    if (r->bytes > s->budget) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->rejected++;
        return srv_fail(s, SIM_E_BUSY, "srv_submit: %d qubits need %llu bytes, budget %llu", n_qubits,
                        (unsigned long long)r->bytes, (unsigned long long)s->budget);
    }
    // plan on the caller's thread, with the autotuned width and front choice for this size and
    // depth class when srv_autotune measured one (an explicit kmax in the options still wins)
    int tuned_front = -1;  // -1: the fixed rule below
    int tuned_kmax = 0;
    if (!r->packed) {
        std::lock_guard<std::mutex> lk(s->tune_mu);
        auto it = s->tune.find({n_qubits, depth_bucket(n_qubits, n_gates)});
        if (it != s->tune.end()) {
            tuned_kmax = it->second.kmax;
            tuned_front = it->second.front;
        }
    }
    sim_plan_opts po{};
    po.kmax = s->o.kmax ? s->o.kmax : (tuned_kmax ? tuned_kmax : auto_kmax(n_qubits, r->packed, r->precision));
    if (r->packed) po.kmax = std::min(po.kmax, kPackMaxK);
    po.precision = r->precision;
    po.search = kSrvPlanSearch;
    // contraction deferral (Sect. 2) for large circuits: the gates up to the (pairs + 1)-th across
    // the bipartition split_choose picks run as two tensors and one contraction (tcgen05 in the
    // tensor-core modes, CUDA cores in FP32; front_pairs_for), when that front holds a large
    // enough share of the circuit
    int front = 0;
    std::vector<int> side(n_qubits, 0);
    const int pairs = front_pairs_for(s, r->precision);
    const bool want_front = pairs > 0 && (tuned_front >= 0 ? tuned_front == 1 : n_qubits >= kFrontMinQubits);
    // a repeated circuit replays its CUDA graph (created at its second submission)
    const bool graph_ok = !r->packed && n_qubits <= kGraphMaxQubits && !want_front;
    if (graph_ok) {
        uint64_t key = 0xcbf29ce484222325ull;  // FNV-1a over the size, the options and the gate records
        auto mix = [&](const void *p, size_t nb) {
            const unsigned char *c = static_cast<const unsigned char *>(p);
            for (size_t i = 0; i < nb; i++) key = (key ^ c[i]) * 0x100000001b3ull;
        };
        mix(&n_qubits, sizeof n_qubits);
        mix(&po.kmax, sizeof po.kmax);
        mix(&po.precision, sizeof po.precision);
        mix(gates, sizeof(sim_gate) * (size_t)n_gates);
        std::lock_guard<std::mutex> glk(s->graph_mu);
        auto it = s->graphs.find(key);
        if (it == s->graphs.end() && ++s->seen[key] >= 2 && (int)s->graphs.size() < kGraphMaxEntries) {
            const int grc = make_graph_entry(s, key, n_qubits, n_gates, gates, po);
            if (grc == SIM_OK) it = s->graphs.find(key);
        }
        if (it != s->graphs.end()) {
            r->graph = it->second;
            r->bytes = 0;  // the entry's memory was reserved when it was made
            return enqueue_request(s, r, ticket);
        }
    }
    if (!r->packed && want_front) {
        int nf = 0;
        if (split_choose(n_qubits, n_gates, gates, pairs, 7, side.data(), &nf, n_qubits) == SIM_OK &&
            nf >= front_min_share(r->precision) * n_gates)
            front = nf;
    }
    sim_split_t *sp = nullptr;
    if (front && sim_split_create(n_qubits, front, gates, side.data(), &sp) == SIM_OK) {
        uint64_t extra = contraction_scratch_bytes(sp);
        for (int t = 0; t < 2; t++) extra += sizeof(float2) << (sp->n_side[t] + 2 * sp->n_pairs);
        if (r->bytes + extra <= s->budget) {
            r->split.reset(sp, [](sim_split_s *p) { sim_split_destroy(p); });
            r->bytes += extra;
        } else {
            sim_split_destroy(sp);
        }
    }
    if (!r->split) front = 0;
    sim_plan_t *plan = nullptr;  // the gates after the front (all of them without one)
    int rc = sim_plan_create(n_qubits, n_gates - front, gates + front, &po, &plan);
    sim_plan_t *tplan[2] = {nullptr, nullptr};
    for (int t = 0; rc == SIM_OK && r->split && t < 2; t++) {
        r->nw[t] = r->split->n_side[t] + 2 * r->split->n_pairs;
        rc = sim_plan_create(r->nw[t], (int)r->split->gates[t].size(), r->split->gates[t].data(), &po, &tplan[t]);
    }
    if (rc != SIM_OK) {
        for (auto *tp : tplan)
            if (tp) sim_plan_destroy(tp);
        if (plan) sim_plan_destroy(plan);
        std::lock_guard<std::mutex> lk(s->mu);
        s->rejected++;
        return srv_fail(s, rc, "srv_submit: %s", sim_last_error(nullptr));
    }
    // where the qubits sit: the identity for packed circuits (one CTA each, no HBM passes); for
    // the others the layout sim_plan_layout picks, the state permuted back before a readout
    int phys[kMaxQubits];
    for (int q = 0; q < kMaxQubits; q++) phys[q] = q;
    if (!r->packed) {
        if (r->split)
            sim_plan_layout_front(plan, r->split.get(), phys, nullptr);
        else
            sim_plan_layout(plan, phys, nullptr);
        bool ident = true;
        for (int q = 0; q < n_qubits; q++) ident = ident && phys[q] == q;
        if (!ident && out_amps) {
            r->back.assign(n_qubits, 0);
            for (int q = 0; q < n_qubits; q++) r->back[phys[q]] = q;
        }
    }
    // blocks: tensor 1's, tensor 2's (each tensor laid out as the contraction into phys wants),
    // then the rest's
    auto prepare = [&](const sim_plan_t *p, const int *phys_of, int nq) {
        for (const PlanBlock &b : p->blocks) {
            Prepared pb;
            pb.k = (int)b.qubits.size();
            pb.mat.resize((size_t)1 << (2 * pb.k));
            const int prc = prepare_block_map(s->slots[0], pb.k, b.qubits.data(), b.mat.data(), phys_of, nq, pb.tpos,
                                              pb.mat.data(), nq);
            if (prc != SIM_OK) return prc;
            r->blocks.push_back(std::move(pb));
        }
        return (int)SIM_OK;
    };
    if (r->split) {
        r->out_bit_of.assign(phys, phys + n_qubits);
        for (int t = 0; rc == SIM_OK && t < 2; t++) {
            int lay[kMaxQubits];
            front_tensor_layout(r->split.get(), tplan[t], t, phys, lay);
            r->t_lay[t].assign(lay, lay + r->nw[t]);
            rc = prepare(tplan[t], lay, r->nw[t]);
            r->nt[t] = (int)tplan[t]->blocks.size();
        }
    }
    if (rc == SIM_OK) rc = prepare(plan, phys, n_qubits);
    for (auto *tp : tplan)
        if (tp) sim_plan_destroy(tp);
    sim_plan_destroy(plan);
    if (rc != SIM_OK) return srv_fail(s, rc, "srv_submit: block preparation failed");
    return enqueue_request(s, r, ticket);
}

// Make the graph entry of a repeated circuit (caller's thread, graph_mu held): the plan as
// srv_submit plans it without a front, a handle of n qubits in the layout sim_plan_layout picks,
// the plan captured on it; its memory is taken from the budget.
static int make_graph_entry(srv_t *s, uint64_t key, int n, int n_gates, const sim_gate *gates,
                            const sim_plan_opts &po)
{
    const uint64_t bytes = (sizeof(float2) << n) + (1u << 20);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->used + bytes > s->budget) return SIM_E_BUSY;
        s->budget -= bytes;
    }
    auto E = std::make_shared<GraphEntry>();
    E->bytes = bytes;
    int rc = sim_plan_create(n, n_gates, gates, &po, &E->plan);
    int phys[kMaxQubits];
    if (rc == SIM_OK) rc = sim_plan_layout(E->plan, phys, nullptr);
    if (rc == SIM_OK) {
        sim_opts so{};
        so.device = s->o.device;
        rc = sim_create(n, 0, &so, &E->h);
    }
    if (rc == SIM_OK) rc = sim_set_layout(E->h, phys);
    if (rc == SIM_OK) rc = sim_graph_create(E->h, E->plan, &E->g);
    if (rc != SIM_OK) {
        if (E->g) sim_graph_destroy(E->g);
        if (E->plan) sim_plan_destroy(E->plan);
        if (E->h) sim_destroy(E->h);
        std::lock_guard<std::mutex> lk(s->mu);
        s->budget += bytes;
        return rc;
    }
    bool ident = true;
    for (int q = 0; q < n; q++) ident = ident && phys[q] == q;
    if (!ident) {
        E->back.assign(n, 0);
        for (int q = 0; q < n; q++) E->back[phys[q]] = q;
    }
    s->graphs[key] = E;
    return SIM_OK;
}

// Queue a planned (or graph-replay) request: its completion event, a ticket, the queue.
static int enqueue_request(srv_t *s, const std::shared_ptr<Req> &r, uint64_t *ticket)
{
    cudaError_t ee;
    {
        DeviceScope dev_scope(s->o.device);
        ee = dev_scope.err != cudaSuccess ? dev_scope.err : cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
    }
    if (ee != cudaSuccess) return srv_fail(s, SIM_E_CUDA, "srv_submit: event");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return srv_fail(s, SIM_E_BUSY, "srv_submit: server is stopping");
        r->ticket = s->next_ticket++;
        r->h_res = s->h_results + 2 * (r->ticket % kResultRing);
        if (r->t_submit == Clock::time_point{}) r->t_submit = Clock::now();
        if (s->submitted == 0) s->t_first = r->t_submit;
        s->submitted++;
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return SIM_OK;
}

int srv_wait(srv_t *s, uint64_t ticket, int timeout_ms, double *norm, double *sum_p2_scaled, double *latency_ms)
{
    if (!s) return srv_fail(nullptr, SIM_E_INVAL, "srv_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return srv_fail(s, SIM_E_INVAL, "srv_wait: unknown ticket %llu", (unsigned long long)ticket);
    auto r = it->second;
    auto done = [&] { return r->status != 1; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return srv_fail(s, SIM_E_TIMEOUT, "srv_wait: ticket %llu not done after %d ms", (unsigned long long)ticket,
                        timeout_ms);
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
    s->reqs.erase(it);
    if (r->status != SIM_OK) return srv_fail(s, r->status, "srv_wait: request failed");
    if (norm) *norm = r->norm;
    if (sum_p2_scaled) *sum_p2_scaled = std::ldexp(r->s2, r->n);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    return SIM_OK;
}

// One candidate of the autotuner on a scratch handle: plan as srv_submit would (block width kmax,
// the contraction-deferral front or not, the layout sim_plan_layout picks), run it twice from the
// start state and return the second run's device time in *ms.  SIM_E_UNSUPPORTED when the front
// does not apply to this circuit.
static int tune_candidate(srv_t *s, sim_t *h, int n, int ng, const sim_gate *gates, int kmax, bool front,
                          cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    sim_plan_opts po{};
    po.kmax = kmax;
    po.precision = s->o.precision;
    po.search = kSrvPlanSearch;
    int nf = 0;
    std::vector<int> side(n, 0);
    sim_split_t *sp = nullptr;
    sim_front_t *fr = nullptr;
    sim_plan_t *plan = nullptr;
    int rc = SIM_OK;
    if (front) {
        rc = split_choose(n, ng, gates, front_pairs_for(s, s->o.precision), 7, side.data(), &nf, n);
        if (rc == SIM_OK && nf < front_min_share(s->o.precision) * ng) rc = SIM_E_UNSUPPORTED;
        if (rc == SIM_OK) rc = sim_split_create(n, nf, gates, side.data(), &sp);
        if (rc == SIM_OK) rc = sim_front_create(h, sp, &po, &fr);
    }
    if (rc == SIM_OK) rc = sim_plan_create(n, ng - nf, gates + nf, &po, &plan);
    int perm[kMaxQubits];
    if (rc == SIM_OK) rc = sim_plan_layout(plan, perm, nullptr);
    for (int rep = 0; rep < 2 && rc == SIM_OK; rep++) {  // the first run warms up
        rc = sim_set_layout(h, perm);
        if (rc == SIM_OK) rc = cudaEventRecord(e0, h->stream) == cudaSuccess ? SIM_OK : SIM_E_CUDA;
        if (rc == SIM_OK) rc = fr ? sim_front_run(h, fr) : sim_reset(h, 0);
        if (rc == SIM_OK) rc = sim_apply_plan(h, plan);
        if (rc == SIM_OK) rc = cudaEventRecord(e1, h->stream) == cudaSuccess ? SIM_OK : SIM_E_CUDA;
        if (rc == SIM_OK) rc = cudaEventSynchronize(e1) == cudaSuccess ? SIM_OK : SIM_E_CUDA;
        if (rc == SIM_OK) rc = cudaEventElapsedTime(ms, e0, e1) == cudaSuccess ? SIM_OK : SIM_E_CUDA;
    }
    if (plan) sim_plan_destroy(plan);
    if (fr) sim_front_destroy(fr);
    if (sp) sim_split_destroy(sp);
    return rc;
}

int srv_autotune(srv_t *s, int n_samples, const int *n_qubits, const int *n_gates, const sim_gate *const *gates,
                 int *kmax_out, int *front_out, double *ms_out)
{
    if (!s || n_samples < 0 || (n_samples > 0 && (!n_qubits || !n_gates || !gates)))
        return srv_fail(s, SIM_E_INVAL, "srv_autotune: NULL argument");
    DeviceScope dev_scope(s->o.device);
    if (dev_scope.err != cudaSuccess) return srv_fail(s, SIM_E_CUDA, "srv_autotune: device unavailable");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return srv_fail(s, SIM_E_CUDA, "srv_autotune: events");
    }
    int rc = SIM_OK;
    for (int i = 0; i < n_samples && rc == SIM_OK; i++) {
        const int n = n_qubits[i], ng = n_gates[i];
        if (kmax_out) kmax_out[i] = 0;
        if (front_out) front_out[i] = 0;
        if (ms_out) ms_out[i] = 0.0;
        if (n <= s->o.small_n) continue;  // packed: one CTA per circuit, blocks of <= 5 qubits
        sim_opts so{};
        so.device = s->o.device;
        sim_t *h = nullptr;
        rc = sim_create(n, 0, &so, &h);
        if (rc != SIM_OK) {
            srv_fail(s, rc, "srv_autotune: scratch state of %d qubits: %s", n, sim_last_error(nullptr));
            break;
        }
        srv_s::Tune best;
        best.ms = 1e300;
        const bool can_front = front_pairs_for(s, s->o.precision) > 0 && n >= 22;
        for (int kmax = 4; kmax <= kMaxK && rc == SIM_OK; kmax++)
            for (int front = 0; front <= (can_front ? 1 : 0) && rc == SIM_OK; front++) {
                float ms = 0.f;
                const int crc = tune_candidate(s, h, n, ng, gates[i], kmax, front == 1, e0, e1, &ms);
                if (crc == SIM_E_UNSUPPORTED) continue;
                if (crc != SIM_OK) {
                    rc = srv_fail(s, crc, "srv_autotune: sample %d (k_max %d, front %d): %s", i, kmax, front,
                                  h->err.c_str());
                    break;
                }
                if (ms < best.ms) {
                    best.ms = ms;
                    best.kmax = kmax;
                    best.front = front;
                }
            }
        sim_destroy(h);
        if (rc != SIM_OK) break;
        {
            std::lock_guard<std::mutex> lk(s->tune_mu);
            s->tune[{n, depth_bucket(n, ng)}] = best;
        }
        if (kmax_out) kmax_out[i] = best.kmax;
        if (front_out) front_out[i] = best.front;
        if (ms_out) ms_out[i] = best.ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int srv_stats(srv_t *s, srv_stats_t *out)
{
    if (!s || !out) return srv_fail(s, SIM_E_INVAL, "srv_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->in_flight = s->submitted - s->completed;
    std::vector<double> v = s->lat_ms;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->circuits_per_s = span > 0 ? (double)s->completed / span : 0.0;
    }
    out->hbm_budget = s->budget;
    out->hbm_used = s->used;
    out->graph_replays = s->graph_replays;
    return SIM_OK;
}

}  // extern "C"
