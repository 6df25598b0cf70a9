// internal.h -- shared internals of the sycsim library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "../../include/sycsim.h"

namespace sycsim {

constexpr int kMaxQubits = 40;
constexpr int kMaxK = 6;
constexpr int kReduceBlocks = 152 * 4;   // persistent reduction grid: 4 CTAs per SM
constexpr uint64_t kStageAmps = 1ull << 23;  // 64 MiB readout/load staging buffer

// Thread-local error text for failures not tied to a handle.
void set_thread_error(const char *fmt, ...);
const char *thread_error();

}  // namespace sycsim

struct sim_s {
    int n = 0;            // qubits
    int s = 0;            // sliced (top) physical bits
    int store = SIM_STORE_DEVICE;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    float2 *d_state = nullptr;  // 2^n amplitudes, physical order
    bool own_state = false;
    uint64_t amps = 0;

    int bit_of[sycsim::kMaxQubits];    // logical qubit -> physical bit
    int qubit_at[sycsim::kMaxQubits];  // physical bit -> logical qubit

    // reduction scratch: per-CTA partials and the final (sum p, sum p^2)
    double *d_partials = nullptr;
    double *d_result = nullptr;       // 8 doubles: [0..1] sums, [4..6] sim_reduce_async's outputs
    double *h_result = nullptr;  // pinned

    // staging for logical-order readout / load
    float2 *d_stage = nullptr;

    // k = 6 matrices go through device memory (the kernel-parameter space holds k <= 5)
    static constexpr int kMat6Slots = 16;
    float2 *d_mat6 = nullptr;
    float2 *h_mat6 = nullptr;  // pinned staging
    cudaEvent_t mat6_ev[kMat6Slots] = {};
    int mat6_next = 0;

    int *d_errflag = nullptr;  // set by kernels whose bounded waits ran out

    // tensor-core contraction into this handle: FP16 operand images and the two scales, kept
    // between calls (grown when a larger split needs more)
    uint8_t *d_contract = nullptr;
    size_t contract_bytes = 0;

    // tensor-core B fragments (fragment-major R^T, hi/lo) go through a device ring
    static constexpr int kFragSlots = 8;
    static constexpr int kFragWords = 2 * 16 * 16 * 64;  // k = 6, split: 128 KiB
    uint32_t *d_frag = nullptr;
    uint32_t *h_frag = nullptr;  // pinned staging
    cudaEvent_t frag_ev[kFragSlots] = {};
    int frag_next = 0;

    // fused reduction: sim_apply_plan's last block (tcgen05) leaves each CTA's (sum p, sum p^2) in
    // d_partials; sim_reduce then only combines them, while no call has written the state since
    // (write_epoch counts the calls that may write it) and the state's memory is the handle's own
    // and was never handed out (state_exposed: sim_state_ptr returned its address)
    uint64_t write_epoch = 1, red_epoch = 0;
    int red_blocks = 0;
    mutable bool state_exposed = false;

    // a whole plan's staged block operands (sim_apply_plan), uploaded in one copy: two slots, each
    // a pinned source and its device copy, reused once the plan that last used it has run
    char *h_plan[2] = {};
    char *d_plan[2] = {};
    size_t plan_bytes[2] = {};
    cudaEvent_t plan_ev[2] = {};
    int plan_next = 0;

    // profiling: CUDA-event pairs around kernel launches, per kernel class
    struct ProfSlot {
        cudaEvent_t a = nullptr, b = nullptr;
        int cls = 0;
        double bytes = 0.0;
    };
    std::vector<ProfSlot> prof;
    int prof_used = 0;
    bool prof_on = false;
    uint64_t launches = 0;  // kernels this handle launched

    // host store (SIM_STORE_HOST, Sect. 4 secondary storage): pinned 2^n amplitudes in the
    // host layout [rest qubits | set B | set A] and device slots of 2^(n - s) amplitudes
    static constexpr int kMaxSlots = 4;
    float2 *h_store = nullptr;   // pinned: the store's regions 0 .. host_regions-1
    float2 *d_store = nullptr;   // device: regions host_regions .. 2^s - 1 (hybrid store)
    uint64_t host_regions = 0;   // regions (one per value of set A, 2^(n-s) amplitudes each) on the host
    cudaEvent_t ev_inplace = nullptr;  // after the latest in-place compute on a device region
    char *h_ops = nullptr;             // pinned: a phase's staged block operands, uploaded once
    size_t h_ops_bytes = 0;
    cudaEvent_t ev_ops = nullptr;      // after the upload from h_ops
    int nslots = 0;
    float2 *d_slot[kMaxSlots] = {};
    cudaStream_t st_in = nullptr, st_out = nullptr;
    cudaEvent_t ev_in[kMaxSlots] = {}, ev_done[kMaxSlots] = {}, ev_out[kMaxSlots] = {};
    int out_set[kMaxSlots] = {-1, -1, -1, -1};  // (set, value) of each slot's last copy-out
    uint64_t out_val[kMaxSlots] = {};
    int set[2][8] = {};                       // sliced sets A (0) and B (1), logical qubits
    int slice_phys[2][sycsim::kMaxQubits];    // phase with set X sliced: qubit -> slot bit (-1: sliced)
    double *h_partials = nullptr;             // pinned, 2 per slice (host-mode reduction)

    std::string err;
};

struct PlanBlock {
    std::vector<int> qubits;  // ascending logical qubits
    std::vector<int> gates;   // gate indices, circuit order
    std::vector<double> mat;  // 2 * D * D, row-major interleaved
};

struct sim_graph_s {
    sim_t *h = nullptr;
    void *d_staged = nullptr;  // every block's staged operands
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> bit_of;  // layout the targets were resolved with
    int n_blocks = 0;
};

struct sim_plan_s {
    int n = 0, n_gates = 0, kmax = 0, precision = 0;
    std::vector<PlanBlock> blocks;
};

struct sim_phases_s {
    int n = 0, s = 0;
    int set_a[8] = {}, set_b[8] = {};
    std::vector<int> set_of;          // sliced set of each phase (0 = A, 1 = B)
    std::vector<sim_plan_t *> plans;  // blocks of each phase
};

// Contraction deferral (split.cpp builds it, contract.cu reads it).
struct sim_split_s {
    int n = 0;
    int n_side[2] = {0, 0};
    int n_pairs = 0;
    std::vector<int> side;            // side of each qubit
    std::vector<sim_gate> gates[2];   // each tensor's gate list over its wires
    std::vector<int> wire_at[2];      // canonical position -> wire
};

namespace sycsim {

// Record an error on h (or the thread when h is null) and return `code`.
int fail(sim_t *h, int code, const char *fmt, ...);

// Makes device `dev` current for the rest of the enclosing scope and gives the calling thread
// its previous current device back when the scope ends, so no call leaves the caller (another
// framework, say) on a device it did not choose.
struct DeviceScope {
    int prev = -1;  // device to restore, or -1
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) err = cudaSetDevice(dev);
        if (prev == dev || err != cudaSuccess) prev = -1;
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
};

#define SIM_DEVICE_SCOPE(h, dev)                                                              \
    ::sycsim::DeviceScope dev_scope_(dev);                                                    \
    if (dev_scope_.err != cudaSuccess)                                                        \
    return ::sycsim::fail((h), SIM_E_CUDA, "cudaSetDevice(%d) failed: %s", (int)(dev),         \
                          cudaGetErrorString(dev_scope_.err))

#define SIM_CUDA_TRY(h, call)                                                           \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::sycsim::fail((h), SIM_E_CUDA, "%s failed: %s (%s:%d)", #call,      \
                                  cudaGetErrorString(e_), __FILE__, __LINE__);           \
    } while (0)

// True if the layout is the identity map.
bool layout_is_identity(const sim_t *h);

// Physical index of a logical index under h's layout.
uint64_t logical_to_physical(const sim_t *h, uint64_t i);

// Profiling brackets: prof_begin records a start event for kernel class `cls` (SIM_PROF_*)
// when profiling is on and returns the slot (or -1); prof_end records the stop event.
int prof_begin(sim_t *h, int cls, double alg_bytes, cudaStream_t st);
void prof_end(sim_t *h, int slot, cudaStream_t st);

// apply.cu: block preparation (targets -> sorted physical bits, FP32 matrix in that order)
// and enqueueing on an arbitrary buffer/stream.
int prepare_block_map(sim_t *h, int k, const int *targets, const double *matrix, const int *phys_of,
                      int nlocal, int *tpos, float2 *mat, int nq = -1);
int prepare_block(sim_t *h, int k, const int *targets, const double *matrix, int *tpos, float2 *mat);
// cudaFuncSetAttribute acts on the current device only: a kernel that needs more than 48 KiB of
// dynamic shared memory is opted in once per device (bit d of `done` records device d < 64;
// higher device numbers are opted in on every call), so a process driving several GPUs can
// launch it on each.
template <typename Kern>
inline bool smem_opt_in(Kern kern, int bytes, std::atomic<uint64_t> &done)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return true;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
    done.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}

// One-time launch configuration of a kernel instantiation (kept in a function-local static).
struct LaunchCfg {
    int sms = 0;
    int occ = 1;  // resident CTAs per SM
    bool ok = false;
};

enum class BlockPath { CudaCore, MmaSync, Tcgen05 };
BlockPath block_path(int nbits, int k, const int *tpos, int precision);
// true if enqueue_block_on would not have to wait for a matrix-staging slot (non-blocking check)
bool staging_slot_free(sim_t *h, int nbits, int k, const int *tpos, int precision);
size_t block_staged_bytes(int nbits, int k, const int *tpos, int precision);
void block_build_staged(int nbits, int k, const int *tpos, const float2 *mat, int precision, void *h_out);
// red / red_grid: as for tcgen05_launch_staged, taken only by tcgen05 blocks (*red_grid stays 0
// for the others)
int launch_block_staged(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat,
                        int precision, const void *d_staged, cudaStream_t st, double *red = nullptr,
                        int *red_grid = nullptr);
int enqueue_block_on(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat,
                     int precision, cudaStream_t st);
int enqueue_block(sim_t *h, int k, const int *tpos, const float2 *mat, int precision);

bool precision_ok(int precision);
// a call is about to write (or may write) the handle's state: partial sums left by a fused
// reduction no longer describe it
inline void state_written(sim_t *h) { h->write_epoch++; }
// the final combine of the reduction over nblocks (sum p, sum p^2) pairs (reduce.cu)
int launch_reduce_final(const double *partials, int nblocks, double *d_result, cudaStream_t st);
// Entries first .. first + count - 1 (logical indices through bit_of, or physical ones when bit_of
// is NULL) whose physical index p lies in [lo, hi): buf[j] = base[p - lo] (scatter: the reverse);
// the others untouched.  The device part of a hybrid host store's readout and load.
int launch_gather_region(float2 *base, uint64_t lo, uint64_t hi, float2 *buf, uint64_t first, uint64_t count, int n,
                         const int *bit_of, int scatter, cudaStream_t st);
// d_result[4..6] = {d_result[0], scale * d_result[1], scale * d_result[1] - 1} (one thread)
int launch_result3(double *d_result, double scale, cudaStream_t st);
// the modes whose 4- to 6-qubit blocks take the tcgen05 kernel where it is eligible
inline bool tmem_mode(int precision) { return precision == SIM_FP16X3_TMEM || precision == SIM_BF16X3; }
// the modes whose mma.sync blocks use the 3xFP16 kernel (BF16X3 hands it what tcgen05 leaves)
inline bool f16x3_mode(int precision)
{
    return precision == SIM_FP16X3 || precision == SIM_FP16X3_TMEM || precision == SIM_BF16X3;
}

// ---- apply_tcgen05.cu (5th-generation tensor cores, TMEM) ----
bool tcgen05_eligible(int nbits, int k, const int *tpos);
// operands staged once in device memory (CUDA graphs): B hi/lo of one block
size_t tcgen05_staged_bytes(int k);
void tcgen05_build_staged(int k, const float2 *mat, bool bf16, void *h_out);
// red (may be NULL): the kernel also writes each CTA's (sum p, sum p^2) of its results at
// red[2 cta]; *grid_out (may be NULL) receives the number of CTAs
int tcgen05_launch_staged(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, bool bf16,
                          const void *d_staged, cudaStream_t st, double *red = nullptr, int *grid_out = nullptr);
int launch_apply_tcgen05(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat, bool bf16,
                         cudaStream_t st);

// ---- apply_tc.cu (tensor cores) ----
bool tc_eligible(int nbits, int k, const int *tpos);
bool tc_eligible_low4(int nbits, int k);
size_t tc_staged_bytes(int k, int precision);
void tc_build_staged(int k, const float2 *mat, int precision, void *h_out);
int tc_launch_staged(float2 *psi, int nbits, int k, const int *tpos, int precision, const void *d_staged,
                     cudaStream_t st);
int launch_apply_tc(sim_t *h, float2 *psi, int nbits, int k, const int *tpos, const float2 *mat,
                    int precision, cudaStream_t st);

// ---- kernel launchers (apply.cu) ----
// Apply a 2^k x 2^k FP32 matrix (row-major complex64, bit j <-> tpos[j], tpos ascending
// physical bits) to a buffer of 2^nbits amplitudes.  mat6_dev: device copy of the
// matrix, used only for k == 6.
int launch_apply_fp32(sim_t *h, float2 *psi, int nbits, int k, const int *tpos,
                      const float2 *mat, const float2 *mat6_dev, cudaStream_t st);

// ---- permute.cu ----
// In-place bit permutation of 2^nbits amplitudes: element i moves to pi(i) where pi
// moves bit b to bit perm[b].
int launch_permute(sim_t *h, float2 *psi, int nbits, const int *perm, cudaStream_t st);

// ---- reduce.cu ----
int launch_reduce(sim_t *h, const float2 *psi, uint64_t amps, double *d_partials,
                  double *d_result, cudaStream_t st);
int launch_gather_logical(const float2 *psi, float2 *dst, uint64_t first, uint64_t count,
                          int n, const int *bit_of, int scatter, cudaStream_t st);
int launch_set_basis(float2 *psi, uint64_t amps, uint64_t phys, cudaStream_t st);

// ---- store.cu (host store) ----
int host_store_create(sim_t *h, const sim_opts &o);
void host_store_release(sim_t *h);
int host_reset(sim_t *h, uint64_t basis);
int host_amplitudes(sim_t *h, uint64_t first, uint64_t count, void *out, int dtype, int physical);
int host_load(sim_t *h, uint64_t first, uint64_t count, const void *src, int physical);
int host_reduce(sim_t *h, double *s1, double *s2);

// ---- contract.cu ----
// Physical bit of each wire of tensor t for a contraction into a state whose layout is out_bit_of
// (and the side qubit at each of the side's bits, if side_qubit is not NULL).
void contract_layout(const sim_split_s *s, const int *out_bit_of, int t, int *bit_of_wire, int *side_qubit);
// sim_split_choose's search from max_seeds seed qubits spread over 0 .. n-1 (the public call
// tries every qubit).
int split_choose(int n_qubits, int n_gates, const sim_gate *gates, int max_pairs, int min_side, int *side,
                 int *n_front, int max_seeds);
// Device bytes of the tensor-core contraction's scratch (operand images, scales) for a split.
size_t contraction_scratch_bytes(const sim_split_s *s);
// Whether tensor t, its wires at tensor_bit_of, can be contracted into a state of layout
// out_bit_of as it is: its side wires on bits 0 .. n_side-1 in any order, the entanglement wires
// above in pair order (as contract_layout places them), and for tensor 1 the same qubits on its
// lowest min(5, n_side) bits as contract_layout puts there (a warp's 32 consecutive x then land on
// 32 consecutive amplitudes of the output).
// With top > 0 the side's top `top` bits must also hold the wires contract_layout puts there (the
// sliced qubits of a contraction into a store, which select the slice).
bool contract_ready(const sim_split_s *s, const int *out_bit_of, int t, const int *tensor_bit_of, int top = 0);
// A contraction prepared once and launched per slice: each side keeps its top top[t] bits fixed
// per launch (the qubits that select a slice of the output), its other n_free[t] bits land at the
// offsets xbit (side 0) / ybit (side 1) of the launch's output buffer.  contract_job_prepare
// computes the scales and operand images (tcgen05) on st; the tensors and the scratch must stay
// unchanged until the last launch has run.
struct ContractJob {
    bool tensor_cores = false, bf16 = false;
    int n_side[2] = {0, 0}, n_free[2] = {0, 0}, e_bits = 0;
    uint32_t ks = 0;                              // k-steps of 16 entanglement values
    const float2 *t[2] = {nullptr, nullptr};
    const uint8_t *img[2] = {nullptr, nullptr};   // operand images (tcgen05)
    const float *amax = nullptr;                  // the two tensors' largest components (tcgen05)
    uint64_t xbit[kMaxQubits] = {}, ybit[kMaxQubits] = {};
};
int contract_job_prepare(sim_t *h, const sim_split_s *s, const float2 *t1, const float2 *t2,
                         const int *const *tensor_bit_of, const int *out_bit_of, int precision, const int *top,
                         uint8_t *scratch, cudaStream_t st, ContractJob *job);
// psi (the output buffer) = the slice with side 0's top bits = fix0 and side 1's = fix1.
int contract_job_launch(sim_t *h, const ContractJob &job, float2 *psi, uint64_t fix0, uint64_t fix1, cudaStream_t st);
// psi (layout out_bit_of) = the contraction of the tensors t1, t2, on stream st: tcgen05 when
// precision is not SIM_FP32 and both sides have >= 7 qubits (scratch: a buffer of
// contraction_scratch_bytes, or NULL for h's own), else the FP32 kernel.  tensor_bit_of[t] is
// tensor t's layout (contract_ready), or NULL (or tensor_bit_of NULL) for contract_layout's.
int enqueue_contraction(sim_t *h, const sim_split_s *s, const float2 *t1, const float2 *t2, float2 *psi,
                        const int *out_bit_of, int precision, uint8_t *scratch, cudaStream_t st,
                        const int *const *tensor_bit_of = nullptr);

// ---- store.cu ----
// The layout a slice of sliced set `set` (0 = A, 1 = B) of host store h is written in, extended
// to all n qubits: the others as in the store, the other set where the slot keeps it (bits
// n-2s ..), the sliced set on top (n-s ..: its value selects the slice).  For set A it is the
// store's own layout.
void store_fill_layout(const sim_t *h, int set, int *lay);
// Relabel a host store's qubits outside its sliced sets (perm as for sim_set_layout; sets A and B
// must keep their bits, else false and nothing changes): the host layout and both slot layouts.
bool host_store_relabel(sim_t *h, const int *perm);
// One phase over a host store (sim_run_phase's body): fill, when given, makes each slice v of the
// sliced set in place of its copy-in ((*fill)(dst, v) enqueues it into dst on the handle's stream);
// p may then be NULL (no blocks).
int run_phase(sim_t *h, int set, const sim_plan_t *p, const std::function<int(float2 *, uint64_t)> *fill);

// ---- split.cpp ----
// Tensor t's layout (wire -> bit) for a contraction into a state of layout out_bit_of: the
// layout contract_layout gives, with the 4 side wires on bits 0-3 chosen so that the tensor's
// blocks (plan, over its wires) run on the fastest kernels (the tcgen05 applies take at most one
// target below bit 4).  Tensor 1 keeps the same qubits on bits 0-4, so that the contraction's
// stores stay whole; its choice is which of them sits on bit 4.  Tensor 2 may put any 4 of its
// side wires there.  The top `top` side bits keep contract_layout's wires (a store's sliced
// qubits).  Scored by the plan's pass estimates; ties keep contract_layout's.  The result
// satisfies contract_ready(..., top).
void front_tensor_layout(const sim_split_s *s, const sim_plan_s *plan, int t, const int *out_bit_of, int *lay,
                         int top = 0);

// ---- plan.cpp ----
// The plan's estimated time per 2^30 amplitudes (sum of its blocks' pass estimates, ms) with
// qubit q on physical bit bit_of[q].
double plan_estimate_ms(const sim_plan_s *p, const int *bit_of);

// ---- gates.cpp ----
// Matrix of a gate record (2x2 or 4x4 complex128, row-major); returns the dimension or 0.
int gate_matrix(const sim_gate &g, double *out /* 32 doubles */);

}  // namespace sycsim
