/*
 * sycsim.h -- C ABI of the GB300 (sm_103a) slice-and-store state-vector
 * simulator for random Sycamore-pattern circuits, after Pednault et al.,
 * "Leveraging Secondary Storage to Simulate Deep 54-qubit Sycamore Circuits"
 * (arXiv:1910.09534).
 *
 * Problem statement (Abstract; Sect. 5): simulate a circuit and output all of
 * its amplitudes.  The method (Sect. 2, 4, 5): evolve the full state
 * ("Schroedinger approach"), with gates aggregated into k-qubit blocks whose
 * 2^k x 2^k matrices are applied to the state (Sect. 5); qubits split into
 * local and sliced ("global") ones, reorganised between phases (Sect. 4); and
 * slices kept in secondary storage -- here pinned host memory -- and streamed
 * through device memory phase by phase (Sect. 4, logical files).
 *
 * Conventions shared by every call:
 *  - Every call returns an int status: SIM_OK (0) or a negative SIM_E_* code.
 *    Nothing aborts, traps or exits.  sim_last_error(h) gives a message for the
 *    last failure on handle h (on the calling thread when h is NULL).
 *  - Qubit q is bit q of the LOGICAL amplitude index (little-endian).  The
 *    library may store the state under another bit order (its layout); calls
 *    that read or write amplitudes say which order they use.
 *  - Matrices are row-major, interleaved complex128 (re, im); bit j of a
 *    row/column index is the value of targets[j].
 *  - The library copies every input array before returning; the caller may
 *    free or reuse it at once.  Output buffers belong to the caller.
 *  - Asynchronous calls are ordered on the handle's CUDA stream; sim_sync()
 *    waits for them.  A handle must not be used by two host threads at once.
 *  - A call works on its handle's device whatever device is current on the
 *    calling thread, and leaves the thread's current device as it found it.
 */
#ifndef SYCSIM_H
#define SYCSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SIM_OK 0
#define SIM_E_INVAL (-1)      /* bad argument (range, duplicate target, non-bijection, ...) */
#define SIM_E_NOMEM_DEV (-2)  /* device allocation failed */
#define SIM_E_NOMEM_HOST (-3) /* pinned host allocation failed */
#define SIM_E_NONLOCAL (-4)   /* a target qubit is currently sliced (Sect. 4: gates act on local qubits) */
#define SIM_E_CUDA (-5)       /* a CUDA call failed; see sim_last_error */
#define SIM_E_TIMEOUT (-6)    /* a bounded wait ran out */
#define SIM_E_BUSY (-7)       /* resource exhausted right now (e.g. serving budget) */
#define SIM_E_UNSUPPORTED (-8)/* valid request this build does not implement */
#define SIM_E_IO (-9)         /* a file could not be opened, read or written */

/* ---- arithmetic of the gate apply ------------------------------------ */
#define SIM_FP32 0   /* CUDA-core FP32 FMA (the default) */
#define SIM_TF32 1   /* tensor cores, TF32 inputs, FP32 accumulate (~1e-3 relative per pass) */
#define SIM_TF32X3 2 /* tensor cores, 3xTF32 split (hi*hi + hi*lo + lo*hi), ~FP32 accuracy */
#define SIM_FP16X3 3 /* tensor cores, 3xFP16 split with a per-tile power-of-two scale, ~FP32 accuracy */
#define SIM_FP16X3_TMEM 4 /* 3xFP16 on tcgen05.mma with tensor-memory accumulators, operands moved
                             by bulk copies (k = 5 and 6 with at most one target below bit 4,
                             k = 4 with none; at least 2^(k+7) amplitudes); other blocks of
                             k = 4..6 as SIM_FP16X3 on mma.sync, narrower ones on CUDA cores */
#define SIM_BF16X3 5 /* BF16x3 on tcgen05.mma: the FP32 operands split into BF16 pieces (8 significant
                        bits each), hi*hi + hi*lo + lo*hi accumulated in FP32; the same kernels and
                        blocks as SIM_FP16X3_TMEM, with what tcgen05 leaves as SIM_FP16X3.  About
                        2^-16 relative per product instead of 3xFP16's 2^-22: a stated-bound mode
                        like SIM_TF32, not FP32-equivalent (Sect. 5 stores FP32 amplitudes) */
/* The mma.sync tensor-core modes apply to blocks with k >= 5 (measured: for k <= 4 the CUDA-core
 * FP32 kernel is faster); narrower blocks run on CUDA cores in FP32. */

/* ---- amplitude dtypes for readout/load ------------------------------- */
#define SIM_C64 0    /* complex64: 2 x float32, interleaved */
#define SIM_C128 1   /* complex128: 2 x float64, interleaved */

/* ---- state storage ---------------------------------------------------- */
#define SIM_STORE_DEVICE 0 /* whole state resident in device memory (HBM) */
#define SIM_STORE_HOST 1   /* whole state in pinned host memory -- the secondary storage of
                              Sect. 4 -- streamed through device slots one slice at a time */

/* ---- slice transfer directions ---------------------------------------- */
#define SIM_H2D 0
#define SIM_D2H 1

typedef struct sim_s sim_t;

typedef struct sim_opts {
    int store;          /* SIM_STORE_DEVICE */
    int device;         /* CUDA device ordinal */
    void *stream;       /* cudaStream_t to order work on; NULL = library-owned stream */
    void *ext_state;    /* optional caller-owned device buffer for the state (>= 8 * 2^n bytes),
                           e.g. a torch tensor's storage; NULL = library allocates */
    uint64_t ext_bytes; /* size of ext_state in bytes */
    int slots;          /* SIM_STORE_HOST: device slice buffers, 2..4 (0 = 3) */
    int set_a[8];       /* SIM_STORE_HOST: the two sliced qubit sets A and B (Sect. 4: the */
    int set_b[8];       /* sliced qubits alternate between two sets); slice_bits qubits each, disjoint */
    int store_device_regions; /* SIM_STORE_HOST: of the 2^slice_bits regions of the store (one per
                           value of set A), how many (the highest values of A) live in device
                           memory instead of pinned host memory, for states larger than the
                           host's memory; 0 = all on the host.  Slice copies then mix
                           host->device and device->device moves. */
    int reserved[7];
} sim_opts;

/* Message for the last failure on h (h == NULL: the calling thread's last failure
 * not tied to a handle).  The string is owned by the library and valid until the
 * next call on h. */
const char *sim_last_error(const sim_t *h);

/* Library version string, and the CUDA device architecture it was built for. */
const char *sim_version(void);

/* Create a simulator for n_qubits (1..40) with `slice_bits` sliced qubits
 * (Sect. 4: the top slice_bits physical bits address 2^slice_bits slices of
 * 2^(n - slice_bits) amplitudes; gates may only target local qubits).
 * The state starts as |0...0>.  opts may be NULL (device 0, own stream, own
 * buffer).  On success *out is a handle to pass to sim_destroy().
 *
 * SIM_STORE_HOST (Sect. 4, secondary storage organised as logical files indexed
 * by the sliced qubits): 1 <= slice_bits <= 8 and 2*slice_bits < n_qubits; the
 * state lives in pinned host memory in the layout [other qubits, ascending |
 * set_b in order | set_a in order] (bit 0 first), so that the 2^(2 slice_bits)
 * "files" (fixed values of A and B) are contiguous runs; the device holds
 * `slots` buffers of 2^(n - slice_bits) amplitudes.  Gates run through
 * sim_run_phase / sim_run_phases only. */
int sim_create(int n_qubits, int slice_bits, const sim_opts *opts, sim_t **out);
int sim_destroy(sim_t *h);

/* n_qubits, slice_bits and the current layout: bit_of[q] = physical bit that
 * holds logical qubit q (array of n_qubits ints, may be NULL). */
int sim_info(const sim_t *h, int *n_qubits, int *slice_bits, int *bit_of);

/* Device pointer of the state buffer (physical order, complex64) and the
 * cudaStream_t the handle orders its work on (either output may be NULL).  Once
 * the state's address has been handed out, sim_reduce always reads the state
 * (see sim_reduce). */
int sim_state_ptr(const sim_t *h, void **dptr, void **stream);

/* Set the state to the computational basis state |basis> (logical index),
 * asynchronously on the handle's stream. */
int sim_reset(sim_t *h, uint64_t basis);

/* Aggregated-gate apply (Sect. 5: gates aggregated into k-qubit kernels given by
 * 2^k x 2^k unitary matrices, applied to the state as matrix-vector products).
 * For every group of 2^k amplitudes that differ only in the target bits,
 * psi_g <- M psi_g, in place.  k in 1..6; targets: k distinct logical qubits, all
 * local (SIM_E_NONLOCAL otherwise); matrix: 2^k x 2^k complex128, row-major,
 * bit j of its index <-> targets[j]; precision: SIM_FP32 .. SIM_BF16X3
 * (Sect. 5 suggests GPUs for the matrix-vector products; the tensor-core modes
 * treat a tile of 16 groups as a real GEMM with [[Re M, -Im M], [Im M, Re M]]).
 * Asynchronous. */
int sim_apply_fused(sim_t *h, int k, const int *targets, const double *matrix, int precision);

/* Qubit reorganisation (Sect. 4: between phases the memory layout is changed so
 * that other qubits become local/global).  perm[q] = new physical bit of logical
 * qubit q; must be a bijection on 0..n-1.  The logical state is unchanged; the
 * amplitudes move so that physical index pi(i) holds what i held, pi moving bit
 * bit_of[q] to bit perm[q].  Bit-exact (pure data movement), in place.
 * Asynchronous. */
int sim_permute(sim_t *h, const int *perm);

/* Copy `count` amplitudes starting at index `first` to host memory `out`
 * (dtype SIM_C64 or SIM_C128), in logical order (physical_order = 0) or in
 * the stored physical order (physical_order = 1).  Synchronous: returns when
 * out is filled.  out may be pageable or pinned (pinned is faster). */
int sim_amplitudes(sim_t *h, uint64_t first, uint64_t count, void *out, int dtype,
                   int physical_order);

/* Readout without waiting (not in the paper: it lets a caller overlap reading one circuit's
 * result with computing the next on another handle).  Enqueues the copy of `count`
 * complex64 amplitudes starting at `first` into host memory `out` on the handle's stream and
 * returns.  out must stay valid until sim_sync(h) returns, and should be pinned (pageable
 * memory makes the copy synchronous).  Logical order requires the identity layout (no
 * permutation pending); physical_order = 1 always works.  SIM_E_UNSUPPORTED for host-store
 * handles or a logical read of a permuted layout (use sim_amplitudes); SIM_E_INVAL for a bad
 * range or NULL out.  Later calls on h are ordered after the copy. */
int sim_amplitudes_async(sim_t *h, uint64_t first, uint64_t count, void *out, int physical_order);

/* Overwrite `count` amplitudes starting at `first` with complex64 values from
 * host memory `src` (logical or physical order as above).  Synchronous. */
int sim_load_amplitudes(sim_t *h, uint64_t first, uint64_t count, const void *src,
                        int physical_order);

/* Reductions over p_i = |psi_i|^2 (used to check simulations; not in the paper):
 * norm = sum p, sum_p2_scaled = 2^n sum p^2 (Porter-Thomas: about 2), and
 * xeb = 2^n sum p^2 - 1 (linear cross-entropy of the ideal distribution).
 * Per-thread partial sums in FP32 over 16 amplitudes, combined in FP64 in a
 * fixed order (deterministic).  Synchronous.  Any output pointer may be NULL.
 * When the last call that wrote the state was sim_apply_plan and its last block
 * ran on tcgen05, that kernel has already summed its results (FP32 per tile and
 * thread, FP64 per thread and CTA, a fixed order): only those CTA sums are
 * combined.  That is skipped -- the state is read again -- for handles on a
 * caller's buffer (ext_state) or whose state address sim_state_ptr handed out. */
int sim_reduce(sim_t *h, double *norm, double *sum_p2_scaled, double *xeb);

/* sim_reduce without waiting (not in the paper: it lets a caller queue the next circuit on the
 * handle before this one's result is back, so the device never idles between circuits).
 * Enqueues on the handle's stream what sim_reduce computes, then the copy of {norm,
 * 2^n sum p^2, xeb} into out (3 doubles of host memory, caller-owned; pinned memory keeps the
 * call from waiting), and returns.  out holds the result once the stream has passed the copy:
 * after sim_sync(h), or after an event the caller records on the handle's stream (sim_state_ptr
 * gives the stream) after this call; it must stay valid until then.  Work queued later on h
 * (a new circuit overwriting the state) does not change the result.  SIM_E_UNSUPPORTED for
 * host-store handles (use sim_reduce); SIM_E_INVAL for NULL h or out. */
int sim_reduce_async(sim_t *h, double *out);

/* Allocation-free reduction (the paper has no counterpart; it serves callers that
 * cannot allocate device memory -- for example code running inside a framework
 * that owns all device memory through its own pool, or code that must not risk
 * the implicit device synchronisation of cudaMalloc/cudaFree).  Computes what
 * sim_reduce computes, over a caller-owned complex64 device buffer:
 * d_out[0] = sum p, d_out[1] = n_amps * sum p^2, d_out[2] = d_out[1] - 1, with
 * d_out a caller-owned device array of 3 doubles; asynchronous on `stream`
 * (cudaStream_t, NULL = legacy default stream) on the current device.
 * d_state: 16-byte aligned, n_amps even, 2 <= n_amps <= 2^40; d_out: 8-byte
 * aligned (SIM_E_INVAL otherwise, before anything is launched).  It calls no
 * allocator: its scratch is one fixed 9.5 KiB array (1216 doubles, one pair per
 * CTA) in the library's device memory, which every GPU that loads the library
 * holds until the process exits.  The first call on a device looks up that
 * array's device address and caches it for the process (make that first call
 * outside any stream capture); a cudaDeviceReset of that device invalidates the
 * cached address, so the call must not be used on a device after it has been
 * reset.  All calls share the array and fully overwrite what they use, so
 * nothing needs clearing; calls that overlap on the GPU (other streams, other
 * threads) race on it and must be serialised by the caller. */
int sim_reduce_noalloc(const void *d_state, uint64_t n_amps, double *d_out, void *stream);

/* Wait for all work queued on the handle's stream, at most timeout_ms
 * milliseconds (< 0: no limit).  SIM_E_TIMEOUT if it did not finish. */
int sim_sync(sim_t *h, int timeout_ms);

/* ---- per-launch profiling (kernel durations on the handle's stream) ------
 * sim_profile_enable(h, 1) clears the counters and brackets every kernel
 * launch that follows with a pair of CUDA events; sim_profile_read() waits for
 * the stream and returns, for one kernel class, the number of launches, their
 * summed device time in ms and their algorithmic bytes (apply: 16 B per
 * amplitude; permute: 16 B per amplitude moved; reduce: 8 B per amplitude;
 * contract (sim_contract's GEMM, compute-bound): the field holds its algorithmic
 * FLOPs instead, 8 per complex multiply-add).
 * sim_launch_count() is the number of kernels the handle has launched. */
#define SIM_PROF_APPLY 0
#define SIM_PROF_PERMUTE 1
#define SIM_PROF_REDUCE 2
#define SIM_PROF_OTHER 3
#define SIM_PROF_CONTRACT 4
int sim_profile_enable(sim_t *h, int on);
int sim_profile_read(sim_t *h, int cls, uint64_t *launches, double *total_ms, double *alg_bytes);
int sim_launch_count(const sim_t *h, uint64_t *n);

/* Pinned host memory helpers for callers that want fast copies. */
int sim_host_alloc(size_t bytes, void **out);
int sim_host_free(void *p);

/* ---- circuits and the aggregation planner ----------------------------- */

/* Gate kinds (Sect. 3): single-qubit sqrt(X), sqrt(Y), sqrt(W) -- read as
 * (I - iP)/sqrt(2) -- and the two-qubit fSim of Eq. 1 with theta, phi and
 * the detunings D+, D-, D-,off; plus caller-given 1- and 2-qubit matrices. */
#define SIM_GATE_SQRT_X 0
#define SIM_GATE_SQRT_Y 1
#define SIM_GATE_SQRT_W 2
#define SIM_GATE_FSIM 3
#define SIM_GATE_U1 4 /* u[0..7]: 2x2 complex128 row-major interleaved */
#define SIM_GATE_U2 5 /* u[0..31]: 4x4 complex128, index b(q0) + 2 b(q1) */

typedef struct sim_gate {
    int32_t kind;
    int32_t q0, q1; /* q1 ignored for single-qubit kinds */
    int32_t reserved;
    double theta, phi, dplus, dminus, dminus_off; /* fSim parameters (Eq. 1) */
    double u[32];                                 /* SIM_GATE_U1 / SIM_GATE_U2 matrix */
} sim_gate;

/* Matrix of one gate record (2x2 or 4x4 complex128, row-major interleaved, 32
 * doubles of room).  Returns the dimension (2 or 4) or SIM_E_INVAL.  Host-only. */
int sim_gate_matrix(const sim_gate *g, double *out);

typedef struct sim_plan_s sim_plan_t;

typedef struct sim_plan_opts {
    int kmax;      /* largest block width, 1..6 (Sect. 5 uses k_max = 5) */
    int precision; /* arithmetic for the blocks' apply: SIM_FP32, SIM_TF32, SIM_TF32X3, SIM_FP16X3 */
    int search;    /* beam width of the block search, 0..256: 0 = the default (16), 1 = the greedy
                      schedule alone; wider searches may find fewer blocks and take longer */
    int reserved[5];
} sim_plan_opts;

/* Aggregation planner (Sect. 5: gates grouped into blocks of at most k_max
 * qubits; Appendix A "new cache" lines list such groups).  Partitions the gate
 * list into blocks that respect gate order on every qubit and composes each
 * block's 2^k x 2^k matrix in FP64 (later gates multiply from the left).
 * Blocks are formed greedily, each from the seed unit that lets it take the most
 * gates; with o->search > 1 (the default, 0, means 16) a beam search over those
 * seeds replaces that schedule when it finds one of fewer blocks.
 * Host-side; the plan is immutable and may be applied to many handles. */
int sim_plan_create(int n_qubits, int n_gates, const sim_gate *gates, const sim_plan_opts *o,
                    sim_plan_t **out);
int sim_plan_destroy(sim_plan_t *p);

/* Number of blocks, number of gates planned and the widest block. */
int sim_plan_info(const sim_plan_t *p, int *n_blocks, int *n_gates, int *max_k);

/* Block i: its width k, its targets (k ints, ascending logical qubits) and its
 * matrix (2^k x 2^k complex128, bit j <-> targets[j]); any output may be NULL. */
int sim_plan_block(const sim_plan_t *p, int i, int *k, int *targets, double *matrix);

/* Apply every block of the plan in order (each as sim_apply_fused).  Async. */
int sim_apply_plan(sim_t *h, const sim_plan_t *p);

/* ---- CUDA graphs (not in the paper) ----------------------------------------
 * Capture the block launches of a plan on h once and replay them.  For a plan run many times
 * (the same circuit from several initial states, repeated runs) a replay skips the per-block host
 * work -- matrix rounding, operand staging, the launch itself -- which dominates below ~2^24
 * amplitudes.  Every block's staged operands (tensor-core B fragments, 6-qubit matrices) are
 * uploaded once into device memory that the graph owns.  A graph is bound to h (its state
 * buffer, stream and layout): sim_graph_launch refuses with SIM_E_INVAL on another handle or
 * once h's layout has changed (sim_permute), and a graph must be destroyed before its handle.
 * SIM_E_UNSUPPORTED for host-store handles or a handle on the legacy default stream.
 * sim_graph_create is synchronous (uploads, captures, instantiates); it does not touch the
 * state.  sim_graph_launch is asynchronous on h's stream, like sim_apply_plan. */
/* Where the qubits should sit for a plan (not in the paper).  The fused-apply kernels' speed on
 * GB300 depends on which physical bits a block targets: in SIM_FP16X3_TMEM, 5- and 6-qubit blocks
 * with two or more targets below bit 4 (and 4-qubit blocks with one) leave the tcgen05 kernel for
 * a slower one, and tcgen05 blocks with no target below bit 8 move their tiles in 1 KiB pieces
 * instead of 2 KiB; in SIM_FP32 targets below bit 5 cost register exchanges.  sim_plan_layout
 * searches layouts (pairwise swaps from 4 seeded starts) for the smallest sum over the
 * plan's blocks of a per-pass time estimate (measured per kernel path on 2^30 amplitudes; other
 * precisions: every layout costs the same and the identity is returned), and writes perm[q] = the
 * physical bit for qubit q (a bijection on 0..n-1, as sim_permute takes) and, if est_ms is not
 * NULL, the estimate for that layout and for the identity (est_ms[0], est_ms[1]).  Host only. */
int sim_plan_layout(const sim_plan_t *p, int *perm, double *est_ms);

typedef struct sim_split_s sim_split_t;
/* The same search for a plan whose state is written by the contraction of split s (Sect. 2's
 * contraction deferral; sim_front_run, sim_contract): the contraction stores psi in the state's
 * layout with the 32 lanes of a warp on 32 consecutive values of the side-0 qubits (ordered by
 * their physical bits), so physical bits 0-4 are kept on side-0 qubits -- each store is then one
 * 256-byte run (measured: 13.4 ms instead of 15.8 for the 30-qubit front's contraction).  s must
 * be a split of the same n.  Host only. */
int sim_plan_layout_front(const sim_plan_t *p, const sim_split_t *s, int *perm, double *est_ms);

/* Relabel the physical bits without moving any amplitude (perm as for sim_permute): the logical
 * state changes, so this belongs before sim_reset, sim_front_run or sim_contract, which overwrite
 * every amplitude -- the way to start a plan in the layout sim_plan_layout chose without a
 * permutation pass.  Device-resident handles (with slice_bits > 0 the qubits then on the top bits
 * are the sliced ones), and host stores as long as perm keeps both sliced sets on the bits the
 * store gives them (only the other qubits' order changes: the host layout and the slots'
 * [others | B] / [others | A] layouts alike; sim_phases_layout chooses it); SIM_E_INVAL
 * otherwise. */
int sim_set_layout(sim_t *h, const int *perm);

typedef struct sim_graph_s sim_graph_t;
int sim_graph_create(sim_t *h, const sim_plan_t *p, sim_graph_t **out);
int sim_graph_launch(sim_t *h, const sim_graph_t *g);
int sim_graph_destroy(sim_graph_t *g);

/* Autotuner (not in the paper; Sect. 5 fixes k_max = 5 for its CPUs): plans the
 * given circuit with every candidate block width (k_max 3..6) and arithmetic the
 * accuracy class allows -- SIM_TUNE_FP32: FP32 only; SIM_TUNE_FP32_EQUIVALENT:
 * also the split tensor-core modes (3xFP16 on mma.sync and on tcgen05, 3xTF32); SIM_TUNE_ANY: also plain
 * TF32 -- runs each from |0...0> on h's state (twice; the second run is timed
 * with CUDA events) and writes the fastest options to *best (and its time in
 * ms to *best_ms, may be NULL).  Synchronous; leaves h in |0...0>.  Needs a
 * device-resident handle without sliced bits. */
#define SIM_TUNE_FP32 0
#define SIM_TUNE_FP32_EQUIVALENT 1
#define SIM_TUNE_ANY 2
int sim_autotune(sim_t *h, int n_gates, const sim_gate *gates, int accuracy, sim_plan_opts *best,
                 double *best_ms);

/* ---- secondary storage: slices and phases (Sect. 4) ------------------------ */

/* Move slice `value` of sliced set `set` (0 = A, 1 = B; value's bit i is the value
 * of set[i]) between the host store and device slot `slot` (0..slots-1), dir
 * SIM_H2D or SIM_D2H.  Asynchronous; copies run on the handle's copy streams and
 * are ordered by events against the compute work on that slot.  Bit-exact.
 * SIM_E_UNSUPPORTED if the handle has no host store. */
int sim_stream_slice(sim_t *h, int set, uint64_t value, int dir, int slot);

/* Device pointer of slot `slot` (2^(n - slice_bits) complex64 amplitudes; with set
 * A sliced its layout is [rest | B], with set B sliced [rest | A]). */
int sim_slot_ptr(const sim_t *h, int slot, void **dptr);

/* Copy `count` complex64 amplitudes of slot `slot` starting at `first` to host
 * memory `out`, after the slot's pending copy-in.  Synchronous. */
int sim_slot_read(sim_t *h, int slot, uint64_t first, uint64_t count, void *out);

/* One phase (Sect. 4: for each value of the sliced qubits, read the slice, apply
 * the phase's gates, write it back): for every value of set `set`, stream the
 * slice in, apply every block of plan p (whose qubits must avoid that set --
 * SIM_E_NONLOCAL otherwise), stream it out; slices rotate through the slots so
 * copies overlap compute.  On a device-resident handle the plan is applied to
 * the whole state instead.  Asynchronous. */
int sim_run_phase(sim_t *h, int set, const sim_plan_t *p);

/* Phase planner (Sect. 4: sliced qubits alternate between two sets; gates are
 * applied while their qubits are local).  Splits the gate list into phases that
 * alternate between slicing set A and set B: a phase takes, in order, every
 * remaining gate that avoids its sliced set and does not follow a deferred gate
 * on one of its qubits.  Each phase's gates are aggregated as by
 * sim_plan_create.  SIM_E_NONLOCAL if a gate couples a qubit of A with one of B. */
typedef struct sim_phases_s sim_phases_t;
int sim_phases_create(int n_qubits, int n_gates, const sim_gate *gates, const sim_plan_opts *o,
                      int slice_bits, const int *set_a, const int *set_b, sim_phases_t **out);
/* Choose the two sliced sets for a circuit (not spelled out in the paper, which fixes them by
 * hand at the two ends of the lattice, Sect. 4): every pair of disjoint windows of slice_bits
 * consecutive qubit numbers (on a row-major lattice: the two ends, the middle rows, ...) that no
 * gate couples is split into phases as sim_phases_create does, each phase grouped into fused blocks
 * (o->kmax, default 4), and scored phases * phase_weight + blocks; the best pair is written to
 * set_a / set_b (slice_bits entries each), its phase and block counts to *n_phases / *n_blocks
 * (either may be NULL).  phase_weight is the cost of streaming the state out and back once, in
 * fused passes (<= 0: 32, about HBM / host-link bandwidth on a GB300 node).  Host only; no device
 * is touched.  SIM_E_INVAL for bad arguments or when no pair can phase the circuit. */
int sim_phases_choose_sets(int n_qubits, int n_gates, const sim_gate *gates, int slice_bits,
                           const sim_plan_opts *o, double phase_weight, int *set_a, int *set_b, int *n_phases,
                           int *n_blocks);
int sim_phases_destroy(sim_phases_t *ph);
int sim_phases_info(const sim_phases_t *ph, int *n_phases, int *total_blocks);
int sim_phases_get(const sim_phases_t *ph, int i, int *set, const sim_plan_t **plan);

/* Run every phase in order (sim_run_phase); the handle's sets must be the
 * phases' sets.  On a device-resident handle created with slice_bits > 0, each
 * phase first permutes its sliced set into the top slice_bits physical bits
 * (sim_permute), so the gates of the phase act on local bits only -- the
 * in-memory analogue of Sect. 4's reorganisation between phases.  The same pass
 * also exchanges pairs of the other bits where the per-pass estimates of
 * sim_plan_layout say the phase's blocks run faster (disjoint exchanges, so still
 * one pass; without a sliced-set move only if they save more than a pass).
 * Asynchronous. */
int sim_run_phases(sim_t *h, const sim_phases_t *ph);

/* Where the qubits outside the two sliced sets should sit for the phases ph (not in the paper;
 * as sim_plan_layout, the fused kernels' speed depends on which qubits sit on the low physical
 * bits).  perm[q] for every qubit: the others on 0 .. n-2s-1 in the order that minimises the
 * per-pass estimates summed over every phase's blocks (local search from the ascending order and
 * from seeded random orders), the two sets above them in set order: for a host store
 * (resident = 0) set B on n-2s .. n-s-1 and set A on n-s .. n-1, where the store keeps them; for
 * a device-resident handle with slice_bits = s (resident = 1) the first phase's sliced set on
 * top, so that sim_run_phases needs no move before it, and the other set below.  front (may be
 * NULL): a split whose contraction writes the state first (sim_front_run, sim_contract_phase);
 * bits 0 .. 4 then hold side-0 qubits (as far as there are five outside the sets), so that the
 * contraction's stores stay whole.  est_ms (may be NULL): {chosen, starting order}.  Apply it
 * with sim_set_layout before the state is written (sim_reset, sim_front_run,
 * sim_contract_phase).  Host only. */
int sim_phases_layout(const sim_phases_t *ph, const sim_split_t *front, int resident, int *perm, double *est_ms);

/* ---- contraction deferral: two subcircuits joined by entanglement indices -----
 * Sect. 2 (contraction deferral: subcircuits simulated separately, each with the Schroedinger
 * approach, bridging gates deferred) and the Appendix (the synthesized operations EI and E2Q and
 * the contraction that eliminates the entanglement indices).  side[q] = 0 puts qubit q in
 * tensor 1, 1 in tensor 2 (both sides non-empty).  Gates within one side act on that side's
 * tensor.  The j-th gate G bridging qubit a (side 0) and qubit b (side 1) adds the pair of
 * entanglement indices (a'_j, a_j) to both tensors:
 *   EI on tensor 1:  T1'[a'', a', a] = delta(a'', a') T1[a]
 *   E2Q on tensor 2: T2'[b'', a', a] = sum_b G[a', b''; a, b] T2[b]
 * (G[x'', y''; x, y]: the gate's element from input (a = x, b = y) to output (x'', y'')) and
 *   psi[.., a'', b'', ..] = sum over all pairs (a'_j, a_j) of T1' T2'.
 *
 * sim_split_create turns this into two ordinary gate lists over "wires", which the planner and
 * every apply path run like any circuit on a handle with n_wires[t] qubits started in |0..0>:
 * tensor t has its side's qubits (wires 0.., in increasing qubit order) plus two fresh wires per
 * bridging gate.  EI is a fan-out gate (SIM_GATE_U2 whose first column is |00> + |11>) on two
 * fresh wires: the first becomes qubit a's wire, the second holds a', and a's previous wire now
 * holds a.  E2Q is the same fan-out on two fresh wires followed by G with the first of them in
 * the role of qubit a: afterwards it holds a' and the second holds a.  Each tensor's canonical
 * layout puts its side's qubits at positions 0 .. n_side[t]-1 (increasing qubit order) and pair j
 * at n_side[t] + 2j (a'_j) and n_side[t] + 2j + 1 (a_j).  Host only; the split copies its inputs.
 *   sim_split_info: n_side[2] qubits per side, n_wires[2] = n_side + 2 * n_pairs, n_pairs
 *     bridging gates, n_gates[2] records per tensor (any pointer may be NULL).
 *   sim_split_gates: tensor t's gate records (n_gates[t] of them) into out.
 *   sim_split_canonical: wire_at[p] = the wire at canonical position p of tensor t
 *     (n_wires[t] entries).
 * SIM_E_INVAL for a bad side vector or gate, or more than 40 wires on a side. */
int sim_split_create(int n_qubits, int n_gates, const sim_gate *gates, const int *side, sim_split_t **out);
int sim_split_info(const sim_split_t *s, int *n_side, int *n_wires, int *n_pairs, int *n_gates);
int sim_split_gates(const sim_split_t *s, int t, sim_gate *out);
int sim_split_canonical(const sim_split_t *s, int t, int *wire_at);
int sim_split_destroy(sim_split_t *s);

/* Choose the bipartition and the first phase for contraction deferral (the paper draws its
 * partitions by hand).  Among splits whose sides have at least min_side qubits (<= 0: 7, the
 * tensor-core contraction's minimum; clamped to n_qubits / 2) and lie within max(1, n/8) qubits
 * of an even split, searches -- from a half grown breadth-first over the circuit's couplings
 * around every qubit, then the best single-qubit moves and exchanges while they help -- for the
 * longest prefix of the gate list that crosses the split at most max_pairs times (ties: the later
 * following crossings, then the more even split).  Writes side[q] (0 or 1) and *n_front: gates
 * [0, n_front) are the split's gate list for sim_split_create, the rest run on the contracted
 * state.  Host only.  SIM_E_INVAL for bad arguments. */
int sim_split_choose(int n_qubits, int n_gates, const sim_gate *gates, int max_pairs, int min_side, int *side,
                     int *n_front);

/* The contraction (Appendix: the sum over the entanglement indices): psi = sum_pairs T1 T2 into
 * `out`.  t1 / t2: device-resident handles of n_wires[0] / n_wires[1] qubits holding the two
 * tensors (their gate lists applied); out: a device-resident handle of n_qubits qubits, not
 * sliced, distinct from both.  First permutes t1 and t2 (on their own streams; the tensors' logical
 * content is unchanged) so that each side's qubits sit at bits 0 .. n_side-1 in the order of their
 * physical bits in out and the pairs above in pair order (the canonical layout when out's layout
 * is the identity), which keeps psi's stores coalesced in any layout of out; then, on out's
 * stream after both, one
 * complex GEMM over the 4^n_pairs entanglement values writes every amplitude of psi, in out's
 * current layout (out's layout map is unchanged; its previous amplitudes are overwritten).
 * t1's and t2's streams wait for the GEMM before any later work on them.
 * precision: SIM_FP32 (CUDA cores, FP32 products and sums), or SIM_FP16X3 / SIM_FP16X3_TMEM
 * (tcgen05 tensor cores: each tensor scaled by one power of two, split into FP16 hi + lo, the
 * products hi*hi + hi*lo + lo*hi summed in FP32; needs n_side[0] >= 7 and n_side[1] >= 7,
 * otherwise the FP32 kernel runs), or SIM_BF16X3 (the same with BF16 pieces).  Asynchronous.  SIM_E_INVAL for handles that do not fit s. */
int sim_contract(sim_t *out, sim_t *t1, sim_t *t2, const sim_split_t *s, int precision);

/* The first phase of a sliced run with its state made by the contraction (Sect. 4: tensors 1
 * and 2 are contracted slice by slice straight into the secondary-storage state of subcircuit 3).
 * out: a host-store handle (sim_create with SIM_STORE_HOST); for every slice of the sliced set
 * `set` (0 = A, 1 = B, as for sim_run_phase), the slice of psi is contracted from t1 and t2 into
 * a device slot (set A on a hybrid store: its device regions in place), the blocks of p are
 * applied to it (a plan over qubits outside that set, as for sim_run_phase; NULL for none), and
 * it is written to the store once: no slice is read, and the store's earlier contents do not
 * matter.  t1, t2, s, precision: as for sim_contract (each tensor is permuted first unless its
 * layout already puts its side's qubits of the sliced set on its top side bits, in set order;
 * sim_front_run_phase lays them out that way).  With a device-resident out it is sim_contract
 * followed by sim_apply_plan.  Asynchronous like sim_run_phase; the tensors must not change until
 * sim_sync(out).  SIM_E_INVAL for NULL or shared handles, mismatched sizes, a set other than 0
 * or 1 or a plan for another qubit count; SIM_E_NONLOCAL for a plan with a block on a qubit of
 * the sliced set (nothing is queued then). */
int sim_contract_phase(sim_t *out, sim_t *t1, sim_t *t2, const sim_split_t *s, int precision, int set,
                       const sim_plan_t *p);

/* A split made ready to run (Sect. 2's subcircuits 1 and 2 and their contraction as one reusable
 * unit).  sim_front_create plans both tensors' gate lists (o as for sim_plan_create; NULL: k_max
 * 4, SIM_FP32) and creates their device states (2^n_wires[t] amplitudes each) on out's device and
 * stream; it keeps its own copy of the split.  sim_front_run enqueues on out's stream: both tensors
 * reset to |0..0>, their blocks applied, and sim_contract into out -- on the tensor cores
 * (SIM_FP16X3_TMEM) when o->precision is SIM_FP16X3 or SIM_FP16X3_TMEM, in BF16x3 when it is
 * SIM_BF16X3, else in FP32.  out must
 * have the split's n_qubits qubits and live on the front's device; it is device-resident, or a
 * host store (the contraction then goes slice by slice into the store: sim_contract_phase with
 * no plan).  Asynchronous like sim_apply_plan; the tensors' kernels count in out's
 * sim_launch_count.  sim_front_destroy waits for the front's work. */
typedef struct sim_front_s sim_front_t;
int sim_front_create(sim_t *out, const sim_split_t *s, const sim_plan_opts *o, sim_front_t **f);
int sim_front_run(sim_t *out, sim_front_t *f);

/* sim_front_run, then the blocks of p on the contracted state, in one pass when out is a host
 * store: the contraction fills each slice of sliced set `set` (0 = A, 1 = B) and p's blocks
 * (qubits outside that set, as for sim_run_phase) run on it before it is written
 * (sim_contract_phase) -- the first phase of sim_phases_create's list, whichever set it slices.
 * For a device-resident out: sim_front_run then sim_apply_plan.  p may be NULL.  The tensors'
 * layouts keep each side's qubits of the sliced set on their top side bits.  sim_front_run(out,
 * f) is sim_front_run_phase(out, f, 0, NULL).  Errors as sim_front_run and sim_contract_phase. */
int sim_front_run_phase(sim_t *out, sim_front_t *f, int set, const sim_plan_t *p);
int sim_front_destroy(sim_front_t *f);

/* ---- a state sharded over global qubits on 2^g ranks (Sect. 4) ------------------------------
 * Sect. 4 splits the state over many memories by "global" qubits, applies gates to the local ones
 * and reorganises the memory layout between phases with an all-to-all (the Appendix's `all2all`
 * lines), so that the next phase's gates find their qubits local.  This call is the schedule of
 * one such exchange; the data moves through the caller's collective library (NCCL or gloo
 * all-to-all with per-rank split sizes) and, locally, sim_permute.
 * Layout: position p < n - g is bit p of a rank's local index, position n - g + j bit j of the
 * rank number.  bit_of[q] = current position of qubit q (a bijection on 0..n-1); next_global: the
 * g qubits that must be global afterwards (any order).  Writes local_perm[p] (p < n - g): the new
 * local position of the amplitude bit now at local position p -- apply it to every rank's local
 * state first (the moving qubits O end at the top m local positions); bit_of_after[q]: the
 * positions after the all-to-all; *chunk_mask (may be NULL): the rank bits R that change.  The
 * all-to-all: a rank's local state is 2^m contiguous chunks of 2^(n-g-m) amplitudes; chunk c goes
 * to the rank that equals the sender outside R and holds c in R (bits of c in R's ascending order),
 * and the chunk from rank s is placed at index (s's bits in R); every other rank exchanges nothing.
 * Returns m (0: nothing moves, no collective needed) or a negative SIM_E_* code (SIM_E_INVAL for a
 * non-bijective bit_of, a repeated or out-of-range next_global entry, or g outside 0 .. n/2).
 * Host only. */
int sim_shard_exchange_plan(int n_qubits, int global_bits, const int *bit_of, const int *next_global,
                            int *local_perm, int *bit_of_after, uint64_t *chunk_mask);

/* ---- checkpoint / resume (not in the paper) --------------------------------
 * Save the whole state to a file, and load it back, e.g. at a phase boundary of a long streamed
 * run (sim_phases_get + sim_run_phase), to resume it in another process.  The file holds a header
 * (n, slice_bits, the sliced sets, the physical layout) and the 2^n complex64 amplitudes in
 * physical order: a host store's regions, device regions included, or the device state.
 * sim_state_load needs the same n and slice_bits; a device-store handle takes the file's layout,
 * a host-store handle must have the layout of the file (the same sliced sets).  Both are
 * synchronous: they wait for h's work and move the data through a bounded pinned buffer.
 * SIM_E_IO if the file cannot be opened, read or written, SIM_E_INVAL if it is not a state file
 * or does not fit h. */
int sim_state_save(sim_t *h, const char *path);
int sim_state_load(sim_t *h, const char *path);

/* ---- serving: many circuits on one GPU (no counterpart in the paper) --------
 * A continuous-batching server.  srv_submit plans the circuit (aggregation as
 * sim_plan_create) on the caller's thread and queues it; a scheduler thread
 * admits queued circuits in arrival order while their device footprint
 * (8 * 2^n bytes + 64 KiB) fits the HBM budget -- a circuit that does not fit
 * can be overtaken by at most 64 later ones -- and runs them concurrently:
 * circuits with n <= small_n go through a device-side queue served by a
 * persistent worker kernel (one thread block per circuit: reset, every block,
 * reduction; circuits published while it runs are taken up without a new launch,
 * and it ends after 200 us without work); larger ones run on `slots` streams with
 * stream-ordered memory.  A circuit always takes the same path and
 * plan, so its result does not depend on what else is in flight (srv_autotune fixes the
 * choices for the sizes it measured before any is served). */
typedef struct srv_s srv_t;

typedef struct srv_opts {
    int device;
    int slots;           /* concurrent circuits above small_n (0 = 6, max 32) */
    int small_n;         /* circuits with n <= small_n are packed (0 = 20, max 24) */
    int max_pack;        /* most circuits per packed launch (0 = 1024) */
    int kmax;            /* aggregation width (0 = 6 in SIM_FP16X3_TMEM and SIM_BF16X3, else 5, or 4 for n > 24
                          * in SIM_FP32); circuits above small_n run in the qubit layout
                          * sim_plan_layout picks and are permuted back before a readout */
    int precision;       /* circuits above small_n: any SIM_FP32 .. SIM_BF16X3 */
    uint64_t hbm_budget; /* device bytes for states (0 = 80% of free memory at creation) */
    int front_pairs;     /* contraction deferral for circuits of >= 26 qubits: the gates up to the
                          * (front_pairs + 1)-th across the bipartition sim_split_choose picks run
                          * as two tensors and one contraction -- in SIM_FP16X3_TMEM / SIM_BF16X3 on
                          * the tensor cores when they are >= 30% of the circuit (0 = 5); in
                          * SIM_FP32 on CUDA cores with at most 2 bridging gates when they are
                          * >= 10% (its cost grows 4x per bridging gate); < 0 = off; none in the
                          * other modes.  The tensors and the contraction's scratch count in the
                          * footprint */
    int max_large;       /* most circuits of >= 27 qubits running at once (0: 1 in SIM_FP32, 2 in the
                          * tensor-core modes -- each is HBM-bound, and sharing the bandwidth among
                          * more of them only delays them all; < 0: unlimited) */
    int reserved[6];
} srv_opts;

typedef struct srv_stats_t {
    uint64_t submitted, completed, rejected, in_flight;
    double p50_ms, p99_ms, mean_ms; /* latency: srv_submit's call (its planning included) ->
                                     * completion */
    double circuits_per_s;          /* completed / (last completion - first srv_submit call) */
    uint64_t hbm_budget, hbm_used;
    uint64_t graph_replays;         /* requests served by replaying a repeated circuit's CUDA graph */
} srv_stats_t;

int srv_create(const srv_opts *o, srv_t **out);
/* Finishes every queued circuit, then frees the server. */
int srv_destroy(srv_t *s);
const char *srv_last_error(const srv_t *s);

/* Queue one circuit (gate records as for sim_plan_create); out_amps, if not NULL,
 * receives all 2^n complex64 amplitudes (logical order) and must stay valid until
 * srv_wait returns for this ticket (pinned memory is faster).  SIM_E_BUSY if the
 * circuit can never fit the budget; SIM_E_INVAL for a bad gate list. */
int srv_submit(srv_t *s, int n_qubits, int n_gates, const sim_gate *gates, void *out_amps,
               uint64_t *ticket);

/* Wait at most timeout_ms (< 0: no limit) for a ticket; SIM_E_TIMEOUT if not done.
 * On success returns the circuit's norm, 2^n sum p^2 and its latency; the ticket
 * is then forgotten. */
int srv_wait(srv_t *s, uint64_t ticket, int timeout_ms, double *norm, double *sum_p2_scaled,
             double *latency_ms);

/* Counters and the latency distribution of completed circuits. */
int srv_stats(srv_t *s, srv_stats_t *out);

/* Autotuner of the server (not in the paper): for each sample circuit above small_n, measures on a
 * scratch state of its size every candidate the server could run it with -- block width k_max 4,
 * 5 and 6, and in SIM_FP16X3_TMEM / SIM_BF16X3 / SIM_FP32 from 22 qubits also with and without
 * the contraction-deferral front (unless front_pairs < 0) -- planned as srv_submit plans (the layout
 * sim_plan_layout picks), each run twice from the start state, the second timed with CUDA events;
 * the fastest is cached for the sample's (n, depth class) and used by every later srv_submit of a
 * circuit of that size and class (depth class: gates per qubit < 18, < 24, or more; an explicit
 * kmax in srv_opts still wins).  Writes the choice per sample (kmax_out, front_out: 0 / 1, ms_out:
 * its device time; 0 for samples the server packs); any output may be NULL.  Synchronous; call it
 * while the server is idle (its scratch states, 8 * 2^n bytes, are allocated outside the budget,
 * and its timings assume an idle device).  gates[i] points at sample i's n_gates[i] records. */
int srv_autotune(srv_t *s, int n_samples, const int *n_qubits, const int *n_gates, const sim_gate *const *gates,
                 int *kmax_out, int *front_out, double *ms_out);

#ifdef __cplusplus
}
#endif
#endif /* SYCSIM_H */
