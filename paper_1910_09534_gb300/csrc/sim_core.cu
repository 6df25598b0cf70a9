// sim_core.cu -- handle lifecycle, layout bookkeeping, readout/load, reductions, sync.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <thread>

#include "internal.h"

namespace sycsim {

static thread_local std::string t_err;

void set_thread_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
}

const char *thread_error() { return t_err.c_str(); }

int fail(sim_t *h, int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        t_err = buf;
    return code;
}

bool layout_is_identity(const sim_t *h)
{
    for (int q = 0; q < h->n; q++)
        if (h->bit_of[q] != q) return false;
    return true;
}

uint64_t logical_to_physical(const sim_t *h, uint64_t i)
{
    uint64_t j = 0;
    for (int q = 0; q < h->n; q++)
        if ((i >> q) & 1) j |= 1ull << h->bit_of[q];
    return j;
}

int prof_begin(sim_t *h, int cls, double alg_bytes, cudaStream_t st)
{
    h->launches++;
    if (!h->prof_on) return -1;
    if (h->prof_used == (int)h->prof.size()) {
        if (h->prof.size() >= 65536) return -1;  // bounded: later launches go untimed
        sim_s::ProfSlot s;
        if (cudaEventCreate(&s.a) != cudaSuccess || cudaEventCreate(&s.b) != cudaSuccess) return -1;
        h->prof.push_back(s);
    }
    const int i = h->prof_used++;
    h->prof[i].cls = cls;
    h->prof[i].bytes = alg_bytes;
    cudaEventRecord(h->prof[i].a, st);
    return i;
}

void prof_end(sim_t *h, int slot, cudaStream_t st)
{
    if (slot >= 0) cudaEventRecord(h->prof[slot].b, st);
}

static void release(sim_t *h)
{
    if (!h) return;
    DeviceScope dev_scope(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto &s : h->prof) {
        cudaEventDestroy(s.a);
        cudaEventDestroy(s.b);
    }
    host_store_release(h);
    if (h->own_state && h->d_state) cudaFree(h->d_state);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->d_result) cudaFree(h->d_result);
    if (h->h_result) cudaFreeHost(h->h_result);
    if (h->d_stage) cudaFree(h->d_stage);
    if (h->d_mat6) cudaFree(h->d_mat6);
    if (h->h_mat6) cudaFreeHost(h->h_mat6);
    for (auto &e : h->mat6_ev)
        if (e) cudaEventDestroy(e);
    if (h->d_frag) cudaFree(h->d_frag);
    for (int i = 0; i < 2; i++) {
        if (h->h_plan[i]) cudaFreeHost(h->h_plan[i]);
        if (h->d_plan[i]) cudaFree(h->d_plan[i]);
        if (h->plan_ev[i]) cudaEventDestroy(h->plan_ev[i]);
    }
    if (h->d_errflag) cudaFree(h->d_errflag);
    if (h->d_contract) cudaFree(h->d_contract);
    if (h->h_frag) cudaFreeHost(h->h_frag);
    for (auto &e : h->frag_ev)
        if (e) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // namespace sycsim

using namespace sycsim;

extern "C" {

const char *sim_last_error(const sim_t *h) { return h ? h->err.c_str() : thread_error(); }

const char *sim_version(void) { return "sycsim 0.1 (sm_103a)"; }

int sim_create(int n_qubits, int slice_bits, const sim_opts *opts, sim_t **out)
{
    if (!out) return fail(nullptr, SIM_E_INVAL, "sim_create: out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > kMaxQubits)
        return fail(nullptr, SIM_E_INVAL, "sim_create: n_qubits=%d outside 1..%d", n_qubits,
                    kMaxQubits);
    if (slice_bits < 0 || slice_bits >= n_qubits)
        return fail(nullptr, SIM_E_INVAL, "sim_create: slice_bits=%d outside 0..n-1", slice_bits);
    sim_opts o{};
    if (opts) o = *opts;
    if (o.store != SIM_STORE_DEVICE && o.store != SIM_STORE_HOST)
        return fail(nullptr, SIM_E_INVAL, "sim_create: store mode %d", o.store);

    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0)
        return fail(nullptr, SIM_E_CUDA, "sim_create: no CUDA device (%s)", cudaGetErrorString(ce));
    if (o.device < 0 || o.device >= ndev)
        return fail(nullptr, SIM_E_INVAL, "sim_create: device %d outside 0..%d", o.device, ndev - 1);

    sim_t *h = new sim_t();
    h->n = n_qubits;
    h->s = slice_bits;
    h->store = o.store;
    h->device = o.device;
    h->amps = 1ull << n_qubits;
    for (int q = 0; q < n_qubits; q++) h->bit_of[q] = h->qubit_at[q] = q;

#define CREATE_TRY(call, code)                                                            \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            int c_ = fail(nullptr, (code), "sim_create: %s failed: %s", #call,             \
                          cudaGetErrorString(e_));                                        \
            release(h);                                                                   \
            return c_;                                                                    \
        }                                                                                 \
    } while (0)

    DeviceScope dev_scope(h->device);
    CREATE_TRY(dev_scope.err, SIM_E_CUDA);
    if (o.stream) {
        h->stream = (cudaStream_t)o.stream;
    } else {
        CREATE_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), SIM_E_CUDA);
        h->own_stream = true;
    }
    const uint64_t bytes = h->amps * sizeof(float2);
    if (h->store == SIM_STORE_HOST) {
        const int rc = host_store_create(h, o);
        if (rc != SIM_OK) {
            release(h);
            return rc;
        }
    } else if (o.ext_state) {
        if (o.ext_bytes < bytes || ((uintptr_t)o.ext_state & 15)) {
            release(h);
            return fail(nullptr, SIM_E_INVAL,
                        "sim_create: ext_state needs >= %llu bytes, 16-byte aligned",
                        (unsigned long long)bytes);
        }
        h->d_state = (float2 *)o.ext_state;
    } else {
        CREATE_TRY(cudaMalloc(&h->d_state, bytes), SIM_E_NOMEM_DEV);
        h->own_state = true;
    }
    CREATE_TRY(cudaMalloc(&h->d_partials, sizeof(double) * 2 * kReduceBlocks), SIM_E_NOMEM_DEV);
    CREATE_TRY(cudaMalloc(&h->d_result, sizeof(double) * 8), SIM_E_NOMEM_DEV);
    CREATE_TRY(cudaHostAlloc(&h->h_result, sizeof(double) * 4, cudaHostAllocDefault),
               SIM_E_NOMEM_HOST);
    const uint64_t stage = h->amps < kStageAmps ? h->amps : kStageAmps;
    if (h->store == SIM_STORE_DEVICE)
        CREATE_TRY(cudaMalloc(&h->d_stage, stage * sizeof(float2)), SIM_E_NOMEM_DEV);
    CREATE_TRY(cudaMalloc(&h->d_mat6, sizeof(float2) * 4096 * sim_s::kMat6Slots), SIM_E_NOMEM_DEV);
    CREATE_TRY(cudaHostAlloc(&h->h_mat6, sizeof(float2) * 4096 * sim_s::kMat6Slots,
                             cudaHostAllocDefault),
               SIM_E_NOMEM_HOST);
    for (auto &e : h->mat6_ev) CREATE_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), SIM_E_CUDA);
    CREATE_TRY(cudaMalloc(&h->d_frag, sizeof(uint32_t) * sim_s::kFragWords * sim_s::kFragSlots),
               SIM_E_NOMEM_DEV);
    CREATE_TRY(cudaHostAlloc(&h->h_frag, sizeof(uint32_t) * sim_s::kFragWords * sim_s::kFragSlots,
                             cudaHostAllocDefault),
               SIM_E_NOMEM_HOST);
    for (auto &e : h->frag_ev) CREATE_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), SIM_E_CUDA);
    CREATE_TRY(cudaMalloc(&h->d_errflag, sizeof(int)), SIM_E_NOMEM_DEV);
    CREATE_TRY(cudaMemset(h->d_errflag, 0, sizeof(int)), SIM_E_CUDA);
#undef CREATE_TRY

    int rc = sim_reset(h, 0);
    if (rc != SIM_OK) {
        fail(nullptr, rc, "sim_create: reset failed: %s", h->err.c_str());
        release(h);
        return rc;
    }
    *out = h;
    return SIM_OK;
}

int sim_destroy(sim_t *h)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_destroy: NULL handle");
    release(h);
    return SIM_OK;
}

int sim_info(const sim_t *h, int *n_qubits, int *slice_bits, int *bit_of)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_info: NULL handle");
    if (n_qubits) *n_qubits = h->n;
    if (slice_bits) *slice_bits = h->s;
    if (bit_of)
        for (int q = 0; q < h->n; q++) bit_of[q] = h->bit_of[q];
    return SIM_OK;
}

int sim_state_ptr(const sim_t *h, void **dptr, void **stream)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_state_ptr: NULL handle");
    if (h->store != SIM_STORE_DEVICE)
        return fail(nullptr, SIM_E_UNSUPPORTED, "sim_state_ptr: state is in the host store (sim_slot_ptr)");
    if (dptr) {
        *dptr = h->d_state;
        h->state_exposed = true;  // the caller may write it behind the handle's back
    }
    if (stream) *stream = (void *)h->stream;
    return SIM_OK;
}

int sim_reset(sim_t *h, uint64_t basis)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_reset: NULL handle");
    state_written(h);
    if (h->n < 64 && (basis >> h->n) != 0)
        return fail(h, SIM_E_INVAL, "sim_reset: basis index has bits above n=%d", h->n);
    SIM_DEVICE_SCOPE(h, h->device);
    if (h->store == SIM_STORE_HOST) return host_reset(h, basis);
    SIM_CUDA_TRY(h, cudaMemsetAsync(h->d_state, 0, h->amps * sizeof(float2), h->stream));
    const int ps = prof_begin(h, SIM_PROF_OTHER, 0.0, h->stream);
    const int rc = launch_set_basis(h->d_state, h->amps, logical_to_physical(h, basis), h->stream);
    prof_end(h, ps, h->stream);
    return rc == 0 ? SIM_OK
                   : fail(h, SIM_E_CUDA, "sim_reset: launch failed: %s",
                          cudaGetErrorString(cudaGetLastError()));
}

// After the handle's streams are idle: report (and clear) a kernel's bounded wait running out.
static int check_device_error(sim_t *h)
{
    int flag = 0;
    SIM_CUDA_TRY(h, cudaMemcpy(&flag, h->d_errflag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        SIM_CUDA_TRY(h, cudaMemset(h->d_errflag, 0, sizeof(int)));
        return fail(h, SIM_E_TIMEOUT, "a tensor-core apply gave up waiting for its MMAs; state is invalid");
    }
    return SIM_OK;
}

int sim_sync(sim_t *h, int timeout_ms)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_sync: NULL handle");
    SIM_DEVICE_SCOPE(h, h->device);
    if (timeout_ms < 0) {
        if (h->st_in) SIM_CUDA_TRY(h, cudaStreamSynchronize(h->st_in));
        SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        if (h->st_out) SIM_CUDA_TRY(h, cudaStreamSynchronize(h->st_out));
        return check_device_error(h);
    }
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(h->stream);
        if (e == cudaSuccess && h->st_in) e = cudaStreamQuery(h->st_in);
        if (e == cudaSuccess && h->st_out) e = cudaStreamQuery(h->st_out);
        if (e == cudaSuccess) return check_device_error(h);
        if (e != cudaErrorNotReady)
            return fail(h, SIM_E_CUDA, "sim_sync: %s", cudaGetErrorString(e));
        auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                      std::chrono::steady_clock::now() - t0)
                      .count();
        if (ms >= timeout_ms)
            return fail(h, SIM_E_TIMEOUT, "sim_sync: stream still busy after %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Expand n complex64 values at the front of buf into complex128, in place (back to front).
static void expand_c64_to_c128(void *buf, uint64_t n)
{
    const float *src = (const float *)buf;
    double *dst = (double *)buf;
    for (uint64_t i = n; i-- > 0;) {
        double re = src[2 * i], im = src[2 * i + 1];
        dst[2 * i] = re;
        dst[2 * i + 1] = im;
    }
}

int sim_amplitudes(sim_t *h, uint64_t first, uint64_t count, void *out, int dtype,
                   int physical_order)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_amplitudes: NULL handle");
    if (dtype != SIM_C64 && dtype != SIM_C128)
        return fail(h, SIM_E_INVAL, "sim_amplitudes: dtype %d", dtype);
    if (first > h->amps || count > h->amps - first)
        return fail(h, SIM_E_INVAL, "sim_amplitudes: range [%llu, +%llu) outside 2^%d",
                    (unsigned long long)first, (unsigned long long)count, h->n);
    if (count == 0) return SIM_OK;
    if (!out) return fail(h, SIM_E_INVAL, "sim_amplitudes: out is NULL");
    SIM_DEVICE_SCOPE(h, h->device);
    if (h->store == SIM_STORE_HOST) return host_amplitudes(h, first, count, out, dtype, physical_order);
    char *dst = (char *)out;
    if (physical_order || layout_is_identity(h)) {
        SIM_CUDA_TRY(h, cudaMemcpyAsync(dst, h->d_state + first, count * sizeof(float2),
                                        cudaMemcpyDeviceToHost, h->stream));
    } else {
        const uint64_t stage = h->amps < kStageAmps ? h->amps : kStageAmps;
        for (uint64_t done = 0; done < count; done += stage) {
            uint64_t c = count - done < stage ? count - done : stage;
            const int ps = prof_begin(h, SIM_PROF_OTHER, 16.0 * c, h->stream);
            const int rc = launch_gather_logical(h->d_state, h->d_stage, first + done, c, h->n,
                                                 h->bit_of, 0, h->stream);
            prof_end(h, ps, h->stream);
            if (rc != 0)
                return fail(h, SIM_E_CUDA, "sim_amplitudes: gather launch failed: %s",
                            cudaGetErrorString(cudaGetLastError()));
            SIM_CUDA_TRY(h, cudaMemcpyAsync(dst + done * sizeof(float2), h->d_stage,
                                            c * sizeof(float2), cudaMemcpyDeviceToHost, h->stream));
            SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // staging is reused
        }
    }
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (dtype == SIM_C128) expand_c64_to_c128(out, count);
    return SIM_OK;
}

int sim_amplitudes_async(sim_t *h, uint64_t first, uint64_t count, void *out, int physical_order)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_amplitudes_async: NULL handle");
    if (first > h->amps || count > h->amps - first)
        return fail(h, SIM_E_INVAL, "sim_amplitudes_async: range [%llu, +%llu) outside 2^%d",
                    (unsigned long long)first, (unsigned long long)count, h->n);
    if (count == 0) return SIM_OK;
    if (!out) return fail(h, SIM_E_INVAL, "sim_amplitudes_async: out is NULL");
    if (h->store == SIM_STORE_HOST)
        return fail(h, SIM_E_UNSUPPORTED, "sim_amplitudes_async: host-store handle (use sim_amplitudes)");
    if (!physical_order && !layout_is_identity(h))
        return fail(h, SIM_E_UNSUPPORTED,
                    "sim_amplitudes_async: logical order of a permuted layout (use sim_amplitudes)");
    SIM_DEVICE_SCOPE(h, h->device);
    SIM_CUDA_TRY(h, cudaMemcpyAsync(out, h->d_state + first, count * sizeof(float2), cudaMemcpyDeviceToHost,
                                    h->stream));
    return SIM_OK;
}

int sim_load_amplitudes(sim_t *h, uint64_t first, uint64_t count, const void *src,
                        int physical_order)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_load_amplitudes: NULL handle");
    state_written(h);
    if (first > h->amps || count > h->amps - first)
        return fail(h, SIM_E_INVAL, "sim_load_amplitudes: range outside the state");
    if (count == 0) return SIM_OK;
    if (!src) return fail(h, SIM_E_INVAL, "sim_load_amplitudes: src is NULL");
    SIM_DEVICE_SCOPE(h, h->device);
    if (h->store == SIM_STORE_HOST) return host_load(h, first, count, src, physical_order);
    const char *s = (const char *)src;
    if (physical_order || layout_is_identity(h)) {
        SIM_CUDA_TRY(h, cudaMemcpyAsync(h->d_state + first, s, count * sizeof(float2),
                                        cudaMemcpyHostToDevice, h->stream));
    } else {
        const uint64_t stage = h->amps < kStageAmps ? h->amps : kStageAmps;
        for (uint64_t done = 0; done < count; done += stage) {
            uint64_t c = count - done < stage ? count - done : stage;
            SIM_CUDA_TRY(h, cudaMemcpyAsync(h->d_stage, s + done * sizeof(float2),
                                            c * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
            const int ps = prof_begin(h, SIM_PROF_OTHER, 16.0 * c, h->stream);
            const int rc = launch_gather_logical(h->d_state, h->d_stage, first + done, c, h->n,
                                                 h->bit_of, 1, h->stream);
            prof_end(h, ps, h->stream);
            if (rc != 0)
                return fail(h, SIM_E_CUDA, "sim_load_amplitudes: scatter launch failed: %s",
                            cudaGetErrorString(cudaGetLastError()));
            SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        }
    }
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SIM_OK;
}

}  // extern "C"

namespace {

// (sum p, sum p^2) of h's state into d_result[0..1] on h's stream: the combine of the partial sums
// the plan's last block left when they are of exactly this state, else the full reduction.
int enqueue_reduce(sim_t *h)
{
    if (h->red_epoch == h->write_epoch && h->red_blocks > 0) {
        h->launches++;
        return launch_reduce_final(h->d_partials, h->red_blocks, h->d_result, h->stream);
    }
    const int ps = prof_begin(h, SIM_PROF_REDUCE, 8.0 * (double)h->amps, h->stream);
    h->launches++;  // the reduction is two kernels (partials + final)
    const int rc = launch_reduce(h, h->d_state, h->amps, h->d_partials, h->d_result, h->stream);
    prof_end(h, ps, h->stream);
    return rc;
}

}  // namespace

extern "C" {

int sim_reduce_async(sim_t *h, double *out)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_reduce_async: NULL handle");
    if (!out) return fail(h, SIM_E_INVAL, "sim_reduce_async: out is NULL");
    if (h->store != SIM_STORE_DEVICE)
        return fail(h, SIM_E_UNSUPPORTED, "sim_reduce_async: host-store state: use sim_reduce");
    SIM_DEVICE_SCOPE(h, h->device);
    if (enqueue_reduce(h) != 0 || launch_result3(h->d_result, std::ldexp(1.0, h->n), h->stream) != 0)
        return fail(h, SIM_E_CUDA, "sim_reduce_async: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    h->launches++;
    SIM_CUDA_TRY(h, cudaMemcpyAsync(out, h->d_result + 4, sizeof(double) * 3, cudaMemcpyDeviceToHost, h->stream));
    return SIM_OK;
}

int sim_reduce(sim_t *h, double *norm, double *sum_p2_scaled, double *xeb)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_reduce: NULL handle");
    SIM_DEVICE_SCOPE(h, h->device);
    if (h->store == SIM_STORE_HOST) {
        double a = 0.0, b = 0.0;
        const int rc = host_reduce(h, &a, &b);
        if (rc != SIM_OK) return rc;
        if (norm) *norm = a;
        if (sum_p2_scaled) *sum_p2_scaled = ldexp(b, h->n);
        if (xeb) *xeb = ldexp(b, h->n) - 1.0;
        return SIM_OK;
    }
    if (enqueue_reduce(h) != 0)
        return fail(h, SIM_E_CUDA, "sim_reduce: launch failed: %s",
                    cudaGetErrorString(cudaGetLastError()));
    SIM_CUDA_TRY(h, cudaMemcpyAsync(h->h_result, h->d_result, sizeof(double) * 2,
                                    cudaMemcpyDeviceToHost, h->stream));
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const double s1 = h->h_result[0], s2 = ldexp(h->h_result[1], h->n);
    if (norm) *norm = s1;
    if (sum_p2_scaled) *sum_p2_scaled = s2;
    if (xeb) *xeb = s2 - 1.0;
    return SIM_OK;
}

int sim_profile_enable(sim_t *h, int on)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_profile_enable: NULL handle");
    SIM_DEVICE_SCOPE(h, h->device);
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->prof_on = on != 0;
    h->prof_used = 0;
    return SIM_OK;
}

int sim_profile_read(sim_t *h, int cls, uint64_t *launches, double *total_ms, double *alg_bytes)
{
    if (!h) return fail(nullptr, SIM_E_INVAL, "sim_profile_read: NULL handle");
    SIM_DEVICE_SCOPE(h, h->device);
    SIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    uint64_t n = 0;
    double ms = 0.0, bytes = 0.0;
    for (int i = 0; i < h->prof_used; i++) {
        if (h->prof[i].cls != cls) continue;
        float e = 0.f;
        SIM_CUDA_TRY(h, cudaEventElapsedTime(&e, h->prof[i].a, h->prof[i].b));
        n++;
        ms += e;
        bytes += h->prof[i].bytes;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    if (alg_bytes) *alg_bytes = bytes;
    return SIM_OK;
}

int sim_launch_count(const sim_t *h, uint64_t *n)
{
    if (!h || !n) return fail(nullptr, SIM_E_INVAL, "sim_launch_count: NULL argument");
    *n = h->launches;
    return SIM_OK;
}

int sim_host_alloc(size_t bytes, void **out)
{
    if (!out) return fail(nullptr, SIM_E_INVAL, "sim_host_alloc: out is NULL");
    cudaError_t e = cudaHostAlloc(out, bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(nullptr, SIM_E_NOMEM_HOST, "sim_host_alloc(%zu): %s", bytes,
                    cudaGetErrorString(e));
    }
    return SIM_OK;
}

int sim_host_free(void *p)
{
    cudaError_t e = cudaFreeHost(p);
    if (e != cudaSuccess)
        return fail(nullptr, SIM_E_CUDA, "sim_host_free: %s", cudaGetErrorString(e));
    return SIM_OK;
}

}  // extern "C"
