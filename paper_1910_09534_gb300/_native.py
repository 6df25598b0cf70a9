"""ctypes binding of libsycsim.so (the C ABI in include/sycsim.h).

Argument marshalling only: every function forwards to the native library with the
same name.  Failures raise ``SimError`` carrying the status code and the library's
message.  Importing this module does not need a GPU; calling anything that touches
the device does.  If the library has not been built, ``lib()`` raises -- there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsycsim.so")

SIM_OK = 0
SIM_E_INVAL = -1
SIM_E_NOMEM_DEV = -2
SIM_E_NOMEM_HOST = -3
SIM_E_NONLOCAL = -4
SIM_E_CUDA = -5
SIM_E_TIMEOUT = -6
SIM_E_BUSY = -7
SIM_E_UNSUPPORTED = -8
SIM_E_IO = -9

SIM_FP32 = 0
SIM_TF32 = 1
SIM_TF32X3 = 2
SIM_FP16X3 = 3
SIM_FP16X3_TMEM = 4
SIM_BF16X3 = 5
SIM_C64 = 0
SIM_C128 = 1
SIM_STORE_DEVICE = 0
SIM_STORE_HOST = 1
SIM_H2D = 0
SIM_D2H = 1

SIM_GATE_SQRT_X = 0
SIM_GATE_SQRT_Y = 1
SIM_GATE_SQRT_W = 2
SIM_GATE_FSIM = 3
SIM_GATE_U1 = 4
SIM_GATE_U2 = 5

# numpy mirror of struct sim_gate
GATE_DTYPE = np.dtype([("kind", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("reserved", "<i4"),
                       ("theta", "<f8"), ("phi", "<f8"), ("dplus", "<f8"), ("dminus", "<f8"),
                       ("dminus_off", "<f8"), ("u", "<f8", (32,))], align=True)


class SimOpts(ctypes.Structure):
    _fields_ = [("store", ctypes.c_int), ("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("ext_state", ctypes.c_void_p), ("ext_bytes", ctypes.c_uint64),
                ("slots", ctypes.c_int), ("set_a", ctypes.c_int * 8), ("set_b", ctypes.c_int * 8),
                ("store_device_regions", ctypes.c_int), ("reserved", ctypes.c_int * 7)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("kmax", ctypes.c_int), ("precision", ctypes.c_int), ("search", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class SrvOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("slots", ctypes.c_int), ("small_n", ctypes.c_int),
                ("max_pack", ctypes.c_int), ("kmax", ctypes.c_int), ("precision", ctypes.c_int),
                ("hbm_budget", ctypes.c_uint64), ("front_pairs", ctypes.c_int), ("max_large", ctypes.c_int),
                ("reserved", ctypes.c_int * 6)]


class SrvStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("in_flight", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("circuits_per_s", ctypes.c_double), ("hbm_budget", ctypes.c_uint64),
                ("hbm_used", ctypes.c_uint64), ("graph_replays", ctypes.c_uint64)]


class SimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lib = None

_SIGS = {
    # name: (restype, argtypes)
    "sim_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "sim_version": (ctypes.c_char_p, []),
    "sim_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sim_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_state_ptr": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_reset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "sim_apply_fused": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int]),
    "sim_permute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_amplitudes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "sim_amplitudes_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_int]),
    "sim_load_amplitudes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_void_p, ctypes.c_int]),
    "sim_reduce": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_reduce_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sim_reduce_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "sim_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sim_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "sim_launch_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_host_alloc": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_void_p]),
    "sim_host_free": (ctypes.c_int, [ctypes.c_void_p]),
    "sim_gate_matrix": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "sim_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sim_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_plan_block": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "sim_apply_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_plan_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_set_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_graph_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "sim_graph_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_graph_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sim_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "sim_stream_slice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_int]),
    "sim_slot_ptr": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sim_slot_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_void_p]),
    "sim_run_phase": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sim_phases_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_phases_choose_sets": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sim_split_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "sim_split_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "sim_split_gates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sim_split_canonical": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sim_split_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "srv_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_plan_layout_front": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_shard_exchange_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_split_choose": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "sim_contract": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int]),
    "sim_front_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "sim_front_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_front_run_phase": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sim_phases_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "sim_contract_phase": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "sim_front_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sim_state_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "sim_state_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "sim_phases_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sim_phases_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_phases_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_run_phases": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "srv_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "srv_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "srv_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "srv_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "srv_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p]),
    "srv_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
}


def lib():
    """The loaded native library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_1910_09534_gb300.build.build() "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return a


def _check(rc: int, handle=None):
    if rc < 0:
        msg = lib().sim_last_error(handle)
        raise SimError(rc, msg.decode() if msg else "")
    return rc


# ---------------------------------------------------------------- C ABI, same names

def sim_version() -> str:
    return lib().sim_version().decode()


def sim_create(n_qubits: int, slice_bits: int = 0, device: int = 0, stream: int | None = None,
               ext_state: int | None = None, ext_bytes: int = 0, store: int = SIM_STORE_DEVICE,
               set_a=(), set_b=(), slots: int = 0, store_device_regions: int = 0):
    o = SimOpts()
    o.store_device_regions = store_device_regions
    o.store = store
    o.device = device
    o.stream = stream
    o.ext_state = ext_state
    o.ext_bytes = ext_bytes
    o.slots = slots
    for i, q in enumerate(set_a):
        o.set_a[i] = q
    for i, q in enumerate(set_b):
        o.set_b[i] = q
    h = ctypes.c_void_p()
    _check(lib().sim_create(n_qubits, slice_bits, ctypes.byref(o), ctypes.byref(h)))
    return h


def sim_destroy(h) -> None:
    _check(lib().sim_destroy(h))


def sim_info(h):
    n, s = ctypes.c_int(), ctypes.c_int()
    _check(lib().sim_info(h, ctypes.byref(n), ctypes.byref(s), None), h)
    bit_of = np.zeros(n.value, dtype=np.int32)
    _check(lib().sim_info(h, None, None, _ptr(bit_of)), h)
    return n.value, s.value, bit_of


def sim_state_ptr(h):
    p, st = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().sim_state_ptr(h, ctypes.byref(p), ctypes.byref(st)), h)
    return p.value, st.value


def sim_stream(h):
    """The handle's cudaStream_t only (sim_state_ptr without asking for the state's address)."""
    st = ctypes.c_void_p()
    _check(lib().sim_state_ptr(h, None, ctypes.byref(st)), h)
    return st.value


def sim_reset(h, basis: int = 0) -> None:
    _check(lib().sim_reset(h, basis), h)


def sim_apply_fused(h, targets, matrix, precision: int = SIM_FP32) -> None:
    t = np.ascontiguousarray(targets, dtype=np.int32)
    m = np.ascontiguousarray(matrix, dtype=np.complex128)
    if m.shape != (1 << t.size, 1 << t.size):
        raise ValueError("matrix must be 2^k x 2^k")
    _check(lib().sim_apply_fused(h, int(t.size), _ptr(t), _ptr(m), precision), h)


def sim_permute(h, perm) -> None:
    p = np.ascontiguousarray(perm, dtype=np.int32)
    _check(lib().sim_permute(h, _ptr(p)), h)


def sim_amplitudes(h, first: int = 0, count: int | None = None, dtype: int = SIM_C64,
                   physical_order: bool = False, out: np.ndarray | None = None) -> np.ndarray:
    n, _, _ = sim_info(h)
    if count is None:
        count = (1 << n) - first
    npdt = np.complex64 if dtype == SIM_C64 else np.complex128
    if out is None:
        out = np.empty(count, dtype=npdt)
    assert out.dtype == npdt and out.size >= count and out.flags.c_contiguous
    _check(lib().sim_amplitudes(h, first, count, _ptr(out), dtype, int(physical_order)), h)
    return out


def sim_amplitudes_async(h, out: np.ndarray, first: int = 0, physical_order: bool = False) -> np.ndarray:
    """Enqueue the readout of out.size complex64 amplitudes into `out` (keep it alive and
    untouched until sim_sync(h)); pinned memory (pinned_array) keeps the copy asynchronous."""
    assert out.dtype == np.complex64 and out.flags.c_contiguous
    _check(lib().sim_amplitudes_async(h, first, out.size, _ptr(out), int(physical_order)), h)
    return out


def sim_load_amplitudes(h, src: np.ndarray, first: int = 0, physical_order: bool = False) -> None:
    a = np.ascontiguousarray(src, dtype=np.complex64)
    _check(lib().sim_load_amplitudes(h, first, a.size, _ptr(a), int(physical_order)), h)


def sim_reduce(h):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().sim_reduce(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), h)
    return a.value, b.value, c.value


def sim_reduce_async(h, out: np.ndarray) -> None:
    """Enqueue sim_reduce's result {norm, 2^n sum p^2, xeb} into out (3 float64, ideally pinned:
    pinned_array); out is filled once the handle's stream has passed this point."""
    if out.dtype != np.float64 or out.size < 3 or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be a contiguous float64 array of at least 3 elements")
    _check(lib().sim_reduce_async(h, _ptr(out)), h)


def sim_reduce_noalloc(d_state: int, n_amps: int, d_out: int, stream: int | None = None) -> None:
    """Reduction over a caller-owned device buffer; writes 3 doubles to device memory d_out."""
    _check(lib().sim_reduce_noalloc(ctypes.c_void_p(d_state), n_amps, ctypes.c_void_p(d_out),
                                    ctypes.c_void_p(stream) if stream else None))


def sim_sync(h, timeout_ms: int = -1) -> None:
    _check(lib().sim_sync(h, timeout_ms), h)


SIM_PROF_APPLY = 0
SIM_PROF_PERMUTE = 1
SIM_PROF_REDUCE = 2
SIM_PROF_OTHER = 3
SIM_PROF_CONTRACT = 4


def sim_profile_enable(h, on: bool = True) -> None:
    _check(lib().sim_profile_enable(h, int(on)), h)


def sim_profile_read(h, cls: int):
    """(launches, total_ms, algorithmic_bytes) of one kernel class since profiling was enabled."""
    n, ms, b = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
    _check(lib().sim_profile_read(h, cls, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b)), h)
    return n.value, ms.value, b.value


def sim_launch_count(h) -> int:
    n = ctypes.c_uint64()
    _check(lib().sim_launch_count(h, ctypes.byref(n)), h)
    return n.value


def sim_host_alloc(nbytes: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().sim_host_alloc(nbytes, ctypes.byref(p)))
    return p.value


def sim_host_free(p: int) -> None:
    _check(lib().sim_host_free(ctypes.c_void_p(p)))


def pinned_array(count: int, dtype=np.complex64):
    """numpy array over pinned host memory; free with sim_host_free(arr.ctypes.data)."""
    nbytes = int(count) * np.dtype(dtype).itemsize
    p = sim_host_alloc(max(nbytes, 1))
    buf = (ctypes.c_char * max(nbytes, 1)).from_address(p)
    return np.frombuffer(buf, dtype=dtype, count=count)


def gates_array(circuit) -> np.ndarray:
    """struct sim_gate records of a syc_inputs.Circuit (or of (kind, q0, q1, theta, phi) tuples,
    optionally followed by the fSim detunings dplus, dminus, dminus_off)."""
    gates = circuit.gates if hasattr(circuit, "gates") else circuit
    a = np.zeros(len(gates), dtype=GATE_DTYPE)
    for i, g in enumerate(gates):
        a[i]["kind"], a[i]["q0"], a[i]["q1"] = g[0], g[1], g[2]
        a[i]["theta"], a[i]["phi"] = g[3], g[4]
        if len(g) > 5:
            a[i]["dplus"], a[i]["dminus"], a[i]["dminus_off"] = g[5], g[6], g[7]
    return a


def sim_gate_matrix(gate) -> np.ndarray:
    g = np.zeros(1, dtype=GATE_DTYPE)
    g[0] = gate
    out = np.zeros(32, dtype=np.float64)
    d = _check(lib().sim_gate_matrix(_ptr(g), _ptr(out)))
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def sim_plan_create(n_qubits: int, gates: np.ndarray, kmax: int = 4, precision: int = SIM_FP32, search: int = 0):
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    o = PlanOpts()
    o.kmax = kmax
    o.precision = precision
    o.search = search
    p = ctypes.c_void_p()
    _check(lib().sim_plan_create(n_qubits, int(g.size), _ptr(g), ctypes.byref(o), ctypes.byref(p)))
    return p


def sim_plan_destroy(p) -> None:
    _check(lib().sim_plan_destroy(p))


def sim_plan_info(p):
    nb, ng, mk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().sim_plan_info(p, ctypes.byref(nb), ctypes.byref(ng), ctypes.byref(mk)))
    return nb.value, ng.value, mk.value


def sim_plan_block(p, i: int):
    k = ctypes.c_int()
    _check(lib().sim_plan_block(p, i, ctypes.byref(k), None, None))
    t = np.zeros(k.value, dtype=np.int32)
    m = np.zeros((1 << k.value, 1 << k.value), dtype=np.complex128)
    _check(lib().sim_plan_block(p, i, None, _ptr(t), _ptr(m)))
    return t, m


def sim_plan_layout(p, n_qubits: int):
    """(perm, estimated ms for it, estimated ms for the identity layout) of a plan on n_qubits."""
    perm = np.zeros(n_qubits, dtype=np.int32)
    est = np.zeros(2, dtype=np.float64)
    _check(lib().sim_plan_layout(p, _ptr(perm), _ptr(est)))
    return [int(x) for x in perm], float(est[0]), float(est[1])


def sim_plan_layout_front(p, s, n_qubits: int):
    """(perm, estimate, identity estimate) for a plan whose state the contraction of split s writes."""
    perm = np.zeros(n_qubits, dtype=np.int32)
    est = np.zeros(2, dtype=np.float64)
    _check(lib().sim_plan_layout_front(p, s, _ptr(perm), _ptr(est)))
    return [int(x) for x in perm], float(est[0]), float(est[1])


def sim_set_layout(h, perm) -> None:
    pm = np.ascontiguousarray(perm, dtype=np.int32)
    _check(lib().sim_set_layout(h, _ptr(pm)), h)


def sim_apply_plan(h, p) -> None:
    _check(lib().sim_apply_plan(h, p), h)


def sim_graph_create(h, p):
    """CUDA graph of the plan's block launches on h (replay with sim_graph_launch)."""
    g = ctypes.c_void_p()
    _check(lib().sim_graph_create(h, p, ctypes.byref(g)), h)
    return g


def sim_graph_launch(h, g) -> None:
    _check(lib().sim_graph_launch(h, g), h)


def sim_graph_destroy(g) -> None:
    _check(lib().sim_graph_destroy(g))


SIM_TUNE_FP32 = 0
SIM_TUNE_FP32_EQUIVALENT = 1
SIM_TUNE_ANY = 2


def sim_autotune(h, gates: np.ndarray, accuracy: int = SIM_TUNE_FP32_EQUIVALENT):
    """(kmax, precision, ms) of the fastest plan for this circuit on h's device."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    o = PlanOpts()
    ms = ctypes.c_double()
    _check(lib().sim_autotune(h, int(g.size), _ptr(g), accuracy, ctypes.byref(o), ctypes.byref(ms)), h)
    return o.kmax, o.precision, ms.value


def sim_stream_slice(h, set_: int, value: int, direction: int, slot: int) -> None:
    _check(lib().sim_stream_slice(h, set_, value, direction, slot), h)


def sim_slot_ptr(h, slot: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().sim_slot_ptr(h, slot, ctypes.byref(p)))
    return p.value


def sim_slot_read(h, slot: int, first: int = 0, count: int | None = None) -> np.ndarray:
    n, s, _ = sim_info(h)
    if count is None:
        count = (1 << (n - s)) - first
    out = np.empty(count, dtype=np.complex64)
    _check(lib().sim_slot_read(h, slot, first, count, _ptr(out)), h)
    return out


def sim_run_phase(h, set_: int, plan) -> None:
    _check(lib().sim_run_phase(h, set_, plan), h)


def sim_phases_create(n_qubits: int, gates: np.ndarray, slice_bits: int, set_a, set_b, kmax: int = 4,
                      precision: int = SIM_FP32, search: int = 0):
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    a = np.ascontiguousarray(set_a, dtype=np.int32)
    b = np.ascontiguousarray(set_b, dtype=np.int32)
    o = PlanOpts()
    o.kmax = kmax
    o.precision = precision
    o.search = search
    p = ctypes.c_void_p()
    _check(lib().sim_phases_create(n_qubits, int(g.size), _ptr(g), ctypes.byref(o), slice_bits, _ptr(a),
                                   _ptr(b), ctypes.byref(p)))
    return p


def sim_phases_choose_sets(n_qubits: int, gates: np.ndarray, slice_bits: int, kmax: int = 4,
                           phase_weight: float = 0.0, search: int = 0):
    """(set_a, set_b, n_phases, n_blocks) chosen for the circuit; host only."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    o = PlanOpts()
    o.kmax = kmax
    o.search = search
    a = np.zeros(slice_bits, dtype=np.int32)
    b = np.zeros(slice_bits, dtype=np.int32)
    nph, nbl = ctypes.c_int(), ctypes.c_int()
    _check(lib().sim_phases_choose_sets(n_qubits, int(g.size), _ptr(g), slice_bits, ctypes.byref(o),
                                        float(phase_weight), _ptr(a), _ptr(b), ctypes.byref(nph),
                                        ctypes.byref(nbl)))
    return [int(x) for x in a], [int(x) for x in b], nph.value, nbl.value


def sim_split_create(n_qubits: int, gates: np.ndarray, side):
    """Contraction-deferral split of a gate list (side[q] = 0: tensor 1, 1: tensor 2)."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    sd = np.ascontiguousarray(side, dtype=np.int32)
    if sd.size != n_qubits:
        raise ValueError("side needs one entry per qubit")
    p = ctypes.c_void_p()
    _check(lib().sim_split_create(n_qubits, int(g.size), _ptr(g), _ptr(sd), ctypes.byref(p)))
    return p


def sim_split_info(s):
    """(n_side[2], n_wires[2], n_pairs, n_gates[2])."""
    ns = np.zeros(2, dtype=np.int32)
    nw = np.zeros(2, dtype=np.int32)
    ng = np.zeros(2, dtype=np.int32)
    npairs = ctypes.c_int()
    _check(lib().sim_split_info(s, _ptr(ns), _ptr(nw), ctypes.byref(npairs), _ptr(ng)))
    return [int(x) for x in ns], [int(x) for x in nw], npairs.value, [int(x) for x in ng]


def sim_split_gates(s, t: int) -> np.ndarray:
    ng = sim_split_info(s)[3][t]
    out = np.zeros(ng, dtype=GATE_DTYPE)
    _check(lib().sim_split_gates(s, t, _ptr(out) if ng else _ptr(np.zeros(1, dtype=GATE_DTYPE))))
    return out


def sim_split_canonical(s, t: int):
    nw = sim_split_info(s)[1][t]
    out = np.zeros(nw, dtype=np.int32)
    _check(lib().sim_split_canonical(s, t, _ptr(out)))
    return [int(x) for x in out]


def sim_split_choose(n_qubits: int, gates: np.ndarray, max_pairs: int = 5, min_side: int = 0):
    """(side, n_front): a bipartition and the gate-list prefix for contraction deferral."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    side = np.zeros(n_qubits, dtype=np.int32)
    nf = ctypes.c_int()
    _check(lib().sim_split_choose(n_qubits, int(g.size), _ptr(g), max_pairs, min_side, _ptr(side), ctypes.byref(nf)))
    return [int(x) for x in side], nf.value


def sim_split_destroy(s) -> None:
    _check(lib().sim_split_destroy(s))


def sim_contract(out, t1, t2, s, precision: int = SIM_FP32) -> None:
    _check(lib().sim_contract(out, t1, t2, s, precision), out)


def sim_front_create(out, s, kmax: int = 4, precision: int = SIM_FP32):
    """Both tensors of split s planned and allocated on out's device and stream."""
    o = PlanOpts()
    o.kmax = kmax
    o.precision = precision
    f = ctypes.c_void_p()
    _check(lib().sim_front_create(out, s, ctypes.byref(o), ctypes.byref(f)), out)
    return f


def sim_front_run(out, f) -> None:
    _check(lib().sim_front_run(out, f), out)


def sim_front_run_phase(out, f, set_: int = 0, plan=None) -> None:
    """sim_front_run, then plan's blocks on the contracted state (one pass into a host store whose
    phase slices set_: 0 = A, 1 = B)."""
    _check(lib().sim_front_run_phase(out, f, set_, plan), out)


def sim_contract_phase(out, t1, t2, s, precision: int = SIM_FP32, set_: int = 0, plan=None) -> None:
    """Contraction slice by slice into a host store's slices of set_ (0 = A, 1 = B), plan's blocks
    on each, one write."""
    _check(lib().sim_contract_phase(out, t1, t2, s, precision, set_, plan), out)


def sim_front_destroy(f) -> None:
    _check(lib().sim_front_destroy(f))


def sim_state_save(h, path: str) -> None:
    _check(lib().sim_state_save(h, os.fsencode(path)), h)


def sim_state_load(h, path: str) -> None:
    _check(lib().sim_state_load(h, os.fsencode(path)), h)


def sim_phases_destroy(ph) -> None:
    _check(lib().sim_phases_destroy(ph))


def sim_phases_info(ph):
    n, t = ctypes.c_int(), ctypes.c_int()
    _check(lib().sim_phases_info(ph, ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def sim_phases_layout(ph, n_qubits: int, front=None, resident: bool = False):
    """(perm, estimate, starting estimate): the order of the qubits outside the sliced sets for the
    phases ph -- a host store's (resident False) or a device-resident sliced handle's (the first
    phase's set on top); front: the split whose contraction writes the state first, or None."""
    perm = np.zeros(n_qubits, dtype=np.int32)
    est = np.zeros(2, dtype=np.float64)
    _check(lib().sim_phases_layout(ph, front, 1 if resident else 0, _ptr(perm), _ptr(est)))
    return [int(x) for x in perm], float(est[0]), float(est[1])


def sim_phases_get(ph, i: int):
    s, p = ctypes.c_int(), ctypes.c_void_p()
    _check(lib().sim_phases_get(ph, i, ctypes.byref(s), ctypes.byref(p)))
    return s.value, p


def sim_run_phases(h, ph) -> None:
    _check(lib().sim_run_phases(h, ph), h)


def _srv_check(rc: int, srv=None):
    if rc < 0:
        msg = lib().srv_last_error(srv)
        raise SimError(rc, msg.decode() if msg else "")
    return rc


def srv_create(device: int = 0, slots: int = 0, small_n: int = 0, max_pack: int = 0, kmax: int = 0,
               precision: int = SIM_FP32, hbm_budget: int = 0, front_pairs: int = 0, max_large: int = 0):
    o = SrvOpts()
    o.device, o.slots, o.small_n, o.max_pack, o.kmax, o.precision = device, slots, small_n, max_pack, kmax, precision
    o.hbm_budget = hbm_budget
    o.front_pairs = front_pairs
    o.max_large = max_large
    srv = ctypes.c_void_p()
    _srv_check(lib().srv_create(ctypes.byref(o), ctypes.byref(srv)))
    return srv


def srv_destroy(srv) -> None:
    _srv_check(lib().srv_destroy(srv))


def srv_submit(srv, n_qubits: int, gates: np.ndarray, out_amps: np.ndarray | None = None) -> int:
    """Queue a circuit; out_amps (complex64, 2^n, kept alive by the caller) receives the amplitudes."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    if out_amps is not None:
        assert out_amps.dtype == np.complex64 and out_amps.size >= (1 << n_qubits) and out_amps.flags.c_contiguous
    t = ctypes.c_uint64()
    _srv_check(lib().srv_submit(srv, n_qubits, int(g.size), _ptr(g), _ptr(out_amps), ctypes.byref(t)), srv)
    return t.value


def srv_wait(srv, ticket: int, timeout_ms: int = -1):
    """(norm, 2^n sum p^2, latency_ms) of a finished circuit."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _srv_check(lib().srv_wait(srv, ticket, timeout_ms, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), srv)
    return a.value, b.value, c.value


def srv_stats(srv) -> dict:
    st = SrvStats()
    _srv_check(lib().srv_stats(srv, ctypes.byref(st)), srv)
    return {f: getattr(st, f) for f, _ in SrvStats._fields_}


def sim_shard_exchange_plan(n_qubits: int, global_bits: int, bit_of, next_global):
    """Schedule of one exchange of a sharded state: (m, local_perm, bit_of_after, chunk_mask)."""
    b = np.ascontiguousarray(bit_of, dtype=np.int32)
    ng = np.ascontiguousarray(next_global, dtype=np.int32)
    lp = np.zeros(max(n_qubits - global_bits, 1), dtype=np.int32)
    after = np.zeros(n_qubits, dtype=np.int32)
    mask = ctypes.c_uint64()
    m = _check(lib().sim_shard_exchange_plan(n_qubits, global_bits, _ptr(b), _ptr(ng) if ng.size else None,
                                             _ptr(lp), _ptr(after), ctypes.byref(mask)))
    return m, [int(x) for x in lp[: n_qubits - global_bits]], [int(x) for x in after], int(mask.value)


def srv_autotune(s, circuits):
    """circuits: (n_qubits, gate records) samples; returns [(kmax, front, ms)] per sample (0s for
    circuits the server packs)."""
    k = len(circuits)
    nq = np.array([c[0] for c in circuits], dtype=np.int32)
    arrs = [np.ascontiguousarray(c[1], dtype=GATE_DTYPE) for c in circuits]
    ng = np.array([a.size for a in arrs], dtype=np.int32)
    ptrs = (ctypes.c_void_p * max(k, 1))(*[a.ctypes.data for a in arrs])
    km = np.zeros(max(k, 1), dtype=np.int32)
    fr = np.zeros(max(k, 1), dtype=np.int32)
    ms = np.zeros(max(k, 1), dtype=np.float64)
    rc = lib().srv_autotune(s, k, _ptr(nq), _ptr(ng), ptrs, _ptr(km), _ptr(fr), _ptr(ms))
    if rc < 0:
        raise SimError(rc, lib().srv_last_error(s).decode())
    return [(int(km[i]), int(fr[i]), float(ms[i])) for i in range(k)]


def exported_symbols() -> list:
    return list(_SIGS)
