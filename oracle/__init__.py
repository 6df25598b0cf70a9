"""CPU oracle for the fused-gate state-vector path (arXiv:1910.09534).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this package; the product library never
does, and it shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C, complex128, gate by gate); this
module only loads it with ctypes and converts numpy arrays.  Every function is
pinned in ``tests/test_oracle_pins.py`` against closed forms, invariants and
brute-force full-operator products; the contraction-deferral tensors (``split_tensors``,
``contract``) against full-operator products of detuned (qubit-order-sensitive) circuits,
outer products, the EI copy structure and the tensors' norms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP on) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fcx-limited-range", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.orc_set_threads.argtypes = [i32]
        L.orc_max_threads.restype = i32
        L.orc_gate_matrix.argtypes = [i32, f64, f64, f64, f64, f64, P]
        L.orc_gate_matrix.restype = i32
        L.orc_apply_1q.argtypes = [P, i32, i32, P]
        L.orc_apply_2q.argtypes = [P, i32, i32, i32, P]
        L.orc_apply_kq.argtypes = [P, i32, i32, P, P]
        L.orc_apply_kq.restype = i32
        L.orc_basis_state.argtypes = [P, i32, u64]
        L.orc_apply_gates.argtypes = [P, i32, i32, P, P, P, P, P, P, P, P]
        L.orc_apply_gates.restype = i32
        L.orc_permute.argtypes = [P, P, i32, P, i32]
        L.orc_permute.restype = i32
        L.orc_slice_move.argtypes = [P, P, i32, i32, P, u64, i32, i32]
        L.orc_slice_move.restype = i32
        L.orc_reduce.argtypes = [P, i32, P, P, P]
        L.orc_split_tensors.argtypes = [i32, i32, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_split_tensors.restype = i32
        L.orc_contract.argtypes = [P, i32, P, i32, i32, P, P, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _nq(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    if psi.size != (1 << n):
        raise ValueError("state length is not a power of two")
    return n


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def gate_matrix(kind: int, theta: float = 0.0, phi: float = 0.0, dplus: float = 0.0,
                dminus: float = 0.0, dminus_off: float = 0.0) -> np.ndarray:
    """2x2 (sqrt X/Y/W) or 4x4 (fSim, Eq. 1) complex128 matrix."""
    out = np.zeros(16, dtype=np.complex128)
    d = lib().orc_gate_matrix(int(kind), theta, phi, dplus, dminus, dminus_off, _ptr(out))
    if d == 0:
        raise ValueError(f"unknown gate kind {kind}")
    return out[: d * d].reshape(d, d).copy()


def apply_1q(psi: np.ndarray, q: int, u: np.ndarray) -> None:
    u = np.ascontiguousarray(u, dtype=np.complex128)
    lib().orc_apply_1q(_ptr(psi), _nq(psi), int(q), _ptr(u))


def apply_2q(psi: np.ndarray, q0: int, q1: int, u: np.ndarray) -> None:
    u = np.ascontiguousarray(u, dtype=np.complex128)
    lib().orc_apply_2q(_ptr(psi), _nq(psi), int(q0), int(q1), _ptr(u))


def apply_kq(psi: np.ndarray, targets, u: np.ndarray) -> None:
    """In place: the fused k-qubit block u on `targets` (bit j of u's index = targets[j])."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    t = np.ascontiguousarray(targets, dtype=np.int32)
    u = np.ascontiguousarray(u, dtype=np.complex128)
    rc = lib().orc_apply_kq(_ptr(psi), _nq(psi), int(t.size), _ptr(t), _ptr(u))
    if rc != 0:
        raise ValueError("bad targets")


def basis_state(n: int, basis: int = 0) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().orc_basis_state(_ptr(psi), int(n), int(basis))
    return psi


def apply_gates(psi: np.ndarray, circuit) -> None:
    """Apply a syc_inputs.Circuit (or a sequence of gate tuples, fSim detunings D+, D-, D-,off
    as elements 5..7 where present) gate by gate, in place."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    cols = [np.ascontiguousarray(c) for c in _gate_columns(circuit)]
    kind = cols[0]
    rc = lib().orc_apply_gates(_ptr(psi), _nq(psi), int(kind.size), *[_ptr(c) for c in cols])
    if rc != 0:
        raise ValueError(f"bad gate at index {-rc - 1}")


def run_circuit(circuit, basis: int = 0, n_qubits: int | None = None) -> np.ndarray:
    """psi = U_G ... U_1 |basis>, complex128 (n_qubits: needed for a plain gate sequence)."""
    psi = basis_state(circuit.n_qubits if n_qubits is None else n_qubits, basis)
    apply_gates(psi, circuit)
    return psi


def permute(psi: np.ndarray, perm) -> np.ndarray:
    """out[pi(i)] = psi[i] with pi moving bit q to bit perm[q]; any dtype, bit-exact."""
    psi = np.ascontiguousarray(psi)
    out = np.empty_like(psi)
    p = np.ascontiguousarray(perm, dtype=np.int32)
    if lib().orc_permute(_ptr(psi), _ptr(out), _nq(psi), _ptr(p), psi.itemsize) != 0:
        raise ValueError("perm is not a bijection")
    return out


def gather_slice(full: np.ndarray, sliced, value: int) -> np.ndarray:
    """Amplitudes whose `sliced` bits equal `value`, remaining bits in increasing order."""
    full = np.ascontiguousarray(full)
    s = np.ascontiguousarray(sliced, dtype=np.int32)
    n = _nq(full)
    out = np.empty(1 << (n - s.size), dtype=full.dtype)
    if lib().orc_slice_move(_ptr(full), _ptr(out), n, int(s.size), _ptr(s), int(value),
                            full.itemsize, 0) != 0:
        raise ValueError("bad sliced set")
    return out


def scatter_slice(full: np.ndarray, sliced, value: int, slice_: np.ndarray) -> None:
    """Inverse of gather_slice, in place on `full`."""
    s = np.ascontiguousarray(sliced, dtype=np.int32)
    slice_ = np.ascontiguousarray(slice_, dtype=full.dtype)
    if lib().orc_slice_move(_ptr(full), _ptr(slice_), _nq(full), int(s.size), _ptr(s),
                            int(value), full.itemsize, 1) != 0:
        raise ValueError("bad sliced set")


def reduce(psi: np.ndarray):
    """(sum p, 2^n sum p^2, 2^n sum p^2 - 1) in float64 over p = |psi|^2."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    vals = (ctypes.c_double(), ctypes.c_double(), ctypes.c_double())
    lib().orc_reduce(_ptr(psi), _nq(psi), *[ctypes.byref(v) for v in vals])
    return tuple(v.value for v in vals)


def _gate_columns(gates):
    """(kind, q0, q1, theta, phi, dplus, dminus, dminus_off) columns from a syc_inputs
    Circuit or from a sequence of 5- or 8-tuples (missing detunings are 0)."""
    g = list(gates.gates if hasattr(gates, "gates") else gates)
    cols = [np.array([x[i] for x in g], dtype=np.int32) for i in range(3)]
    cols += [np.array([x[i] if len(x) > i else 0.0 for x in g], dtype=np.float64) for i in range(3, 8)]
    return tuple(cols)


def split_tensors(n: int, gates, side):
    """Tensors 1 and 2 of the contraction-deferral split (Sect. 2; Appendix, EI and E2Q).

    Returns (t1, t2, c): c bridging gates; t1 over the side-0 qubits (increasing order) then
    the 2c entanglement bits, pair j's (a', a) at n1 + 2j, n1 + 2j + 1; t2 likewise."""
    cols = _gate_columns(gates)
    sd = np.ascontiguousarray(side, dtype=np.int32)
    ptrs = [_ptr(np.ascontiguousarray(a)) for a in cols]
    c = lib().orc_split_tensors(int(n), int(cols[0].size), *ptrs, _ptr(sd), None, None)
    if c < 0:
        raise ValueError(f"bad split input ({c})")
    n1 = int((sd == 0).sum())
    n2 = n - n1
    t1 = np.empty(1 << (n1 + 2 * c), dtype=np.complex128)
    t2 = np.empty(1 << (n2 + 2 * c), dtype=np.complex128)
    rc = lib().orc_split_tensors(int(n), int(cols[0].size), *ptrs, _ptr(sd), _ptr(t1), _ptr(t2))
    if rc != c:
        raise ValueError(f"split failed ({rc})")
    return t1, t2, c


def contract(t1: np.ndarray, t2: np.ndarray, n1: int, n2: int, qa, qb) -> np.ndarray:
    """psi over n1 + n2 qubits (logical order) = the sum over the shared entanglement bits of
    t1 * t2; qa / qb: qubit at each qubit position of t1 / t2."""
    t1 = np.ascontiguousarray(t1, dtype=np.complex128)
    t2 = np.ascontiguousarray(t2, dtype=np.complex128)
    e = _nq(t1) - n1
    if e < 0 or _nq(t2) - n2 != e or len(qa) != n1 or len(qb) != n2:
        raise ValueError("tensor shapes do not match")
    a = np.ascontiguousarray(qa, dtype=np.int32)
    b = np.ascontiguousarray(qb, dtype=np.int32)
    psi = np.empty(1 << (n1 + n2), dtype=np.complex128)
    lib().orc_contract(_ptr(t1), int(n1), _ptr(t2), int(n2), int(e), _ptr(a), _ptr(b), _ptr(psi))
    return psi
