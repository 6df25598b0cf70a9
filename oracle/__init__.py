"""CPU oracle for the fused-gate state-vector path (arXiv:1910.09534).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this package; the product library never
does, and it shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C, complex128, gate by gate); this
module only loads it with ctypes and converts numpy arrays.  Every function is
pinned in ``tests/test_oracle_pins.py`` against closed forms, invariants and
brute-force full-operator products.
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
        L.orc_apply_gates.argtypes = [P, i32, i32, P, P, P, P, P]
        L.orc_apply_gates.restype = i32
        L.orc_permute.argtypes = [P, P, i32, P, i32]
        L.orc_permute.restype = i32
        L.orc_slice_move.argtypes = [P, P, i32, i32, P, u64, i32, i32]
        L.orc_slice_move.restype = i32
        L.orc_reduce.argtypes = [P, i32, P, P, P]
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
    """Apply a syc_inputs.Circuit gate by gate, in place."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    kind, q0, q1, theta, phi = circuit.arrays()
    rc = lib().orc_apply_gates(_ptr(psi), _nq(psi), int(kind.size), _ptr(kind), _ptr(q0),
                               _ptr(q1), _ptr(theta), _ptr(phi))
    if rc != 0:
        raise ValueError(f"bad gate at index {-rc - 1}")


def run_circuit(circuit, basis: int = 0) -> np.ndarray:
    """psi = U_G ... U_1 |basis>, complex128."""
    psi = basis_state(circuit.n_qubits, basis)
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
