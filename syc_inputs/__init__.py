"""Seeded synthetic inputs shared by the CUDA path, the tests, the bench and the oracle.

This module only *draws* inputs: which gate sits where (random circuit
structure), random state vectors and random unitaries for kernel tests, and
request arrival times for the serving stream.  It holds none of the method's
arithmetic: no gate matrix, no state update, no fusion, no reduction.  A gate is
emitted as a record ``(kind, q0, q1, theta, phi)``; each consumer builds the
matrix itself from the gate definitions of Sect. 3 (Eq. 1 for fSim).

Random circuit structure (Sect. 3, "Sycamore circuits"):

* a cycle is one layer of single-qubit gates on every qubit followed by one
  layer of two-qubit fSim gates; a final single-qubit layer follows the last
  cycle;
* single-qubit gates are drawn from {sqrt(X), sqrt(Y), sqrt(W)};
* the two-qubit layers follow the coupler patterns in the order ABCDCDAB.

Readings taken where the paper is silent (its lattice figures are missing):

* sites of an R x C rectangular grid, kept sites numbered row-major; qubit q is
  bit q of the state index (little-endian);
* pattern A = horizontal couplers (r,c)-(r,c+1) with r+c even, B = horizontal
  with r+c odd, C = vertical couplers (r,c)-(r+1,c) with r+c even, D = vertical
  with r+c odd; each pattern is a matching and the four cover every coupler once;
* cycle t uses pattern "ABCDCDAB"[t mod 8]; every coupler of the pattern whose two
  sites are kept gets an fSim gate, first-listed qubit = the lower-numbered site;
* single-qubit choice: uniform over the three gates in the first layer, then
  uniform over the two gates that differ from the previous gate on that qubit;
* pseudo-random numbers: SplitMix64 (Steele, Lea, Flood 2014) seeded with the
  circuit seed; an integer below m is ``(x * m) >> 64``.

Per-location, per-depth two-qubit gates (Sect. 3: the hardware's two-qubit
unitaries vary with both the coupler and the cycle; Eq. 1 gives their form):
``detuned_sycamore_circuit`` emits the same gate structure as
``sycamore_circuit`` for the same seed, but each fSim record carries its own
draw of (theta, phi, D+, D-, D-,off) as an 8-tuple
``(kind, q0, q1, theta, phi, dplus, dminus, dminus_off)``: theta = pi/2 + U(-0.1, 0.1),
phi = pi/6 + U(-0.1, 0.1), each detuning U(-pi, pi), from a second SplitMix64
stream seeded with ``seed ^ DETUNE_SEED_XOR``, drawn in gate order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Gate kinds as emitted in gate records.
SQRT_X = 0
SQRT_Y = 1
SQRT_W = 2
FSIM = 3
KIND_NAMES = {SQRT_X: "sqrtX", SQRT_Y: "sqrtY", SQRT_W: "sqrtW", FSIM: "fSim"}

PATTERN_ORDER = "ABCDCDAB"
DETUNE_SEED_XOR = 0xD37D37D37D37D37D

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014; constants as published)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def below(self, m: int) -> int:
        return (self.next_u64() * m) >> 64

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


@dataclass
class Grid:
    rows: int
    cols: int
    removed: tuple = ()
    limit: int | None = None  # keep only the first `limit` sites (row-major)

    def sites(self) -> list:
        out = [(r, c) for r in range(self.rows) for c in range(self.cols)
               if (r, c) not in set(self.removed)]
        if self.limit is not None:
            out = out[: self.limit]
        return out

    def qubit_of(self) -> dict:
        return {s: q for q, s in enumerate(self.sites())}

    @property
    def n_qubits(self) -> int:
        return len(self.sites())

    def pattern(self, name: str) -> list:
        """Couplers (q_lo, q_hi) of pattern A/B/C/D on this grid."""
        qof = self.qubit_of()
        horizontal = name in "AB"
        parity = 0 if name in "AC" else 1
        out = []
        for (r, c), q in qof.items():
            if (r + c) % 2 != parity:
                continue
            nb = (r, c + 1) if horizontal else (r + 1, c)
            if nb in qof:
                a, b = q, qof[nb]
                out.append((min(a, b), max(a, b)))
        return sorted(out)


@dataclass
class Circuit:
    """A gate list in application order.  Records are (kind, q0, q1, theta, phi);
    q1 = -1 and theta = phi = 0 for single-qubit gates."""
    n_qubits: int
    gates: list = field(default_factory=list)
    name: str = ""

    @property
    def n_gates(self) -> int:
        return len(self.gates)

    def arrays(self):
        """Columns as numpy arrays: kind/q0/q1 int32, theta/phi float64."""
        g = self.gates
        kind = np.array([x[0] for x in g], dtype=np.int32)
        q0 = np.array([x[1] for x in g], dtype=np.int32)
        q1 = np.array([x[2] for x in g], dtype=np.int32)
        theta = np.array([x[3] for x in g], dtype=np.float64)
        phi = np.array([x[4] for x in g], dtype=np.float64)
        return kind, q0, q1, theta, phi

    def detunings(self):
        """fSim detunings (dplus, dminus, dminus_off) as float64 columns (0 for 5-tuples)."""
        g = self.gates
        return tuple(np.array([x[i] if len(x) > i else 0.0 for x in g], dtype=np.float64)
                     for i in (5, 6, 7))

    def count(self, kind: int) -> int:
        return sum(1 for x in self.gates if x[0] == kind)


def sycamore_circuit(grid: Grid, cycles: int, seed: int, theta: float = math.pi / 2,
                     phi: float = math.pi / 6, name: str = "") -> Circuit:
    """Random Sycamore-pattern circuit on `grid` (see module docstring)."""
    rng = SplitMix64(seed)
    n = grid.n_qubits
    patterns = {p: grid.pattern(p) for p in "ABCD"}
    prev = [-1] * n
    gates = []

    def one_qubit_layer():
        for q in range(n):
            if prev[q] < 0:
                g = rng.below(3)
            else:
                g = (prev[q] + 1 + rng.below(2)) % 3  # one of the two other gates
            prev[q] = g
            gates.append((g, q, -1, 0.0, 0.0))

    for t in range(cycles):
        one_qubit_layer()
        for (a, b) in patterns[PATTERN_ORDER[t % 8]]:
            gates.append((FSIM, a, b, float(theta), float(phi)))
    one_qubit_layer()
    return Circuit(n_qubits=n, gates=gates, name=name)


def detuned_sycamore_circuit(grid: Grid, cycles: int, seed: int, theta_spread: float = 0.1,
                             phi_spread: float = 0.1, name: str = "") -> Circuit:
    """``sycamore_circuit(grid, cycles, seed)`` with every fSim gate's parameters drawn for that
    gate instance (see the module docstring), so that its matrix depends on the coupler and the
    cycle."""
    base = sycamore_circuit(grid, cycles, seed, name=name)
    rng = SplitMix64(seed ^ DETUNE_SEED_XOR)

    def u(lo, hi):
        return lo + (hi - lo) * rng.uniform()

    gates = []
    for g in base.gates:
        if g[0] == FSIM:
            th = math.pi / 2 + u(-theta_spread, theta_spread)
            ph = math.pi / 6 + u(-phi_spread, phi_spread)
            gates.append((FSIM, g[1], g[2], th, ph, u(-math.pi, math.pi), u(-math.pi, math.pi),
                          u(-math.pi, math.pi)))
        else:
            gates.append(g)
    return Circuit(n_qubits=base.n_qubits, gates=gates, name=name)


# Named workloads (rows, cols, removed sites, cycles).
WORKLOADS = {
    "syc12_3x4_d8": dict(grid=Grid(3, 4), cycles=8),
    "syc30_5x6_d20": dict(grid=Grid(5, 6), cycles=20),
    "syc33_6x6m3_d20": dict(grid=Grid(6, 6, removed=((0, 0), (0, 5), (5, 0))), cycles=20),
    "syc28_4x7_d20": dict(grid=Grid(4, 7), cycles=20),
    "syc35_5x7_d16": dict(grid=Grid(5, 7), cycles=16),
    # 35 qubits need a 256 GiB host store; hosts with less memory run the same pattern on the
    # 5x7 grid minus one corner site (34 qubits, 128 GiB)
    "syc34_5x7m1_d16": dict(grid=Grid(5, 7, removed=((4, 6),)), cycles=16),
}


def workload_circuit(name: str, seed: int = 0) -> Circuit:
    w = WORKLOADS[name]
    return sycamore_circuit(w["grid"], w["cycles"], seed, name=name)


def near_square_grid(n: int) -> Grid:
    """Serving-stream grid for n qubits: R = floor(sqrt n), C = ceil(n / R), first n sites."""
    r = int(math.isqrt(n))
    c = -(-n // r)
    return Grid(r, c, limit=n)


def serving_stream(count: int, base_seed: int, rate_hz: float, n_lo: int = 16, n_hi: int = 30,
                   d_lo: int = 8, d_hi: int = 20):
    """Requests of the serving workload: list of (arrival_s, Circuit).

    Qubit count uniform in [n_lo, n_hi], depth uniform in [d_lo, d_hi], Poisson
    arrivals at `rate_hz`; circuit i uses seed base_seed + i."""
    rng = SplitMix64(base_seed ^ 0x5EED5EED5EED5EED)
    t = 0.0
    out = []
    for i in range(count):
        n = n_lo + rng.below(n_hi - n_lo + 1)
        d = d_lo + rng.below(d_hi - d_lo + 1)
        t += -math.log(1.0 - rng.uniform()) / rate_hz
        out.append((t, sycamore_circuit(near_square_grid(n), d, base_seed + i,
                                        name=f"srv{i}_n{n}_d{d}")))
    return out


def random_state(n_qubits: int, seed: int) -> np.ndarray:
    """Normalised complex64 state with i.i.d. Gaussian components (seeded PCG64)."""
    rng = np.random.default_rng(seed)
    dim = 1 << n_qubits
    v = rng.standard_normal(2 * dim, dtype=np.float32).view(np.complex64)
    v /= np.float32(np.sqrt(np.sum(np.abs(v.astype(np.complex128)) ** 2)))
    return v


def random_unitary(k: int, seed: int) -> np.ndarray:
    """Haar-random 2^k x 2^k complex128 unitary (QR of a Gaussian, phases fixed)."""
    rng = np.random.default_rng(seed)
    d = 1 << k
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diagonal(r) / np.abs(np.diagonal(r))
    return q * ph[None, :]


def random_targets(n_qubits: int, k: int, seed: int) -> list:
    """k distinct qubits drawn uniformly, in random order."""
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.choice(n_qubits, size=k, replace=False)]


def random_permutation(n_qubits: int, seed: int) -> list:
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.permutation(n_qubits)]
