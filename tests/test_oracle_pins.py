"""Pins for the CPU oracle: closed forms, invariants and brute force (no GPU).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a swapped qubit order, a transposed matrix, a wrong bit in the
permutation or slice maps) fails at least one of them.  Brute-force operators
are built here from the definition "a gate acts on its target bits and is the
identity on the rest", independently of the oracle's pair/quad enumeration.
"""
import math
import os

import numpy as np
import pytest

import syc_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
H = np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)


def full_operator(n, targets, u):
    """2^n x 2^n operator of u on `targets` (bit j of u's index <-> targets[j]), by definition:
    <i'|U|i> = u[r(i'), r(i)] when i' and i agree on every non-target bit, else 0."""
    idx = np.arange(1 << n)
    r = np.zeros_like(idx)
    tmask = 0
    for j, t in enumerate(targets):
        r |= ((idx >> t) & 1) << j
        tmask |= 1 << t
    rest = idx & ~tmask
    return u[r[:, None], r[None, :]] * (rest[:, None] == rest[None, :])


def kron_1q(n, q, u):
    """Single-qubit operator by Kronecker products (little-endian: qubit 0 is the last factor)."""
    return np.kron(np.kron(np.eye(1 << (n - q - 1)), u), np.eye(1 << q))


def rand_state128(n, seed):
    return si.random_state(n, seed).astype(np.complex128)


# --------------------------------------------------------------------------- gate library

def test_sqrt_gates_square_to_minus_i_pauli(oracle_mod):
    W = (X + Y) / math.sqrt(2)
    for kind, P in ((si.SQRT_X, X), (si.SQRT_Y, Y), (si.SQRT_W, W)):
        s = oracle_mod.gate_matrix(kind)
        assert np.allclose(s @ s, -1j * P, atol=1e-15)
        assert np.allclose(s.conj().T @ s, np.eye(2), atol=1e-15)


def test_fsim_special_cases(oracle_mod):
    assert np.allclose(oracle_mod.gate_matrix(si.FSIM, 0.0, 0.0), np.eye(4), atol=1e-15)
    iswap_like = np.array([[1, 0, 0, 0], [0, 0, -1j, 0], [0, -1j, 0, 0], [0, 0, 0, 1]])
    assert np.allclose(oracle_mod.gate_matrix(si.FSIM, math.pi / 2, 0.0), iswap_like, atol=1e-15)
    # the conditional phase acts on |11> only
    cz_like = np.diag([1, 1, 1, np.exp(-1j * 0.7)])
    assert np.allclose(oracle_mod.gate_matrix(si.FSIM, 0.0, 0.7), cz_like, atol=1e-15)


def test_fsim_golden_eq1(oracle_mod):
    want = np.zeros((4, 4), dtype=complex)
    for line in open(os.path.join(GOLDEN, "fsim_eq1_theta90_phi30.txt")):
        if line.startswith("#") or not line.strip():
            continue
        r, c, re, im = line.split()
        want[int(r), int(c)] = float(re) + 1j * float(im)
    got = oracle_mod.gate_matrix(si.FSIM, math.pi / 2, math.pi / 6)
    assert np.allclose(got, want, atol=1e-15)


def test_fsim_group_laws(oracle_mod):
    f = lambda t, p: oracle_mod.gate_matrix(si.FSIM, t, p)
    assert np.allclose(f(0.3, 0.0) @ f(0.9, 0.0), f(1.2, 0.0), atol=1e-14)
    assert np.allclose(f(0.0, 0.4) @ f(0.0, 1.1), f(0.0, 1.5), atol=1e-14)
    assert np.allclose(f(0.3, 0.2) @ f(0.9, 0.5), f(1.2, 0.7), atol=1e-14)


def test_fsim_detuning_is_phase_dressing(oracle_mod):
    # Eq. 1 with detunings equals diag phases (a product of single-qubit phase gates) on both
    # sides of the undetuned fSim: D_L fSim(theta, phi) D_R.
    rng = np.random.default_rng(5)
    for _ in range(5):
        th, ph, dp, dm, do = rng.uniform(-3, 3, 5)
        a1, a2, b2 = dp + dm, dp + do, -dm - do
        DL = np.diag(np.exp(1j * np.array([0, a1, a2, a1 + a2])))
        DR = np.diag(np.exp(1j * np.array([0, 0, b2, b2])))
        got = oracle_mod.gate_matrix(si.FSIM, th, ph, dp, dm, do)
        assert np.allclose(got, DL @ oracle_mod.gate_matrix(si.FSIM, th, ph) @ DR, atol=1e-14)
        assert np.allclose(got.conj().T @ got, np.eye(4), atol=1e-14)


# --------------------------------------------------------------------------- gate application

@pytest.mark.parametrize("n,q", [(1, 0), (5, 0), (5, 2), (7, 6)])
def test_apply_1q_matches_kron(oracle_mod, n, q):
    u = si.random_unitary(1, seed=10 + q)
    psi = rand_state128(n, seed=n)
    want = kron_1q(n, q, u) @ psi
    oracle_mod.apply_1q(psi, q, u)
    assert np.allclose(psi, want, atol=1e-14)


@pytest.mark.parametrize("n,q0,q1", [(2, 0, 1), (2, 1, 0), (6, 4, 1), (7, 0, 6), (7, 5, 2)])
def test_apply_2q_matches_brute_force(oracle_mod, n, q0, q1):
    u = si.random_unitary(2, seed=q0 * 7 + q1)  # not symmetric: catches swapped q0/q1 or u.T
    psi = rand_state128(n, seed=3)
    want = full_operator(n, [q0, q1], u) @ psi
    oracle_mod.apply_2q(psi, q0, q1, u)
    assert np.allclose(psi, want, atol=1e-14)


@pytest.mark.parametrize("n,targets", [(3, [0, 1, 2]), (6, [5, 0, 3]), (8, [1, 7, 4, 2]),
                                        (8, [6, 0, 2, 7, 3]), (7, [3, 1, 6, 0, 5, 2])])
def test_apply_kq_matches_brute_force(oracle_mod, n, targets):
    u = si.random_unitary(len(targets), seed=sum(targets))
    psi = rand_state128(n, seed=11)
    want = full_operator(n, targets, u) @ psi
    oracle_mod.apply_kq(psi, targets, u)
    assert np.allclose(psi, want, atol=1e-13)


def test_apply_kq_rejects_bad_targets(oracle_mod):
    psi = rand_state128(4, 0)
    with pytest.raises(ValueError):
        oracle_mod.apply_kq(psi, [1, 1], np.eye(4))
    with pytest.raises(ValueError):
        oracle_mod.apply_kq(psi, [4], np.eye(2))


def test_fused_block_equals_gate_sequence(oracle_mod):
    # Aggregation (Sect. 5): the block matrix of a gate run, composed on the block's own
    # k-qubit space with later gates multiplying from the left, acts like the run itself.
    n, targets = 7, [5, 1, 3, 6]
    gates = [(si.SQRT_X, [5]), (si.FSIM, [5, 1]), (si.SQRT_W, [3]), (si.FSIM, [1, 3]),
             (si.SQRT_Y, [6]), (si.FSIM, [6, 5]), (si.SQRT_X, [1])]
    k = len(targets)
    block = np.eye(1 << k, dtype=complex)
    psi_seq = rand_state128(n, seed=21)
    psi_blk = psi_seq.copy()
    for kind, qs in gates:
        u = oracle_mod.gate_matrix(kind, 1.1, 0.4)
        local = [targets.index(q) for q in qs]
        block = full_operator(k, local, u) @ block
        if len(qs) == 1:
            oracle_mod.apply_1q(psi_seq, qs[0], u)
        else:
            oracle_mod.apply_2q(psi_seq, qs[0], qs[1], u)
    oracle_mod.apply_kq(psi_blk, targets, block)
    assert np.allclose(psi_blk, psi_seq, atol=1e-13)


# --------------------------------------------------------------------------- worked states

@pytest.mark.parametrize("n", [2, 5, 9])
def test_ghz(oracle_mod, n):
    # H on qubit 0 then a CNOT chain gives (|0..0> + |1..1>)/sqrt 2.  CNOT with control =
    # first-listed qubit (index bit 0), target = second (index bit 1).
    cnot = np.zeros((4, 4))
    cnot[0, 0] = cnot[2, 2] = cnot[3, 1] = cnot[1, 3] = 1
    psi = oracle_mod.basis_state(n, 0)
    oracle_mod.apply_1q(psi, 0, H)
    for q in range(n - 1):
        oracle_mod.apply_2q(psi, q, q + 1, cnot)
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.allclose(psi, want, atol=1e-15)
    # the same through the generic k-qubit block on reversed target order
    psi2 = oracle_mod.basis_state(n, 0)
    oracle_mod.apply_kq(psi2, [0], H)
    swapped = full_operator(2, [1, 0], cnot)  # control on index bit 1
    for q in range(n - 1):
        oracle_mod.apply_kq(psi2, [q + 1, q], swapped)
    assert np.allclose(psi2, want, atol=1e-15)


@pytest.mark.parametrize("n", [1, 6, 10])
def test_uniform_hadamard_layer(oracle_mod, n):
    psi = oracle_mod.basis_state(n, 0)
    for q in range(n):
        oracle_mod.apply_1q(psi, q, H)
    assert np.allclose(psi, np.full(1 << n, 2.0 ** (-n / 2)), atol=1e-15)


def test_basis_state(oracle_mod):
    psi = oracle_mod.basis_state(5, 19)
    assert psi[19] == 1 and np.count_nonzero(psi) == 1


# --------------------------------------------------------------------------- circuits

def test_generator_gate_counts():
    for line in open(os.path.join(GOLDEN, "sycamore_gate_counts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, n, cyc, n1, n2, a, b, c, d = line.split()
        w = si.WORKLOADS[name]
        assert w["grid"].n_qubits == int(n) and w["cycles"] == int(cyc)
        circ = si.workload_circuit(name, seed=0)
        assert circ.n_gates == int(n1) + int(n2)
        assert circ.count(si.FSIM) == int(n2)
        assert [len(w["grid"].pattern(p)) for p in "ABCD"] == [int(a), int(b), int(c), int(d)]


def test_generator_patterns_are_matchings_covering_all_couplers():
    for g in (si.Grid(3, 4), si.Grid(5, 6), si.Grid(6, 6, removed=((0, 0), (0, 5), (5, 0))),
              si.near_square_grid(23)):
        allp = []
        for p in "ABCD":
            e = g.pattern(p)
            qs = [q for pair in e for q in pair]
            assert len(qs) == len(set(qs))  # matching
            allp += e
        qof = g.qubit_of()
        every = {tuple(sorted((qof[s], qof[(s[0] + dr, s[1] + dc)])))
                 for s in qof for dr, dc in ((0, 1), (1, 0)) if (s[0] + dr, s[1] + dc) in qof}
        assert sorted(allp) == sorted(every)


def test_generator_no_immediate_repeat_and_determinism():
    c1 = si.workload_circuit("syc12_3x4_d8", seed=7)
    c2 = si.workload_circuit("syc12_3x4_d8", seed=7)
    assert c1.gates == c2.gates
    assert c1.gates != si.workload_circuit("syc12_3x4_d8", seed=8).gates
    last = {}
    for kind, q0, q1, _, _ in c1.gates:
        if kind != si.FSIM:
            assert last.get(q0) != kind
            last[q0] = kind


def test_run_circuit_matches_operator_product(oracle_mod):
    grid = si.Grid(2, 4)
    circ = si.sycamore_circuit(grid, cycles=6, seed=3)
    n = circ.n_qubits
    U = np.eye(1 << n, dtype=complex)
    for kind, q0, q1, th, ph in circ.gates:
        u = oracle_mod.gate_matrix(kind, th, ph)
        U = full_operator(n, [q0] if kind != si.FSIM else [q0, q1], u) @ U
    psi = oracle_mod.run_circuit(circ)
    assert np.allclose(psi, U[:, 0], atol=1e-13)
    psi5 = oracle_mod.run_circuit(circ, basis=5)
    assert np.allclose(psi5, U[:, 5], atol=1e-13)


def test_norm_preserved_on_workload(oracle_mod):
    psi = oracle_mod.run_circuit(si.workload_circuit("syc12_3x4_d8", seed=0))
    norm, _, _ = oracle_mod.reduce(psi)
    assert abs(norm - 1.0) < 1e-12


def test_porter_thomas(oracle_mod):
    # Random-circuit output probabilities approach the Porter-Thomas (exponential)
    # distribution: 2^n sum p^2 -> 2 (2 * 2^n / (2^n + 1) for Haar states), std ~ sqrt(20 / 2^n).
    circ = si.sycamore_circuit(si.Grid(4, 4), cycles=20, seed=1)
    _, s2, xeb = oracle_mod.reduce(oracle_mod.run_circuit(circ))
    assert abs(s2 - 2.0) < 0.1
    assert abs(xeb - 1.0) < 0.1
    # a circuit with no entangling cycle is far from it: one single-qubit layer of sqrt(X/Y/W)
    # on |0..0> gives p = 2^-n everywhere, so 2^n sum p^2 = 1 exactly
    shallow = si.sycamore_circuit(si.Grid(4, 4), cycles=0, seed=1)
    _, s2_0, _ = oracle_mod.reduce(oracle_mod.run_circuit(shallow))
    assert abs(s2_0 - 1.0) < 1e-12


# --------------------------------------------------------------------------- permutation / slices

def _pi(i, perm):
    j = 0
    for q, p in enumerate(perm):
        if (i >> q) & 1:
            j |= 1 << p
    return j


@pytest.mark.parametrize("n,seed", [(1, 0), (4, 1), (9, 2), (12, 3)])
def test_permute_closed_form(oracle_mod, n, seed):
    perm = si.random_permutation(n, seed)
    data = np.arange(1 << n, dtype=np.int64)
    out = oracle_mod.permute(data, perm)
    want = np.empty_like(data)
    for i in range(1 << n):
        want[_pi(i, perm)] = i
    assert np.array_equal(out, want)
    inv = [0] * n
    for q, p in enumerate(perm):
        inv[p] = q
    assert np.array_equal(oracle_mod.permute(out, inv), data)


def test_permute_commutes_with_gates(oracle_mod):
    # relabelling qubits: a gate on qubit q before the permutation equals the same gate on
    # bit perm[q] after it
    n = 7
    perm = si.random_permutation(n, 4)
    u = si.random_unitary(2, 9)
    psi = rand_state128(n, 2)
    a = psi.copy()
    oracle_mod.apply_2q(a, 1, 5, u)
    a = oracle_mod.permute(a, perm)
    b = oracle_mod.permute(psi, perm)
    oracle_mod.apply_2q(b, perm[1], perm[5], u)
    assert np.allclose(a, b, atol=1e-15)


def test_permute_rejects_non_bijection(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.permute(np.zeros(8, dtype=np.complex64), [0, 0, 1])


def test_slice_gather_scatter(oracle_mod):
    n, sliced = 8, [6, 2, 7]
    data = np.arange(1 << n, dtype=np.int64)
    seen = []
    for v in range(1 << len(sliced)):
        sl = oracle_mod.gather_slice(data, sliced, v)
        rest = [q for q in range(n) if q not in sliced]
        for j in range(sl.size):
            i = 0
            for b, q in enumerate(rest):
                i |= ((j >> b) & 1) << q
            for b, q in enumerate(sliced):
                i |= ((v >> b) & 1) << q
            assert sl[j] == i
        seen.append(sl)
    assert np.array_equal(np.sort(np.concatenate(seen)), data)
    back = np.zeros_like(data)
    for v in range(1 << len(sliced)):
        oracle_mod.scatter_slice(back, sliced, v, seen[v])
    assert np.array_equal(back, data)


# --------------------------------------------------------------------------- reductions

def test_reduce_closed_forms(oracle_mod):
    n = 10
    norm, s2, xeb = oracle_mod.reduce(oracle_mod.basis_state(n, 77))
    assert (norm, s2, xeb) == (1.0, 2.0 ** n, 2.0 ** n - 1)
    norm, s2, xeb = oracle_mod.reduce(np.full(1 << n, 2.0 ** (-n / 2), dtype=complex))
    assert abs(norm - 1) < 1e-14 and abs(s2 - 1) < 1e-12 and abs(xeb) < 1e-12
    psi = rand_state128(n, 5) * 1.5
    p = np.abs(psi) ** 2
    norm, s2, _ = oracle_mod.reduce(psi)
    assert abs(norm - p.sum()) < 1e-12 and abs(s2 - (1 << n) * (p ** 2).sum()) < 1e-10


def test_threads_do_not_change_results(oracle_mod):
    circ = si.sycamore_circuit(si.Grid(3, 5), cycles=6, seed=2)
    oracle_mod.set_threads(1)
    a = oracle_mod.run_circuit(circ)
    oracle_mod.set_threads(4)
    b = oracle_mod.run_circuit(circ)
    oracle_mod.set_threads(os.cpu_count() or 1)
    assert np.array_equal(a, b)


# ---- contraction deferral: EI / E2Q tensors and the contraction (Sect. 2; Appendix) ----

def _detuned_circuit(n, n_gates, seed):
    """Random gate list of 8-tuples with fSim detunings, so the gate is not symmetric under
    exchanging its qubits (a swapped role of a and b then changes the result)."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(n_gates):
        if rng.random() < 0.5:
            gates.append((int(rng.integers(3)), int(rng.integers(n)), -1, 0.0, 0.0))
        else:
            q0, q1 = (int(x) for x in rng.choice(n, 2, replace=False))
            gates.append((si.FSIM, q0, q1, *(float(x) for x in rng.uniform(-np.pi, np.pi, 5))))
    return gates


def _plain_by_operators(oracle_mod, n, gates):
    """psi = U_G ... U_1 |0>, each gate as its full 2^n x 2^n operator (definition)."""
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0
    for g in gates:
        kind, q0, q1 = g[0], g[1], g[2]
        u = oracle_mod.gate_matrix(kind, *g[3:])
        psi = full_operator(n, [q0] if kind != si.FSIM else [q0, q1], u) @ psi
    return psi


@pytest.mark.parametrize("n,n_gates,seed", [(3, 12, 11), (5, 30, 12), (7, 40, 13)])
def test_apply_gates_detuned_matches_operator_product(oracle_mod, n, n_gates, seed):
    # Sect. 3 / Eq. 1 with per-gate detunings: the oracle's gate-by-gate run of 8-tuple records
    # equals the product of the gates' full 2^n x 2^n operators (a dropped detuning, a swapped
    # q0/q1 role or a wrong sign of one of them fails this: the detuned gate is not symmetric)
    gates = _detuned_circuit(n, n_gates, seed)
    psi = oracle_mod.run_circuit(gates, n_qubits=n)
    assert np.allclose(psi, _plain_by_operators(oracle_mod, n, gates), atol=1e-12)


def test_detuned_sycamore_circuit_by_operators(oracle_mod):
    # the generator's per-location, per-cycle fSim records through the oracle, against full
    # operators; and the detunings matter (the undetuned circuit gives another state)
    circ = si.detuned_sycamore_circuit(si.Grid(2, 4), cycles=6, seed=3)
    psi = oracle_mod.run_circuit(circ)
    assert np.allclose(psi, _plain_by_operators(oracle_mod, 8, circ.gates), atol=1e-12)
    plain = oracle_mod.run_circuit(si.sycamore_circuit(si.Grid(2, 4), cycles=6, seed=3))
    assert np.linalg.norm(psi - plain) > 0.1


def test_detuned_generator_structure():
    # same gate structure as the undetuned generator for the seed; every fSim instance has its
    # own parameters, inside the stated ranges; deterministic
    grid = si.Grid(3, 4)
    a = si.detuned_sycamore_circuit(grid, cycles=8, seed=9)
    b = si.sycamore_circuit(grid, cycles=8, seed=9)
    assert [g[:3] for g in a.gates] == [g[:3] for g in b.gates]
    assert a.gates == si.detuned_sycamore_circuit(grid, cycles=8, seed=9).gates
    fs = [g for g in a.gates if g[0] == si.FSIM]
    assert len(fs) == 34 and all(len(g) == 8 for g in fs)
    assert all(abs(g[3] - np.pi / 2) <= 0.1 and abs(g[4] - np.pi / 6) <= 0.1 for g in fs)
    assert all(all(-np.pi <= x < np.pi for x in g[5:]) for g in fs)
    assert len({g[3:] for g in fs}) == len(fs)
    d = a.detunings()
    assert d[0].shape == (a.n_gates,) and np.count_nonzero(d[0]) == len(fs)


def _contract_logical(oracle_mod, n, side, t1, t2):
    qa = [q for q in range(n) if side[q] == 0]
    qb = [q for q in range(n) if side[q] == 1]
    return oracle_mod.contract(t1, t2, len(qa), len(qb), qa, qb)


@pytest.mark.parametrize("n,n_gates,seed", [(2, 6, 0), (4, 14, 1), (5, 18, 2), (6, 16, 3)])
def test_split_contraction_equals_full_operator_product(oracle_mod, n, n_gates, seed):
    gates = _detuned_circuit(n, n_gates, seed)
    rng = np.random.default_rng(100 + seed)
    side = [0] * n
    while len(set(side)) < 2:
        side = [int(x) for x in rng.integers(0, 2, n)]
    t1, t2, c = oracle_mod.split_tensors(n, gates, side)
    assert c == sum(1 for g in gates if g[0] == si.FSIM and side[g[1]] != side[g[2]])
    assert c > 0
    psi = _contract_logical(oracle_mod, n, side, t1, t2)
    assert np.allclose(psi, _plain_by_operators(oracle_mod, n, gates), atol=1e-12)


def test_split_sycamore_prefix_equals_plain_run(oracle_mod):
    # 3 x 4 grid split between columns 1 and 2: the first two cycles (patterns A, B) bridge
    # the cut with 1 + 2 gates, the next four (C, D, C, D) stay on either side.
    circ = si.sycamore_circuit(si.Grid(3, 4), cycles=6, seed=4)
    side = [0 if (q % 4) < 2 else 1 for q in range(12)]
    t1, t2, c = oracle_mod.split_tensors(12, circ, side)
    assert c == 3
    assert t1.size == 1 << (6 + 6) and t2.size == 1 << (6 + 6)
    psi = _contract_logical(oracle_mod, 12, side, t1, t2)
    assert np.allclose(psi, oracle_mod.run_circuit(circ), atol=1e-12)


def test_split_without_bridging_gates_is_an_outer_product(oracle_mod):
    # gates never cross the cut: psi = T1 (x) T2 with the qubits placed by the sides
    n = 5
    side = [0, 1, 1, 0, 1]
    gates = [(0, 0, -1, 0, 0), (si.FSIM, 0, 3, 0.3, 0.2, 0.1, -0.4, 0.7), (1, 2, -1, 0, 0),
             (si.FSIM, 4, 1, 1.1, -0.5, 0.2, 0.3, -0.1), (2, 3, -1, 0, 0), (si.FSIM, 2, 4, 0.7, 0.9)]
    t1, t2, c = oracle_mod.split_tensors(n, gates, side)
    assert c == 0 and t1.size == 4 and t2.size == 8
    psi = _contract_logical(oracle_mod, n, side, t1, t2)
    assert np.allclose(psi, _plain_by_operators(oracle_mod, n, gates), atol=1e-13)
    # the same from numpy: kron over qubit order 4, 3, 2, 1, 0 (little-endian)
    t1q = {0: 0, 3: 1}
    t2q = {1: 0, 2: 1, 4: 2}
    full = np.einsum("ab,cde->abcde", t1.reshape(2, 2).T, t2.reshape(2, 2, 2).transpose(2, 1, 0))
    # full[a0, a3, b1, b2, b4] -> psi index sum q bit_q 2^q
    psi2 = np.zeros(1 << n, dtype=complex)
    for i in range(1 << n):
        b = [(i >> q) & 1 for q in range(n)]
        psi2[i] = full[b[0], b[3], b[1], b[2], b[4]]
    assert t1q and t2q and np.allclose(psi, psi2, atol=1e-15)


def test_split_ei_structure_and_norms(oracle_mod):
    # EI copies a'' = a' (entries with a'' != a' vanish right after it) and doubles the squared
    # norm; E2Q also doubles it (sum over a of |G (e_a x chi)|^2 = 2 |chi|^2 for unitary G).
    n = 2
    gates = [(0, 0, -1, 0, 0), (2, 1, -1, 0, 0), (si.FSIM, 1, 0, 0.8, 0.4, 0.3, 0.6, -0.2)]
    t1, t2, c = oracle_mod.split_tensors(n, gates, [0, 1])
    assert c == 1 and t1.size == 8 and t2.size == 8
    for i in range(8):
        app, ap = i & 1, (i >> 1) & 1
        if app != ap:
            assert t1[i] == 0
    phi = oracle_mod.gate_matrix(0)[:, 0]  # sqrt(X)|0>
    for a in range(2):
        for v in range(2):
            assert t1[v + 2 * v + 4 * a] == pytest.approx(phi[a], abs=1e-15)
    assert np.vdot(t1, t1).real == pytest.approx(2.0, abs=1e-13)
    assert np.vdot(t2, t2).real == pytest.approx(2.0, abs=1e-13)
    circ = si.sycamore_circuit(si.Grid(3, 4), cycles=6, seed=5)
    side = [0 if (q % 4) < 2 else 1 for q in range(12)]
    t1, t2, c = oracle_mod.split_tensors(12, circ, side)
    assert np.vdot(t1, t1).real == pytest.approx(2.0 ** c, rel=1e-12)
    assert np.vdot(t2, t2).real == pytest.approx(2.0 ** c, rel=1e-12)


def test_contract_matches_einsum(oracle_mod):
    rng = np.random.default_rng(7)
    n1, n2, e = 3, 2, 4
    t1 = rng.normal(size=1 << (n1 + e)) + 1j * rng.normal(size=1 << (n1 + e))
    t2 = rng.normal(size=1 << (n2 + e)) + 1j * rng.normal(size=1 << (n2 + e))
    qa, qb = [4, 0, 2], [3, 1]
    psi = oracle_mod.contract(t1, t2, n1, n2, qa, qb)
    m = np.einsum("kx,ky->xy", t1.reshape(1 << e, 1 << n1), t2.reshape(1 << e, 1 << n2))
    for x in range(1 << n1):
        for y in range(1 << n2):
            li = sum(((x >> i) & 1) << qa[i] for i in range(n1)) + sum(((y >> j) & 1) << qb[j] for j in range(n2))
            assert psi[li] == pytest.approx(m[x, y], abs=1e-12)


def test_split_rejects_bad_sides(oracle_mod):
    gates = [(0, 0, -1, 0, 0)]
    with pytest.raises(ValueError):
        oracle_mod.split_tensors(2, gates, [0, 0])
    with pytest.raises(ValueError):
        oracle_mod.split_tensors(2, gates, [0, 2])
    with pytest.raises(ValueError):
        oracle_mod.split_tensors(2, [(si.FSIM, 0, 0, 1.0, 1.0)], [0, 1])
