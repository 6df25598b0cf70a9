"""Host-side checks of the native library (no GPU): it loads, exports every symbol declared in
include/*.h, validates arguments without touching the device, and its host logic -- gate
matrices and the aggregation planner -- agrees with the CPU oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import syc_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as p
    p.lib()
    return p


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\([^;]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(pkg):
    names = declared_functions()
    assert len(names) >= 20
    L = pkg.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding wraps each of them
    assert sorted(set(names) - set(pkg._native.exported_symbols())) == []


def test_version(pkg):
    assert "sm_103a" in pkg.sim_version()


def test_errors_without_touching_device(pkg):
    L = pkg.lib()
    h = ctypes.c_void_p()
    assert L.sim_create(0, 0, None, ctypes.byref(h)) == pkg.SIM_E_INVAL
    assert b"n_qubits" in L.sim_last_error(None)
    assert L.sim_create(10, 10, None, ctypes.byref(h)) == pkg.SIM_E_INVAL
    assert L.sim_amplitudes_async(None, 0, 1, None, 0) == pkg.SIM_E_INVAL
    assert L.sim_destroy(None) == pkg.SIM_E_INVAL
    assert L.sim_apply_fused(None, 1, None, None, 0) == pkg.SIM_E_INVAL
    assert L.sim_plan_create(4, 1, None, None, ctypes.byref(h)) == pkg.SIM_E_INVAL


def test_gate_matrices_match_oracle(pkg, oracle_mod):
    rng = np.random.default_rng(0)
    for kind in (si.SQRT_X, si.SQRT_Y, si.SQRT_W):
        g = np.zeros(1, dtype=pkg._native.GATE_DTYPE)[0]
        g["kind"] = kind
        assert np.allclose(pkg.sim_gate_matrix(g), oracle_mod.gate_matrix(kind), atol=1e-15)
    for _ in range(5):
        th, ph, dp, dm, do = rng.uniform(-3, 3, 5)
        g = np.zeros(1, dtype=pkg._native.GATE_DTYPE)[0]
        g["kind"], g["theta"], g["phi"] = si.FSIM, th, ph
        g["dplus"], g["dminus"], g["dminus_off"] = dp, dm, do
        assert np.allclose(pkg.sim_gate_matrix(g), oracle_mod.gate_matrix(si.FSIM, th, ph, dp, dm, do),
                           atol=1e-15)


def plan_blocks(pkg, plan):
    nb, _, _ = pkg.sim_plan_info(plan)
    return [pkg.sim_plan_block(plan, i) for i in range(nb)]


@pytest.mark.parametrize("kmax", [2, 3, 4, 5, 6])
def test_planner_blocks_reproduce_circuit(pkg, oracle_mod, kmax):
    # Sect. 5 aggregation: applying the composed blocks in plan order equals applying the
    # gates one by one (oracle), up to FP64 rounding.
    circ = si.sycamore_circuit(si.Grid(3, 4), cycles=8, seed=4)
    plan = pkg.sim_plan_create(circ.n_qubits, pkg.gates_array(circ), kmax=kmax)
    try:
        nb, ng, mk = pkg.sim_plan_info(plan)
        assert ng == circ.n_gates and mk <= kmax and nb >= 1
        psi = oracle_mod.basis_state(circ.n_qubits, 0)
        for t, m in plan_blocks(pkg, plan):
            assert list(t) == sorted(t) and len(set(t)) == len(t) <= kmax
            assert np.allclose(m.conj().T @ m, np.eye(m.shape[0]), atol=1e-12)
            oracle_mod.apply_kq(psi, t, m)
        want = oracle_mod.run_circuit(circ)
        assert np.linalg.norm(psi - want) < 1e-12
    finally:
        pkg.sim_plan_destroy(plan)


@pytest.mark.parametrize("kmax", [2, 4, 6])
def test_planner_blocks_reproduce_detuned_circuit(pkg, oracle_mod, kmax):
    # per-location, per-cycle detuned fSim gates (Sect. 3, Eq. 1): the planner's FP64 blocks
    # reproduce the oracle's gate-by-gate run
    circ = si.detuned_sycamore_circuit(si.Grid(3, 4), cycles=8, seed=6)
    plan = pkg.sim_plan_create(circ.n_qubits, pkg.gates_array(circ), kmax=kmax)
    try:
        psi = oracle_mod.basis_state(circ.n_qubits, 0)
        for t, m in plan_blocks(pkg, plan):
            oracle_mod.apply_kq(psi, t, m)
        assert np.linalg.norm(psi - oracle_mod.run_circuit(circ)) < 1e-12
    finally:
        pkg.sim_plan_destroy(plan)


def test_planner_counts_on_30q_circuit(pkg):
    # Wider blocks -> fewer passes over the state (Sect. 5, Tables 1-2 count "5Q kernels").
    circ = si.workload_circuit("syc30_5x6_d20", seed=0)
    counts = {}
    for kmax in (2, 3, 4, 5, 6):
        plan = pkg.sim_plan_create(circ.n_qubits, pkg.gates_array(circ), kmax=kmax)
        counts[kmax] = pkg.sim_plan_info(plan)[0]
        pkg.sim_plan_destroy(plan)
    assert counts[2] <= 245  # at most one block per fSim once single-qubit gates merge in
    assert counts[2] > counts[3] > counts[4] > counts[5] >= counts[6]


@pytest.mark.parametrize("grid,cycles,kmax", [((3, 4), 12, 5), ((4, 4), 12, 3), ((3, 5), 20, 5)])
def test_planner_search_finds_fewer_blocks_that_reproduce_circuit(pkg, oracle_mod, grid, cycles, kmax):
    # the beam search over block seeds (sim_plan_opts.search): never more blocks than the greedy
    # schedule (search=1), fewer on these circuits at the default width, and its blocks still
    # reproduce the gate-by-gate run
    circ = si.sycamore_circuit(si.Grid(*grid), cycles=cycles, seed=8)
    g = pkg.gates_array(circ)
    want = oracle_mod.run_circuit(circ)
    counts = {}
    for w in (1, 2, 16, 64, 0):
        plan = pkg.sim_plan_create(circ.n_qubits, g, kmax=kmax, search=w)
        try:
            nb, ng, mk = pkg.sim_plan_info(plan)
            assert ng == circ.n_gates and mk <= kmax
            counts[w] = nb
            psi = oracle_mod.basis_state(circ.n_qubits, 0)
            for t, m in plan_blocks(pkg, plan):
                assert list(t) == sorted(t) and len(set(t)) == len(t) <= kmax
                oracle_mod.apply_kq(psi, t, m)
            assert np.linalg.norm(psi - want) < 1e-12
        finally:
            pkg.sim_plan_destroy(plan)
    assert all(counts[w] <= counts[1] for w in counts)
    assert counts[0] == counts[16] < counts[1]  # 0 = the default width, 16


def test_planner_search_on_the_33_qubit_phases(pkg):
    # the 33-qubit, 20-cycle workload after its 3-pair front, phased over the lattice's two ends:
    # the default search plans fewer blocks than the greedy schedule; bad widths are refused
    circ = si.workload_circuit("syc33_6x6m3_d20", seed=0)
    n, g = circ.n_qubits, pkg.gates_array(circ)
    _, nf = pkg.sim_split_choose(n, g, 3)
    blocks = {}
    for w in (1, 0):
        ph = pkg.sim_phases_create(n, g[nf:], 3, [0, 1, 2], [n - 3, n - 2, n - 1], kmax=6, search=w)
        blocks[w] = pkg.sim_phases_info(ph)
        pkg.sim_phases_destroy(ph)
    assert blocks[0][0] == blocks[1][0] == 3
    assert blocks[0][1] < blocks[1][1]
    for bad in (-1, 257):
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_plan_create(n, g, kmax=6, search=bad)
        assert e.value.code == pkg.SIM_E_INVAL


def test_planner_custom_matrices(pkg, oracle_mod):
    n = 5
    rng = np.random.default_rng(2)
    recs = np.zeros(6, dtype=pkg._native.GATE_DTYPE)
    psi = oracle_mod.basis_state(n, 3)
    for i in range(6):
        if i % 2 == 0:
            q = int(rng.integers(n))
            u = si.random_unitary(1, seed=i)
            recs[i]["kind"], recs[i]["q0"] = pkg.SIM_GATE_U1, q
            recs[i]["u"][:8] = u.view(np.float64).ravel()
            oracle_mod.apply_1q(psi, q, u)
        else:
            q0, q1 = (int(x) for x in rng.choice(n, 2, replace=False))
            u = si.random_unitary(2, seed=i)
            recs[i]["kind"], recs[i]["q0"], recs[i]["q1"] = pkg.SIM_GATE_U2, q0, q1
            recs[i]["u"][:] = u.view(np.float64).ravel()
            oracle_mod.apply_2q(psi, q0, q1, u)
    plan = pkg.sim_plan_create(n, recs, kmax=3)
    got = oracle_mod.basis_state(n, 3)
    for t, m in plan_blocks(pkg, plan):
        oracle_mod.apply_kq(got, t, m)
    pkg.sim_plan_destroy(plan)
    assert np.linalg.norm(got - psi) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_planner_random_pairs_and_lone_qubits(pkg, oracle_mod, seed):
    # arbitrary one- and two-qubit unitaries on random (not lattice) pairs of 7 qubits, two of
    # which only ever see single-qubit gates (units of one qubit): at every width and search,
    # the blocks -- composed on the qubits met so far, in the order met, then reordered --
    # reproduce the gate-by-gate run
    n, lone = 7, (2, 5)
    rng = np.random.default_rng(40 + seed)
    paired = [q for q in range(n) if q not in lone]
    recs = np.zeros(60, dtype=pkg._native.GATE_DTYPE)
    psi = oracle_mod.basis_state(n, 0)
    for i in range(recs.size):
        if rng.random() < 0.4:
            q = int(rng.integers(n))
            u = si.random_unitary(1, seed=1000 * seed + i)
            recs[i]["kind"], recs[i]["q0"] = pkg.SIM_GATE_U1, q
            recs[i]["u"][:8] = u.view(np.float64).ravel()
            oracle_mod.apply_1q(psi, q, u)
        else:
            q0, q1 = (int(x) for x in rng.choice(paired, 2, replace=False))
            u = si.random_unitary(2, seed=1000 * seed + i)
            recs[i]["kind"], recs[i]["q0"], recs[i]["q1"] = pkg.SIM_GATE_U2, q0, q1
            recs[i]["u"][:] = u.view(np.float64).ravel()
            oracle_mod.apply_2q(psi, q0, q1, u)
    for kmax in (2, 3, 4, 5, 6):
        for search in (1, 3, 16):
            plan = pkg.sim_plan_create(n, recs, kmax=kmax, search=search)
            try:
                got = oracle_mod.basis_state(n, 0)
                for t, m in plan_blocks(pkg, plan):
                    assert list(t) == sorted(t) and len(t) <= kmax
                    oracle_mod.apply_kq(got, t, m)
                assert np.linalg.norm(got - psi) < 1e-12, (kmax, search)
            finally:
                pkg.sim_plan_destroy(plan)


def test_planner_rejects_bad_gates(pkg):
    recs = np.zeros(1, dtype=pkg._native.GATE_DTYPE)
    recs[0]["kind"], recs[0]["q0"], recs[0]["q1"] = si.FSIM, 2, 2
    with pytest.raises(pkg.SimError):
        pkg.sim_plan_create(4, recs)
    recs[0]["kind"] = 77
    with pytest.raises(pkg.SimError):
        pkg.sim_plan_create(4, recs)
    with pytest.raises(pkg.SimError):
        pkg.sim_plan_create(4, np.zeros(0, dtype=pkg._native.GATE_DTYPE), kmax=7)


def phase_list(pkg, ph):
    n_ph, _ = pkg.sim_phases_info(ph)
    out = []
    for i in range(n_ph):
        s, plan = pkg.sim_phases_get(ph, i)
        nb = pkg.sim_plan_info(plan)[0]
        out.append((s, [pkg.sim_plan_block(plan, j) for j in range(nb)]))
    return out


@pytest.mark.parametrize("grid,cycles,s", [((3, 4), 8, 2), ((4, 5), 12, 3), ((5, 7), 16, 4)])
def test_phases_reproduce_circuit_and_avoid_sliced_sets(pkg, oracle_mod, grid, cycles, s):
    # Sect. 4: phases alternate the sliced set; within a phase no gate touches it.
    circ = si.sycamore_circuit(si.Grid(*grid), cycles=cycles, seed=5)
    n = circ.n_qubits
    set_a = list(range(s))                 # one end of the lattice
    set_b = list(range(n - s, n))          # the other end
    ph = pkg.sim_phases_create(n, pkg.gates_array(circ), s, set_a, set_b, kmax=4)
    try:
        phases = phase_list(pkg, ph)
        assert all(phases[i][0] != phases[i + 1][0] for i in range(len(phases) - 1))
        if n <= 20:
            psi = oracle_mod.basis_state(n, 0)
        for which, blocks in phases:
            sliced = set(set_a if which == 0 else set_b)
            for t, m in blocks:
                assert not sliced & set(int(q) for q in t)
                if n <= 20:
                    oracle_mod.apply_kq(psi, t, m)
        if n <= 20:
            assert np.linalg.norm(psi - oracle_mod.run_circuit(circ)) < 1e-12
        assert sum(len(b) for _, b in phases) == pkg.sim_phases_info(ph)[1]
    finally:
        pkg.sim_phases_destroy(ph)


def test_phases_reject_gate_across_sets(pkg):
    recs = np.zeros(1, dtype=pkg._native.GATE_DTYPE)
    recs[0]["kind"], recs[0]["q0"], recs[0]["q1"] = si.FSIM, 0, 5
    with pytest.raises(pkg.SimError) as e:
        pkg.sim_phases_create(8, recs, 1, [0], [5])
    assert e.value.code == pkg.SIM_E_NONLOCAL


def _phase_cost(pkg, circ, s, a, b, kmax, weight):
    try:
        ph = pkg.sim_phases_create(circ.n_qubits, pkg.gates_array(circ), s, a, b, kmax=kmax)
    except pkg.SimError:
        return None
    nph, nbl = pkg.sim_phases_info(ph)
    pkg.sim_phases_destroy(ph)
    return weight * nph + nbl, nph, nbl


@pytest.mark.parametrize("grid,cycles,s,kmax", [((3, 4), 8, 2, 4), ((4, 4), 10, 2, 5), ((3, 5), 12, 3, 4)])
def test_phase_set_choice_is_the_best_window_pair(pkg, grid, cycles, s, kmax):
    # brute force over every pair of disjoint windows of s consecutive qubits, through
    # sim_phases_create: the chooser's cost must be the minimum, and its pair must reach it
    circ = si.sycamore_circuit(si.Grid(*grid), cycles=cycles, seed=21)
    n, weight = circ.n_qubits, 32.0
    a, b, nph, nbl = pkg.sim_phases_choose_sets(n, pkg.gates_array(circ), s, kmax=kmax, phase_weight=weight)
    assert len(set(a) | set(b)) == 2 * s
    costs = []
    for i in range(n - s + 1):
        for j in range(i + s, n - s + 1):
            c = _phase_cost(pkg, circ, s, list(range(i, i + s)), list(range(j, j + s)), kmax, weight)
            if c is not None:
                costs.append(c[0])
    chosen = _phase_cost(pkg, circ, s, a, b, kmax, weight)
    assert chosen == (weight * nph + nbl, nph, nbl)
    assert chosen[0] == min(costs)
    ends = _phase_cost(pkg, circ, s, list(range(s)), list(range(n - s, n)), kmax, weight)
    assert ends is None or chosen[0] <= ends[0]


def test_phase_set_choice_weights_and_errors(pkg):
    circ = si.sycamore_circuit(si.Grid(4, 5), cycles=12, seed=3)
    n = circ.n_qubits
    # a huge phase weight minimises the number of phases first
    _, _, nph_heavy, _ = pkg.sim_phases_choose_sets(n, pkg.gates_array(circ), 2, kmax=4, phase_weight=1e9)
    best = None
    for i in range(n - 1):
        for j in range(i + 2, n - 1):
            c = _phase_cost(pkg, circ, 2, [i, i + 1], [j, j + 1], 4, 1.0)
            if c is not None and (best is None or c[1] < best):
                best = c[1]
    assert nph_heavy == best
    for bad in ((n, 0), (n, 9), (1, 1)):
        with pytest.raises(pkg.SimError):
            pkg.sim_phases_choose_sets(bad[0], pkg.gates_array(circ), bad[1])


# ---- contraction deferral: the split's gate lists against the oracle's EI / E2Q tensors ----

def _records_from_tuples(pkg, gates):
    recs = np.zeros(len(gates), dtype=pkg._native.GATE_DTYPE)
    for i, g in enumerate(gates):
        recs[i]["kind"], recs[i]["q0"], recs[i]["q1"] = g[0], g[1], g[2]
        for j, f in enumerate(("theta", "phi", "dplus", "dminus", "dminus_off")):
            recs[i][f] = g[3 + j] if len(g) > 3 + j else 0.0
    return recs


def _run_records_on_oracle(pkg, oracle_mod, n, recs):
    """The oracle applies a gate-record list one gate at a time (matrices of the standard kinds
    from the oracle; caller-given U1/U2 matrices as stored in the records)."""
    psi = oracle_mod.basis_state(n, 0)
    for r in recs:
        kind = int(r["kind"])
        if kind == pkg.SIM_GATE_U2:
            oracle_mod.apply_2q(psi, int(r["q0"]), int(r["q1"]), r["u"].view(np.complex128).reshape(4, 4))
        elif kind == pkg.SIM_GATE_U1:
            oracle_mod.apply_1q(psi, int(r["q0"]), r["u"][:8].view(np.complex128).reshape(2, 2))
        elif kind == si.FSIM:
            u = oracle_mod.gate_matrix(kind, r["theta"], r["phi"], r["dplus"], r["dminus"], r["dminus_off"])
            oracle_mod.apply_2q(psi, int(r["q0"]), int(r["q1"]), u)
        else:
            oracle_mod.apply_1q(psi, int(r["q0"]), oracle_mod.gate_matrix(kind))
    return psi


def _split_cases():
    rng = np.random.default_rng(11)
    cases = []
    for seed, n in ((0, 4), (1, 6), (2, 7)):
        gates = []
        for _ in range(3 * n):
            if rng.random() < 0.4:
                gates.append((int(rng.integers(3)), int(rng.integers(n)), -1))
            else:
                q0, q1 = (int(x) for x in rng.choice(n, 2, replace=False))
                gates.append((si.FSIM, q0, q1, *(float(x) for x in rng.uniform(-3, 3, 5))))
        side = [int(x) for x in rng.permutation([0] * (n // 2) + [1] * (n - n // 2))]
        cases.append((n, gates, side))
    circ = si.sycamore_circuit(si.Grid(3, 4), cycles=6, seed=4)
    cases.append((12, [tuple(g) for g in circ.gates], [0 if (q % 4) < 2 else 1 for q in range(12)]))
    return cases


@pytest.mark.parametrize("case", range(4))
def test_split_gate_lists_reproduce_oracle_tensors(pkg, oracle_mod, case):
    n, gates, side = _split_cases()[case]
    recs = _records_from_tuples(pkg, gates)
    s = pkg.sim_split_create(n, recs, side)
    try:
        n_side, n_wires, pairs, n_gates = pkg.sim_split_info(s)
        o1, o2, c = oracle_mod.split_tensors(n, gates, side)
        assert pairs == c and n_side == [side.count(0), side.count(1)]
        assert n_wires == [n_side[0] + 2 * c, n_side[1] + 2 * c]
        for t, want in ((0, o1), (1, o2)):
            tg = pkg.sim_split_gates(s, t)
            assert tg.size == n_gates[t]
            wire_at = pkg.sim_split_canonical(s, t)
            assert sorted(wire_at) == list(range(n_wires[t]))
            perm = [0] * n_wires[t]
            for p, w in enumerate(wire_at):
                perm[w] = p
            got = oracle_mod.permute(_run_records_on_oracle(pkg, oracle_mod, n_wires[t], tg), perm)
            assert np.linalg.norm(got - want) < 1e-12 * max(1.0, np.linalg.norm(want))
            # and through the aggregation planner: fused blocks of the tensor's gate list
            plan = pkg.sim_plan_create(n_wires[t], tg, kmax=4)
            psi = oracle_mod.basis_state(n_wires[t], 0)
            for tt, m in plan_blocks(pkg, plan):
                oracle_mod.apply_kq(psi, tt, m)
            pkg.sim_plan_destroy(plan)
            assert np.linalg.norm(oracle_mod.permute(psi, perm) - want) < 1e-11 * max(1.0, np.linalg.norm(want))
    finally:
        pkg.sim_split_destroy(s)


def test_split_rejects_bad_input(pkg):
    recs = _records_from_tuples(pkg, [(0, 0, -1), (si.FSIM, 0, 1, 1.0, 0.5)])
    for side in ([0, 0], [1, 1], [0, 2], [-1, 1]):
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_split_create(2, recs, side)
        assert e.value.code == pkg.SIM_E_INVAL
    bad = _records_from_tuples(pkg, [(si.FSIM, 1, 1, 1.0, 0.5)])
    with pytest.raises(pkg.SimError):
        pkg.sim_split_create(2, bad, [0, 1])
    # 20 bridging gates on one pair of qubits: 1 + 40 wires per tensor exceeds the 40-qubit limit
    many = _records_from_tuples(pkg, [(si.FSIM, 0, 1, 1.0, 0.5)] * 20)
    with pytest.raises(pkg.SimError):
        pkg.sim_split_create(2, many, [0, 1])
    L = pkg.lib()
    assert L.sim_contract(None, None, None, None, 0) == pkg.SIM_E_INVAL
    assert L.sim_front_create(None, None, None, None) == pkg.SIM_E_INVAL
    assert L.sim_front_run(None, None) == pkg.SIM_E_INVAL
    assert L.sim_front_destroy(None) == pkg.SIM_E_INVAL
    assert L.sim_split_info(None, None, None, None, None) == pkg.SIM_E_INVAL


def test_plan_layout_is_a_bijection_no_worse_than_identity(pkg):
    circ = si.workload_circuit("syc30_5x6_d20", seed=0)
    g = pkg.gates_array(circ)
    for kmax, prec in ((6, pkg.SIM_FP16X3_TMEM), (5, pkg.SIM_FP16X3_TMEM), (4, pkg.SIM_FP32), (5, pkg.SIM_TF32X3)):
        plan = pkg.sim_plan_create(30, g, kmax=kmax, precision=prec)
        try:
            perm, est, ident = pkg.sim_plan_layout(plan, 30)
            assert sorted(perm) == list(range(30))
            assert est <= ident + 1e-9
            if prec == pkg.SIM_TF32X3:  # no cost model: identity
                assert perm == list(range(30)) and est == ident
            if kmax == 6:
                assert est < 0.9 * ident  # the 6-qubit blocks gain from leaving bits 0-3
            assert pkg.sim_plan_layout(plan, 30)[0] == perm  # deterministic
        finally:
            pkg.sim_plan_destroy(plan)
    L = pkg.lib()
    assert L.sim_plan_layout(None, None, None) == pkg.SIM_E_INVAL
    assert L.sim_set_layout(None, None) == pkg.SIM_E_INVAL


def _front_len(gates, side, max_pairs):
    pairs = 0
    for i, g in enumerate(gates):
        if g[2] >= 0 and side[g[1]] != side[g[2]]:
            if pairs == max_pairs:
                return i
            pairs += 1
    return len(gates)


@pytest.mark.parametrize("shape,cycles,seed,max_pairs", [((2, 4), 8, 1, 3), ((3, 3), 8, 2, 4), ((2, 5), 10, 3, 3),
                                                         ((3, 4), 8, 4, 5), ((2, 6), 10, 5, 4)])
def test_split_choice_matches_brute_force(pkg, shape, cycles, seed, max_pairs):
    # the search's front equals the longest over every bipartition in the allowed size window
    import itertools
    circ = si.sycamore_circuit(si.Grid(*shape), cycles, seed)
    n = circ.n_qubits
    side, nf = pkg.sim_split_choose(n, pkg.gates_array(circ), max_pairs, min_side=3)
    slack = max(1, n // 8)
    lo, hi = max(min(3, n // 2), n // 2 - slack), min(n - min(3, n // 2), (n + 1) // 2 + slack)
    assert lo <= side.count(0) <= hi
    assert nf == _front_len(circ.gates, side, max_pairs)
    best = 0
    for k in range(lo, hi + 1):
        for comb in itertools.combinations(range(n), k):
            sd = [1] * n
            for q in comb:
                sd[q] = 0
            best = max(best, _front_len(circ.gates, sd, max_pairs))
    assert nf == best


def test_split_choice_on_the_30_qubit_workload(pkg):
    # the lattice's middle column: 5 crossings in the first 6 cycles, 284 gates
    circ = si.workload_circuit("syc30_5x6_d20", seed=0)
    side, nf = pkg.sim_split_choose(30, pkg.gates_array(circ), 5)
    assert nf == 284 and side.count(0) == 15
    bridging = [g for g in circ.gates[:nf] if g[2] >= 0 and side[g[1]] != side[g[2]]]
    assert len(bridging) == 5
    g = circ.gates[nf]
    assert g[2] >= 0 and side[g[1]] != side[g[2]]  # the sixth crossing ends the front
    s = pkg.sim_split_create(30, pkg.gates_array(circ)[:nf], side)
    try:
        assert pkg.sim_split_info(s)[2] == 5
    finally:
        pkg.sim_split_destroy(s)
    L = pkg.lib()
    assert L.sim_split_choose(1, 0, None, 5, 0, None, None) == pkg.SIM_E_INVAL


@pytest.mark.parametrize("name,s,kmax", [("syc34_5x7m1_d16", 3, 6), ("syc35_5x7_d16", 4, 6)])
def test_phases_layout_keeps_sliced_sets_and_lowers_estimate(pkg, name, s, kmax):
    # the host-store order of the qubits outside the sliced sets: a bijection with set B on bits
    # n-2s .. n-s-1 and set A on n-s .. n-1 in set order, never worse than the ascending order,
    # and the same on every call (seeded)
    circ = si.workload_circuit(name, seed=0)
    n = circ.n_qubits
    gates = pkg.gates_array(circ)
    a, b, _, _ = pkg.sim_phases_choose_sets(n, gates, s, kmax=kmax)
    ph = pkg.sim_phases_create(n, gates, s, a, b, kmax=kmax, precision=pkg.SIM_FP16X3_TMEM)
    side, nf = pkg.sim_split_choose(n, gates, 4)
    sp = pkg.sim_split_create(n, gates[:nf], side)
    try:
        perm, est, est_asc = pkg.sim_phases_layout(ph, n)
        again = pkg.sim_phases_layout(ph, n)
        pf, estf, _ = pkg.sim_phases_layout(ph, n, sp)
        pr, _, _ = pkg.sim_phases_layout(ph, n, sp, resident=True)
        first = pkg.sim_phases_get(ph, 0)[0]
    finally:
        pkg.sim_phases_destroy(ph)
        pkg.sim_split_destroy(sp)
    for p_ in (perm, pf, pr):
        assert sorted(p_) == list(range(n))
    assert [perm[q] for q in b] == list(range(n - 2 * s, n - s))
    assert [perm[q] for q in a] == list(range(n - s, n))
    assert est <= est_asc + 1e-9 and est < est_asc  # these circuits have blocks with low targets
    assert again == (perm, est, est_asc)
    # with a front: the sets where a host store keeps them, side-0 qubits on bits 0-4
    assert [pf[q] for q in a] == list(range(n - s, n))
    low = sorted(range(n), key=lambda q: pf[q])[:5]
    assert all(side[q] == 0 for q in low)
    # resident: the first phase's sliced set on top, the other below, side-0 qubits low
    top, below = (a, b) if first == 0 else (b, a)
    assert [pr[q] for q in top] == list(range(n - s, n))
    assert [pr[q] for q in below] == list(range(n - 2 * s, n - s))
    assert all(side[q] == 0 for q in sorted(range(n), key=lambda q: pr[q])[:5])
    assert estf < est_asc
