"""GPU: the contraction straight into a sliced host store (Sect. 4: tensors 1 and 2 are contracted
slice by slice into the secondary-storage state of subcircuit 3).

sim_contract_phase and sim_front_run_phase fill every slice of the sliced set (A, or B) from the
two tensors (in a device slot, or in place for a hybrid store's device regions), optionally run a
phase's blocks on it, and write it once.  Every amplitude, read back in logical order, is compared
with the oracle's plain simulation of the same gates: the sliced set's qubits on both sides, on one
side only (the side left too narrow for the tensor-core kernel takes the FP32 one), 2 and 3 sliced
bits, slices of set A and of set B, a hybrid store, FP32 and 3xFP16 on tcgen05, with and without
the fused phase, the other phases after it, and a store laid out by sim_phases_layout.
"""
import numpy as np
import pytest

import syc_inputs as si

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as p
    return p


def front_length(grid, cycles):
    """Gate records in the first `cycles` cycles (a 1q layer plus the cycle's pattern each)."""
    n = grid.n_qubits
    return sum(n + len(grid.pattern(si.PATTERN_ORDER[t % 8])) for t in range(cycles))


def column_sides(grid, cut):
    return [0 if c < cut else 1 for (r, c) in grid.sites()]


def tensor_handles(pkg, s, kmax, precision):
    _, n_wires, _, _ = pkg.sim_split_info(s)
    hs = []
    for t in range(2):
        h = pkg.sim_create(n_wires[t])
        plan = pkg.sim_plan_create(n_wires[t], pkg.sim_split_gates(s, t), kmax=kmax, precision=precision)
        pkg.sim_apply_plan(h, plan)
        pkg.sim_plan_destroy(plan)
        hs.append(h)
    return hs


def avoiding(circ, start, count, qubits):
    """Indices of up to `count` gates from `start` on that touch none of `qubits`."""
    bad = set(qubits)
    out = []
    for i in range(start, len(circ.gates)):
        g = circ.gates[i]
        qs = {g[1]} if g[2] < 0 else {g[1], g[2]}  # one-qubit gates carry q1 = -1
        if not qs & bad:
            out.append(i)
            if len(out) == count:
                break
    return out


def err2(got, want):
    d = got.astype(np.complex128) - want
    return float(np.sqrt(np.vdot(d, d).real))


GRID, CYCLES, CUT = (4, 5), 4, 2  # 20 qubits; side 0 = columns 0-1 (8 qubits), side 1 = 12 qubits


@pytest.mark.parametrize("set_a,set_b,regions,prec,fill", [
    ([1, 13], [8, 12], 0, "tmem", 0),     # one set-A qubit per side, tcgen05 (7 + 11 free side bits)
    ([1, 13], [8, 12], 0, "fp32", 0),     # the FP32 kernel on strided sub-ranges
    ([13, 18], [2, 7], 2, "tmem", 0),     # both on side 1; hybrid store: 2 of 4 regions in place
    ([0, 6], [13, 18], 0, "tmem", 0),     # both on side 0: 6 free bits there, the FP32 kernel
    ([1, 13, 19], [7, 8, 12], 3, "tmem", 0),  # 3 sliced bits, 8 slices, 3 in device memory
    ([1, 13], [8, 12], 0, "tmem", 1),     # slices of set B: each slot scattered as files
    ([13, 18], [2, 7], 2, "fp32", 1),     # set B's qubits both on side 1, hybrid store
])
def test_contraction_into_store_matches_oracle(pkg, oracle_mod, set_a, set_b, regions, prec, fill):
    grid = si.Grid(*GRID)
    circ = si.sycamore_circuit(grid, CYCLES + 2, seed=31)
    n = circ.n_qubits
    gates = pkg.gates_array(circ)
    nf = front_length(grid, CYCLES)
    precision = pkg.SIM_FP32 if prec == "fp32" else pkg.SIM_FP16X3_TMEM
    s = pkg.sim_split_create(n, gates[:nf], column_sides(grid, CUT))
    t1, t2 = tensor_handles(pkg, s, 4, precision)
    out = pkg.sim_create(n, len(set_a), store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=2,
                         store_device_regions=regions)
    try:
        pkg.sim_contract_phase(out, t1, t2, s, precision, fill)
        pkg.sim_sync(out)
        got = pkg.sim_amplitudes(out, dtype=pkg.SIM_C128)
        norm, s2, _ = pkg.sim_reduce(out)
    finally:
        for h in (out, t1, t2):
            pkg.sim_destroy(h)
        pkg.sim_split_destroy(s)
    want = oracle_mod.run_circuit(circ.gates[:nf], n_qubits=n)
    assert err2(got, want) <= TOL
    onorm, os2, _ = oracle_mod.reduce(want)
    assert abs(norm - onorm) < 1e-5 and abs(s2 - os2) < 1e-4


@pytest.mark.parametrize("regions", [0, 2])
def test_fused_phase_then_set_b_phase_match_oracle(pkg, oracle_mod, regions):
    # the front runner contracts into the store with the first phase's blocks (gates avoiding set
    # A) fused; a set-B phase (gates avoiding set B) follows through sim_run_phase
    grid = si.Grid(*GRID)
    circ = si.sycamore_circuit(grid, CYCLES + 6, seed=32)
    n = circ.n_qubits
    gates = pkg.gates_array(circ)
    nf = front_length(grid, CYCLES)
    set_a, set_b = [1, 13], [8, 12]
    ph1 = avoiding(circ, nf, 60, set_a)
    ph2 = avoiding(circ, ph1[-1] + 1, 60, set_b)
    s = pkg.sim_split_create(n, gates[:nf], column_sides(grid, CUT))
    out = pkg.sim_create(n, 2, store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=3,
                         store_device_regions=regions)
    fr = pkg.sim_front_create(out, s, kmax=5, precision=pkg.SIM_FP16X3_TMEM)
    p1 = pkg.sim_plan_create(n, gates[ph1], kmax=5, precision=pkg.SIM_FP16X3_TMEM)
    p2 = pkg.sim_plan_create(n, gates[ph2], kmax=5, precision=pkg.SIM_FP16X3_TMEM)
    try:
        n0 = pkg.sim_launch_count(out)
        pkg.sim_front_run_phase(out, fr, 0, p1)
        pkg.sim_run_phase(out, 1, p2)
        pkg.sim_sync(out)
        assert pkg.sim_launch_count(out) > n0
        got = pkg.sim_amplitudes(out, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_front_destroy(fr)
        for p in (p1, p2):
            pkg.sim_plan_destroy(p)
        pkg.sim_destroy(out)
        pkg.sim_split_destroy(s)
    want = oracle_mod.run_circuit([circ.gates[i] for i in list(range(nf)) + ph1 + ph2], n_qubits=n)
    assert err2(got, want) <= TOL


def test_front_run_into_store_twice_overwrites(pkg, oracle_mod):
    # the store's earlier contents do not matter: a second front run gives the same state
    grid = si.Grid(*GRID)
    circ = si.sycamore_circuit(grid, CYCLES, seed=33)
    n = circ.n_qubits
    gates = pkg.gates_array(circ)
    nf = front_length(grid, CYCLES)
    s = pkg.sim_split_create(n, gates[:nf], column_sides(grid, CUT))
    out = pkg.sim_create(n, 2, store=pkg.SIM_STORE_HOST, set_a=[1, 13], set_b=[8, 12], slots=2)
    fr = pkg.sim_front_create(out, s, kmax=4, precision=pkg.SIM_FP16X3_TMEM)
    try:
        pkg.sim_reset(out, 5)
        pkg.sim_front_run(out, fr)
        pkg.sim_sync(out)
        first = pkg.sim_amplitudes(out, dtype=pkg.SIM_C128)
        pkg.sim_front_run(out, fr)
        pkg.sim_sync(out)
        second = pkg.sim_amplitudes(out, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_front_destroy(fr)
        pkg.sim_destroy(out)
        pkg.sim_split_destroy(s)
    assert np.array_equal(first, second)
    assert err2(first, oracle_mod.run_circuit(circ.gates[:nf], n_qubits=n)) <= TOL


def test_plan_on_set_a_is_rejected_and_device_out_contracts(pkg, oracle_mod):
    grid = si.Grid(*GRID)
    circ = si.sycamore_circuit(grid, CYCLES + 1, seed=34)
    n = circ.n_qubits
    gates = pkg.gates_array(circ)
    nf = front_length(grid, CYCLES)
    s = pkg.sim_split_create(n, gates[:nf], column_sides(grid, CUT))
    t1, t2 = tensor_handles(pkg, s, 4, pkg.SIM_FP16X3_TMEM)
    store = pkg.sim_create(n, 2, store=pkg.SIM_STORE_HOST, set_a=[1, 13], set_b=[8, 12], slots=2)
    dev = pkg.sim_create(n)
    rest = gates[nf:]  # touches every qubit, set A's too
    p = pkg.sim_plan_create(n, rest, kmax=4, precision=pkg.SIM_FP16X3_TMEM)
    try:
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_contract_phase(store, t1, t2, s, pkg.SIM_FP16X3_TMEM, 0, p)
        assert e.value.code == pkg.SIM_E_NONLOCAL
        # a device-resident out: the contraction, then the plan
        pkg.sim_contract_phase(dev, t1, t2, s, pkg.SIM_FP16X3_TMEM, 0, p)
        got = pkg.sim_amplitudes(dev, dtype=pkg.SIM_C128)
    finally:
        for h in (store, dev, t1, t2):
            pkg.sim_destroy(h)
        pkg.sim_plan_destroy(p)
        pkg.sim_split_destroy(s)
    assert err2(got, oracle_mod.run_circuit(circ, n_qubits=n)) <= TOL


@pytest.mark.parametrize("regions", [0, 1])
def test_chosen_store_layout_front_and_phases_match_oracle(pkg, oracle_mod, regions, tmp_path):
    # the whole circuit: the front contracted into a store laid out by sim_phases_layout, fused
    # with the first phase, the other phases after it; then a checkpoint of that store loaded into
    # a fresh store in the ascending layout (it takes the file's order of the other qubits)
    grid = si.Grid(*GRID)
    circ = si.sycamore_circuit(grid, 12, seed=35)
    n = circ.n_qubits
    gates = pkg.gates_array(circ)
    nf = front_length(grid, CYCLES)
    rest = gates[nf:]
    prec = pkg.SIM_FP16X3_TMEM
    a, b, _, _ = pkg.sim_phases_choose_sets(n, rest, 2, kmax=5)
    ph = pkg.sim_phases_create(n, rest, 2, a, b, kmax=5, precision=prec)
    s = pkg.sim_split_create(n, gates[:nf], column_sides(grid, CUT))
    perm, est, est_asc = pkg.sim_phases_layout(ph, n, s)
    assert est <= est_asc
    out = pkg.sim_create(n, 2, store=pkg.SIM_STORE_HOST, set_a=a, set_b=b, slots=2, store_device_regions=regions)
    fresh = pkg.sim_create(n, 2, store=pkg.SIM_STORE_HOST, set_a=a, set_b=b, slots=2)
    fr = pkg.sim_front_create(out, s, kmax=5, precision=prec)
    path = str(tmp_path / "store.ckpt")
    try:
        pkg.sim_set_layout(out, perm)
        assert [int(x) for x in pkg.sim_info(out)[2]] == perm
        n_phases, _ = pkg.sim_phases_info(ph)
        set0, p0 = pkg.sim_phases_get(ph, 0)  # whichever set the first phase slices
        pkg.sim_front_run_phase(out, fr, set0, p0)
        for i in range(1, n_phases):
            pkg.sim_run_phase(out, *pkg.sim_phases_get(ph, i))
        pkg.sim_sync(out)
        got = pkg.sim_amplitudes(out, dtype=pkg.SIM_C128)
        pkg.sim_state_save(out, path)
        pkg.sim_state_load(fresh, path)
        assert [int(x) for x in pkg.sim_info(fresh)[2]] == perm
        loaded = pkg.sim_amplitudes(fresh, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_front_destroy(fr)
        pkg.sim_destroy(out)
        pkg.sim_destroy(fresh)
        pkg.sim_split_destroy(s)
        pkg.sim_phases_destroy(ph)
    assert err2(got, oracle_mod.run_circuit(circ)) <= TOL
    assert np.array_equal(got, loaded)


def test_store_layout_must_keep_sliced_sets(pkg):
    n = 20
    out = pkg.sim_create(n, 2, store=pkg.SIM_STORE_HOST, set_a=[1, 13], set_b=[8, 12], slots=2)
    try:
        bits = [int(x) for x in pkg.sim_info(out)[2]]
        moved = list(bits)
        moved[1], moved[0] = bits[0], bits[1]  # qubit 1 (set A) trades bits with qubit 0
        with pytest.raises(pkg.SimError):
            pkg.sim_set_layout(out, moved)
        swapped = list(bits)
        swapped[0], swapped[2] = bits[2], bits[0]  # two qubits outside both sets: allowed
        pkg.sim_set_layout(out, swapped)
        assert [int(x) for x in pkg.sim_info(out)[2]] == swapped
    finally:
        pkg.sim_destroy(out)


@pytest.mark.parametrize("side0,set_a,set_b,prec,tol", [
    ([0, 1], [0, 1], [18, 19], "fp32", TOL),          # side 0 entirely sliced: no free x bit
    (None, [0, 1, 2, 3, 10, 11, 12, 13], [5, 6, 7, 8, 15, 16, 17, 18], "tmem", TOL),  # 8 sliced bits
    (None, [1, 13], [8, 12], "bf16x3", 1e-4),          # BF16x3 into a store (its stated bound)
])
def test_store_contraction_edges(pkg, oracle_mod, side0, set_a, set_b, prec, tol):
    grid = si.Grid(*GRID)
    circ = si.sycamore_circuit(grid, CYCLES, seed=36)
    n = circ.n_qubits
    gates = pkg.gates_array(circ)
    nf = front_length(grid, CYCLES)
    side = column_sides(grid, CUT) if side0 is None else [0 if q in side0 else 1 for q in range(n)]
    precision = {"fp32": pkg.SIM_FP32, "tmem": pkg.SIM_FP16X3_TMEM, "bf16x3": pkg.SIM_BF16X3}[prec]
    s = pkg.sim_split_create(n, gates[:nf], side)
    t1, t2 = tensor_handles(pkg, s, 4, pkg.SIM_FP32 if prec == "fp32" else precision)
    out = pkg.sim_create(n, len(set_a), store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=2)
    try:
        pkg.sim_contract_phase(out, t1, t2, s, precision)
        pkg.sim_sync(out)
        got = pkg.sim_amplitudes(out, dtype=pkg.SIM_C128)
    finally:
        for h in (out, t1, t2):
            pkg.sim_destroy(h)
        pkg.sim_split_destroy(s)
    assert err2(got, oracle_mod.run_circuit(circ.gates[:nf], n_qubits=n)) <= tol


def test_front_into_sliced_resident_state_then_phases(pkg, oracle_mod):
    # a device-resident state with 2 sliced bits (Sect. 4 in HBM): the contraction writes the
    # whole state in the layout sim_phases_layout chose (the first phase's sliced set already on
    # top, so no move before it), then sim_run_phases runs the rest, against the oracle
    grid = si.Grid(*GRID)
    circ = si.sycamore_circuit(grid, 12, seed=37)
    n = circ.n_qubits
    gates = pkg.gates_array(circ)
    nf = front_length(grid, CYCLES)
    prec = pkg.SIM_FP16X3_TMEM
    a, b = [0, 1], [18, 19]
    ph = pkg.sim_phases_create(n, gates[nf:], 2, a, b, kmax=5, precision=prec)
    s = pkg.sim_split_create(n, gates[:nf], column_sides(grid, CUT))
    perm, _, _ = pkg.sim_phases_layout(ph, n, s, resident=True)
    h = pkg.sim_create(n, 2)
    fr = pkg.sim_front_create(h, s, kmax=5, precision=prec)
    try:
        n_phases, _ = pkg.sim_phases_info(ph)
        for _ in range(2):  # twice: the layout is set again before each run
            pkg.sim_set_layout(h, perm)
            pkg.sim_profile_enable(h, True)
            pkg.sim_front_run(h, fr)
            pkg.sim_run_phases(h, ph)
            perms = pkg.sim_profile_read(h, pkg.SIM_PROF_PERMUTE)[0]
            pkg.sim_profile_enable(h, False)
            got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
            assert perms <= n_phases - 1  # no move before the first phase
            assert err2(got, oracle_mod.run_circuit(circ)) <= TOL
    finally:
        pkg.sim_front_destroy(fr)
        pkg.sim_destroy(h)
        pkg.sim_split_destroy(s)
        pkg.sim_phases_destroy(ph)
