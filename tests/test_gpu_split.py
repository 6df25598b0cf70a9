"""GPU: contraction deferral (Sect. 2; Appendix, EI / E2Q and the contraction).

* Tensors 1 and 2, computed by running the split's gate lists through the planner and the fused
  apply kernels, against the oracle's EI / E2Q tensors, element by element.
* sim_contract (FP32 CUDA cores and tcgen05 3xFP16) against the oracle's plain simulation of the
  same gates: ||psi - psi_oracle||_2 <= 1e-5 (the tensors carry squared norm 2^c each; the
  contraction brings psi back to norm 1).
* The whole circuit: its first cycles through the split and the contraction, the rest through
  the fused blocks on the contracted state, against the oracle.
* Edge cases: no bridging gate (a single entanglement value: an outer product), sides narrower
  than a tile (ragged x / y), sides too narrow for the tensor-core kernel.
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
    """side 0 for lattice columns < cut, 1 for the rest (qubits numbered row-major)."""
    return [0 if c < cut else 1 for (r, c) in grid.sites()]


def tensor_states(pkg, s, kmax, precision):
    """Run each tensor's gate list on its own handle; returns the two handles."""
    _, n_wires, _, _ = pkg.sim_split_info(s)
    hs = []
    for t in range(2):
        h = pkg.sim_create(n_wires[t])
        plan = pkg.sim_plan_create(n_wires[t], pkg.sim_split_gates(s, t), kmax=kmax, precision=precision)
        pkg.sim_apply_plan(h, plan)
        pkg.sim_plan_destroy(plan)
        hs.append(h)
    return hs


def contracted_front(pkg, n, gates, side, kmax, precision, contract_precision):
    """psi after the gate list, through the split and the contraction (returns handle, split)."""
    s = pkg.sim_split_create(n, gates, side)
    h1, h2 = tensor_states(pkg, s, kmax, precision)
    out = pkg.sim_create(n)
    try:
        pkg.sim_contract(out, h1, h2, s, contract_precision)
        pkg.sim_sync(out)
    finally:
        pkg.sim_destroy(h1)
        pkg.sim_destroy(h2)
    return out, s


def err2(got64, want128):
    d = got64.astype(np.complex128) - want128
    return float(np.sqrt(np.vdot(d, d).real))


@pytest.mark.parametrize("precision", ["fp32", "tmem"])
def test_tensors_match_oracle(pkg, oracle_mod, precision):
    grid = si.Grid(3, 4)
    circ = si.sycamore_circuit(grid, cycles=6, seed=4)
    side = column_sides(grid, 2)
    prec, kmax = (pkg.SIM_FP32, 4) if precision == "fp32" else (pkg.SIM_FP16X3_TMEM, 5)
    s = pkg.sim_split_create(12, pkg.gates_array(circ), side)
    try:
        _, n_wires, c, _ = pkg.sim_split_info(s)
        o1, o2, oc = oracle_mod.split_tensors(12, circ, side)
        assert c == oc == 3
        hs = tensor_states(pkg, s, kmax, prec)
        for t, want in ((0, o1), (1, o2)):
            got = pkg.sim_amplitudes(hs[t])  # logical (wire) order
            wire_at = pkg.sim_split_canonical(s, t)
            want_w = oracle_mod.permute(want, wire_at)  # canonical position p -> wire wire_at[p]
            rel = err2(got, want_w) / float(np.linalg.norm(want))
            print(f"tensor {t + 1} ({precision}): relative error {rel:.2e}")
            assert rel <= TOL
        for h in hs:
            pkg.sim_destroy(h)
    finally:
        pkg.sim_split_destroy(s)


@pytest.mark.parametrize("cprec", ["fp32", "tmem", "bf16x3"])
@pytest.mark.parametrize("shape,cycles,cut", [((3, 4), 6, 2), ((4, 4), 4, 2), ((4, 5), 6, 2), ((4, 6), 6, 3)])
def test_contraction_matches_plain_simulation(pkg, oracle_mod, shape, cycles, cut, cprec):
    grid = si.Grid(*shape)
    circ = si.sycamore_circuit(grid, cycles=cycles, seed=sum(shape) + cycles)
    n = grid.n_qubits
    side = column_sides(grid, cut)
    gates = pkg.gates_array(circ)
    cp = {"fp32": pkg.SIM_FP32, "tmem": pkg.SIM_FP16X3_TMEM, "bf16x3": pkg.SIM_BF16X3}[cprec]
    out, s = contracted_front(pkg, n, gates, side, 4, pkg.SIM_FP32, cp)
    try:
        pairs = pkg.sim_split_info(s)[2]
        got = pkg.sim_amplitudes(out)
        norm = pkg.sim_reduce(out)[0]
    finally:
        pkg.sim_destroy(out)
        pkg.sim_split_destroy(s)
    want = oracle_mod.run_circuit(circ)
    e = err2(got, want)
    print(f"{shape} {cycles} cycles, {pairs} bridging gates, {cprec}: ||dpsi|| = {e:.2e}, norm {norm:.8f}")
    # BF16x3: pieces of 8 significant bits, about 2^-16 relative per product (measured 0.2-4.5e-6
    # on these fronts; bound 2e-5 as for one BF16x3 pass)
    tol = 2e-5 if cprec == "bf16x3" else TOL
    assert pairs > 0 and e <= tol and abs(norm - 1) < (2e-5 if cprec == "bf16x3" else 1e-5)


@pytest.mark.parametrize("cprec", ["fp32", "tmem"])
def test_front_then_fused_blocks_matches_oracle(pkg, oracle_mod, cprec):
    # 20 qubits, 14 cycles: the first 6 through the split (patterns A, B bridge the column cut),
    # the remaining gates as fused blocks on the contracted state (its layout puts side-0 qubits
    # low), against the oracle for the whole circuit.
    grid = si.Grid(4, 5)
    circ = si.sycamore_circuit(grid, cycles=14, seed=9)
    n = grid.n_qubits
    f = front_length(grid, 6)
    gates = pkg.gates_array(circ)
    cp, prec, kmax = ((pkg.SIM_FP32, pkg.SIM_FP32, 4) if cprec == "fp32"
                      else (pkg.SIM_FP16X3_TMEM, pkg.SIM_FP16X3_TMEM, 5))
    out, s = contracted_front(pkg, n, gates[:f], column_sides(grid, 2), kmax, prec, cp)
    try:
        _, _, bit_of = pkg.sim_info(out)
        assert sorted(bit_of) == list(range(n))
        plan = pkg.sim_plan_create(n, gates[f:], kmax=kmax, precision=prec)
        pkg.sim_apply_plan(out, plan)
        pkg.sim_plan_destroy(plan)
        got = pkg.sim_amplitudes(out)
    finally:
        pkg.sim_destroy(out)
        pkg.sim_split_destroy(s)
    e = err2(got, oracle_mod.run_circuit(circ))
    print(f"20q 14 cycles, split front of 6 ({cprec}): ||dpsi|| = {e:.2e}")
    assert e <= TOL


@pytest.mark.parametrize("cprec", ["fp32", "tmem"])
def test_no_bridging_gate_is_outer_product(pkg, oracle_mod, cprec):
    # 3 x 4 grid, cycles C, D (t = 2, 3 of ABCDCDAB) only: vertical couplers never cross a
    # column cut, so the contraction has one entanglement value
    grid = si.Grid(3, 4)
    circ = si.sycamore_circuit(grid, cycles=4, seed=1)
    n = 12
    keep = [g for g in circ.gates if g[0] != si.FSIM or abs(g[1] - g[2]) != 1]  # drop horizontal
    gates = pkg.gates_array(keep)
    cp = pkg.SIM_FP32 if cprec == "fp32" else pkg.SIM_FP16X3_TMEM
    out, s = contracted_front(pkg, n, gates, column_sides(grid, 2), 4, pkg.SIM_FP32, cp)
    try:
        assert pkg.sim_split_info(s)[2] == 0
        got = pkg.sim_amplitudes(out)
    finally:
        pkg.sim_destroy(out)
        pkg.sim_split_destroy(s)
    psi = oracle_mod.basis_state(n, 0)
    for g in keep:
        u = oracle_mod.gate_matrix(g[0], g[3], g[4])
        if g[0] == si.FSIM:
            oracle_mod.apply_2q(psi, g[1], g[2], u)
        else:
            oracle_mod.apply_1q(psi, g[1], u)
    assert err2(got, psi) <= TOL


@pytest.mark.parametrize("cprec", ["fp32", "tmem"])
def test_ragged_and_narrow_sides(pkg, oracle_mod, cprec):
    # sides of 3 and 9 qubits (x tiles ragged for the CUDA-core kernel; too narrow for tcgen05,
    # which then leaves the work to the FP32 kernel), and 7 + 9 (tcgen05's smallest)
    cp = pkg.SIM_FP32 if cprec == "fp32" else pkg.SIM_FP16X3_TMEM
    for shape, cut in (((3, 4), 1), ((4, 4), 2)):
        grid = si.Grid(*shape)
        circ = si.sycamore_circuit(grid, cycles=3, seed=2)
        n = grid.n_qubits
        side = column_sides(grid, cut)
        if shape == (4, 4):
            side = [1 if (r, c) == (0, 1) else sd for sd, (r, c) in zip(side, grid.sites())]
        out, s = contracted_front(pkg, n, pkg.gates_array(circ), side, 4, pkg.SIM_FP32, cp)
        try:
            got = pkg.sim_amplitudes(out)
        finally:
            pkg.sim_destroy(out)
            pkg.sim_split_destroy(s)
        assert err2(got, oracle_mod.run_circuit(circ)) <= TOL, (shape, cut)


def test_contract_rejects_mismatched_handles(pkg):
    grid = si.Grid(3, 4)
    circ = si.sycamore_circuit(grid, cycles=2, seed=0)
    s = pkg.sim_split_create(12, pkg.gates_array(circ), column_sides(grid, 1))  # 3 + 9 qubits
    _, n_wires, _, _ = pkg.sim_split_info(s)
    h1, h2 = pkg.sim_create(n_wires[0]), pkg.sim_create(n_wires[1])
    wrong = pkg.sim_create(11)
    out = pkg.sim_create(12)
    try:
        for args in ((wrong, h1, h2), (out, h2, h1), (out, out, h2), (out, h1, wrong)):
            with pytest.raises(pkg.SimError) as e:
                pkg.sim_contract(*args, s)
            assert e.value.code == pkg.SIM_E_INVAL
        with pytest.raises(pkg.SimError):
            pkg.sim_contract(out, h1, h2, s, pkg.SIM_TF32)
    finally:
        for h in (h1, h2, wrong, out):
            pkg.sim_destroy(h)
        pkg.sim_split_destroy(s)


@pytest.mark.parametrize("cprec", ["fp32", "tmem"])
def test_front_runner_into_permuted_layout(pkg, oracle_mod, cprec):
    # sim_front_run writes psi in out's current layout (here a random permutation, left as it is),
    # the rest of the circuit then runs on it; a second run gives the same bits (deterministic)
    grid = si.Grid(4, 5)
    circ = si.sycamore_circuit(grid, cycles=9, seed=12)
    n = grid.n_qubits
    f = front_length(grid, 6)
    gates = pkg.gates_array(circ)
    prec, kmax = (pkg.SIM_FP32, 4) if cprec == "fp32" else (pkg.SIM_FP16X3_TMEM, 5)
    s = pkg.sim_split_create(n, gates[:f], column_sides(grid, 2))
    out = pkg.sim_create(n)
    perm = [int(x) for x in np.random.default_rng(3).permutation(n)]
    pkg.sim_permute(out, perm)
    fr = pkg.sim_front_create(out, s, kmax=kmax, precision=prec)
    plan = pkg.sim_plan_create(n, gates[f:], kmax=kmax, precision=prec)
    try:
        runs = []
        for _ in range(2):
            pkg.sim_front_run(out, fr)
            pkg.sim_apply_plan(out, plan)
            assert [int(b) for b in pkg.sim_info(out)[2]] == perm
            runs.append(pkg.sim_amplitudes(out))
    finally:
        pkg.sim_plan_destroy(plan)
        pkg.sim_front_destroy(fr)
        pkg.sim_destroy(out)
        pkg.sim_split_destroy(s)
    assert np.array_equal(runs[0], runs[1])
    e = err2(runs[0], oracle_mod.run_circuit(circ))
    print(f"front runner into a permuted layout ({cprec}): ||dpsi|| = {e:.2e}")
    assert e <= TOL
