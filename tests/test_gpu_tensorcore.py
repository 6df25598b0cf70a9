"""GPU: tensor-core apply (SIM_TF32, SIM_TF32X3, SIM_FP16X3, SIM_FP16X3_TMEM, SIM_BF16X3) against
the oracle.

Tolerances (unit-norm states): 3xTF32 and 3xFP16 (per-tile power-of-two scale) recover ~21-22
mantissa bits, so they are held to the FP32 bound 1e-5; plain TF32 keeps 10 mantissa bits (2^-11 ~
4.9e-4 relative per rounded input), and a single pass is held to 5e-3, a whole 12-qubit circuit to
3e-2.  BF16x3 splits each FP32 operand into two BF16 pieces of 8 significant bits: hi + lo keeps
~16 bits (2^-16 ~ 1.5e-5 relative at worst, rounding errors of random sign average down) and the
dropped lo*lo product is of the same order; measured on GB300 4.4-4.6e-6 per pass on unit-norm
random states and 1.4-1.7e-5 on a 20-qubit circuit, so a single pass is held to 2e-5 and a whole
circuit to 1e-4.  The measured errors are printed so that the per-result bound can be quoted.
"""
import numpy as np
import pytest

import syc_inputs as si

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "fp16x3": 1e-5, "fp16x3_tmem": 1e-5, "tf32": 5e-3, "bf16x3": 2e-5}


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as p
    return p


def mode(pkg, name):
    return {"fp32": pkg.SIM_FP32, "tf32": pkg.SIM_TF32, "tf32x3": pkg.SIM_TF32X3, "fp16x3": pkg.SIM_FP16X3,
            "fp16x3_tmem": pkg.SIM_FP16X3_TMEM, "bf16x3": pkg.SIM_BF16X3}[name]


@pytest.mark.parametrize("name", ["tf32x3", "fp16x3", "fp16x3_tmem", "tf32", "bf16x3"])
@pytest.mark.parametrize("n,targets", [(14, [6, 13, 9, 4, 10]), (20, [19, 5, 12, 8, 16]), (16, [4, 5, 6, 7, 8, 9]),
                                       (21, [20, 6, 14, 9, 17, 11]), (12, [0, 1, 2, 3, 4]), (15, [3, 0, 9, 1, 14]),
                                       (18, [0, 1, 2, 3, 4, 5]), (17, [16, 2, 8, 0, 11, 5]), (9, [0, 2, 4, 6, 8]),
                                       (16, [0, 7, 9, 12])])  # last: k = 4 -> FP32 CUDA cores
def test_tensor_core_apply_matches_oracle(pkg, oracle_mod, name, n, targets):
    k = len(targets)
    u = si.random_unitary(k, seed=7 * n + k)
    psi = si.random_state(n, seed=n)
    h = pkg.sim_create(n)
    try:
        pkg.sim_load_amplitudes(h, psi)
        pkg.sim_apply_fused(h, targets, u, precision=mode(pkg, name))
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
    want = psi.astype(np.complex128)
    oracle_mod.apply_kq(want, targets, u)
    err = np.linalg.norm(got - want)
    print(f"{name} n={n} k={k} err={err:.3e}")
    # k = 4: CUDA cores in the mma.sync modes; the tcgen05 modes take it when no target is below
    # bit 4 (then BF16x3 arithmetic)
    narrow = k < 5 and not (name == "bf16x3" and min(targets) >= 4 and n >= k + 7)
    assert err <= (TOL["fp32"] if narrow else TOL[name]), err


@pytest.mark.parametrize("name,kmax,tol", [("tf32x3", 5, 1e-5), ("tf32x3", 6, 1e-5), ("fp16x3", 5, 1e-5),
                                          ("fp16x3", 6, 1e-5), ("fp16x3_tmem", 5, 1e-5), ("fp16x3_tmem", 6, 1e-5),
                                          ("tf32", 5, 3e-2), ("bf16x3", 5, 1e-4), ("bf16x3", 6, 1e-4)])
def test_tensor_core_circuit_matches_oracle(pkg, oracle_mod, name, kmax, tol):
    circ = si.sycamore_circuit(si.Grid(4, 5), cycles=14, seed=8)
    plan = pkg.sim_plan_create(circ.n_qubits, pkg.gates_array(circ), kmax=kmax, precision=mode(pkg, name))
    h = pkg.sim_create(circ.n_qubits)
    try:
        pkg.sim_apply_plan(h, plan)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    err = np.linalg.norm(got - oracle_mod.run_circuit(circ))
    print(f"{name} kmax={kmax} 20-qubit circuit err={err:.3e}")
    assert err <= tol, err


def test_fp16x3_tiny_and_zero_amplitudes(pkg, oracle_mod):
    # the per-tile scale must keep tiles of tiny amplitudes accurate and leave zero tiles at zero
    n = 14
    psi = si.random_state(n, 3)
    psi[: 1 << 12] *= np.float32(1e-20)   # a whole region of tiny amplitudes
    psi[1 << 13: (1 << 13) + (1 << 11)] = 0
    u = si.random_unitary(5, 4)
    h = pkg.sim_create(n)
    try:
        pkg.sim_load_amplitudes(h, psi)
        pkg.sim_apply_fused(h, [4, 6, 8, 10, 12], u, precision=pkg.SIM_FP16X3)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
    want = psi.astype(np.complex128)
    oracle_mod.apply_kq(want, [4, 6, 8, 10, 12], u)
    assert np.linalg.norm(got - want) <= 1e-5
    tiny = np.abs(want) < 1e-15
    assert np.all(np.abs(got[tiny] - want[tiny]) <= 1e-5 * np.abs(want[tiny]) + 1e-30)


@pytest.mark.parametrize("n,targets", [
    # tcgen05 path (no target below bit 4).  128-group tiles (bit 7 a target or inside the run):
    (12, [4, 5, 6, 7]), (22, [21, 5, 13, 8, 17]), (16, [15, 8, 4, 11]), (20, [4, 5, 6, 7, 8]),
    (21, [5, 9, 10, 15, 20]), (24, [23, 6, 11, 7, 16]),
    # 256-group tiles (two M = 128 sub-tiles; bit 7 becomes a row bit), one tile at 13 qubits; at
    # 24 and 25 qubits every CTA takes many tiles, so the stage ring and both TMEM sets wrap
    (25, [9, 10, 11, 12]), (20, [12, 13, 14, 15, 16]), (13, [8, 9, 10, 11, 12]), (19, [8, 10, 12, 14]),
    # k = 5 with one target below bit 4: rows read through the per-row member XOR, results
    # stored from registers
    (24, [23, 2, 11, 7, 16]), (20, [3, 4, 5, 7, 8]),
    # more targets below bit 4 (k = 5), or any (k = 4): the same mode runs on the mma.sync 3xFP16
    # kernel; one tile at 11 qubits
    (19, [1, 6, 7, 12]),
    (13, [0, 12, 3, 7, 9]), (23, [0, 1, 2, 3, 4]), (22, [0, 2, 4, 6]), (11, [0, 1, 2, 3]),
    (21, [1, 2, 3, 12, 13]),
    # k = 6 (128-group tiles, 2-stage ring, results drained 16 columns at a time): one tile at
    # 13 qubits; all targets above bit 7 (1 KiB runs); mixed; targets from bit 4 up; many tiles
    # per CTA at 24-25 qubits
    (13, [7, 8, 9, 10, 11, 12]), (24, [23, 16, 12, 10, 9, 8]), (22, [21, 5, 13, 8, 17, 10]),
    (20, [4, 5, 6, 7, 8, 9]), (25, [4, 9, 14, 19, 22, 24]),
    # k = 6 with one target below bit 4 (per-row member XOR), and with two (mma.sync 3xFP16)
    (22, [2, 8, 11, 15, 19, 21]), (20, [3, 4, 5, 7, 8, 9]), (25, [0, 9, 13, 17, 21, 24]),
    (19, [2, 3, 9, 11, 14, 18])])
@pytest.mark.parametrize("name", ["fp16x3_tmem", "bf16x3"])
def test_tcgen05_tiles_match_oracle(pkg, oracle_mod, n, targets, name):
    # the tcgen05 path takes k = 4, 5 or 6 and >= 2^(k+7) amplitudes (one 128-group tile); the
    # BF16x3 mode runs the same tiles with BF16 pieces (what tcgen05 leaves: 3xFP16 on mma.sync)
    k = len(targets)
    u = si.random_unitary(k, seed=n + 3 * k)
    psi = si.random_state(n, seed=2 * n)
    h = pkg.sim_create(n)
    try:
        pkg.sim_load_amplitudes(h, psi)
        pkg.sim_apply_fused(h, targets, u, precision=mode(pkg, name))
        pkg.sim_sync(h)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
    want = psi.astype(np.complex128)
    oracle_mod.apply_kq(want, targets, u)
    err = np.linalg.norm(got - want)
    print(f"tcgen05 {name} n={n} targets={targets}: err {err:.3e}")
    assert err <= TOL[name], err


@pytest.mark.parametrize("accuracy", ["fp32", "fp32_equivalent", "any"])
def test_autotune_picks_a_valid_plan(pkg, oracle_mod, accuracy):
    circ = si.sycamore_circuit(si.Grid(4, 5), cycles=10, seed=12)
    acc = {"fp32": pkg.SIM_TUNE_FP32, "fp32_equivalent": pkg.SIM_TUNE_FP32_EQUIVALENT,
           "any": pkg.SIM_TUNE_ANY}[accuracy]
    h = pkg.sim_create(circ.n_qubits)
    try:
        kmax, prec, ms = pkg.sim_autotune(h, pkg.gates_array(circ), acc)
        assert 3 <= kmax <= 6 and ms > 0
        fp32_class = (pkg.SIM_FP32, pkg.SIM_FP16X3, pkg.SIM_FP16X3_TMEM, pkg.SIM_TF32X3)
        if accuracy == "fp32":
            assert prec == pkg.SIM_FP32
        elif accuracy == "fp32_equivalent":
            assert prec in fp32_class
        else:  # the stated-bound modes join the candidates
            assert prec in fp32_class + (pkg.SIM_TF32, pkg.SIM_BF16X3)
        assert pkg.sim_amplitudes(h, count=2)[0] == 1  # left in |0...0>
        plan = pkg.sim_plan_create(circ.n_qubits, pkg.gates_array(circ), kmax=kmax, precision=prec)
        pkg.sim_apply_plan(h, plan)
        pkg.sim_plan_destroy(plan)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
    bound = {pkg.SIM_TF32: 3e-2, pkg.SIM_BF16X3: 1e-4}.get(prec, 1e-5)
    assert np.linalg.norm(got - oracle_mod.run_circuit(circ)) <= bound


@pytest.mark.parametrize("name,kmax", [("fp16x3_tmem", 6), ("fp16x3_tmem", 5), ("fp32", 4), ("bf16x3", 6)])
def test_chosen_layout_runs_the_same_circuit(pkg, oracle_mod, name, kmax):
    # sim_plan_layout picks where the qubits sit; sim_set_layout relabels without moving data, so
    # it goes before the reset; the plan then runs in that layout and reads out in logical order
    circ = si.sycamore_circuit(si.Grid(4, 5), cycles=14, seed=8)
    n = circ.n_qubits
    plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=kmax, precision=mode(pkg, name))
    perm, est, est_identity = pkg.sim_plan_layout(plan, n)
    assert sorted(perm) == list(range(n)) and est <= est_identity
    h = pkg.sim_create(n)
    try:
        pkg.sim_set_layout(h, perm)
        pkg.sim_reset(h)
        pkg.sim_apply_plan(h, plan)
        assert [int(b) for b in pkg.sim_info(h)[2]] == perm
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
        pkg.sim_permute(h, list(range(n)))  # back to the identity: the same state, bit for bit
        again = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    assert np.array_equal(got, again)
    err = np.linalg.norm(got - oracle_mod.run_circuit(circ))
    print(f"{name} kmax {kmax}, chosen layout (estimate {est:.1f} vs {est_identity:.1f}): err {err:.2e}")
    assert err <= (1e-4 if name == "bf16x3" else 1e-5)
