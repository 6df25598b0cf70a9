"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerances: the FP32 gate path must satisfy ||psi - psi_oracle||_2 <= 1e-5 for a unit-norm
state (one FP32 pass rounds each output of a 2^k-term sum: relative error <~ 2^k * 2^-24 per
pass); permutations, slice moves, loads and readouts are pure data movement and must be
bit-exact.
"""
import numpy as np
import pytest

import syc_inputs as si

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as p
    return p


def load_state(pkg, n, seed, slice_bits=0):
    psi = si.random_state(n, seed)
    h = pkg.sim_create(n, slice_bits)
    pkg.sim_load_amplitudes(h, psi)
    return h, psi


APPLY_CASES = [
    # (n, targets) -- low (< 5), high, mixed, ragged small states, top bits
    (1, [0]), (2, [1]), (2, [0, 1]), (3, [2, 0, 1]), (6, [5, 0, 3, 1, 2, 4]),
    (10, [0]), (10, [9]), (10, [4, 5]), (12, [3, 11, 0]), (12, [7, 2, 9, 4]),
    (14, [0, 1, 2, 3]), (14, [10, 11, 12, 13]), (14, [13, 0, 6, 2, 9]),
    (16, [5, 8, 15]), (16, [6, 7, 8, 9, 10]), (16, [0, 1, 2, 3, 4]), (16, [15, 4, 0, 12, 3, 8]),
    (18, [17, 16, 15, 14, 13, 12]), (18, [0, 1, 2, 3, 4, 5]), (20, [5, 19]), (20, [4, 18, 1, 11]),
    (20, [2, 19, 7, 13, 0, 16]), (21, [6, 9, 12, 20, 8]),
]


@pytest.mark.parametrize("n,targets", APPLY_CASES)
def test_apply_fused_matches_oracle(pkg, oracle_mod, n, targets):
    k = len(targets)
    u = si.random_unitary(k, seed=n * 100 + sum(targets))
    h, psi = load_state(pkg, n, seed=n + k)
    try:
        pkg.sim_apply_fused(h, targets, u)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
    want = psi.astype(np.complex128)
    oracle_mod.apply_kq(want, targets, u)
    err = np.linalg.norm(got - want)
    assert err <= TOL_FP32, err


@pytest.mark.parametrize("kmax", [2, 3, 4, 5, 6])
def test_circuit_12q_matches_oracle(pkg, oracle_mod, kmax):
    circ = si.workload_circuit("syc12_3x4_d8", seed=kmax)
    plan = pkg.sim_plan_create(circ.n_qubits, pkg.gates_array(circ), kmax=kmax)
    h = pkg.sim_create(circ.n_qubits)
    try:
        pkg.sim_apply_plan(h, plan)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
        norm, s2, xeb = pkg.sim_reduce(h)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    want = oracle_mod.run_circuit(circ)
    assert np.linalg.norm(got - want) <= TOL_FP32
    onorm, os2, _ = oracle_mod.reduce(want)
    assert abs(norm - 1.0) < 1e-5 and abs(s2 - os2) < 1e-4 * os2


def test_circuit_20q_deep_matches_oracle(pkg, oracle_mod):
    circ = si.sycamore_circuit(si.Grid(4, 5), cycles=14, seed=3)
    plan = pkg.sim_plan_create(circ.n_qubits, pkg.gates_array(circ), kmax=5)
    h = pkg.sim_create(circ.n_qubits)
    try:
        pkg.sim_apply_plan(h, plan)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    want = oracle_mod.run_circuit(circ)
    assert np.linalg.norm(got - want) <= TOL_FP32


@pytest.mark.parametrize("n,seed", [(3, 0), (9, 1), (14, 2), (20, 3), (22, 4)])
def test_permute_bit_exact(pkg, oracle_mod, n, seed):
    perm = si.random_permutation(n, seed)
    h, psi = load_state(pkg, n, seed)
    try:
        pkg.sim_permute(h, perm)
        phys = pkg.sim_amplitudes(h, physical_order=True)
        logical = pkg.sim_amplitudes(h)
        _, _, bit_of = pkg.sim_info(h)
    finally:
        pkg.sim_destroy(h)
    assert list(bit_of) == perm
    want = oracle_mod.permute(psi, perm)
    assert np.array_equal(phys.view(np.uint64), want.view(np.uint64))
    assert np.array_equal(logical.view(np.uint64), psi.view(np.uint64))


@pytest.mark.parametrize("perm_kind", ["swap_high", "swap_low_high", "low_only", "cycle_all", "reverse"])
def test_permute_structured_bit_exact(pkg, oracle_mod, perm_kind):
    n = 18
    perm = list(range(n))
    if perm_kind == "swap_high":      # the slice-phase exchange: top 3 bits <-> 3 middle bits
        for a, b in ((15, 8), (16, 9), (17, 10)):
            perm[a], perm[b] = b, a
    elif perm_kind == "swap_low_high":
        for a, b in ((0, 17), (2, 12), (4, 6)):
            perm[a], perm[b] = b, a
    elif perm_kind == "low_only":
        perm[:5] = [3, 0, 4, 1, 2]
    elif perm_kind == "cycle_all":
        perm = [(q + 1) % n for q in range(n)]
    else:
        perm = perm[::-1]
    h, psi = load_state(pkg, n, 7)
    try:
        pkg.sim_permute(h, perm)
        phys = pkg.sim_amplitudes(h, physical_order=True)
        # a second permutation composes with the first
        pkg.sim_permute(h, list(range(n)))
        back = pkg.sim_amplitudes(h, physical_order=True)
    finally:
        pkg.sim_destroy(h)
    assert np.array_equal(phys.view(np.uint64), oracle_mod.permute(psi, perm).view(np.uint64))
    assert np.array_equal(back.view(np.uint64), psi.view(np.uint64))


def test_gates_follow_layout_after_permute(pkg, oracle_mod):
    n = 16
    perm = si.random_permutation(n, 11)
    u = si.random_unitary(4, 5)
    targets = [0, 7, 15, 3]
    h, psi = load_state(pkg, n, 2)
    try:
        pkg.sim_permute(h, perm)
        pkg.sim_apply_fused(h, targets, u)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
    want = psi.astype(np.complex128)
    oracle_mod.apply_kq(want, targets, u)
    assert np.linalg.norm(got - want) <= TOL_FP32


def test_sliced_qubits_are_not_local(pkg, oracle_mod):
    # Sect. 4: gates apply to local qubits only; a reorganisation makes sliced qubits local.
    n, s = 14, 3
    h, psi = load_state(pkg, n, 1, slice_bits=s)
    u = si.random_unitary(2, 0)
    try:
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_apply_fused(h, [12, 2], u)
        assert e.value.code == pkg.SIM_E_NONLOCAL
        perm = list(range(n))
        for a, b in ((11, 5), (12, 6), (13, 7)):
            perm[a], perm[b] = b, a
        pkg.sim_permute(h, perm)
        pkg.sim_apply_fused(h, [12, 2], u)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
    want = psi.astype(np.complex128)
    oracle_mod.apply_kq(want, [12, 2], u)
    assert np.linalg.norm(got - want) <= TOL_FP32


@pytest.mark.parametrize("n", [1, 5, 12, 21])
def test_reduce_matches_oracle(pkg, oracle_mod, n):
    h, psi = load_state(pkg, n, n)
    try:
        norm, s2, xeb = pkg.sim_reduce(h)
        norm2, _, _ = pkg.sim_reduce(h)
    finally:
        pkg.sim_destroy(h)
    onorm, os2, oxeb = oracle_mod.reduce(psi.astype(np.complex128))
    assert norm == norm2  # deterministic
    assert abs(norm - onorm) <= 1e-6 * onorm
    assert abs(s2 - os2) <= 1e-5 * os2
    assert abs(xeb - oxeb) <= 1e-5 * os2


@pytest.mark.parametrize("n,basis", [(1, 1), (7, 0), (7, 93), (16, 40000)])
def test_reset_basis_exact(pkg, n, basis):
    h = pkg.sim_create(n)
    try:
        pkg.sim_reset(h, basis)
        a = pkg.sim_amplitudes(h)
        perm = list(reversed(range(n)))
        pkg.sim_permute(h, perm)
        pkg.sim_reset(h, basis)
        b = pkg.sim_amplitudes(h)
    finally:
        pkg.sim_destroy(h)
    want = np.zeros(1 << n, dtype=np.complex64)
    want[basis] = 1
    assert np.array_equal(a, want) and np.array_equal(b, want)


def test_load_readout_roundtrip_bit_exact(pkg):
    n = 15
    psi = si.random_state(n, 3)
    h = pkg.sim_create(n)
    try:
        pkg.sim_permute(h, si.random_permutation(n, 3))
        pkg.sim_load_amplitudes(h, psi)  # logical order under a non-identity layout
        out = pkg.sim_amplitudes(h)
        part = pkg.sim_amplitudes(h, first=1000, count=777)
        part128 = pkg.sim_amplitudes(h, first=5, count=9, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
    assert np.array_equal(out.view(np.uint64), psi.view(np.uint64))
    assert np.array_equal(part, psi[1000:1777])
    assert np.array_equal(part128, psi[5:14].astype(np.complex128))


def test_async_readout_bit_exact_and_overlapping(pkg):
    # two handles: the readout of one is enqueued while the other is being computed
    n = 18
    psi = si.random_state(n, 11)
    ha, hb = pkg.sim_create(n), pkg.sim_create(n)
    outs = [pkg.pinned_array(1 << n), pkg.pinned_array(1 << n)]
    part = pkg.pinned_array(300)
    try:
        pkg.sim_load_amplitudes(ha, psi)
        pkg.sim_amplitudes_async(ha, outs[0])
        pkg.sim_amplitudes_async(ha, part, first=4000)
        pkg.sim_reset(hb)
        circ = si.sycamore_circuit(si.Grid(3, 6), cycles=6, seed=3)
        plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=5, precision=pkg.SIM_FP16X3_TMEM)
        pkg.sim_apply_plan(hb, plan)
        pkg.sim_plan_destroy(plan)
        pkg.sim_amplitudes_async(hb, outs[1])
        pkg.sim_sync(ha)
        assert np.array_equal(outs[0].view(np.uint64), psi.view(np.uint64))
        assert np.array_equal(part, psi[4000:4300])
        pkg.sim_sync(hb)
        assert np.array_equal(outs[1].view(np.uint64), pkg.sim_amplitudes(hb).view(np.uint64))
        # logical order of a permuted layout is refused; physical order is fine
        perm = si.random_permutation(n, 5)
        pkg.sim_permute(ha, perm)
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_amplitudes_async(ha, outs[0])
        assert e.value.code == pkg.SIM_E_UNSUPPORTED
        pkg.sim_amplitudes_async(ha, outs[0], physical_order=True)
        pkg.sim_sync(ha)
        assert np.array_equal(outs[0].view(np.uint64), pkg.sim_amplitudes(ha, physical_order=True).view(np.uint64))
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_amplitudes_async(ha, part, first=(1 << n) - 10)
        assert e.value.code == pkg.SIM_E_INVAL
    finally:
        pkg.sim_destroy(ha)
        pkg.sim_destroy(hb)
        for a in outs + [part]:
            pkg.sim_host_free(a.ctypes.data)


def test_argument_errors(pkg):
    h = pkg.sim_create(8)
    try:
        for targets, code in (([1, 1], pkg.SIM_E_INVAL), ([8], pkg.SIM_E_INVAL), ([-1], pkg.SIM_E_INVAL)):
            with pytest.raises(pkg.SimError) as e:
                pkg.sim_apply_fused(h, targets, np.eye(1 << len(targets)))
            assert e.value.code == code
        with pytest.raises(pkg.SimError):
            pkg.sim_permute(h, [0, 1, 2, 3, 4, 5, 6, 6])
        with pytest.raises(pkg.SimError):
            pkg.sim_reset(h, 256)
        with pytest.raises(pkg.SimError):
            pkg.sim_apply_fused(h, [0], np.eye(2), precision=99)
        pkg.sim_sync(h, 1000)
    finally:
        pkg.sim_destroy(h)


def test_external_torch_buffer_and_stream(pkg, oracle_mod):
    torch = pytest.importorskip("torch")
    n = 12
    buf = torch.zeros(2 << n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    h = pkg.sim_create(n, 0, stream=stream.cuda_stream, ext_state=buf.data_ptr(),
                       ext_bytes=buf.numel() * 4)
    try:
        u = si.random_unitary(3, 1)
        pkg.sim_apply_fused(h, [0, 5, 11], u)
        pkg.sim_sync(h)
        got = buf.cpu().numpy().view(np.complex64).astype(np.complex128)
    finally:
        pkg.sim_destroy(h)
    want = oracle_mod.basis_state(n, 0)
    oracle_mod.apply_kq(want, [0, 5, 11], u)
    assert np.linalg.norm(got - want) <= TOL_FP32
