"""GPU: the reduction fused into a plan's last block.

After sim_apply_plan whose last block runs on tcgen05, sim_reduce combines the per-CTA sums that
block left instead of reading the state again.  Checked against the oracle's FP64 reduction of the
oracle state and against the full reduction of the same device state; a later write (another
block) must make sim_reduce read the state again; handles on a caller's buffer, or whose state
address was handed out, never take the shortcut (the caller could have written the buffer).
"""
import numpy as np
import pytest

import syc_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as p
    return p


@pytest.mark.parametrize("grid,cycles,kmax", [((4, 5), 12, 6), ((4, 6), 10, 5), ((5, 5), 14, 6)])
def test_fused_reduction_matches_oracle_and_full(pkg, oracle_mod, grid, cycles, kmax):
    circ = si.sycamore_circuit(si.Grid(*grid), cycles, seed=sum(grid) + cycles)
    n = circ.n_qubits
    plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=kmax, precision=pkg.SIM_FP16X3_TMEM)
    h = pkg.sim_create(n)
    try:
        perm, _, _ = pkg.sim_plan_layout(plan, n)
        pkg.sim_set_layout(h, perm)
        pkg.sim_reset(h)
        pkg.sim_apply_plan(h, plan)
        n0 = pkg.sim_launch_count(h)
        fused = pkg.sim_reduce(h)
        fused_launches = pkg.sim_launch_count(h) - n0
        pkg.sim_set_layout(h, perm)  # writes nothing, but counts as a write: the next reduce reads the state
        n0 = pkg.sim_launch_count(h)
        full = pkg.sim_reduce(h)
        full_launches = pkg.sim_launch_count(h) - n0
        amps = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    # one combine kernel when the plan's last block ran on tcgen05, the full two-kernel reduction
    # otherwise; a reduction after a write is always the full one
    assert fused_launches in (1, 2) and full_launches == 2
    onorm, os2, oxeb = oracle_mod.reduce(amps)  # the oracle's FP64 sums over the same amplitudes
    for (a, b, c) in (fused, full):
        assert abs(a - onorm) <= 1e-6 * onorm
        assert abs(b - os2) <= 1e-5 * os2
        assert abs(c - oxeb) <= 1e-5 * os2
    assert abs(fused[0] - full[0]) <= 1e-6 and abs(fused[1] - full[1]) <= 1e-5 * full[1]
    # and against the oracle's own run of the circuit
    wnorm, ws2, _ = oracle_mod.reduce(oracle_mod.run_circuit(circ))
    assert abs(fused[0] - wnorm) < 1e-5 and abs(fused[1] - ws2) < 1e-3


def test_later_write_invalidates_fused_sums(pkg, oracle_mod):
    circ = si.sycamore_circuit(si.Grid(4, 5), 10, seed=4)
    n = circ.n_qubits
    plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=6, precision=pkg.SIM_FP16X3_TMEM)
    h = pkg.sim_create(n)
    try:
        pkg.sim_reset(h)
        pkg.sim_apply_plan(h, plan)
        # scale the state by sqrt(2) through a diagonal 1-qubit "gate": the norm becomes 2
        pkg.sim_apply_fused(h, [3], np.sqrt(2.0) * np.eye(2, dtype=np.complex128))
        norm, _, _ = pkg.sim_reduce(h)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    assert abs(norm - 2.0) < 1e-5


def test_caller_buffer_never_takes_the_shortcut(pkg):
    torch = pytest.importorskip("torch")
    circ = si.sycamore_circuit(si.Grid(4, 5), 10, seed=5)
    n = circ.n_qubits
    buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=6, precision=pkg.SIM_FP16X3_TMEM)
    h = pkg.sim_create(n, ext_state=buf.data_ptr(), ext_bytes=buf.numel() * 8)
    try:
        pkg.sim_reset(h)
        pkg.sim_apply_plan(h, plan)
        pkg.sim_sync(h)
        buf.mul_(2.0)  # the caller writes its buffer behind the handle's back
        torch.cuda.synchronize()
        norm, _, _ = pkg.sim_reduce(h)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    assert abs(norm - 4.0) < 1e-4


def test_single_tcgen05_block_plan_takes_the_shortcut(pkg, oracle_mod):
    # every gate inside qubits 12..17: the plan is one 6-qubit block, on tcgen05 (no target below
    # bit 4), so sim_reduce must combine its CTA sums (one kernel)
    n = 20
    rng = np.random.default_rng(3)
    recs = np.zeros(12, dtype=pkg._native.GATE_DTYPE)
    for i in range(12):
        q0, q1 = (int(x) for x in rng.choice(np.arange(12, 18), 2, replace=False))
        recs[i]["kind"], recs[i]["q0"], recs[i]["q1"] = pkg.SIM_GATE_U2, q0, q1
        recs[i]["u"][:32] = si.random_unitary(2, seed=40 + i).view(np.float64).ravel()
    plan = pkg.sim_plan_create(n, recs, kmax=6, precision=pkg.SIM_FP16X3_TMEM)
    psi = si.random_state(n, 11)
    h = pkg.sim_create(n)
    try:
        assert pkg.sim_plan_info(plan)[0] == 1
        pkg.sim_load_amplitudes(h, psi)
        pkg.sim_apply_plan(h, plan)
        n0 = pkg.sim_launch_count(h)
        norm, s2, _ = pkg.sim_reduce(h)
        assert pkg.sim_launch_count(h) - n0 == 1
        amps = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    onorm, os2, _ = oracle_mod.reduce(amps)
    assert abs(norm - onorm) <= 1e-6 * onorm and abs(s2 - os2) <= 1e-5 * os2


def test_reduce_async_matches_sync_and_oracle_when_pipelined(pkg, oracle_mod):
    # two circuits back to back on one handle: the first's reduction is queued, the second circuit
    # is queued behind it (overwriting the state) before the first result is read; each result must
    # be its own circuit's, and equal what sim_reduce returns for the same state
    torch = pytest.importorskip("torch")
    circs = [si.sycamore_circuit(si.Grid(4, 5), 10, seed=21), si.sycamore_circuit(si.Grid(4, 5), 12, seed=22)]
    n = circs[0].n_qubits
    plans = [pkg.sim_plan_create(n, pkg.gates_array(c), kmax=6, precision=pkg.SIM_FP16X3_TMEM) for c in circs]
    outs = [pkg.pinned_array(3, dtype=np.float64) for _ in range(3)]
    h = pkg.sim_create(n)
    try:
        st = torch.cuda.ExternalStream(pkg.sim_stream(h))
        evs = [torch.cuda.Event() for _ in range(2)]
        for i in range(2):
            pkg.sim_reset(h)
            pkg.sim_apply_plan(h, plans[i])
            pkg.sim_reduce_async(h, outs[i])  # the fused combine (last block on tcgen05)
            evs[i].record(st)
        evs[0].synchronize()
        first = [float(x) for x in outs[0][:3]]
        evs[1].synchronize()
        second = [float(x) for x in outs[1][:3]]
        sync2 = pkg.sim_reduce(h)  # the same state, waited for
        pkg.sim_set_layout(h, list(range(n)))  # counts as a write: the full reduction next
        pkg.sim_reduce_async(h, outs[2])
        pkg.sim_sync(h)
        full2 = [float(x) for x in outs[2][:3]]
    finally:
        pkg.sim_destroy(h)
        for p in plans:
            pkg.sim_plan_destroy(p)
        for o in outs:
            pkg.sim_host_free(o.ctypes.data)
    for got, c in ((first, circs[0]), (second, circs[1])):
        onorm, os2, oxeb = oracle_mod.reduce(oracle_mod.run_circuit(c))
        assert abs(got[0] - onorm) < 1e-5 and abs(got[1] - os2) < 1e-3 and abs(got[2] - oxeb) < 1e-3
        assert abs(got[2] - (got[1] - 1.0)) < 1e-12
    assert all(abs(a - b) <= 1e-12 * max(1.0, abs(b)) for a, b in zip(second, sync2))
    assert abs(full2[0] - sync2[0]) < 1e-6 and abs(full2[1] - sync2[1]) < 1e-5


def test_reduce_async_rejects_bad_output(pkg):
    h = pkg.sim_create(12)
    try:
        with pytest.raises(ValueError):
            pkg.sim_reduce_async(h, np.zeros(2, dtype=np.float64))
        assert pkg.lib().sim_reduce_async(h, None) == pkg.SIM_E_INVAL
        assert pkg.lib().sim_reduce_async(None, None) == pkg.SIM_E_INVAL
    finally:
        pkg.sim_destroy(h)
    store = pkg.sim_create(12, 1, store=pkg.SIM_STORE_HOST, set_a=[0], set_b=[11], slots=2)
    try:
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_reduce_async(store, pkg.pinned_array(3, dtype=np.float64))
        assert e.value.code == pkg.SIM_E_UNSUPPORTED
    finally:
        pkg.sim_destroy(store)
