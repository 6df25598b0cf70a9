"""GPU: secondary storage (Sect. 4) -- host store, slice streaming and phases.

Slice moves are pure data movement and must be bit-exact; a streamed run must equal the
device-resident run of the same phases bit for bit (same blocks, same kernels, same order),
and match the oracle within the FP32 tolerance.
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


def expected_slice(oracle_mod, psi, n, sliced, other, value):
    """Slot content for `sliced` = value: the oracle's gather (remaining qubits ascending),
    reordered to the slot layout [rest ascending | other set in order]."""
    sl = oracle_mod.gather_slice(psi, sliced, value)
    remaining = sorted(q for q in range(n) if q not in sliced)
    rest = sorted(q for q in remaining if q not in other)
    layout = rest + list(other)
    perm = [layout.index(q) for q in remaining]
    return oracle_mod.permute(sl, perm)


@pytest.mark.parametrize("n,s,set_a,set_b,slots,dev_regions", [
    (10, 2, [3, 8], [0, 6], 2, 0), (14, 3, [13, 1, 7], [4, 11, 2], 3, 0), (12, 1, [11], [10], 4, 0),
    # hybrid stores: the top regions (values of set A) in device memory, up to all of them
    (10, 2, [3, 8], [0, 6], 2, 1), (14, 3, [13, 1, 7], [4, 11, 2], 3, 5), (12, 1, [11], [10], 4, 2)])
def test_slice_streaming_bit_exact(pkg, oracle_mod, n, s, set_a, set_b, slots, dev_regions):
    psi = si.random_state(n, n)
    h = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=slots,
                       store_device_regions=dev_regions)
    try:
        pkg.sim_load_amplitudes(h, psi)
        assert np.array_equal(pkg.sim_amplitudes(h).view(np.uint64), psi.view(np.uint64))
        for which, (sliced, other) in enumerate(((set_a, set_b), (set_b, set_a))):
            for v in range(1 << s):
                slot = v % slots
                pkg.sim_stream_slice(h, which, v, pkg.SIM_H2D, slot)
                got = pkg.sim_slot_read(h, slot)
                want = expected_slice(oracle_mod, psi, n, sliced, other, v)
                assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (which, v)
                pkg.sim_stream_slice(h, which, v, pkg.SIM_D2H, slot)  # write back unchanged
        pkg.sim_sync(h)
        assert np.array_equal(pkg.sim_amplitudes(h).view(np.uint64), psi.view(np.uint64))
        norm, s2, _ = pkg.sim_reduce(h)
        onorm, os2, _ = oracle_mod.reduce(psi.astype(np.complex128))
        assert abs(norm - onorm) < 1e-6 and abs(s2 - os2) < 1e-5 * os2
    finally:
        pkg.sim_destroy(h)


@pytest.mark.parametrize("grid,cycles,s,dev_regions", [((4, 4), 10, 2, 0), ((4, 6), 12, 3, 0), ((4, 6), 12, 3, 5)])
def test_streamed_phases_equal_resident_bit_exact(pkg, oracle_mod, grid, cycles, s, dev_regions):
    # Streaming only moves data: with the resident state stored in the host store's bit
    # layout, every block sees the same target order, matrix and kernel, so the two runs agree
    # bit for bit.
    circ = si.sycamore_circuit(si.Grid(*grid), cycles=cycles, seed=9)
    n = circ.n_qubits
    set_a, set_b = list(range(s)), list(range(n - s, n))  # the two ends of the lattice
    ph = pkg.sim_phases_create(n, pkg.gates_array(circ), s, set_a, set_b, kmax=4)
    hr = pkg.sim_create(n)
    hh = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b,
                        store_device_regions=dev_regions)
    try:
        assert pkg.sim_phases_info(ph)[0] >= 2
        pkg.sim_permute(hr, list(pkg.sim_info(hh)[2]))
        pkg.sim_run_phases(hr, ph)
        pkg.sim_run_phases(hh, ph)
        pkg.sim_sync(hh)
        a = pkg.sim_amplitudes(hr)
        b = pkg.sim_amplitudes(hh)
    finally:
        pkg.sim_destroy(hr)
        pkg.sim_destroy(hh)
        pkg.sim_phases_destroy(ph)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    want = oracle_mod.run_circuit(circ)
    assert np.linalg.norm(b.astype(np.complex128) - want) <= TOL_FP32


def test_streamed_phases_scrambled_sets_match_oracle(pkg, oracle_mod):
    circ = si.sycamore_circuit(si.Grid(4, 5), cycles=12, seed=2)
    n, s = circ.n_qubits, 2
    set_a, set_b = [0, 1], [18, 19]  # the two ends of the lattice
    ph = pkg.sim_phases_create(n, pkg.gates_array(circ), s, set_a, set_b, kmax=5)
    h = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=2)
    try:
        pkg.sim_run_phases(h, ph)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_phases_destroy(ph)
    assert np.linalg.norm(got - oracle_mod.run_circuit(circ)) <= TOL_FP32


def test_hybrid_store_tensor_core_phases_match_oracle(pkg, oracle_mod):
    # the default arithmetic through a hybrid store: 3 of 8 regions on the device
    circ = si.sycamore_circuit(si.Grid(4, 6), cycles=14, seed=4)
    n, s = circ.n_qubits, 3
    set_a, set_b = [0, 1, 2], [21, 22, 23]
    ph = pkg.sim_phases_create(n, pkg.gates_array(circ), s, set_a, set_b, kmax=5, precision=pkg.SIM_FP16X3_TMEM)
    h = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=3, store_device_regions=3)
    try:
        pkg.sim_run_phases(h, ph)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
        norm, s2, _ = pkg.sim_reduce(h)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_phases_destroy(ph)
    want = oracle_mod.run_circuit(circ)
    assert np.linalg.norm(got - want) <= TOL_FP32
    assert abs(norm - 1.0) < 1e-5


def test_chosen_sets_stream_to_the_oracle(pkg, oracle_mod):
    # sets picked by sim_phases_choose_sets, streamed through a host store
    circ = si.sycamore_circuit(si.Grid(4, 5), cycles=14, seed=8)
    n, s = circ.n_qubits, 2
    set_a, set_b, nph, nbl = pkg.sim_phases_choose_sets(n, pkg.gates_array(circ), s, kmax=5)
    ph = pkg.sim_phases_create(n, pkg.gates_array(circ), s, set_a, set_b, kmax=5, precision=pkg.SIM_FP16X3_TMEM)
    assert pkg.sim_phases_info(ph) == (nph, nbl)
    h = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=3)
    try:
        pkg.sim_run_phases(h, ph)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_phases_destroy(ph)
    assert np.linalg.norm(got - oracle_mod.run_circuit(circ)) <= TOL_FP32


def test_host_store_rejects_sliced_targets_and_device_calls(pkg):
    n, s = 10, 2
    h = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=[0, 1], set_b=[8, 9])
    recs = pkg.gates_array([(si.FSIM, 0, 2, 1.0, 0.5)])
    plan = pkg.sim_plan_create(n, recs)
    try:
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_run_phase(h, 0, plan)  # qubit 0 is in set A
        assert e.value.code == pkg.SIM_E_NONLOCAL
        pkg.sim_run_phase(h, 1, plan)      # fine with set B sliced
        for call in (lambda: pkg.sim_apply_fused(h, [2], np.eye(2)), lambda: pkg.sim_permute(h, list(range(n))),
                     lambda: pkg.sim_apply_plan(h, plan)):
            with pytest.raises(pkg.SimError) as e:
                call()
            assert e.value.code == pkg.SIM_E_UNSUPPORTED
        with pytest.raises(pkg.SimError):
            pkg.sim_stream_slice(h, 0, 4, pkg.SIM_H2D, 0)
    finally:
        pkg.sim_plan_destroy(plan)
        pkg.sim_destroy(h)
    with pytest.raises(pkg.SimError):
        pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=[0, 1], set_b=[1, 9])


@pytest.mark.parametrize("slots", [2, 3, 4])
def test_phase_boundaries_order_copies(pkg, oracle_mod, slots):
    # Every slice of one set meets every slice of the other, so a phase must not read a file
    # before the previous phase has written it back.  Many slices per slot stress the ordering.
    circ = si.sycamore_circuit(si.Grid(4, 6), cycles=14, seed=4)
    n, s = circ.n_qubits, 4
    set_a, set_b = [0, 1, 2, 3], [20, 21, 22, 23]
    ph = pkg.sim_phases_create(n, pkg.gates_array(circ), s, set_a, set_b, kmax=4)
    h = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=slots)
    try:
        assert pkg.sim_phases_info(ph)[0] >= 3
        pkg.sim_run_phases(h, ph)
        norm, _, _ = pkg.sim_reduce(h)
        got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_phases_destroy(ph)
    assert abs(norm - 1.0) < 1e-5
    assert np.linalg.norm(got - oracle_mod.run_circuit(circ)) <= TOL_FP32


@pytest.mark.parametrize("physical", [False, True])
def test_hybrid_store_load_and_readout_in_chunks(pkg, oracle_mod, physical):
    # 26 qubits, 4 regions of 2^24 amplitudes, 2 of them in HBM, relabelled: a load and a readout
    # of all 2^26 amplitudes (four staging chunks; the device regions' entries go through the
    # device, the host regions' in place) and of a ragged range across the regions' boundary are
    # bit-exact, in logical and in physical order
    n, s = 26, 2
    h = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=[3, 17], set_b=[8, 21], slots=2,
                       store_device_regions=2)
    try:
        bits = [int(x) for x in pkg.sim_info(h)[2]]
        others = sorted(range(n), key=lambda q: bits[q])[:n - 2 * s]
        perm = list(bits)
        for q, b in zip(others, reversed(sorted(bits[q] for q in others))):
            perm[q] = b  # the other qubits' order reversed: a relabelling the store allows
        pkg.sim_set_layout(h, perm)
        rng = np.random.default_rng(5)
        psi = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(np.complex64)
        pkg.sim_load_amplitudes(h, psi, physical_order=physical)
        back = pkg.sim_amplitudes(h, dtype=pkg.SIM_C64, physical_order=physical)
        assert np.array_equal(back.view(np.uint64), psi.view(np.uint64))
        first, count = (1 << 25) - 12345, (1 << 24) + 777  # straddles the host / device boundary
        part = pkg.sim_amplitudes(h, first, count, dtype=pkg.SIM_C64, physical_order=physical)
        assert np.array_equal(part.view(np.uint64), psi[first:first + count].view(np.uint64))
        patch = (rng.standard_normal(count) + 1j * rng.standard_normal(count)).astype(np.complex64)
        pkg.sim_load_amplitudes(h, patch, first=first, physical_order=physical)
        psi[first:first + count] = patch
        back = pkg.sim_amplitudes(h, dtype=pkg.SIM_C64, physical_order=physical)
        assert np.array_equal(back.view(np.uint64), psi.view(np.uint64))
    finally:
        pkg.sim_destroy(h)
