"""GPU: the continuous-batching server (srv_*).

Each served result is checked against the oracle; a circuit served alone and served in a mix
of others must give bit-identical amplitudes (same path, plan and kernels); admission must keep
the device footprint under the HBM budget; waits are bounded.
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


def mixed_circuits():
    # packed (n <= 14 with small_n = 14) and stream-path circuits of several depths
    out = []
    for i, (n, d) in enumerate([(10, 8), (12, 12), (14, 10), (15, 9), (17, 14), (11, 20), (16, 8), (13, 16),
                                (18, 10), (14, 8)]):
        out.append(si.sycamore_circuit(si.near_square_grid(n), d, seed=100 + i))
    return out


def serve(pkg, circuits, together, **opts):
    srv = pkg.srv_create(**opts)
    outs = [np.zeros(1 << c.n_qubits, dtype=np.complex64) for c in circuits]
    res = [None] * len(circuits)
    try:
        if together:
            tickets = [pkg.srv_submit(srv, c.n_qubits, pkg.gates_array(c), o) for c, o in zip(circuits, outs)]
            for i, t in enumerate(tickets):
                res[i] = pkg.srv_wait(srv, t, timeout_ms=60000)
        else:
            for i, (c, o) in enumerate(zip(circuits, outs)):
                res[i] = pkg.srv_wait(srv, pkg.srv_submit(srv, c.n_qubits, pkg.gates_array(c), o), 60000)
        stats = pkg.srv_stats(srv)
    finally:
        pkg.srv_destroy(srv)
    return outs, res, stats


def test_served_results_match_oracle_and_alone_equals_mix(pkg, oracle_mod):
    circuits = mixed_circuits()
    mix, res_mix, stats = serve(pkg, circuits, True, small_n=14, slots=3)
    alone, res_alone, _ = serve(pkg, circuits, False, small_n=14, slots=3)
    assert stats["completed"] == len(circuits) and stats["p99_ms"] >= stats["p50_ms"] > 0
    for c, a, b, (norm, s2, lat) in zip(circuits, mix, alone, res_mix):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), c.name
        want = oracle_mod.run_circuit(c)
        assert np.linalg.norm(a.astype(np.complex128) - want) <= TOL_FP32
        onorm, os2, _ = oracle_mod.reduce(want)
        assert abs(norm - 1.0) < 1e-5 and abs(s2 - os2) < 1e-3 * os2 and lat > 0


def test_tensor_core_modes_on_concurrent_streams(pkg, oracle_mod):
    # stream-path circuits on several slot streams at once, in the tcgen05 and mma.sync 3xFP16
    # modes: the shared matrix-staging rings must not be overwritten under a kernel still queued
    # on another stream; served alone and in a mix must agree bit for bit
    circuits = [si.sycamore_circuit(si.near_square_grid(n), d, seed=300 + i)
                for i, (n, d) in enumerate([(16, 12), (18, 10), (17, 14), (19, 8), (16, 16), (18, 12)])]
    for prec in (pkg.SIM_FP16X3_TMEM, pkg.SIM_FP16X3):
        mix, res, stats = serve(pkg, circuits, True, small_n=12, slots=4, kmax=5, precision=prec)
        alone, _, _ = serve(pkg, circuits, False, small_n=12, slots=4, kmax=5, precision=prec)
        assert stats["completed"] == len(circuits)
        for c, a, b, (norm, s2, lat) in zip(circuits, mix, alone, res):
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), (prec, c.name)
            assert np.linalg.norm(a.astype(np.complex128) - oracle_mod.run_circuit(c)) <= TOL_FP32, (prec, c.name)


def test_default_tcgen05_mode_blocks_of_six_in_a_chosen_layout(pkg, oracle_mod):
    # circuits above small_n in SIM_FP16X3_TMEM with the automatic width (6) run in the layout
    # sim_plan_layout picks and are permuted back before the readout: logical-order amplitudes,
    # the same alone and in a mix
    circuits = [si.sycamore_circuit(si.near_square_grid(n), d, seed=500 + i)
                for i, (n, d) in enumerate([(21, 10), (22, 8), (23, 12), (21, 14)])]
    mix, res, stats = serve(pkg, circuits, True, slots=3, precision=pkg.SIM_FP16X3_TMEM)
    alone, _, _ = serve(pkg, circuits, False, slots=3, precision=pkg.SIM_FP16X3_TMEM)
    assert stats["completed"] == len(circuits)
    for c, a, b, (norm, s2, lat) in zip(circuits, mix, alone, res):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), c.name
        err = np.linalg.norm(a.astype(np.complex128) - oracle_mod.run_circuit(c))
        print(f"served {c.n_qubits} qubits, {len(c.gates)} gates (tcgen05, k <= 6, chosen layout): err {err:.2e}")
        assert err <= TOL_FP32 and abs(norm - 1.0) < 1e-5


def test_large_circuits_take_the_contraction_front(pkg, oracle_mod):
    # >= 26 qubits in SIM_FP16X3_TMEM: the first gates as two tensors contracted on the tensor cores
    # (when they are >= 30 % of the circuit), the rest in the chosen layout; logical-order
    # amplitudes match the oracle and are the same alone and in a mix; with front_pairs < 0 the
    # same circuits run without the front
    circuits = [si.sycamore_circuit(si.near_square_grid(n), d, seed=700 + i)
                for i, (n, d) in enumerate([(26, 9), (27, 11), (26, 14)])]
    mix, res, stats = serve(pkg, circuits, True, slots=2, precision=pkg.SIM_FP16X3_TMEM)
    alone, _, _ = serve(pkg, circuits, False, slots=2, precision=pkg.SIM_FP16X3_TMEM)
    plain, _, _ = serve(pkg, circuits, False, slots=2, precision=pkg.SIM_FP16X3_TMEM, front_pairs=-1)
    assert stats["completed"] == len(circuits)
    for c, a, b, p, (norm, s2, lat) in zip(circuits, mix, alone, plain, res):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), c.name
        want = oracle_mod.run_circuit(c)
        err = np.linalg.norm(a.astype(np.complex128) - want)
        err_plain = np.linalg.norm(p.astype(np.complex128) - want)
        side, nf = pkg.sim_split_choose(c.n_qubits, pkg.gates_array(c), 5)
        print(f"served {c.n_qubits} qubits, {len(c.gates)} gates, front of {nf}: err {err:.2e} "
              f"(without the front {err_plain:.2e})")
        assert nf >= 0.3 * len(c.gates)
        assert err <= TOL_FP32 and err_plain <= TOL_FP32 and abs(norm - 1.0) < 1e-5
        assert not np.array_equal(a, p)  # the front did run


def test_large_fp32_circuits_take_a_two_pair_front(pkg, oracle_mod):
    # >= 26 qubits in SIM_FP32: a front of at most 2 bridging gates (its contraction runs on CUDA
    # cores and grows 4x per gate) when it holds >= 10 % of the circuit; amplitudes match the oracle,
    # alone equals mix, and the result differs in its bits from the run without the front
    circuits = [si.sycamore_circuit(si.near_square_grid(n), d, seed=750 + i)
                for i, (n, d) in enumerate([(26, 12), (27, 16)])]
    mix, res, stats = serve(pkg, circuits, True, slots=2, precision=pkg.SIM_FP32)
    alone, _, _ = serve(pkg, circuits, False, slots=2, precision=pkg.SIM_FP32)
    plain, _, _ = serve(pkg, circuits, False, slots=2, precision=pkg.SIM_FP32, front_pairs=-1)
    assert stats["completed"] == len(circuits)
    for c, a, b, p, (norm, s2, lat) in zip(circuits, mix, alone, plain, res):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), c.name
        want = oracle_mod.run_circuit(c)
        err = np.linalg.norm(a.astype(np.complex128) - want)
        err_plain = np.linalg.norm(p.astype(np.complex128) - want)
        side, nf = pkg.sim_split_choose(c.n_qubits, pkg.gates_array(c), 2)
        print(f"served FP32 {c.n_qubits} qubits, {len(c.gates)} gates, front of {nf}: err {err:.2e} "
              f"(without the front {err_plain:.2e})")
        assert nf >= 0.1 * len(c.gates)
        assert err <= TOL_FP32 and err_plain <= TOL_FP32 and abs(norm - 1.0) < 1e-5
        assert not np.array_equal(a, p)  # the front did run


def test_admission_respects_hbm_budget(pkg, oracle_mod):
    # 20-qubit states are 8 MiB; a 20 MiB budget admits two at a time
    circuits = [si.sycamore_circuit(si.near_square_grid(20), 6, seed=s) for s in range(5)]
    outs, res, stats = serve(pkg, circuits, True, small_n=16, slots=4, hbm_budget=20 << 20)
    assert stats["completed"] == 5 and stats["hbm_used"] == 0
    for c, o in zip(circuits, outs):
        assert np.linalg.norm(o.astype(np.complex128) - oracle_mod.run_circuit(c)) <= TOL_FP32
    srv = pkg.srv_create(hbm_budget=20 << 20)
    try:
        big = si.sycamore_circuit(si.near_square_grid(22), 2, seed=1)  # 32 MiB > budget
        with pytest.raises(pkg.SimError) as e:
            pkg.srv_submit(srv, big.n_qubits, pkg.gates_array(big))
        assert e.value.code == pkg.SIM_E_BUSY
        assert pkg.srv_stats(srv)["rejected"] == 1
    finally:
        pkg.srv_destroy(srv)


def test_wait_is_bounded_and_errors_are_reported(pkg):
    srv = pkg.srv_create(small_n=12)
    try:
        c = si.sycamore_circuit(si.near_square_grid(24), 20, seed=3)
        t = pkg.srv_submit(srv, c.n_qubits, pkg.gates_array(c))
        try:
            pkg.srv_wait(srv, t, timeout_ms=0)  # a 24-qubit, 20-cycle circuit is not done at once
            timed_out = False
        except pkg.SimError as e:
            assert e.code == pkg.SIM_E_TIMEOUT
            timed_out = True
        assert timed_out
        norm, _, _ = pkg.srv_wait(srv, t, timeout_ms=60000)
        assert abs(norm - 1) < 1e-5
        with pytest.raises(pkg.SimError):
            pkg.srv_wait(srv, t, timeout_ms=10)  # forgotten after a successful wait
        bad = pkg.gates_array([(si.FSIM, 0, 0, 1.0, 0.5)])
        with pytest.raises(pkg.SimError) as e:
            pkg.srv_submit(srv, 4, bad)
        assert e.value.code == pkg.SIM_E_INVAL
    finally:
        pkg.srv_destroy(srv)


def test_packed_path_many_small_circuits(pkg, oracle_mod):
    circuits = [si.sycamore_circuit(si.near_square_grid(12 + (i % 5)), 6 + (i % 7), seed=i) for i in range(300)]
    outs, res, stats = serve(pkg, circuits, True, small_n=20)
    assert stats["completed"] == 300
    for i in range(0, 300, 37):
        assert np.linalg.norm(outs[i].astype(np.complex128) - oracle_mod.run_circuit(circuits[i])) <= TOL_FP32


def test_autotuned_server_matches_oracle_and_alone_equals_mix(pkg, oracle_mod):
    # srv_autotune measures the candidates per (size, depth class) once; every later circuit of a
    # tuned class takes the cached choice, served alone or in a mix alike
    samples = [si.sycamore_circuit(si.near_square_grid(n), d, seed=900 + n) for n, d in ((21, 10), (24, 10), (26, 14))]
    srv = pkg.srv_create(small_n=20, slots=3, precision=pkg.SIM_FP16X3_TMEM)
    try:
        picks = pkg.srv_autotune(srv, [(c.n_qubits, pkg.gates_array(c)) for c in samples])
        for c, (k, fr, ms) in zip(samples, picks):
            print(f"tuned {c.n_qubits} qubits, {c.n_gates} gates: k_max {k}, front {fr}, {ms:.2f} ms")
            assert 4 <= k <= 6 and fr in (0, 1) and ms > 0
        circuits = [si.sycamore_circuit(si.near_square_grid(n), d, seed=950 + i)
                    for i, (n, d) in enumerate(((21, 9), (24, 11), (26, 13), (18, 8), (21, 11)))]
        outs = [np.zeros(1 << c.n_qubits, dtype=np.complex64) for c in circuits]
        tickets = [pkg.srv_submit(srv, c.n_qubits, pkg.gates_array(c), o) for c, o in zip(circuits, outs)]
        for t in tickets:
            pkg.srv_wait(srv, t, timeout_ms=120000)
        alone = [np.zeros_like(o) for o in outs]
        for c, o in zip(circuits, alone):
            pkg.srv_wait(srv, pkg.srv_submit(srv, c.n_qubits, pkg.gates_array(c), o), 120000)
    finally:
        pkg.srv_destroy(srv)
    for c, a, b in zip(circuits, outs, alone):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), c.name
        assert np.linalg.norm(a.astype(np.complex128) - oracle_mod.run_circuit(c)) <= TOL_FP32


def test_repeated_circuit_replays_its_graph_bit_identically(pkg, oracle_mod):
    # the second submission of the same circuit makes a CUDA-graph entry; later ones replay it
    # with the stream path's kernels, layout and reduction: every result bit-identical, also to the
    # same circuit served once by a fresh server (stream path), and to the oracle within 1e-5
    circ = si.sycamore_circuit(si.near_square_grid(22), 12, seed=777)
    g = pkg.gates_array(circ)
    once = np.zeros(1 << 22, dtype=np.complex64)
    srv = pkg.srv_create(small_n=20, slots=2, precision=pkg.SIM_FP16X3_TMEM)
    try:
        pkg.srv_wait(srv, pkg.srv_submit(srv, 22, g, once), 120000)
        assert pkg.srv_stats(srv)["graph_replays"] == 0
    finally:
        pkg.srv_destroy(srv)
    srv = pkg.srv_create(small_n=20, slots=2, precision=pkg.SIM_FP16X3_TMEM)
    outs = [np.zeros(1 << 22, dtype=np.complex64) for _ in range(5)]
    try:
        for o in outs[:2]:  # the first on the stream path, the second makes and replays the graph
            pkg.srv_wait(srv, pkg.srv_submit(srv, 22, g, o), 120000)
        tickets = [pkg.srv_submit(srv, 22, g, o) for o in outs[2:]]  # queued together: one replay at a time
        res = [pkg.srv_wait(srv, t, 120000) for t in tickets]
        stats = pkg.srv_stats(srv)
    finally:
        pkg.srv_destroy(srv)
    assert stats["graph_replays"] == 4
    for o in outs:
        assert np.array_equal(o.view(np.uint64), once.view(np.uint64))
    assert np.linalg.norm(once.astype(np.complex128) - oracle_mod.run_circuit(circ)) <= TOL_FP32
    assert all(abs(norm - 1.0) < 1e-5 for norm, _, _ in res)
