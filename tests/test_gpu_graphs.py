"""GPU: CUDA graphs of a plan (sim_graph_create / sim_graph_launch).

A replayed graph runs the same kernels on the same staged operands as sim_apply_plan, so its
result must be bit-identical to the direct path, for every kernel family (tcgen05, mma.sync
3xFP16 and 3xTF32, CUDA-core FP32 including the 6-qubit blocks whose matrix is staged in device
memory); replays from different initial states must match the direct path too, and the graph
must refuse a changed layout or another handle.
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


CASES = [("4x5", 12, 5, "fp16x3_tmem"), ("4x5", 10, 4, "fp16x3_tmem"), ("3x6", 10, 6, "fp32"),
         ("4x4", 12, 5, "tf32x3"), ("3x5", 8, 5, "fp16x3")]


def prec_of(pkg, name):
    return {"fp32": pkg.SIM_FP32, "fp16x3": pkg.SIM_FP16X3, "fp16x3_tmem": pkg.SIM_FP16X3_TMEM,
            "tf32x3": pkg.SIM_TF32X3}[name]


@pytest.mark.parametrize("grid,cycles,kmax,prec", CASES)
def test_graph_replay_bit_identical_to_direct(pkg, oracle_mod, grid, cycles, kmax, prec):
    r, c = map(int, grid.split("x"))
    circ = si.sycamore_circuit(si.Grid(r, c), cycles=cycles, seed=r * 10 + c + kmax)
    n = circ.n_qubits
    plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=kmax, precision=prec_of(pkg, prec))
    h = pkg.sim_create(n)
    graph = None
    try:
        graph = pkg.sim_graph_create(h, plan)
        for basis, reps in ((0, 1), (5, 2), ((1 << n) - 1, 1)):
            pkg.sim_reset(h, basis)
            for _ in range(reps):
                pkg.sim_apply_plan(h, plan)
            direct = pkg.sim_amplitudes(h)
            pkg.sim_reset(h, basis)
            for _ in range(reps):
                pkg.sim_graph_launch(h, graph)
            replay = pkg.sim_amplitudes(h)
            assert np.array_equal(replay.view(np.uint64), direct.view(np.uint64)), (basis, prec)
        pkg.sim_sync(h, 10000)
    finally:
        if graph is not None:
            pkg.sim_graph_destroy(graph)
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    if prec in ("fp32", "fp16x3_tmem"):  # and against the oracle
        h = pkg.sim_create(n)
        plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=kmax, precision=prec_of(pkg, prec))
        graph = None
        try:
            graph = pkg.sim_graph_create(h, plan)
            pkg.sim_graph_launch(h, graph)
            got = pkg.sim_amplitudes(h, dtype=pkg.SIM_C128)
        finally:
            if graph is not None:
                pkg.sim_graph_destroy(graph)
            pkg.sim_destroy(h)
            pkg.sim_plan_destroy(plan)
        assert np.linalg.norm(got - oracle_mod.run_circuit(circ)) <= 1e-5


def test_graph_refuses_changed_layout_and_other_handle(pkg):
    circ = si.sycamore_circuit(si.Grid(3, 4), cycles=6, seed=1)
    n = circ.n_qubits
    plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=5, precision=pkg.SIM_FP16X3_TMEM)
    h, h2 = pkg.sim_create(n), pkg.sim_create(n)
    g = pkg.sim_graph_create(h, plan)
    try:
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_graph_launch(h2, g)
        assert e.value.code == pkg.SIM_E_INVAL
        pkg.sim_permute(h, si.random_permutation(n, 2))
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_graph_launch(h, g)
        assert e.value.code == pkg.SIM_E_INVAL
        pkg.sim_permute(h, list(range(n)))  # back to the layout it was captured with
        pkg.sim_graph_launch(h, g)
        pkg.sim_sync(h, 10000)
    finally:
        pkg.sim_graph_destroy(g)
        pkg.sim_destroy(h)
        pkg.sim_destroy(h2)
        pkg.sim_plan_destroy(plan)
