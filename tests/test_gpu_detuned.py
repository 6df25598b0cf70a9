"""GPU parity on circuits whose two-qubit gates vary with location and depth.

Sect. 3 notes that the hardware's fSim unitaries differ from coupler to coupler and from cycle to
cycle; Eq. 1 gives their form with theta, phi and the detunings D+, D-, D-,off.  These circuits
(`syc_inputs.detuned_sycamore_circuit`: every fSim instance draws its own parameters) run through
the CUDA path -- fused blocks in FP32 and in the default split mode (3xFP16 on tcgen05, blocks of
<= 6 qubits in the layout sim_plan_layout picks), the contraction-deferral front, the resident
sliced phases and the server -- and every amplitude is compared with the oracle's gate-by-gate
complex128 run.  A detuned fSim is not symmetric in its two qubits, so a swapped role anywhere
(composition, E2Q's bridging gate, the layout) shows up here.  Bound ||psi - psi_oracle||_2 <= 1e-5.
"""
import os

import numpy as np
import pytest

import syc_inputs as si

pytestmark = pytest.mark.gpu
TOL = 1e-5

CIRCUITS = {
    12: (si.Grid(3, 4), 8),
    20: (si.Grid(4, 5), 14),
    28: (si.Grid(4, 7), 20),
}
_cache = {}


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as p
    return p


def detuned(oracle_mod, n):
    """(circuit, oracle amplitudes) for the n-qubit detuned workload, computed once."""
    if n not in _cache:
        grid, cycles = CIRCUITS[n]
        circ = si.detuned_sycamore_circuit(grid, cycles, seed=40 + n, name=f"detuned{n}")
        oracle_mod.set_threads(os.cpu_count() or 1)
        _cache[n] = (circ, oracle_mod.run_circuit(circ))
    return _cache[n]


def err_and_max(got64, want128, chunk=1 << 26):
    s, m = 0.0, 0.0
    for a in range(0, want128.size, chunk):
        d = got64[a:a + chunk].astype(np.complex128) - want128[a:a + chunk]
        s += float(np.vdot(d, d).real)
        m = max(m, float(np.abs(d).max()))
    return s ** 0.5, m


MODES = [("fp32_k4", 4, "SIM_FP32", False), ("fp16x3_tmem_k6_layout", 6, "SIM_FP16X3_TMEM", True)]


@pytest.mark.parametrize("n", [12, 20, 28])
@pytest.mark.parametrize("mode", MODES, ids=[m[0] for m in MODES])
def test_detuned_fused_blocks_match_oracle(pkg, oracle_mod, n, mode):
    name, kmax, prec_name, layout = mode
    prec = getattr(pkg, prec_name)
    circ, want = detuned(oracle_mod, n)
    plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=kmax, precision=prec)
    h = pkg.sim_create(n)
    try:
        if layout:
            perm, _, _ = pkg.sim_plan_layout(plan, n)
            pkg.sim_set_layout(h, perm)
        pkg.sim_reset(h)
        pkg.sim_apply_plan(h, plan)
        got = pkg.sim_amplitudes(h)
        norm, _, _ = pkg.sim_reduce(h)
    finally:
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
    err, emax = err_and_max(got, want)
    print(f"detuned {n}q {name}: ||psi - psi_oracle||_2 = {err:.3e}, max |d| = {emax:.3e}")
    assert err <= TOL, (n, name, err)
    assert abs(norm - 1.0) < 1e-5


@pytest.mark.parametrize("n", [20, 28])
@pytest.mark.parametrize("prec_name,kmax", [("SIM_FP32", 4), ("SIM_FP16X3_TMEM", 6)])
def test_detuned_contraction_front_matches_oracle(pkg, oracle_mod, n, prec_name, kmax):
    # contraction deferral (Sect. 2; Appendix EI / E2Q): the gates up to the sixth crossing of the
    # chosen bipartition as two tensors, contracted into the state, the rest as fused blocks
    prec = getattr(pkg, prec_name)
    circ, want = detuned(oracle_mod, n)
    gates = pkg.gates_array(circ)
    side, front = pkg.sim_split_choose(n, gates, 5)
    s = pkg.sim_split_create(n, gates[:front], side)
    pairs = pkg.sim_split_info(s)[2]
    assert pairs >= 1
    h = pkg.sim_create(n)
    fr = pkg.sim_front_create(h, s, kmax=kmax, precision=prec)
    plan = pkg.sim_plan_create(n, gates[front:], kmax=kmax, precision=prec)
    try:
        if prec == pkg.SIM_FP16X3_TMEM:
            perm, _, _ = pkg.sim_plan_layout(plan, n)
            pkg.sim_set_layout(h, perm)
        pkg.sim_front_run(h, fr)
        pkg.sim_apply_plan(h, plan)
        got = pkg.sim_amplitudes(h)
    finally:
        pkg.sim_plan_destroy(plan)
        pkg.sim_front_destroy(fr)
        pkg.sim_destroy(h)
        pkg.sim_split_destroy(s)
    err, emax = err_and_max(got, want)
    print(f"detuned {n}q front ({pairs} bridging gates, {front} gates) {prec_name}: "
          f"||psi - psi_oracle||_2 = {err:.3e}, max |d| = {emax:.3e}")
    assert err <= TOL, (n, prec_name, err)


def test_detuned_sliced_phases_match_oracle(pkg, oracle_mod):
    # Sect. 4 in device memory: 8 slices over the 3 top bits, phases alternating the sliced sets
    # at the lattice's two ends, permutation passes between them
    circ, want = detuned(oracle_mod, 20)
    n, s = 20, 3
    set_a, set_b = list(range(s)), list(range(n - s, n))
    for prec, kmax in ((pkg.SIM_FP32, 4), (pkg.SIM_FP16X3_TMEM, 6)):
        ph = pkg.sim_phases_create(n, pkg.gates_array(circ), s, set_a, set_b, kmax=kmax, precision=prec)
        h = pkg.sim_create(n, s)
        try:
            pkg.sim_run_phases(h, ph)
            got = pkg.sim_amplitudes(h)
            assert pkg.sim_phases_info(ph)[0] >= 2
        finally:
            pkg.sim_destroy(h)
            pkg.sim_phases_destroy(ph)
        err, _ = err_and_max(got, want)
        assert err <= TOL, (prec, err)


def test_detuned_served_match_oracle(pkg, oracle_mod):
    # the server: a packed circuit (<= small_n qubits, one CTA per circuit) and two on the stream
    # path (one of them >= 26 qubits would take the front; these stay below), every amplitude
    circuits = [si.detuned_sycamore_circuit(si.near_square_grid(n), d, seed=500 + n)
                for n, d in ((14, 10), (18, 12), (22, 9))]
    srv = pkg.srv_create(small_n=16, slots=2, precision=pkg.SIM_FP16X3_TMEM)
    outs = [np.zeros(1 << c.n_qubits, dtype=np.complex64) for c in circuits]
    try:
        tickets = [pkg.srv_submit(srv, c.n_qubits, pkg.gates_array(c), o) for c, o in zip(circuits, outs)]
        for t in tickets:
            pkg.srv_wait(srv, t, timeout_ms=60000)
    finally:
        pkg.srv_destroy(srv)
    for c, o in zip(circuits, outs):
        err, _ = err_and_max(o, oracle_mod.run_circuit(c))
        assert err <= TOL, (c.n_qubits, err)
