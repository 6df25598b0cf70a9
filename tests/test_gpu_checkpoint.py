"""GPU: checkpoint / resume (sim_state_save / sim_state_load).

Saving and loading only moves data, so a resumed run must equal the uninterrupted one bit for
bit: a device state with a permuted layout round-trips, and a host-store run (one of its regions
in HBM) checkpointed at a phase boundary and resumed in a new handle finishes with the same
amplitudes as the run that never stopped.  Files that do not fit the handle are refused.
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


def test_device_state_round_trip_with_layout(pkg, tmp_path):
    n = 17
    psi = si.random_state(n, 4)
    path = str(tmp_path / "dev.state")
    h = pkg.sim_create(n)
    try:
        pkg.sim_load_amplitudes(h, psi)
        pkg.sim_permute(h, si.random_permutation(n, 9))
        layout = list(pkg.sim_info(h)[2])
        pkg.sim_state_save(h, path)
    finally:
        pkg.sim_destroy(h)
    h2 = pkg.sim_create(n)
    try:
        pkg.sim_state_load(h2, path)
        assert list(pkg.sim_info(h2)[2]) == layout
        assert np.array_equal(pkg.sim_amplitudes(h2).view(np.uint64), psi.view(np.uint64))
    finally:
        pkg.sim_destroy(h2)


def test_host_store_resume_at_a_phase_boundary_is_bit_identical(pkg, tmp_path):
    circ = si.sycamore_circuit(si.Grid(4, 5), cycles=14, seed=13)
    n, s = circ.n_qubits, 2
    set_a, set_b = [0, 1], [18, 19]
    ph = pkg.sim_phases_create(n, pkg.gates_array(circ), s, set_a, set_b, kmax=5, precision=pkg.SIM_FP16X3_TMEM)
    nph = pkg.sim_phases_info(ph)[0]
    assert nph >= 3
    opts = dict(store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=3, store_device_regions=1)
    path = str(tmp_path / "phase.state")
    try:
        h = pkg.sim_create(n, s, **opts)  # uninterrupted
        try:
            pkg.sim_run_phases(h, ph)
            want = pkg.sim_amplitudes(h)
        finally:
            pkg.sim_destroy(h)
        h = pkg.sim_create(n, s, **opts)  # first two phases, then a checkpoint
        try:
            for i in range(2):
                pkg.sim_run_phase(h, *pkg.sim_phases_get(ph, i))
            pkg.sim_state_save(h, path)
        finally:
            pkg.sim_destroy(h)
        h = pkg.sim_create(n, s, **opts)  # resumed elsewhere
        try:
            pkg.sim_state_load(h, path)
            for i in range(2, nph):
                pkg.sim_run_phase(h, *pkg.sim_phases_get(ph, i))
            got = pkg.sim_amplitudes(h)
        finally:
            pkg.sim_destroy(h)
    finally:
        pkg.sim_phases_destroy(ph)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_checkpoint_refusals(pkg, tmp_path):
    n = 12
    good = str(tmp_path / "g.state")
    h = pkg.sim_create(n)
    try:
        pkg.sim_state_save(h, good)
    finally:
        pkg.sim_destroy(h)
    h13 = pkg.sim_create(n + 1)
    try:
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_state_load(h13, good)
        assert e.value.code == pkg.SIM_E_INVAL
        bad = tmp_path / "b.state"
        bad.write_bytes(b"not a state file" * 64)
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_state_load(h13, str(bad))
        assert e.value.code == pkg.SIM_E_INVAL
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_state_load(h13, str(tmp_path / "missing.state"))
        assert e.value.code == pkg.SIM_E_IO
    finally:
        pkg.sim_destroy(h13)
    h = pkg.sim_create(n)
    try:
        trunc = tmp_path / "t.state"
        trunc.write_bytes(open(good, "rb").read()[:-100])
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_state_load(h, str(trunc))
        assert e.value.code == pkg.SIM_E_IO
    finally:
        pkg.sim_destroy(h)
