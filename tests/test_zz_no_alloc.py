"""The allocation-free reduction entry point, checked through the C ABI against the oracle's
reduction and against sim_reduce.

sim_reduce_noalloc is for callers that cannot allocate device memory themselves (their device
memory belongs to another framework's pool, or they must avoid cudaMalloc's implicit device
synchronisation); it keeps its scratch in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run everything else; it
also passes when run alone in a fresh process (the first call then does the per-device set-up).
"""
import numpy as np
import pytest

import oracle
import syc_inputs as si

pytestmark = pytest.mark.gpu

# same tolerances as the reduction parity tests
REL_NORM = 1e-6
REL_S2 = 1e-5


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as p
    return p


def test_reduce_noalloc_matches_sim_reduce(pkg):
    torch = pytest.importorskip("torch")
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")  # caller's output
    torch.cuda.synchronize()
    for n, seed in ((20, 1), (13, 2)):
        psi = si.random_state(n, seed)
        h = pkg.sim_create(n)
        try:
            pkg.sim_load_amplitudes(h, psi)
            norm, s2, xeb = pkg.sim_reduce(h)
            dptr, stream = pkg.sim_state_ptr(h)
            # the oracle's FP64 reduction of the complex64 amplitudes the device holds
            onorm, os2, oxeb = oracle.reduce(psi.astype(np.complex128))
            for _ in range(2):  # two calls in a row share (and reuse) the scratch array
                pkg.sim_reduce_noalloc(dptr, 1 << n, out.data_ptr(), stream)
                pkg.sim_sync(h)
                got = out.cpu().numpy()
                assert abs(got[0] - onorm) <= REL_NORM * onorm
                assert abs(got[1] - os2) <= REL_S2 * os2
                assert abs(got[2] - oxeb) <= REL_S2 * os2
                assert abs(got[0] - norm) <= REL_NORM * norm
                assert abs(got[1] - s2) <= REL_S2 * s2
                assert abs(got[2] - xeb) <= REL_S2 * s2
        finally:
            pkg.sim_destroy(h)


def test_reduce_noalloc_rejects_bad_sizes(pkg):
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for n_amps in (0, 3, (1 << 40) + 2):
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_reduce_noalloc(buf.data_ptr(), n_amps, out.data_ptr())
        assert e.value.code == pkg.SIM_E_INVAL
    # misaligned buffers are refused on the host before any launch
    for d_state, d_out in ((buf.data_ptr() + 8, out.data_ptr()), (buf.data_ptr(), out.data_ptr() + 4)):
        with pytest.raises(pkg.SimError) as e:
            pkg.sim_reduce_noalloc(d_state, 8, d_out)
        assert e.value.code == pkg.SIM_E_INVAL
