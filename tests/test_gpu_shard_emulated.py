"""GPU: the sharded device path (`shard.ShardedState`: sim_permute, relabelling and
sim_apply_fused on each rank's shard, chunk exchanges between the two buffers) with two ranks
emulated by two host threads on one GPU.  Each rank has its own handles and stream; the
exchange is done by device copies between the ranks' buffers while both host threads wait at a
barrier (no kernel ever waits on another rank).  The gathered state must match the oracle's
gate-by-gate run (||psi - psi_oracle||_2 <= 1e-5)."""
import threading

import numpy as np
import pytest

import syc_inputs as si

pytestmark = pytest.mark.gpu


class Hub:
    """An all-to-all for ranks that are threads of one process: every rank posts its buffers and
    split sizes, then copies the chunks addressed to it out of the other ranks' send buffers."""

    def __init__(self, world):
        import torch
        self.torch, self.world = torch, world
        self.barrier = threading.Barrier(world, timeout=120)
        self.src, self.splits = [None] * world, [None] * world

    def make(self, rank):
        def a2a(dst, src, splits):
            self.torch.cuda.synchronize()  # this rank's local permutation has run
            self.src[rank], self.splits[rank] = src, list(splits)
            self.barrier.wait()
            out = 0
            for s in range(self.world):
                cnt = self.splits[s][rank]
                if cnt:
                    off = sum(self.splits[s][:rank])
                    dst[out:out + cnt].copy_(self.src[s][off:off + cnt])
                    out += cnt
            self.torch.cuda.synchronize()
            self.barrier.wait()  # no rank reuses its send buffer before every copy is done
        return a2a


@pytest.mark.parametrize("prec_name,kmax", [("SIM_FP32", 4), ("SIM_FP16X3_TMEM", 6)])
def test_two_emulated_ranks_match_oracle(oracle_mod, prec_name, kmax):
    pytest.importorskip("torch")
    from paper_1910_09534_gb300 import build
    build.build()
    import paper_1910_09534_gb300 as pkg
    from paper_1910_09534_gb300 import shard

    circ = si.detuned_sycamore_circuit(si.Grid(4, 4), cycles=10, seed=21)
    n, g, world = circ.n_qubits, 1, 2
    set_a, set_b = [0], [n - 1]
    prec = getattr(pkg, prec_name)
    ph = pkg.sim_phases_create(n, pkg.gates_array(circ), g, set_a, set_b, kmax=kmax, precision=prec)
    hub = Hub(world)
    states = [shard.ShardedState(n, g, rank=r, world=world, all_to_all=hub.make(r)) for r in range(world)]
    layouts, errors = [None] * world, []

    def rank_main(r):
        try:
            layouts[r] = states[r].run_phases(ph, set_a, set_b, precision=prec)
        except Exception as e:  # noqa: BLE001 -- reported below
            errors.append(e)
            hub.barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    try:
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=300)
        assert not errors, errors[0]
        assert layouts[0] == layouts[1]
        assert pkg.sim_phases_info(ph)[0] >= 2  # at least one exchange
        shards = [st.local_amplitudes() for st in states]
        sums = [st.local_reduce() for st in states]
    finally:
        for st in states:
            st.destroy()
        pkg.sim_phases_destroy(ph)
    got = shard.gather_logical(shards, n, g, layouts[0]).astype(np.complex128)
    want = oracle_mod.run_circuit(circ)
    err = float(np.linalg.norm(got - want))
    print(f"2 emulated ranks, {prec_name}: ||psi - psi_oracle||_2 = {err:.3e}")
    assert err <= 1e-5
    assert abs(sum(s[0] for s in sums) - 1.0) < 1e-5
