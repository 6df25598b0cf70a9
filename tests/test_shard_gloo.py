"""Global-qubit sharding across ranks (Sect. 4: the state split by global qubits, an all-to-all
between phases), as gloo ranks on the CPU: world sizes 2 and 4 (g = 1, 2).

* Exchanges alone: a random state sharded under a random layout goes through a sequence of
  exchanges (the library's schedule, each rank's local permutation, one all_to_all_single with
  the schedule's split sizes); after every exchange the gathered shards equal the oracle's
  permutation of the whole state into the new layout, bit for bit.
* A whole circuit: the library's phase planner (sliced sets at the lattice's two ends, slice_bits
  = g) drives `shard.run_phases`; blocks are applied to each rank's shard with the oracle's k-qubit
  apply (the device path applies them with sim_apply_fused, checked on the GPU elsewhere), and the
  gathered logical state equals the oracle's gate-by-gate run to 1e-12.
"""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def gather(dist, torch, local: np.ndarray, world: int) -> np.ndarray:
    t = torch.from_numpy(np.ascontiguousarray(local).view(np.int64).copy())
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    return np.concatenate([p.numpy() for p in parts]).view(local.dtype)


def ranks_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    import paper_1910_09534_gb300 as pkg
    import syc_inputs as si
    from paper_1910_09534_gb300 import shard

    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
        g = world.bit_length() - 1
        oracle.set_threads(1)

        def make_all_to_all(state):
            def a2a(splits):  # split sizes are in amplitudes; the buffer moves as 8-byte words
                words = [s * (state["buf"].itemsize // 8) for s in splits]
                src = torch.from_numpy(state["buf"].view(np.int64).copy())
                dst = torch.empty_like(src)
                dist.all_to_all_single(dst, src, words, words)
                state["buf"] = dst.numpy().view(state["buf"].dtype).copy()
            return a2a

        def make_permute(state):
            def perm(p):
                state["buf"] = oracle.permute(state["buf"], p)
            return perm

        # ---- exchanges alone, bit for bit ----
        n = 10
        rng = np.random.default_rng(5)
        psi = si.random_state(n, 17)
        bit_of = [int(x) for x in rng.permutation(n)]
        L = n - g
        phys = oracle.permute(psi, bit_of)
        st = {"buf": phys[rank << L:(rank + 1) << L].copy()}
        for step in range(8):
            nxt = [int(x) for x in rng.choice(n, g, replace=False)]
            bit_of = shard.exchange(n, g, bit_of, nxt, rank, world, make_permute(st), make_all_to_all(st))
            assert sorted(bit_of[q] for q in nxt) == list(range(L, n)), (step, bit_of, nxt)
            full = gather(dist, torch, st["buf"], world)
            want = oracle.permute(psi, bit_of)
            assert np.array_equal(full.view(np.uint64), want.view(np.uint64)), step

        # ---- a whole circuit through the phase planner ----
        circ = si.sycamore_circuit(si.Grid(3, 4), cycles=8, seed=3)
        n = circ.n_qubits
        gates = pkg.gates_array(circ)
        set_a, set_b = list(range(g)), list(range(n - g, n))
        ph = pkg.sim_phases_create(n, gates, g, set_a, set_b, kmax=4)
        try:
            n_phases = pkg.sim_phases_info(ph)[0]
            bit_of = shard.initial_layout(n, set_a)
            L = n - g
            st = {"buf": np.zeros(1 << L, dtype=np.complex128)}
            if rank == 0:
                st["buf"][0] = 1.0

            def apply_block(targets, mat):
                oracle.apply_kq(st["buf"], targets, mat)

            bit_of = shard.run_phases(n, g, ph, set_a, set_b, bit_of, rank, world, make_permute(st), apply_block,
                                      make_all_to_all(st))
        finally:
            pkg.sim_phases_destroy(ph)
        full = gather(dist, torch, st["buf"], world)
        got = shard.gather_logical(np.split(full, world), n, g, bit_of)
        err = float(np.abs(got - oracle.run_circuit(circ)).max())
        assert err < 1e-12, err
        dist.destroy_process_group()
        q.put((rank, "ok", n_phases))
    except Exception as e:  # report to the parent instead of hanging it
        import traceback
        q.put((rank, "fail", traceback.format_exc()))


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_exchanges_and_phases_match_oracle(world):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=ranks_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = []
    try:
        for _ in range(world):
            results.append(q.get(timeout=240))
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    fails = [r for r in results if r[1] != "ok"]
    assert not fails, fails[0][2]
    assert all(r[2] >= 2 for r in results)  # the circuit needed at least one exchange


def test_exchange_plan_host_checks():
    import sys
    sys.path.insert(0, ROOT)
    import paper_1910_09534_gb300 as pkg
    from paper_1910_09534_gb300 import shard

    n, g = 8, 2
    ident = list(range(n))
    m, lp, after, mask = pkg.sim_shard_exchange_plan(n, g, ident, [6, 7])
    assert m == 0 and after == ident and lp == list(range(n - g))
    m, lp, after, mask = pkg.sim_shard_exchange_plan(n, g, ident, [0, 7])
    # qubit 6 (rank bit 0) leaves, qubit 0 takes its rank bit; 0 first moves to local position 5
    assert m == 1 and mask == 1 and lp[0] == 5 and after[0] == 6 and after[6] == 5 and after[7] == 7
    assert sorted(lp) == list(range(n - g)) and sorted(after) == list(range(n))
    assert shard.partner_splits(2, 4, 1, 16) == [0, 0, 16, 16]
    for bad in (([0] * n, [6, 7]), (ident, [7, 7]), (ident, [8, 1])):
        with pytest.raises(pkg.SimError):
            pkg.sim_shard_exchange_plan(n, g, *bad)
    with pytest.raises(pkg.SimError):
        pkg.sim_shard_exchange_plan(n, 5, ident, [0, 1, 2, 3, 4])
