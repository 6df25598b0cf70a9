"""A state sharded over global qubits across 2^g ranks (Sect. 4; the Appendix's `all2all`).

The paper splits the state over many memories by g "global" qubits: gates act on the local ones,
and between phases an all-to-all reorganises the layout so that the next phase's gates find their
qubits local.  Here each rank holds 2^(n-g) amplitudes; `sim_shard_exchange_plan` (host, C ABI)
gives the local permutation and the chunk schedule of one exchange, the local permutation runs
on the device (`sim_permute`), and the chunks move in one `all_to_all_single` with per-rank split
sizes (NCCL between GPUs).  The phases come from the library's phase planner with the global set
as the sliced set (`sim_phases_create`): phase i's gates avoid its set, which is made global first.

Layout: position p < n - g is bit p of a rank's local index, position n - g + j bit j of the rank.

The loop (`run_phases`) only sequences calls: it takes the local permutation, the block apply and
the collective as callables, so the same schedule drives the device path (`ShardedState`) and
any other backend of the three operations.
"""
from __future__ import annotations

import numpy as np

from . import _native as N


def partner_splits(rank: int, world: int, mask: int, chunk: int) -> list:
    """Split sizes (amplitudes) of an exchange's all-to-all for `rank`: `chunk` to and from each rank
    that agrees with it outside the changing rank bits `mask`, 0 for every other rank."""
    return [chunk if (d & ~mask) == (rank & ~mask) else 0 for d in range(world)]


def exchange(n: int, g: int, bit_of, next_global, rank: int, world: int, local_permute, all_to_all):
    """One exchange making `next_global` the global qubits.  local_permute(perm) permutes the local
    state's amplitude bits (perm[p] = new local position of bit p); all_to_all(splits) exchanges
    the local state's chunks with those split sizes (the same list in both directions) and makes
    the received chunks the local state.  Returns the layout after the exchange."""
    m, local_perm, after, mask = N.sim_shard_exchange_plan(n, g, bit_of, next_global)
    if m == 0:
        return list(bit_of)
    if local_perm != list(range(n - g)):
        local_permute(local_perm)
    all_to_all(partner_splits(rank, world, mask, 1 << (n - g - m)))
    return after


def initial_layout(n: int, set_a) -> list:
    """A layout with the sliced set A global (A[j] at rank bit j) and the other qubits local in
    increasing order."""
    g = len(set_a)
    bit_of = [0] * n
    p = 0
    for q in range(n):
        if q in set_a:
            bit_of[q] = n - g + list(set_a).index(q)
        else:
            bit_of[q] = p
            p += 1
    return bit_of


def run_phases(n: int, g: int, phases, set_a, set_b, bit_of, rank: int, world: int, local_permute,
               apply_block, all_to_all):
    """Run every phase of a `sim_phases_t` (made with slice_bits = g and sets set_a, set_b) on a
    sharded state: make the phase's sliced set global (an exchange, if it is not already), then
    apply each of its blocks with targets mapped to local positions (apply_block(local_targets,
    matrix)).  Returns the final layout."""
    n_phases, _ = N.sim_phases_info(phases)
    for i in range(n_phases):
        set_id, plan = N.sim_phases_get(phases, i)
        glob = list(set_a) if set_id == 0 else list(set_b)
        bit_of = exchange(n, g, bit_of, glob, rank, world, local_permute, all_to_all)
        nb = N.sim_plan_info(plan)[0]
        for b in range(nb):
            targets, mat = N.sim_plan_block(plan, b)
            local = [bit_of[q] for q in targets]
            if max(local) >= n - g:
                raise ValueError(f"phase {i} block {b}: target qubit is global")
            apply_block(local, mat)
    return bit_of


class ShardedState:
    """The device path: this rank's 2^(n-g) amplitudes in torch CUDA tensors that sim handles use as
    their state (ext_state), ordered on torch's current stream; `group` is a torch.distributed
    process group over the 2^g ranks (NCCL).  Two buffers alternate: an exchange receives into the
    other one, whose handle then holds the state."""

    def __init__(self, n: int, g: int, group=None, device: int = 0, rank: int | None = None,
                 world: int | None = None, all_to_all=None):
        """all_to_all(dst, src, splits): the collective on int64 views of the buffers (one word per
        amplitude); default torch.distributed.all_to_all_single over `group`, with rank and world
        taken from it."""
        import torch

        self.torch, self.group = torch, group
        self.n, self.g = n, g
        if all_to_all is None:
            import torch.distributed as dist
            self.world, self.rank = dist.get_world_size(group), dist.get_rank(group)
            self.collective = lambda dst, src, splits: dist.all_to_all_single(dst, src, splits, splits, group=group)
        else:
            self.world, self.rank, self.collective = world, rank, all_to_all
        if self.world != 1 << g:
            raise ValueError(f"{self.world} ranks for {g} global qubits")
        amps = 1 << (n - g)
        dev = torch.device("cuda", device)
        # one stream orders the library's kernels, torch's buffer operations and the collective
        self.stream = torch.cuda.Stream(dev)
        with torch.cuda.stream(self.stream):
            self.bufs = [torch.zeros(amps, dtype=torch.complex64, device=dev) for _ in range(2)]
        self.hs = [N.sim_create(n - g, 0, device=device, stream=self.stream.cuda_stream, ext_state=b.data_ptr(),
                                ext_bytes=amps * 8) for b in self.bufs]
        self.cur = 0
        self.identity = list(range(n - g))
        self.bit_of = list(range(n))

    @property
    def h(self):
        return self.hs[self.cur]

    def reset(self):
        """|0...0>: amplitude 1 at local index 0 of rank 0 (rank bits are the top positions)."""
        self.cur = 0
        N.sim_set_layout(self.h, self.identity)
        if self.rank == 0:
            N.sim_reset(self.h, 0)
        else:
            with self.torch.cuda.stream(self.stream):
                self.bufs[0].zero_()

    def _local_permute(self, perm):
        N.sim_permute(self.h, perm)
        N.sim_set_layout(self.h, self.identity)  # the data now sits in the new order: relabel

    def _apply_block(self, targets, mat, precision):
        N.sim_apply_fused(self.h, targets, mat, precision=precision)

    def _all_to_all(self, splits):
        src, dst = self.bufs[self.cur], self.bufs[1 - self.cur]
        with self.torch.cuda.stream(self.stream):
            self.collective(dst.view(self.torch.int64), src.view(self.torch.int64), splits)
        self.cur = 1 - self.cur
        N.sim_set_layout(self.h, self.identity)

    def run_phases(self, phases, set_a, set_b, precision=N.SIM_FP32):
        """Start from |0...0> with set A global and run every phase (sim_phases_create with
        slice_bits = g and the same sets)."""
        self.bit_of = initial_layout(self.n, set_a)
        self.reset()
        self.bit_of = run_phases(self.n, self.g, phases, set_a, set_b, self.bit_of, self.rank, self.world,
                                 self._local_permute, lambda t, m: self._apply_block(t, m, precision),
                                 self._all_to_all)
        return self.bit_of

    def local_reduce(self):
        """This rank's (sum p, sum p^2) from sim_reduce."""
        norm, s2_local, _ = N.sim_reduce(self.h)
        return norm, s2_local / (1 << (self.n - self.g))

    def reduce(self):
        """(norm, 2^n sum p^2) over all ranks: each rank's sim_reduce, then one all-reduce."""
        import torch.distributed as dist
        with self.torch.cuda.stream(self.stream):
            v = self.torch.tensor(self.local_reduce(), dtype=self.torch.float64, device=self.bufs[0].device)
            dist.all_reduce(v, group=self.group)
        return float(v[0]), float(v[1]) * (1 << self.n)

    def local_amplitudes(self):
        """This rank's 2^(n-g) amplitudes (complex64, local index order) on the host."""
        return N.sim_amplitudes(self.h, physical_order=True)

    def destroy(self):
        for h in self.hs:
            N.sim_destroy(h)


def gather_logical(shards, n: int, g: int, bit_of) -> np.ndarray:
    """The whole state in logical order from every rank's local amplitudes (rank order): test and
    readout helper for small n."""
    phys = np.concatenate([np.asarray(s) for s in shards])
    idx = np.arange(1 << n, dtype=np.int64)
    logical = np.zeros_like(idx)
    for q in range(n):
        logical |= ((idx >> bit_of[q]) & 1) << q
    out = np.empty_like(phys)
    out[logical] = phys
    return out
