"""One network over several ranks (one device each): subsystem sharding.

Subsystems meet only through transmission lines, and the value a line end
sends at step n is consumed at the far end at step n + d, d the line's
travel time in whole steps (Sec. II-B: the line decouples its two ends; the
paper scales out by running independent work on many devices, Sec. IV-D).
So the subsystems can be dealt out to ranks, cutting only lines:

* plan_shards: groups the units (CTAs of the library, subsystems of any
  other engine) that lines shorter than ``min_window`` steps join, deals the
  groups to ranks (heaviest first, to the lightest rank, preferring the rank
  it shares most cut lines with among equally loaded ones), and sets the
  window D = the shortest cut line;
* a window of w <= D steps reads only values sent before it began, so every
  rank runs it alone; between windows each rank sends each neighbour the
  values its cut line ends sent during the window (point to point, one
  message per neighbour and window, no collective) and writes what it
  receives into its own copy of the rings.

The exchange is engine-agnostic: an engine has ``rank``, ``peers``,
``window``, ``step(w)``, ``pack(w) -> {peer: tensor}``,
``recv_buffers(w) -> {peer: tensor}`` and ``unpack(w, {peer: tensor})``.
``Shard`` is the CUDA engine (through the C ABI); ``run_local`` runs all
ranks' shards in one process (one device, windows one after another: no
kernel waits on another rank's), ``run_distributed`` one shard per process
over torch.distributed (NCCL between devices, gloo on CPU).
"""
from __future__ import annotations

from typing import Dict, List, Optional

import numpy as np

from . import emt


class ShardPlan:
    """Owner rank of every unit, the window, and the cut line ends."""

    def __init__(self, owner, window: int, n_ranks: int, end_unit, end_far):
        self.owner = np.asarray(owner, dtype=np.int32)
        self.window = int(window)
        self.n_ranks = int(n_ranks)
        self.end_unit = np.asarray(end_unit, dtype=np.int64)
        self.end_far = np.asarray(end_far, dtype=np.int64)
        self._end_rank = self.owner[self.end_unit] if self.end_unit.size else np.zeros(0, np.int32)

    def cut_ends(self, src: int, dst: int) -> np.ndarray:
        """Line ends run at rank src whose far end runs at rank dst, ascending:
        what src sends dst after every window."""
        if self.end_unit.size == 0:
            return np.zeros(0, np.int64)
        r = self._end_rank
        return np.nonzero((r == src) & (r[self.end_far] == dst))[0]

    def peers(self, rank: int) -> List[int]:
        """Ranks that share a cut line with ``rank``."""
        if self.end_unit.size == 0:
            return []
        r = self._end_rank
        mine = r == rank
        other = r[self.end_far]
        return sorted(set(other[mine & (other != rank)].tolist()))


def plan_shards(unit_weight, end_unit, end_far, end_d, n_ranks: int, min_window: int = 1,
                owner=None) -> ShardPlan:
    """Deal units to ``n_ranks`` ranks cutting only line ends of at least
    ``min_window`` steps (see the module docstring); ``owner`` (per unit)
    overrides the dealing.  Deterministic: every rank computes the same plan."""
    w = np.asarray(unit_weight, dtype=np.float64)
    n_units = w.size
    end_unit = np.asarray(end_unit, dtype=np.int64)
    end_far = np.asarray(end_far, dtype=np.int64)
    end_d = np.asarray(end_d, dtype=np.int64)
    if n_ranks < 1:
        raise ValueError("n_ranks must be at least 1")
    if min_window < 1:
        raise ValueError("min_window must be at least 1")
    if owner is None:
        parent = list(range(n_units))

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        for e in range(end_unit.size):   # lines too short to cut keep their two sides together
            if end_d[e] < min_window:
                a, b = find(int(end_unit[e])), find(int(end_unit[end_far[e]]))
                if a != b:
                    parent[max(a, b)] = min(a, b)
        root = np.array([find(u) for u in range(n_units)], dtype=np.int64)
        groups = sorted(set(root.tolist()))
        if len(groups) < n_ranks:
            raise ValueError(f"{len(groups)} groups of subsystems joined by lines shorter than {min_window} "
                             f"steps: too few for {n_ranks} ranks")
        gw = {g: float(w[root == g].sum()) for g in groups}
        # line ends between groups, for the affinity tie-break
        link: Dict[int, Dict[int, int]] = {g: {} for g in groups}
        for e in range(end_unit.size):
            a, b = int(root[end_unit[e]]), int(root[end_unit[end_far[e]]])
            if a != b:
                link[a][b] = link[a].get(b, 0) + 1
        load = np.zeros(n_ranks)
        grp_rank: Dict[int, int] = {}
        for g in sorted(groups, key=lambda g: (-gw[g], g)):
            empty = [r for r in range(n_ranks) if load[r] == 0]
            if empty:                      # every rank gets a group first
                best = empty[0]
            else:
                lo = load.min()
                cand = [r for r in range(n_ranks) if load[r] <= lo * (1 + 1e-9) + 1e-12]
                best = max(cand, key=lambda r: (sum(c for h, c in link[g].items() if grp_rank.get(h) == r), -r))
            grp_rank[g] = best
            load[best] += gw[g]
        owner = np.array([grp_rank[int(root[u])] for u in range(n_units)], dtype=np.int32)
    owner = np.asarray(owner, dtype=np.int32)
    if owner.size != n_units or (owner.size and (owner.min() < 0 or owner.max() >= n_ranks)):
        raise ValueError("owner needs one rank in [0, n_ranks) per unit")
    cut = owner[end_unit] != owner[end_unit[end_far]] if end_unit.size else np.zeros(0, bool)
    window = int(end_d[cut].min()) if cut.any() else 2 ** 31 - 1
    return ShardPlan(owner, window, n_ranks, end_unit, end_far)


def windows(n_steps: int, window: int):
    """The window lengths that cover n_steps steps."""
    done = 0
    while done < n_steps:
        w = min(window, n_steps - done)
        yield w
        done += w


# ------------------------------------------------------------------ CUDA engine

class Shard:
    """This rank's part of a network on the current CUDA device: a context of
    the whole network (so that CTAs and line ends are numbered as on every
    other rank) that runs only the CTAs the plan gives this rank."""

    SLOT_BYTES = 16   # one ring slot: tag and value words

    def __init__(self, net, rank: int, n_ranks: int, min_window: int = 1, owner=None, record: bool = True,
                 n_steps: Optional[int] = None, options: Optional[dict] = None):
        import torch
        self.rank, self.n_ranks = int(rank), int(n_ranks)
        self.net = net
        self.ctx = emt.emt_build_network(net)
        for k, v in (options or {}).items():
            emt.emt_set_option(self.ctx, k, v)
        emt.emt_prefactor(self.ctx)
        if record:
            emt.emt_set_recording(self.ctx, None, 1, int(n_steps if n_steps is not None else net.n_steps))
        self.node_cta = emt.emt_get_node_ctas(self.ctx)
        n_cta = emt.emt_get_info(self.ctx, "n_ctas")
        size = np.bincount(self.node_cta, minlength=n_cta).astype(np.float64)
        end_cta, end_far, end_d = emt.emt_get_line_ends(self.ctx)
        # a CTA's step costs about its solve (n^2) plus a fixed part
        self.plan = plan_shards(size ** 2 + 64.0, end_cta, end_far, end_d, self.n_ranks, min_window, owner)
        emt.emt_set_shard(self.ctx, self.plan.owner, self.rank)
        self.window = emt.emt_get_info(self.ctx, "shard_window")
        self.peers = self.plan.peers(self.rank)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        wmax = min(self.window, int(n_steps if n_steps is not None else net.n_steps))
        self._send = {p: torch.empty(self.SLOT_BYTES * len(self.plan.cut_ends(self.rank, p)) * wmax,
                                     dtype=torch.uint8, device=self.dev) for p in self.peers}
        self._recv = {p: torch.empty(self.SLOT_BYTES * len(self.plan.cut_ends(p, self.rank)) * wmax,
                                     dtype=torch.uint8, device=self.dev) for p in self.peers}
        self.owned_nodes = self.plan.owner[self.node_cta] == self.rank

    def _stream(self):
        import torch
        return torch.cuda.current_stream(self.dev)

    def _grow(self, bufs, p, nbytes):
        import torch
        if bufs[p].numel() < nbytes:
            bufs[p] = torch.empty(nbytes, dtype=torch.uint8, device=self.dev)
        return bufs[p][:nbytes]

    def step(self, w: int) -> None:
        emt.emt_step_n(self.ctx, int(w), self._stream())

    def pack(self, w: int) -> Dict[int, "object"]:
        out = {}
        for p in self.peers:
            nbytes = self.SLOT_BYTES * len(self.plan.cut_ends(self.rank, p)) * int(w)
            buf = self._grow(self._send, p, nbytes)
            emt.emt_shard_pack(self.ctx, p, buf, self._stream())
            out[p] = buf
        return out

    def recv_buffers(self, w: int) -> Dict[int, "object"]:
        return {p: self._grow(self._recv, p, self.SLOT_BYTES * len(self.plan.cut_ends(p, self.rank)) * int(w))
                for p in self.peers}

    def unpack(self, w: int, bufs) -> None:
        for p in self.peers:
            emt.emt_shard_unpack(self.ctx, p, bufs[p], bufs[p].numel(), self._stream())

    def waveforms(self, n_rows: Optional[int] = None):
        """Recorded node voltages [rows, n_nodes]; only this rank's nodes
        (``owned_nodes``) are meaningful."""
        n_rows = emt.emt_get_info(self.ctx, "step") if n_rows is None else n_rows
        return emt.emt_read_waveforms(self.ctx, np.arange(self.net.n_nodes, dtype=np.int32), 1, n_rows)[:, 0, :]

    def sync(self):
        return emt.emt_sync(self.ctx)

    def close(self):
        emt.emt_destroy(self.ctx)


# ------------------------------------------------------------------ runners

def run_local(shards, n_steps: int) -> None:
    """All ranks' shards in this process: each window runs on every shard in
    turn, then every shard's sent values go straight into its neighbours'
    buffers (no transport)."""
    by_rank = {s.rank: s for s in shards}
    window = min(s.window for s in shards)
    for w in windows(int(n_steps), window):
        for s in shards:
            s.step(w)
        sent = {s.rank: s.pack(w) for s in shards}
        for s in shards:
            inbox = s.recv_buffers(w)
            for p in s.peers:
                src = sent[p][s.rank] if p in by_rank else None
                if src is None:
                    raise ValueError(f"rank {p} is not among the local shards")
                inbox[p].copy_(src)
            s.unpack(w, inbox)


def run_distributed(engine, n_steps: int, group=None) -> None:
    """One shard per process: after every window, one point-to-point message
    each way per neighbouring rank (torch.distributed isend/irecv)."""
    import torch.distributed as dist
    for w in windows(int(n_steps), int(engine.window)):
        engine.step(w)
        out = engine.pack(w)
        inbox = engine.recv_buffers(w)
        ops = []
        for p in engine.peers:
            ops.append(dist.P2POp(dist.isend, out[p], p, group))
            ops.append(dist.P2POp(dist.irecv, inbox[p], p, group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        engine.unpack(w, inbox)
