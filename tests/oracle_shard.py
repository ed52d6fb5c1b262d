"""The oracle as a shard engine (for the exchange tests of
paper_1903_01081_b300.shard): one rank's subsystems run in an oracle
session, and the line values its cut ends sent during a window are read
from, and the peers' written into, the session's line storage."""
import numpy as np
import torch

import oracle
from paper_1903_01081_b300.shard import plan_shards


class OracleShard:
    def __init__(self, net, rank: int, n_ranks: int, min_window: int = 1, owner=None):
        self.rank = int(rank)
        self.sess = oracle.Session(net)
        sub, n_sub = oracle.partition(net)
        node, far, d = oracle.line_ends(net)
        weight = np.bincount(sub, minlength=n_sub).astype(np.float64) ** 2 + 64.0
        self.plan = plan_shards(weight, sub[node] if node.size else node, far, d, n_ranks, min_window, owner)
        self.active = (self.plan.owner == self.rank).astype(np.uint8)
        self.owned_nodes = self.plan.owner[sub] == self.rank
        self.window = self.plan.window
        self.peers = self.plan.peers(self.rank)
        self.rows = []
        self.n0 = 1

    def step(self, w):
        self.n0 = self.sess.step + 1
        self.rows.append(self.sess.advance(w, self.active))

    def pack(self, w):
        out = {}
        for p in self.peers:
            ends = self.plan.cut_ends(self.rank, p)
            vals = [self.sess.sent(int(e), self.n0, w) for e in ends]
            out[p] = torch.from_numpy(np.concatenate(vals) if vals else np.zeros(0))
        return out

    def recv_buffers(self, w):
        return {p: torch.zeros(len(self.plan.cut_ends(p, self.rank)) * w, dtype=torch.float64) for p in self.peers}

    def unpack(self, w, bufs):
        for p in self.peers:
            vals = bufs[p].numpy().reshape(-1, w)
            for i, e in enumerate(self.plan.cut_ends(p, self.rank)):
                self.sess.set_sent(int(e), self.n0, vals[i])

    def voltages(self):
        return np.concatenate(self.rows) if self.rows else np.zeros((0, len(self.owned_nodes)))
