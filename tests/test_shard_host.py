"""Subsystem sharding on the CPU: the plan (paper_1903_01081_b300.shard) and
the window-by-window exchange of line values, with the oracle as the
engine of every rank.

The run is pinned by the decoupling the method rests on (Sec. II-B: a line
end consumes at step n what the far end sent at step n - d): a network
dealt out to ranks and run window by window, the ranks swapping only the
values their cut line ends sent, gives bitwise the whole network's run.
Covered: plain, coupled three-phase and frequency-dependent lines; two and
three ranks in one process; two ranks over torch.distributed (gloo, world
size 2, 127.0.0.1); and a run whose exchange is left out (a planted
mistake) is far off.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import netgen as g
from paper_1903_01081_b300.shard import plan_shards, run_local, windows

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from oracle_shard import OracleShard  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 700


def base():
    return g.multi_subsystem(77, [4, 5, 3, 6, 4, 5], n_lines=10, n_sources=3, dt=20e-6, n_series_extra=2)


def nets():
    b = base()
    return {"plain": b, "coupled": g.with_coupled_lines(b, seed=1007), "fd": g.with_fd_lines(b, seed=1009)}


def random_graph(seed, n_units=40, n_lines=70):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n_units, n_lines)
    b = (a + rng.integers(1, n_units, n_lines)) % n_units
    d = rng.integers(1, 30, n_lines)
    end_unit = np.stack([a, b], 1).ravel()
    end_far = np.arange(2 * n_lines) ^ 1
    end_d = np.repeat(d, 2)
    return rng.uniform(1, 10, n_units), end_unit, end_far, end_d


@pytest.mark.parametrize("min_window", [1, 8, 15])
def test_plan_cuts_only_lines_of_at_least_the_window(min_window):
    w, eu, ef, ed = random_graph(3)
    for R in (2, 3, 4):
        p = plan_shards(w, eu, ef, ed, R, min_window=min_window)
        r = p.owner[eu]
        cut = r != r[ef]
        assert cut.any()
        assert ed[cut].min() >= min_window and p.window == ed[cut].min()
        assert sorted(set(p.owner.tolist())) == list(range(R))      # every rank runs something
        # the send list of a to b is the receive list of b from a, and covers every cut end
        total = sum(len(p.cut_ends(a, b)) for a in range(R) for b in range(R) if a != b)
        assert total == cut.sum()
        for a in range(R):
            for b in p.peers(a):
                assert a in p.peers(b) and len(p.cut_ends(a, b)) > 0
        again = plan_shards(w, eu, ef, ed, R, min_window=min_window)
        assert np.array_equal(again.owner, p.owner)                  # every rank computes the same plan


def test_plan_balances_equal_units():
    n = 24
    eu = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).ravel()   # a ring of units
    ef = np.arange(2 * n) ^ 1
    p = plan_shards(np.ones(n), eu, ef, np.full(2 * n, 5), 4)
    assert np.bincount(p.owner).tolist() == [6, 6, 6, 6]


def test_plan_owner_override_and_errors():
    w, eu, ef, ed = random_graph(5, n_units=6, n_lines=8)
    own = np.array([0, 1, 0, 1, 0, 1])
    p = plan_shards(w, eu, ef, ed, 2, owner=own)
    assert np.array_equal(p.owner, own)
    with pytest.raises(ValueError):
        plan_shards(w, eu, ef, ed, 2, owner=[0, 1, 2, 0, 1, 0])      # rank out of range
    with pytest.raises(ValueError):
        plan_shards(w, eu, ef, ed, 2, min_window=100)                  # nothing may be cut
    with pytest.raises(ValueError):
        plan_shards(w, eu, ef, ed, 0)
    # no line cut: the window is unbounded
    p = plan_shards(np.ones(2), np.zeros(0, int), np.zeros(0, int), np.zeros(0, int), 2)
    assert p.window == 2 ** 31 - 1 and p.peers(0) == []


def test_windows_cover_the_run():
    assert list(windows(10, 4)) == [4, 4, 2]
    assert list(windows(3, 100)) == [3]
    assert list(windows(0, 4)) == []


def gather(shards, n_nodes):
    got, owned = None, np.zeros(n_nodes, int)
    for s in shards:
        v = s.voltages()
        got = np.zeros_like(v) if got is None else got
        got[:, s.owned_nodes] = v[:, s.owned_nodes]
        owned += s.owned_nodes
    assert np.all(owned == 1)
    return got


@pytest.mark.parametrize("kind", ["plain", "coupled", "fd"])
@pytest.mark.parametrize("R", [2, 3])
def test_sharded_oracle_in_one_process_is_bitwise_the_whole_run(kind, R):
    net = nets()[kind]
    shards = [OracleShard(net, r, R) for r in range(R)]
    assert all(s.peers for s in shards)
    run_local(shards, N)
    assert np.array_equal(gather(shards, net.n_nodes), oracle.simulate(net, N))


def test_longer_windows_cut_fewer_lines_and_still_match():
    net = nets()["coupled"]
    shards = [OracleShard(net, r, 2, min_window=9) for r in range(2)]
    assert shards[0].window >= 9
    run_local(shards, N)
    assert np.array_equal(gather(shards, net.n_nodes), oracle.simulate(net, N))


def test_a_run_without_the_exchange_is_far_off():
    net = nets()["plain"]
    shards = [OracleShard(net, r, 2) for r in range(2)]
    for s in shards:
        s.unpack = lambda w, bufs: None       # the planted mistake: received values dropped
    run_local(shards, N)
    ref = oracle.simulate(net, N)
    assert np.max(np.abs(gather(shards, net.n_nodes) - ref)) > 1e-3 * np.max(np.abs(ref))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("kind,min_window", [("plain", 1), ("coupled", 1), ("fd", 4)])
def test_two_gloo_ranks_reproduce_the_whole_run_bitwise(kind, min_window):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "tests", "shard_gloo_worker.py"), kind, str(N), str(min_window)]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["world"] == 2 and d["peers"] == [1, 1] and d["window"] >= min_window
    assert d["each_node_once"] and min(d["nodes_per_rank"]) > 0
    assert d["bitwise"], d["max_abs_diff"]
