"""Subsystem sharding through the C ABI on one device: two or three shards
of one network (one context each, every context running only its own
CTAs), their windows run one after another, the slots each window wrote
for the other shards packed and unpacked in between
(paper_1903_01081_b300.shard.run_local).  No kernel waits on another
shard's: every value a window reads was unpacked before it started.

Pinned by the decoupling (Sec. II-B: a line end consumes at step n what
the far end sent at step n - d): the merged waveforms are bitwise those of
the whole network in one context, which the other GPU tests hold to the
oracle; the oracle is checked here too.  Plus the protocol's refusals.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g
from paper_1903_01081_b300.shard import Shard, run_local

pytestmark = pytest.mark.gpu
TOL = 1e-10


def base():
    return g.multi_subsystem(77, [4, 5, 3, 6, 4, 5], n_lines=10, n_sources=3, dt=20e-6, n_series_extra=2)


def whole(net, n_steps, options=None):
    ctx = emt.emt_build_network(net)
    for k, v in (options or {}).items():
        emt.emt_set_option(ctx, k, v)
    emt.emt_prefactor(ctx)
    emt.emt_set_recording(ctx, None, 1, n_steps)
    emt.emt_step_n(ctx, n_steps)
    emt.emt_sync(ctx)
    w = emt.emt_read_waveforms(ctx, np.arange(net.n_nodes, dtype=np.int32), 1, n_steps)[:, 0, :]
    emt.emt_destroy(ctx)
    return w


def sharded(net, n_steps, R, **kw):
    shards = [Shard(net, r, R, n_steps=n_steps, **kw) for r in range(R)]
    try:
        run_local(shards, n_steps)
        got = np.zeros((n_steps, net.n_nodes))
        owned = np.zeros(net.n_nodes, int)
        for s in shards:
            s.sync()
            w = s.waveforms(n_steps)
            got[:, s.owned_nodes] = w[:, s.owned_nodes]
            owned += s.owned_nodes
        assert np.all(owned == 1)
        return got, shards[0].window, [len(s.peers) for s in shards]
    finally:
        for s in shards:
            s.close()


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("kind", ["plain", "coupled", "fd", "switched"])
def test_two_shards_are_bitwise_the_whole_network(kind):
    b = base()
    net = {"plain": b, "coupled": g.with_coupled_lines(b, seed=1007), "fd": g.with_fd_lines(b, seed=1009),
           "switched": g.with_rectifier_loads(b, seed=1006, n_rectifiers=4, n_breakers=2)}[kind]
    N = 1500
    got, window, peers = sharded(net, N, 2)
    assert window >= 1 and peers == [1, 1]
    ref = whole(net, N)
    assert np.array_equal(got, ref)
    if kind != "switched":   # (diode decisions near zero crossings: the switched runs' parity is tested elsewhere)
        assert rel(got, oracle.simulate(net, N)) <= TOL


def test_three_shards_and_a_longer_window():
    net = g.with_coupled_lines(base(), seed=1007)
    N = 1200
    got, window, _ = sharded(net, N, 3)
    assert np.array_equal(got, whole(net, N))
    got, window, _ = sharded(net, N, 2, min_window=9)
    assert window >= 9
    assert np.array_equal(got, whole(net, N))


def test_shards_of_the_large_network():
    net = g.large_scale(n_steps=600)
    got, window, peers = sharded(net, 600, 2)
    assert min(peers) >= 1
    assert np.array_equal(got, whole(net, 600))


def test_shards_on_the_warp_per_subsystem_kernel():
    net = base()
    opts = {"warp_per_subsystem": 1}
    got, _, _ = sharded(net, 1000, 2, options=opts)
    ref = whole(net, 1000, opts)
    assert np.array_equal(got, ref)


def test_line_end_export():
    net = g.with_coupled_lines(base(), seed=1007)
    ctx = emt.emt_build_network(net)
    cta, far, d = emt.emt_get_line_ends(ctx)
    node_cta = emt.emt_get_node_ctas(ctx)
    assert cta.size == emt.emt_get_info(ctx, "n_line_ends") > 0
    assert np.array_equal(far[far], np.arange(far.size)) and np.all(far != np.arange(far.size))
    assert np.all(d >= 1) and np.array_equal(d, d[far])
    assert set(cta.tolist()) <= set(node_cta.tolist())
    emt.emt_destroy(ctx)


def test_protocol_refusals():
    net = base()
    s0, s1 = Shard(net, 0, 2, n_steps=400), Shard(net, 1, 2, n_steps=400)
    try:
        W = s0.window
        assert emt.emt_get_info(s0.ctx, "shard_rank") == 0 and emt.emt_get_info(s0.ctx, "shard_window") == W
        assert emt.emt_get_info(s0.ctx, "shard_ctas") + emt.emt_get_info(s1.ctx, "shard_ctas") == \
            emt.emt_get_info(s0.ctx, "n_ctas")
        with pytest.raises(emt.EmtError) as ei:            # longer than the shortest cut line
            s0.step(W + 1)
        assert ei.value.status == emt.EMT_EINVAL
        s0.step(W)
        with pytest.raises(emt.EmtError) as ei:            # the window's values not exchanged yet
            s0.step(1)
        assert ei.value.status == emt.EMT_ESTATE
        out = s0.pack(W)
        with pytest.raises(emt.EmtError) as ei:            # still waiting for rank 1's values
            s0.step(1)
        assert ei.value.status == emt.EMT_ESTATE
        s1.step(W)
        s1.pack(W)
        with pytest.raises(emt.EmtError) as ei:            # a buffer of the wrong size
            emt.emt_shard_unpack(s0.ctx, 1, out[1], out[1].numel() - 16)
        assert ei.value.status == emt.EMT_EINVAL
        s0.unpack(W, {1: s1.pack(W)[0]})
        s0.step(1)                                         # the exchange is complete: the next window runs
        with pytest.raises(emt.EmtError) as ei:
            emt.emt_adjoint(s0.ctx, np.zeros((5, net.n_nodes)), 5)
        assert ei.value.status == emt.EMT_EINVAL
        n_cta = emt.emt_get_info(s0.ctx, "n_ctas")
        with pytest.raises(emt.EmtError) as ei:            # a rank that owns nothing
            emt.emt_set_shard(s0.ctx, np.zeros(n_cta, np.int32), 1)
        assert ei.value.status == emt.EMT_EINVAL
        bad = np.zeros(n_cta, np.int32)
        bad[0] = -1
        with pytest.raises(emt.EmtError):
            emt.emt_set_shard(s0.ctx, bad, 0)
        emt.emt_set_shard(s0.ctx, None, 0)                 # the whole network again
        assert emt.emt_get_info(s0.ctx, "shard_rank") == -1
        emt.emt_reset(s0.ctx)
        emt.emt_step_n(s0.ctx, 3 * W)
        emt.emt_sync(s0.ctx)
    finally:
        s0.close()
        s1.close()


def test_scenario_sets_are_not_sharded():
    net, sc = g.n1_contingency(seed=77, n_scenarios=12, n_buses=40, n_sub=8, n_lines=12, n_sources=3, n_steps=100,
                                fault_step=50, target_branches=240)
    ctx = emt.emt_build_network(net, sc)
    for call in (lambda: emt.emt_set_shard(ctx, np.zeros(emt.emt_get_info(ctx, "n_ctas"), np.int32), 0),
                 lambda: emt.emt_get_line_ends(ctx), lambda: emt.emt_get_node_ctas(ctx)):
        with pytest.raises(emt.EmtError) as ei:
            call()
        assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)
