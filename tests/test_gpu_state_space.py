"""The state-space form of the step (emt_ss.cu) through the C ABI: for
networks of small subsystems with the basic elements, each step is one
product [h(n) | v(n)] = M [h(n-1) | v_src(n) | J(n)], M built on the device
from the prefactored G^-1 in double-double arithmetic.

Held to the oracle (relative error <= 1e-10 over whole runs, including a
100,000-step run for drift) and to the CTA kernel of the same network;
stiff (strong) L branches, switch epochs, shards and a resumed run; the
option's values and refusals.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10


def run(net, n_steps, mode, chunks=1):
    ctx = emt.emt_build_network(net)
    emt.emt_set_option(ctx, "state_space", mode)
    emt.emt_prefactor(ctx)
    emt.emt_set_recording(ctx, None, 1, n_steps)
    for k in range(chunks):
        emt.emt_step_n(ctx, n_steps // chunks + (n_steps % chunks if k == chunks - 1 else 0))
    emt.emt_sync(ctx)
    used = emt.emt_get_info(ctx, "state_space")
    w = emt.emt_read_waveforms(ctx, np.arange(net.n_nodes, dtype=np.int32), 1, n_steps)[:, 0, :]
    emt.emt_destroy(ctx)
    return w, used


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def switched():
    net = g.multi_subsystem(131, [3, 6, 2, 5, 4], n_lines=8, n_sources=2, dt=20e-6, n_series_extra=2)
    nodes = np.random.default_rng(4).choice(net.n_nodes, size=2, replace=False)
    net.sw_k = nodes.astype(np.int32)
    net.sw_m = np.array([-1, int(nodes[0])], np.int32)
    net.sw_r = np.array([0.05, 1.5])
    net.sw_close_step = np.array([300, 500], np.int64)
    net.sw_open_step = np.array([-1, 900], np.int64)
    return net


def stiff():
    """Two sources feeding a ladder through a stiff 0.1 uH link (companion
    conductance 100 S against ~0.1 S around it): a strong branch."""
    b = g.NetworkBuilder()
    b.source(1000.0, 0.3)
    b.source(800.0, -1.1, 50.0)
    b.branch(g.source_node(0), 0, g.KIND_R, 2.0)
    b.branch(0, 1, g.KIND_L, 1e-7)
    b.branch(1, 2, g.KIND_R, 10.0)
    b.branch(2, g.GROUND, g.KIND_C, 20e-6)
    b.branch(1, g.GROUND, g.KIND_R, 50.0)
    b.branch(2, 3, g.KIND_L, 0.02)
    b.branch(3, g.GROUND, g.KIND_R, 30.0)
    b.branch(g.source_node(1), 3, g.KIND_L, 0.01)
    return b.build(20e-6, 4, 6000)


@pytest.mark.parametrize("kind", ["config1", "switched", "strict_500x6", "stiff"])
def test_matches_the_oracle_and_the_cta_kernel(kind):
    net, N = {"config1": (g.single_rlc(), 20000), "switched": (switched(), 3000),
              "strict_500x6": (g.large_scale(strict_500=True, n_steps=2000), 2000), "stiff": (stiff(), 6000)}[kind]
    got, used = run(net, N, 1)
    assert used == 1
    cta, used0 = run(net, N, 0)
    assert used0 == 0
    ref = oracle.simulate(net, N)
    assert rel(got, ref) <= TOL
    assert rel(got, cta) <= TOL


def test_the_stiff_link_is_a_strong_branch():
    ctx = emt.emt_build_network(stiff())
    assert emt.emt_get_info(ctx, "n_strong_branches") >= 1
    emt.emt_destroy(ctx)


def test_no_drift_over_a_long_run():
    net = g.single_rlc(n_steps=100000)
    got, used = run(net, 100000, 1)
    assert used == 1
    assert rel(got, oracle.simulate(net, 100000)) <= TOL


def test_resumed_run_is_bitwise_the_single_launch():
    net = switched()
    one, _ = run(net, 2000, 2)
    four, _ = run(net, 2000, 2, chunks=4)
    assert np.array_equal(one, four)


def test_option_values_and_refusals():
    net = g.single_rlc(n_steps=10)
    ctx = emt.emt_build_network(net)
    for bad in (-1, 3):
        with pytest.raises(emt.EmtError) as ei:
            emt.emt_set_option(ctx, "state_space", bad)
        assert ei.value.status == emt.EMT_EINVAL
    emt.emt_set_option(ctx, "state_space", 2)
    emt.emt_prefactor(ctx)
    assert emt.emt_get_info(ctx, "state_space") == 1
    emt.emt_set_option(ctx, "warp_per_subsystem", 1)     # the explicit choice wins
    assert emt.emt_get_info(ctx, "state_space") == 0
    emt.emt_destroy(ctx)
    # runtime switches are outside the state-space form
    ctl = g.with_rectifier_loads(g.multi_subsystem(77, [4, 5, 3], n_lines=4, n_sources=2, dt=20e-6),
                                 seed=1006, n_rectifiers=2, n_breakers=1)
    ctx = emt.emt_build_network(ctl)
    assert emt.emt_get_info(ctx, "state_space") == 0
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_set_option(ctx, "state_space", 2)
    assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)
