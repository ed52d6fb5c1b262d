"""GPU parity of the control blocks (layered control components driving
controlled current injections) against the oracle: node voltages every
step and the block outputs of the last step."""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def gpu_run(net, N, chunks=None):
    sim = emt.Simulator(net, n_steps=N)
    for c in (chunks or [N]):
        sim.run(c)
    sim.sync()
    w = sim.waveforms()[:, 0, :]
    y = sim.controls()
    sim.close()
    return w, y


def check(net, N, chunks=None, tol=TOL):
    w, y = gpu_run(net, N, chunks)
    ref = oracle.simulate(net, N)
    yr = oracle.controls(net, N)[-1]
    assert rel(w, ref) <= tol
    assert np.max(np.abs(y - yr)) <= 1e-9 * max(np.max(np.abs(yr)), 1e-300)
    return w, y


def test_converters_large_scale():
    net = g.with_converter_controls(g.large_scale(n_steps=3000))
    sim = emt.Simulator(net, n_steps=1)
    assert sim.info("n_control_blocks") == 180 * 24
    assert sim.info("n_control_injections") == 180 * 3
    assert sim.info("max_control_layers") == 11
    sim.close()
    w, y = check(net, 3000)
    assert np.max(np.abs(y[21::24])) > 1.0      # the converters draw current


def test_converters_large_scale_full_length():
    net = g.with_converter_controls(g.large_scale())
    check(net, net.n_steps)


def test_resume_across_launches_is_bitwise():
    net = g.with_converter_controls(g.multi_subsystem(11, [4, 5, 3, 6], n_lines=5, n_sources=3, dt=20e-6),
                                    n_converters=7)
    a, ya = gpu_run(net, 2500)
    b, yb = gpu_run(net, 2500, chunks=[1000, 1, 777, 722])
    assert np.array_equal(a, b) and np.array_equal(ya, yb)
    check(net, 2500)


def test_reset_reproduces():
    net = g.with_converter_controls(g.multi_subsystem(12, [5, 4], n_lines=2, n_sources=2, dt=20e-6), n_converters=3)
    sim = emt.Simulator(net, n_steps=800)
    sim.run(800)
    w1, y1 = sim.waveforms()[:, 0, :].copy(), sim.controls().copy()
    sim.reset()
    sim.run(800)
    w2, y2 = sim.waveforms()[:, 0, :], sim.controls()
    sim.close()
    assert np.array_equal(w1, w2) and np.array_equal(y1, y2)


def test_loop_breaking_and_injection_small():
    """Both block orders of a self-referencing sum, an integrator, a lag and
    a PI, and a proportional current injection, in one subsystem."""
    b = g.NetworkBuilder()
    b.source(1000.0, 0.4, 60.0)
    b.branch(g.source_node(0), 0, g.KIND_R, 2.0)
    b.branch(0, g.GROUND, g.KIND_R, 5.0)
    b.branch(0, 1, g.KIND_L, 0.02)
    b.branch(1, g.GROUND, g.KIND_C, 50e-6)
    s = b.block(g.CB_SUM, 1, 0, p0=1.0, p1=0.5)
    b.block(g.CB_CONST, p0=1.0)
    c = b.block(g.CB_CONST, p0=2.0)
    b.block(g.CB_SUM, c, c + 1, p0=1.0, p1=0.5)
    m = b.block(g.CB_MEAS, node=1)
    b.block(g.CB_INTEG, m, p0=3.0)
    b.block(g.CB_LAG, m, p0=0.5, p1=1e-3)
    pi = b.block(g.CB_PI, m, p0=-0.01, p1=-1.0)
    lim = b.block(g.CB_LIMIT, pi, p0=-20.0, p1=20.0)
    b.injection(lim, 1)
    b.injection(s, 0)
    net = b.build(50e-6, 2)
    check(net, 4000)


def test_wide_and_deep_graphs():
    """A layer of 70 blocks (more than one warp's lanes) and a chain of 60
    layers; a block group that touches no node (runs in subsystem 0)."""
    base = g.multi_subsystem(13, [6, 6, 6], n_lines=3, n_sources=2, dt=20e-6)
    b = g.NetworkBuilder()
    buses = base.meta["bus_nodes"]
    nodes = [x for bus in buses for x in bus]
    sub, _ = oracle.partition(base)
    same = [x for x in nodes if sub[x] == sub[nodes[0]]][:18]
    meas = [b.block(g.CB_MEAS, node=x) for x in (same * 4)[:70]]
    acc = meas[0]
    for i in range(1, 60):
        acc = b.block(g.CB_SUM, acc, meas[i % 70], p0=0.9, p1=0.001)
    b.injection(acc, same[0])
    k = b.block(g.CB_CONST, p0=0.25)
    b.block(g.CB_INTEG, k, p0=1.0)
    ctl = b.build(base.dt, 0)
    net = base.copy()
    for f in ("cb_type", "cb_in0", "cb_in1", "cb_node", "cb_p0", "cb_p1", "ci_block", "ci_node"):
        setattr(net, f, getattr(ctl, f))
    sim = emt.Simulator(net, n_steps=1)
    assert sim.info("max_control_layers") == 60
    sim.close()
    check(net, 3000)


def test_adjoint_rejects_controls():
    net = g.with_converter_controls(g.multi_subsystem(12, [5, 4], n_lines=2, n_sources=2, dt=20e-6), n_converters=2)
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    with pytest.raises(emt.EmtError, match="control blocks have no adjoint"):
        emt.emt_adjoint(ctx, np.zeros((10, net.n_nodes)), 10)
    emt.emt_destroy(ctx)


def test_scenario_set_with_controls():
    """A multi-scenario study with control blocks (40 converter loads on the
    600-node network; per scenario the converters' power set points and a
    fault resistance): sampled scenarios against the oracle, each written
    out as a plain network with its set points; scenarios differ; the block
    outputs are not readable per context."""
    net, sc = g.converter_study(n_scenarios=48, n_steps=3000)
    N = 3000
    sim = emt.Simulator(net, sc, n_steps=N)
    sim.run(N)
    sim.sync()
    w = sim.waveforms()
    with pytest.raises(emt.EmtError, match="per scenario"):
        sim.controls()
    sim.close()
    for s in (0, 13, 47):
        assert rel(w[:, s, :], oracle.simulate(sc.expand(net, s), N)) <= TOL
    assert rel(w[:, 13, :], w[:, 47, :]) > 1e-6


def test_scenario_set_with_controls_resume_and_one_scenario():
    """The same study in two launches equals one launch bit for bit, and a
    set of one scenario matches the single-network kernel on that scenario."""
    net, sc = g.converter_study(n_scenarios=8, n_steps=2000)
    N = 2000
    a = emt.Simulator(net, sc, n_steps=N)
    a.run(N)
    a.sync()
    b = emt.Simulator(net, sc, n_steps=N)
    b.run(700)
    b.run(N - 700)
    b.sync()
    assert np.array_equal(a.waveforms(), b.waveforms())
    a.close()
    b.close()
    one = sc.subset([5])
    c = emt.Simulator(net, one, n_steps=N)
    c.run(N)
    c.sync()
    single = gpu_run(one.expand(net, 0), N)[0]
    assert rel(c.waveforms()[:, 0, :], single) <= TOL
    c.close()
