"""GPU parity of frequency-dependent lines (pole-residue Y_c and propagation
function, trapezoidal recursive convolution, interpolated travel time)
against the oracle."""
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
    sim.close()
    return w


def test_large_scale_lossy_lines():
    net = g.with_fd_lines(g.large_scale(n_steps=3000))
    sim = emt.Simulator(net, n_steps=1)
    assert sim.info("n_fd_lines") == 2100
    sim.close()
    assert rel(gpu_run(net, 3000), oracle.simulate(net, 3000)) <= TOL


def test_large_scale_lossy_lines_full_length():
    net = g.with_fd_lines(g.large_scale())
    N = net.n_steps
    assert rel(gpu_run(net, N), oracle.simulate(net, N)) <= TOL


def small_network():
    dt = 2.0 ** -16
    b = g.NetworkBuilder()
    b.source(1000.0, 0.3, 60.0)
    b.branch(g.source_node(0), 0, g.KIND_R, 5.0)
    b.branch(0, g.GROUND, g.KIND_C, 20e-6)
    b.branch(0, g.GROUND, g.KIND_R, 200.0)
    b.branch(1, g.GROUND, g.KIND_R, 150.0)
    b.branch(1, g.GROUND, g.KIND_L, 0.05)
    b.branch(2, g.GROUND, g.KIND_R, 90.0)
    b.branch(2, g.GROUND, g.KIND_C, 40e-6)
    b.fd_line(0, 1, 37.3 * dt, 1 / 320.0, yq=[-4e3, -6e4], yc=[0.3e3 / 320, 5e3 / 320],
              a0=0.2, ap=[-5e3, -8e4], ar=[0.6 * 5e3, 0.1 * 8e4])
    b.fd_line(1, 2, 12.0 * dt, 1 / 410.0, yq=[-2e4], yc=[3e3 / 410], a0=0.0, ap=[-3e4], ar=[0.9 * 3e4])
    b.fd_line(2, 0, 1.0 * dt, 1 / 250.0, a0=1.0)                   # lossless, shortest travel time
    b.fd_line(1, 0, 3.5 * dt, 1 / 300.0, yq=[-1e4] * 4, yc=[1.0, 2.0, 3.0, 4.0], a0=0.1,
              ap=[-1e4, -2e4, -4e4, -8e4], ar=[1e3, 2e3, 4e3, 8e3])   # four poles each
    return b.build(dt, 3)


def test_small_network_all_pole_counts():
    net = small_network()
    assert rel(gpu_run(net, 6000), oracle.simulate(net, 6000)) <= TOL


def test_resume_across_launches_is_bitwise():
    net = g.with_fd_lines(g.multi_subsystem(21, [4, 5, 3, 6], n_lines=6, n_sources=3, dt=20e-6))
    a = gpu_run(net, 2500)
    b = gpu_run(net, 2500, chunks=[1000, 0, 1, 777, 0, 722])
    assert np.array_equal(a, b)
    assert rel(a, oracle.simulate(net, 2500)) <= TOL


def test_reset_reproduces():
    net = g.with_fd_lines(g.multi_subsystem(22, [5, 4], n_lines=2, n_sources=2, dt=20e-6))
    sim = emt.Simulator(net, n_steps=900)
    sim.run(900)
    w1 = sim.waveforms()[:, 0, :].copy()
    sim.reset()
    sim.run(900)
    w2 = sim.waveforms()[:, 0, :]
    sim.close()
    assert np.array_equal(w1, w2)


def test_adjoint_rejects_fd_lines():
    net = g.with_fd_lines(g.multi_subsystem(22, [5, 4], n_lines=2, n_sources=2, dt=20e-6))
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    with pytest.raises(emt.EmtError, match="frequency-dependent lines have no adjoint"):
        emt.emt_adjoint(ctx, np.zeros((10, net.n_nodes)), 10)
    emt.emt_destroy(ctx)


def test_scenario_set_with_fd_lines():
    """A study on the 600-node network with its lines frequency-dependent
    (per scenario the source amplitudes and angles and a fault resistance):
    sampled scenarios against the oracle, each written out as a plain
    network; two launches equal one bit for bit."""
    N = 3000
    base, _ = g.n1_contingency(n_scenarios=1, n_steps=N)
    net, sc = g.shared_g(n_scenarios=24, n_steps=N, fault_step=1500, base=g.with_fd_lines(base))
    assert net.n_fd_lines > 0 and net.n_lines == 0
    sim = emt.Simulator(net, sc, n_steps=N)
    sim.run(N)
    sim.sync()
    w = sim.waveforms()
    sim.close()
    for s in (0, 11, 23):
        ref = oracle.simulate(sc.expand(net, s), N)
        assert np.max(np.abs(w[:, s, :] - ref)) <= 1e-10 * np.max(np.abs(ref))
    two = emt.Simulator(net, sc, n_steps=N)
    two.run(1234)
    two.run(N - 1234)
    two.sync()
    assert np.array_equal(two.waveforms(), w)
    two.close()
