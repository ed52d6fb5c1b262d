"""GPU parity of coupled three-phase lines (modal Bergeron, interpolated
non-integer travel times) against the oracle, whose line model is pinned
in tests/test_oracle_coupled_lines.py."""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10
DT = 2.0 ** -16


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def gpu_run(net, N, chunks=(None,)):
    sim = emt.Simulator(net, n_steps=N)
    done = 0
    for c in chunks:
        k = N - done if c is None else c
        sim.run(k)
        done += k
    sim.sync()
    w = sim.waveforms()[:, 0, :]
    sim.close()
    return w


def loaded_line(tv, z, tau):
    b = g.NetworkBuilder()
    for p, amp in enumerate((1000.0, 600.0, 1400.0)):
        b.source(amp, 0.2 - 2 * np.pi * p / 3, 60.0)
        b.branch(g.source_node(p), p, 0, 40.0)
        b.branch(p, g.GROUND, 2, 3e-6)
        b.branch(3 + p, g.GROUND, 0, 700.0 + 100 * p)
        b.branch(3 + p, g.GROUND, 1, 0.2)
    b.branch(0, 1, 0, 1500.0)
    b.branch(4, 5, 0, 1500.0)
    b.coupled_line([0, 1, 2], [3, 4, 5], tv, z, tau)
    return b.build(DT, 6, 4000)


@pytest.mark.parametrize("tv,z,steps", [
    (np.eye(3), (400.0, 300.0, 250.0), (3.0, 5.0, 7.0)),
    (np.eye(3), (400.0, 300.0, 250.0), (1.0, 2.5, 9.875)),
    (g.CLARKE, (600.0, 300.0, 300.0), (7.3, 5.6, 5.6)),
    (np.array([[1.0, 0.2, 0.1], [0.3, 1.1, -0.2], [0.1, -0.4, 0.9]]), (500.0, 320.0, 280.0), (4.2, 3.7, 6.05)),
])
def test_single_coupled_line(tv, z, steps):
    net = loaded_line(tv, z, [s * DT for s in steps])
    N = 4000
    assert rel(gpu_run(net, N), oracle.simulate(net, N)) <= TOL


def test_multi_subsystem_with_coupled_lines_resumable():
    base = g.multi_subsystem(161, [3, 4, 2, 3, 5], n_lines=8, n_sources=2, dt=20e-6)
    net = g.with_coupled_lines(base, seed=3)
    N = 3000
    ref = oracle.simulate(net, N)
    one = gpu_run(net, N)
    assert rel(one, ref) <= TOL
    split = gpu_run(net, N, chunks=(777, 1111, None))   # interpolation state carried across launches
    assert np.array_equal(split, one)


def test_large_network_with_coupled_lines():
    net = g.with_coupled_lines(g.large_scale())
    N = 5000
    assert rel(gpu_run(net, N), oracle.simulate(net, N)) <= TOL


def test_coupled_lines_count_and_invalid_travel_time():
    base = g.multi_subsystem(161, [3, 4, 2], n_lines=3, n_sources=2, dt=20e-6)
    net = g.with_coupled_lines(base, seed=3)
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    assert emt.emt_get_info(ctx, "n_coupled_lines") == 3   # three three-phase lines
    emt.emt_destroy(ctx)
    bad = net.copy()
    bad.cl_tau = bad.cl_tau.copy()
    bad.cl_tau[0] = 0.5 * net.dt
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_build_network(bad)
    assert ei.value.status == emt.EMT_EINVAL


def test_scenario_set_with_coupled_lines():
    """A study on the 600-node network with its three-phase lines as coupled
    modal lines with interpolated travel times (per scenario the source
    amplitudes and angles and a fault resistance): sampled scenarios against
    the oracle; two launches equal one bit for bit."""
    N = 3000
    base, _ = g.n1_contingency(n_scenarios=1, n_steps=N)
    net, sc = g.shared_g(n_scenarios=24, n_steps=N, fault_step=1500, base=g.with_coupled_lines(base))
    assert net.n_coupled_lines > 0 and net.n_lines == 0
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
