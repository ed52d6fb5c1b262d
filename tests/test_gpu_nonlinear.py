"""GPU parity of nonlinear resistors solved by the compensation method
(odd piecewise-linear surge-arrester characteristics) against the oracle."""
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


def test_arresters_large_scale():
    net = g.with_arresters(g.large_scale(n_steps=3000))
    sim = emt.Simulator(net, n_steps=1)
    assert sim.info("n_nonlinear") == 40
    sim.close()
    ref = oracle.simulate(net, 3000)
    assert rel(gpu_run(net, 3000), ref) <= TOL
    assert np.max(np.abs(ref[:, net.nl_k])) > g.ARRESTER_V[0]        # some arresters conduct


def test_arresters_large_scale_full_length():
    net = g.with_arresters(g.large_scale())
    assert rel(gpu_run(net, net.n_steps), oracle.simulate(net, net.n_steps)) <= TOL


def test_resistive_circuit_past_the_last_point():
    b = g.NetworkBuilder()
    b.source(20000.0, 0.2, 60.0)
    b.branch(g.source_node(0), 0, g.KIND_R, 2.0)
    b.branch(0, g.GROUND, g.KIND_R, 50.0)
    b.nonlinear_resistor(0, g.GROUND, g.ARRESTER_V, g.ARRESTER_I)
    b.branch(0, 1, g.KIND_L, 0.01)                       # a second node and a dynamic element
    b.branch(1, g.GROUND, g.KIND_C, 30e-6)
    net = b.build(20e-6, 2)
    ref = oracle.simulate(net, 2500)
    assert np.max(np.abs(ref[:, 0])) > g.ARRESTER_V[-1]
    assert rel(gpu_run(net, 2500), ref) <= TOL


def test_node_to_node_element_with_switching():
    """An element between two unknown nodes, in a subsystem whose matrix
    changes with a scheduled switch and a diode (its column follows)."""
    b = g.NetworkBuilder()
    b.source(1500.0, 0.3, 60.0)
    b.branch(g.source_node(0), 0, g.KIND_R, 1.0)
    b.branch(0, 1, g.KIND_L, 0.02)
    b.branch(1, g.GROUND, g.KIND_R, 40.0)
    b.branch(0, g.GROUND, g.KIND_C, 20e-6)
    b.nonlinear_resistor(0, 1, [300.0, 600.0, 900.0], [0.1, 50.0, 400.0])
    b.switch(1, g.GROUND, 2.0, 700, 1600)
    b.diode(1, 2, 0.01, 1e6)
    b.branch(2, g.GROUND, g.KIND_R, 30.0)
    b.branch(2, g.GROUND, g.KIND_C, 50e-6)
    net = b.build(20e-6, 3)
    ref = oracle.simulate(net, 3000)
    a = gpu_run(net, 3000)
    bb = gpu_run(net, 3000, chunks=[650, 1, 1000, 1349])
    assert np.array_equal(a, bb)
    assert rel(a, ref) <= TOL


def test_adjoint_rejects_nonlinear():
    net = g.with_arresters(g.multi_subsystem(41, [4, 5, 3], n_lines=4, n_sources=2, dt=20e-6), n_arresters=1)
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    with pytest.raises(emt.EmtError, match="nonlinear resistors have no adjoint"):
        emt.emt_adjoint(ctx, np.zeros((10, net.n_nodes)), 10)
    emt.emt_destroy(ctx)


def test_scenario_set_with_arresters():
    """Surge arresters in an N-1 study (compensation per scenario against the
    scenario's own solve matrix): sampled scenarios against the oracle, each
    written out as a plain network; the arresters conduct; two launches
    equal one bit for bit."""
    base, sc = g.n1_contingency(n_scenarios=32, n_steps=3000)
    net = g.with_arresters(base, n_arresters=20)
    N = 3000
    sim = emt.Simulator(net, sc, n_steps=N)
    sim.run(N)
    sim.sync()
    w = sim.waveforms()
    sim.close()
    for s in (0, 9, 31):
        assert rel(w[:, s, :], oracle.simulate(sc.expand(net, s), N)) <= TOL
    knee = min(g.ARRESTER_V) * 0.9
    assert np.max(np.abs(w[:, :, np.asarray(net.nl_k)])) > knee
    two = emt.Simulator(net, sc, n_steps=N)
    two.run(1100)
    two.run(N - 1100)
    two.sync()
    assert np.array_equal(two.waveforms(), w)
    two.close()


def test_three_arresters_in_one_subsystem():
    """Arresters on all three phases of a source bus (their knees low enough
    to conduct): the three elements are solved together through their
    Thevenin matrix, against the oracle's piecewise-linear Newton iteration
    on the nodal equations; 3,000 steps, and the same run in three launches
    (the segments carry across launches)."""
    base = g.multi_subsystem(43, [4, 5, 3], n_lines=4, n_sources=2, dt=20e-6)
    net = g.with_bus_arresters(base, n_buses=1, scale=(0.07, 0.09))   # this bus peaks near 120 V
    assert net.n_nonlinear == 3
    N = 3000
    ref = oracle.simulate(net, N)
    knees = np.asarray(net.nl_v).reshape(-1, 8)[:, 0]
    assert np.all(np.max(np.abs(ref[:, net.nl_k]), axis=0) > knees)      # all three conduct
    assert rel(gpu_run(net, N), ref) <= TOL
    assert rel(gpu_run(net, N, chunks=[900, 1300, 800]), ref) <= TOL


def test_four_elements_resistive_ladder():
    """Four elements in one resistive subsystem (one between two nodes), the
    source driving them past their second breakpoints in both signs."""
    vp = [[700.0, 1000.0], [650.0, 900.0], [800.0, 1100.0], [300.0, 500.0]]
    ip = [[1.0, 40.0], [0.5, 60.0], [2.0, 30.0], [0.2, 20.0]]
    b = g.NetworkBuilder()
    b.source(6000.0, 0.2, 60.0)
    b.branch(g.source_node(0), 0, g.KIND_R, 2.0)
    b.branch(0, 1, g.KIND_R, 30.0)
    b.branch(1, 2, g.KIND_R, 30.0)
    for x in range(3):
        b.branch(x, g.GROUND, g.KIND_R, 200.0)
    for (k, m), v_, i_ in zip([(0, g.GROUND), (1, g.GROUND), (2, g.GROUND), (0, 2)], vp, ip):
        b.nonlinear_resistor(k, m, v_, i_)
    net = b.build(20e-6, 3)
    N = 2000
    ref = oracle.simulate(net, N)
    assert np.max(np.abs(ref)) > 1000.0
    assert rel(gpu_run(net, N), ref) <= TOL


def test_bus_arresters_on_the_large_network():
    """Three-phase arrester sets at 20 buses of the 3,000-node network (three
    elements per subsystem), 3,000 steps against the oracle."""
    net = g.with_bus_arresters(g.large_scale(n_steps=3000), n_buses=20)
    assert net.n_nonlinear == 60
    N = 3000
    ref = oracle.simulate(net, N)
    assert rel(gpu_run(net, N), ref) <= TOL


def test_several_per_subsystem_rejected_in_scenario_sets():
    base = g.multi_subsystem(43, [4, 5, 3], n_lines=4, n_sources=2, dt=20e-6)
    net = g.with_bus_arresters(base, n_buses=1)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_build_network(net, g.Scenarios(n_scenarios=2))
    assert ei.value.status == emt.EMT_EINVAL and "scenario set" in str(ei.value)
