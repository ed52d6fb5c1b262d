"""GPU parity of runtime switches (diodes, current-zero breakers) against
the oracle.  Every case first checks on the oracle's waveforms that no
switching decision sits within rounding of its threshold, so that both
sides must take the same decisions."""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10


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


def decision_margin(net, v):
    """Smallest |v_k - v_m| / max(|v_k|, |v_m|) of the diodes over the run:
    how close a decision comes to cancellation, where the two sides'
    rounding (about 1e-12 of the values) could flip its sign.  Values that
    are exactly zero on both ends (a subsystem not yet energised) carry no
    rounding and are left out."""
    node = lambda x: v[:, x] if x >= 0 else np.zeros(len(v))
    m = np.inf
    for w in range(net.n_runtime_switches):
        if net.rs_kind[w] == 0:
            a, b = node(int(net.rs_k[w])), node(int(net.rs_m[w]))
            sc = np.maximum(np.abs(a), np.abs(b))
            ok = sc > 0
            if ok.any():
                m = min(m, np.min(np.abs(a - b)[ok] / sc[ok]))
    return m


def rectifier(cap):
    b = g.NetworkBuilder()
    b.source(1000.0, 0.3, 60.0)
    b.branch(g.source_node(0), 0, 0, 1.0)
    b.diode(0, 1, 0.01, 1e6)
    b.branch(1, g.GROUND, 0, 10.0)
    if cap:
        b.branch(1, g.GROUND, 2, cap)
    return b.build(50e-6, 2, 2000)


@pytest.mark.parametrize("cap", [None, 200e-6])
def test_rectifier(cap):
    net = rectifier(cap)
    N = 2000
    ref = oracle.simulate(net, N)
    assert decision_margin(net, ref) > 1e-9
    assert rel(gpu_run(net, N), ref) <= TOL


def test_breaker_interrupts_at_current_zero():
    b = g.NetworkBuilder()
    b.source(1000.0, 0.3, 60.0)
    b.branch(g.source_node(0), 0, 0, 1.0)
    b.branch(0, 1, 1, 10e-3)
    b.breaker(1, g.GROUND, 1e-3, 1e5, 777)
    b.branch(1, g.GROUND, 2, 1e-6)
    net = b.build(20e-6, 2, 3000)
    N = 3000
    ref = oracle.simulate(net, N)
    st = oracle.runtime_switch_states(net, N)[:, 0]
    assert st[0] == 1 and st[-1] == 0
    assert rel(gpu_run(net, N), ref) <= TOL


def switched_multi():
    base = g.multi_subsystem(151, [3, 4, 2, 3], n_lines=5, n_sources=2, dt=20e-6)
    return g.with_rectifier_loads(base, seed=12, n_rectifiers=6, n_breakers=3, trip_range=(300, 900))


def test_multi_subsystem_with_rectifiers_and_breakers_resumable():
    net = switched_multi()
    N = 2000
    ref = oracle.simulate(net, N)
    assert decision_margin(net, ref) > 1e-9
    st = oracle.runtime_switch_states(net, N)
    assert (st[:, :6].min(axis=0) != st[:, :6].max(axis=0)).any()    # diodes switch
    assert (st[:, 6:].min(axis=0) != st[:, 6:].max(axis=0)).all()    # every breaker opens
    one = gpu_run(net, N)
    assert rel(one, ref) <= TOL
    split = gpu_run(net, N, chunks=(333, 667, None))                   # states carried across launches
    assert np.array_equal(split, one)


def test_large_network_with_runtime_switches():
    net = g.with_rectifier_loads(g.large_scale(), seed=1006)
    N = 5000
    ref = oracle.simulate(net, N)
    assert decision_margin(net, ref) > 1e-9
    assert rel(gpu_run(net, N), ref) <= TOL


def test_runtime_switch_limits():
    b = g.NetworkBuilder()
    b.source(1000.0, 0.0)
    b.branch(g.source_node(0), 0, 0, 1.0)
    for i in range(31):
        b.diode(0, i + 1, 0.01, 1e6)
        b.branch(i + 1, g.GROUND, 0, 10.0)
    net = b.build(50e-6, 32, 10)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_build_network(net)
    assert ei.value.status == emt.EMT_EINVAL and "runtime switches" in str(ei.value)
    # nine in one subsystem of a scenario set (every state prefactored there)
    b = g.NetworkBuilder()
    b.source(1000.0, 0.0)
    b.branch(g.source_node(0), 0, 0, 1.0)
    for i in range(9):
        b.diode(0, i + 1, 0.01, 1e6)
        b.branch(i + 1, g.GROUND, 0, 10.0)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_build_network(b.build(50e-6, 10, 10), g.Scenarios(n_scenarios=2))
    assert ei.value.status == emt.EMT_EINVAL and "scenario set" in str(ei.value)
    net = switched_multi()
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    assert emt.emt_get_info(ctx, "n_runtime_switches") == 9
    emt.emt_destroy(ctx)


def test_scenario_set_with_runtime_switches():
    """An N-1 study of the 600-node network with 10 diode-rectifier loads and
    4 current-zero breakers: each scenario keeps its own state words and
    picks the matching prefactored matrices; sampled scenarios against the
    oracle (each written out as a plain network); the switches change state;
    two launches equal one bit for bit."""
    N = 3000
    base, sc = g.n1_contingency(n_scenarios=32, n_steps=N)
    net = g.with_rectifier_loads(base, n_rectifiers=10, n_breakers=4)
    sim = emt.Simulator(net, sc, n_steps=N)
    sim.run(N)
    sim.sync()
    w = sim.waveforms()
    sim.close()
    for s in (0, 9, 31):
        x = sc.expand(net, s)
        assert rel(w[:, s, :], oracle.simulate(x, N)) <= TOL
    st = oracle.runtime_switch_states(sc.expand(net, 9), N)
    assert np.sum(st[1:] != st[:-1]) > 0
    two = emt.Simulator(net, sc, n_steps=N)
    two.run(1500)
    two.run(N - 1500)
    two.sync()
    assert np.array_equal(two.waveforms(), w)
    two.close()


def station_network(n_stations=1):
    base = g.multi_subsystem(41, [3, 5, 4], n_lines=4, n_sources=2, dt=20e-6)
    return g.with_converter_stations(base, n_stations=n_stations)


def test_two_six_pulse_bridges_in_one_subsystem_factorised_at_run_time():
    """Twelve diodes in one subsystem (two six-pulse bridges): more than the
    eight whose 2^k states are prefactored, so the CTA factorises each switch
    state the first time it meets it.  4,000 steps (about 110 valve
    commutations, 29 distinct states) against the oracle, which factorises G
    again at every state change.  A second run from the de-energised state
    finds every state in the cache and gives the same waveforms bit for bit."""
    net = station_network()
    N = 4000
    ref = oracle.simulate(net, N)
    assert decision_margin(net, ref) > 1e-9
    st = oracle.runtime_switch_states(net, N)
    assert len({tuple(r) for r in st}) > 10
    sim = emt.Simulator(net, n_steps=N)
    assert sim.info("lazy_subsystems") == 1
    before = sim.info("factorised_states")
    sim.run(N)
    sim.sync()
    assert sim.info("factorised_states") > before
    w = sim.waveforms()[:, 0, :]
    assert rel(w, ref) <= TOL
    sim.reset()
    sim.run(N)
    sim.sync()
    assert np.array_equal(sim.waveforms()[:, 0, :], w)
    sim.close()


def test_run_time_factorisation_across_launches():
    net = station_network()
    N = 3000
    ref = oracle.simulate(net, N)
    assert rel(gpu_run(net, N, chunks=(700, 1100, None)), ref) <= TOL


def test_converter_stations_on_the_large_network():
    """Ten two-bridge stations (120 diodes) on the 3,000-node network, one per
    subsystem: 3,000 steps against the oracle."""
    net = g.with_converter_stations(g.large_scale(n_steps=3000), n_stations=10)
    N = 3000
    ref = oracle.simulate(net, N)
    assert decision_margin(net, ref) > 1e-9
    sim = emt.Simulator(net, n_steps=N)
    assert sim.info("lazy_subsystems") == 10
    sim.run(N)
    sim.sync()
    assert rel(sim.waveforms()[:, 0, :], ref) <= TOL
    sim.close()


def test_adjoint_rejects_states_factorised_at_run_time():
    net = station_network()
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_adjoint(ctx, np.zeros((10, net.n_nodes)), 10, 0)
    assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)
