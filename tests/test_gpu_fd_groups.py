"""Frequency-dependent line groups on the GPU (three frequency-dependent
conductors as the modes of one three-phase line through T_v): each end is a
coupled end whose modes run the frequency-dependent line equations on modal
quantities.  Held to the oracle at a peak-normalised 1e-10, also across
launches (the modal histories are folded into the phase slots when a launch
starts), over the full 50,000 steps of the large-scale network, together
with the extended kernel code, and in a scenario set."""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel_err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def base_net():
    return g.multi_subsystem(161, [3, 4, 2, 3, 5], n_lines=8, n_sources=2, dt=20e-6)


def gpu_run(net, chunks):
    sim = emt.Simulator(net, n_steps=sum(chunks))
    for n in chunks:
        sim.run(n)
    sim.sync()
    w = sim.waveforms()[:, 0, :]
    sim.close()
    return w


def test_small_network_matches_the_oracle_across_launches():
    net = g.with_fd_line_groups(base_net())
    N = 4000
    ref = oracle.simulate(net, N)
    assert rel_err(gpu_run(net, [N]), ref) <= TOL
    assert rel_err(gpu_run(net, [1, 1499, 2500]), ref) <= TOL


def test_lossless_groups_are_the_coupled_line():
    cnet = g.with_coupled_lines(base_net(), seed=3)
    net = g.fd_groups_from_coupled(cnet, lossless=True)
    N = 3000
    got = gpu_run(net, [N])
    assert rel_err(got, oracle.simulate(net, N)) <= TOL
    assert rel_err(got, gpu_run(cnet, [N])) <= TOL


def test_large_scale_network_full_length():
    net = g.with_fd_line_groups(g.large_scale())
    N = net.n_steps
    got = gpu_run(net, [N])
    ref = oracle.simulate(net, N)
    assert rel_err(got, ref) <= TOL


def test_scenario_set_with_line_groups():
    """A study on the 600-node network with its three-phase lines as line
    groups (per scenario the source amplitudes and angles and a fault
    resistance): sampled scenarios against the oracle, each written out as a
    plain network; two launches equal one bit for bit."""
    N = 3000
    base, _ = g.n1_contingency(n_scenarios=1, n_steps=N)
    net, sc = g.shared_g(n_scenarios=24, n_steps=N, fault_step=1500, base=g.with_fd_line_groups(base))
    assert len(net.fg_line) > 0 and net.n_lines == 0
    sim = emt.Simulator(net, sc, n_steps=N)
    sim.run(N)
    sim.sync()
    w = sim.waveforms()
    sim.close()
    for s in (0, 11, 23):
        ref = oracle.simulate(sc.expand(net, s), N)
        assert rel_err(w[:, s, :], ref) <= TOL, s
    two = emt.Simulator(net, sc, n_steps=N)
    two.run(1234)
    two.run(N - 1234)
    two.sync()
    assert np.array_equal(two.waveforms(), w)
    two.close()


def test_groups_with_run_time_factorisation_and_arrester_sets():
    """Line groups on a network that also needs the extended kernel code
    (converter stations whose subsystems are factorised at run time, and
    three-phase arrester sets: several nonlinear resistors per subsystem):
    the kernel build that carries both, across launches, against the oracle."""
    base = g.with_converter_stations(g.large_scale(n_steps=3000), n_stations=10)
    net = g.with_fd_line_groups(g.with_bus_arresters(base, n_buses=20))
    N = 3000
    ref = oracle.simulate(net, N)
    sim = emt.Simulator(net, n_steps=N)
    sim.run(1000)
    sim.run(N - 1000)
    sim.sync()
    assert sim.info("lazy_subsystems") == 10
    got = sim.waveforms()[:, 0, :]
    sim.close()
    assert rel_err(got, ref) <= TOL


def test_groups_are_refused_by_the_adjoint():
    net = g.with_fd_line_groups(base_net())
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_adjoint(ctx, np.zeros((10, net.n_nodes)), 10, 0)
    assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)
