"""Pins of the oracle's discrete adjoint.

The adjoint is checked against two methods that share none of its code:
the complex-step derivative (the same forward loop run in complex
arithmetic, exact to rounding) and central finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import netgen as g


def adjoint_case(seed=41, n_steps=400):
    net = g.multi_subsystem(seed, [2, 3, 2], n_lines=4, n_sources=2, dt=20e-6, n_series_extra=2,
                            delay_range=(1, 6))
    # a fault switch at fixed times inside the window
    node = int(net.meta["bus_nodes"][1][0])
    net.sw_k = np.array([node], np.int32)
    net.sw_m = np.array([g.GROUND], np.int32)
    net.sw_r = np.array([0.05])
    net.sw_close_step = np.array([150], np.int64)
    net.sw_open_step = np.array([320], np.int64)
    br_t, amp_t = g.adjoint_target(net, seed=seed + 1000)
    target = oracle.simulate(net.with_params(br_t, amp_t), n_steps)
    return net, target


@pytest.fixture(scope="module")
def case():
    net, target = adjoint_case()
    grad, J = oracle.adjoint(net, 400, target)
    return net, target, grad, J


def test_adjoint_loss_matches_forward(case):
    net, target, grad, J = case
    assert J == pytest.approx(oracle.loss(net, 400, target), rel=1e-14)
    assert J > 0


def test_adjoint_vs_complex_step_all_parameters(case):
    net, target, grad, J = case
    n_par = net.n_branches + net.n_sources
    cs = np.array([oracle.loss_complex_step(net, 400, target, p)[1] for p in range(n_par)])
    # compare in the parameter-scaled form p dJ/dp (units of J)
    p = np.concatenate([net.br_value, net.src_amp])
    err = np.abs(p * (grad - cs)) / J
    assert np.max(err) < 1e-9, np.max(err)


def test_adjoint_vs_central_differences(case):
    net, target, grad, J = case
    p0 = np.concatenate([net.br_value, net.src_amp])
    scaled = np.abs(p0 * grad)
    # FD is unreliable where p dJ/dp is tiny next to J (cancellation); draw
    # only among parameters with |p dJ/dp| >= 1e-6 J
    cand = np.nonzero(scaled >= 1e-6 * J)[0]
    rng = np.random.default_rng(5)
    pick = rng.choice(cand, size=min(12, len(cand)), replace=False)
    nb = net.n_branches
    for i in pick:
        h = 1e-5 * abs(p0[i])
        vals = []
        for sgn in (+1, -1):
            p = p0.copy()
            p[i] += sgn * h
            vals.append(oracle.loss(net.with_params(p[:nb], p[nb:]), 400, target))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * abs(grad[i]), (i, fd, grad[i])


def test_adjoint_zero_at_target():
    net, _ = adjoint_case(seed=43, n_steps=200)
    target = oracle.simulate(net, 200)
    grad, J = oracle.adjoint(net, 200, target)
    assert J == 0.0
    assert np.all(grad == 0.0)


def switched_adjoint_case(n_steps=500):
    """Diode rectifier loads and breakers (runtime switches) on a small
    three-subsystem network."""
    base = g.multi_subsystem(43, [2, 3, 2], n_lines=4, n_sources=2, dt=20e-6, n_series_extra=2,
                             delay_range=(1, 6))
    net = g.with_rectifier_loads(base, seed=7, n_rectifiers=3, n_breakers=2, trip_range=(100, 300))
    br_t, amp_t = g.adjoint_target(net, seed=1043)
    target = oracle.simulate(net.with_params(br_t, amp_t), n_steps)
    return net, target


def test_adjoint_with_runtime_switches_vs_complex_step():
    """The reverse sweep replays the forward's switch states; the complex-step
    derivative (decisions taken on the real part) is the same derivative."""
    net, target = switched_adjoint_case()
    st = oracle.runtime_switch_states(net, 500)
    assert (st.min(axis=0) != st.max(axis=0)).any()          # the switches do switch
    grad, J = oracle.adjoint(net, 500, target)
    n_par = net.n_branches + net.n_sources
    cs = np.array([oracle.loss_complex_step(net, 500, target, p)[1] for p in range(n_par)])
    p = np.concatenate([net.br_value, net.src_amp])
    assert np.max(np.abs(p * (grad - cs)) / J) < 1e-9
