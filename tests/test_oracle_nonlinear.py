"""Pins of the oracle's nonlinear resistors (odd piecewise-linear i = f(v),
solved by the compensation method against the linear solution).

* a resistive circuit: each step's node voltage is the root of
  u + R_th f(u) = v_th found by bisection on f itself (f evaluated from the
  breakpoints by numpy interpolation), including negative half-waves and
  voltages past the last breakpoint;
* a one-segment characteristic is a plain resistor (an independent, already
  pinned code path);
* a series-L circuit against a hand-written implicit trapezoidal recursion
  solved by bisection every step;
* monolithic and partitioned solves agree; invalid descriptions are
  rejected.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import netgen as g

A, F, PHI, DT = 2000.0, 60.0, 0.2, 20e-6
V_PTS = [800.0, 950.0, 1050.0, 1150.0, 1300.0, 1500.0]
I_PTS = [1e-3, 1.0, 50.0, 300.0, 1500.0, 4000.0]


def f(u):
    """The odd piecewise-linear characteristic, continued with the last slope."""
    v = np.concatenate([[0.0], V_PTS])
    i = np.concatenate([[0.0], I_PTS])
    x = np.abs(u)
    last = (i[-1] - i[-2]) / (v[-1] - v[-2])
    y = np.where(x <= v[-1], np.interp(x, v, i), i[-1] + last * (x - v[-1]))
    return np.sign(u) * y


def bisect(h, lo, hi, iters=200):
    """Root of an increasing scalar function on [lo, hi]."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if h(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def vsrc(n):
    return A * np.sin(2 * np.pi * F * n * DT + PHI)


def test_resistive_circuit_matches_bisection():
    rs, r, amp = 2.0, 50.0, 20000.0     # a source strong enough to drive the arrester past its last point
    b = g.NetworkBuilder()
    b.source(amp, PHI, F)
    b.branch(g.source_node(0), 0, g.KIND_R, rs)
    b.branch(0, g.GROUND, g.KIND_R, r)
    b.nonlinear_resistor(0, g.GROUND, V_PTS, I_PTS)
    net = b.build(DT, 1)
    N = 1200
    v = oracle.simulate(net, N)[:, 0]
    rth = rs * r / (rs + r)
    want = np.array([bisect(lambda u, vt=vsrc(n) * amp / A * r / (rs + r): u + rth * f(u) - vt, -amp, amp)
                     for n in range(1, N + 1)])
    assert np.max(np.abs(v - want)) <= 1e-12 * np.max(np.abs(want))
    assert np.max(np.abs(v)) > V_PTS[-1] and np.min(v) < -V_PTS[-1]     # past the last point, both signs


def test_one_segment_is_a_resistor():
    g_lin = 0.02
    nets = []
    for nl in (True, False):
        b = g.NetworkBuilder()
        b.source(1000.0, PHI, F)
        b.branch(g.source_node(0), 0, g.KIND_L, 0.01)
        b.branch(0, 1, g.KIND_C, 50e-6)
        b.branch(1, g.GROUND, g.KIND_R, 20.0)
        if nl:
            b.nonlinear_resistor(0, 1, [100.0], [100.0 * g_lin])
        else:
            b.branch(0, 1, g.KIND_R, 1.0 / g_lin)
        nets.append(b.build(DT, 2))
    a, r = oracle.simulate(nets[0], 3000), oracle.simulate(nets[1], 3000)
    assert np.max(np.abs(a - r)) <= 1e-12 * np.max(np.abs(r))


def test_series_inductor_against_scalar_recursion():
    lval, r = 0.005, 100.0
    b = g.NetworkBuilder()
    b.source(A, PHI, F)
    b.branch(g.source_node(0), 0, g.KIND_L, lval)
    b.branch(0, g.GROUND, g.KIND_R, r)
    b.nonlinear_resistor(0, g.GROUND, V_PTS, I_PTS)
    net = b.build(DT, 1)
    N = 2500
    v = oracle.simulate(net, N)[:, 0]
    k = DT / (2 * lval)
    want = np.zeros(N)
    i_prev, v_prev, vs_prev = 0.0, 0.0, 0.0
    for n in range(1, N + 1):
        vs = vsrc(n)
        rhs = lambda u: u / r + f(u) - (i_prev + k * (vs - u + vs_prev - v_prev))
        u = bisect(rhs, -3 * A, 3 * A)
        i_prev = u / r + f(u)
        v_prev, vs_prev = u, vs
        want[n - 1] = u
    assert np.max(np.abs(v - want)) <= 1e-10 * np.max(np.abs(want))
    assert np.max(np.abs(v)) > V_PTS[0]


def test_monolithic_equals_partitioned_with_one_arrester():
    base = g.multi_subsystem(41, [4, 5, 3], n_lines=4, n_sources=2, dt=DT)
    net = g.with_arresters(base, n_arresters=1)
    assert net.n_nonlinear == 1
    a = oracle.simulate(net, 2000)
    m = oracle.simulate(net, 2000, monolithic=True)
    assert np.max(np.abs(a - m)) <= 1e-11 * np.max(np.abs(a))


def test_invalid_nonlinear_rejected():
    base = g.multi_subsystem(41, [4, 5, 3], n_lines=4, n_sources=2, dt=DT)
    net = g.with_arresters(base, n_arresters=2)

    def bad(**kw):
        x = net.copy()
        for k_, v_ in kw.items():
            setattr(x, k_, v_)
        with pytest.raises(oracle.OracleError):
            oracle.simulate(x, 5)

    sub, _ = oracle.partition(net)
    same = [x for x in range(net.n_nodes) if sub[x] == sub[net.nl_k[0]] and x != net.nl_k[0]][0]
    k = net.nl_k.copy(); k[1] = same
    bad(nl_k=k)                                     # two in one subsystem
    v = net.nl_v.copy(); v[1] = v[0]
    bad(nl_v=v)                                     # breakpoints not increasing
    i = net.nl_i.copy(); i[2] = 0.0
    bad(nl_i=i)                                     # current decreasing
    bad(nl_np=np.array([9, 6], np.int32))
    bad(nl_k=np.array([-1, net.nl_k[1]], np.int32))  # both ends ground
    with pytest.raises(oracle.OracleError):
        oracle.adjoint(net, 5, np.zeros((5, net.n_nodes)))
