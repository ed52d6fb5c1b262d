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
  rejected;
* several elements in one subsystem (the piecewise-linear Newton iteration
  on the nodal equations): on a resistive network every step is a static
  problem, and each step's solution is the one consistent assignment found
  by trying every combination of segments.
"""
import itertools
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

    v = net.nl_v.copy(); v[1] = v[0]
    bad(nl_v=v)                                     # breakpoints not increasing
    i = net.nl_i.copy(); i[2] = 0.0
    bad(nl_i=i)                                     # current decreasing
    bad(nl_np=np.array([9, 6], np.int32))
    bad(nl_k=np.array([-1, net.nl_k[1]], np.int32))  # both ends ground
    with pytest.raises(oracle.OracleError):
        oracle.adjoint(net, 5, np.zeros((5, net.n_nodes)))


def three_arrester_ladder(amp=6000.0):
    """Source -> 2 ohm -> node 0 -> 30 ohm -> node 1 -> 30 ohm -> node 2, 200 ohm
    loads to ground at each node and an arrester to ground at each node,
    plus one between nodes 0 and 2: four nonlinear resistors in one
    subsystem, no storage elements (each step is a static problem)."""
    vp = [[700.0, 1000.0], [650.0, 900.0], [800.0, 1100.0], [300.0, 500.0]]
    ip = [[1.0, 40.0], [0.5, 60.0], [2.0, 30.0], [0.2, 20.0]]
    b = g.NetworkBuilder()
    b.source(amp, PHI, F)
    b.branch(g.source_node(0), 0, g.KIND_R, 2.0)
    b.branch(0, 1, g.KIND_R, 30.0)
    b.branch(1, 2, g.KIND_R, 30.0)
    for x in range(3):
        b.branch(x, g.GROUND, g.KIND_R, 200.0)
    for (k, m), v_, i_ in zip([(0, g.GROUND), (1, g.GROUND), (2, g.GROUND), (0, 2)], vp, ip):
        b.nonlinear_resistor(k, m, v_, i_)
    return b.build(DT, 3), vp, ip


def brute_force_step(vs, vp, ip):
    """Node voltages of the ladder at source voltage vs: every assignment of
    the four elements to segments (sign x segment) linearised and solved;
    the assignments whose solution lies on their own segments."""
    ends = [(0, -1), (1, -1), (2, -1), (0, 2)]
    G0 = np.zeros((3, 3))
    def stamp(Gm, k, m, gg):
        for a in (k, m):
            if a >= 0:
                Gm[a, a] += gg
        if k >= 0 and m >= 0:
            Gm[k, m] -= gg
            Gm[m, k] -= gg
    stamp(G0, 0, -1, 1 / 2.0); stamp(G0, 0, 1, 1 / 30.0); stamp(G0, 1, 2, 1 / 30.0)
    for x in range(3):
        stamp(G0, x, -1, 1 / 200.0)
    segs = []
    for v_, i_ in zip(vp, ip):
        pts_v, pts_i = [0.0] + v_, [0.0] + i_
        lines = []
        for j in range(3):   # two breakpoints: three segments, the last continued
            q = min(j, 1)
            slope = (pts_i[q + 1] - pts_i[q]) / (pts_v[q + 1] - pts_v[q])
            lo, hi = pts_v[j], (pts_v[j + 1] if j < 2 else np.inf)
            for sg in (1.0, -1.0):
                lines.append((sg, lo, hi, slope, sg * (pts_i[j] - slope * pts_v[j])))
        segs.append(lines)
    sols = []
    for combo in itertools.product(*segs):
        Gm = G0.copy()
        r = np.array([vs / 2.0, 0.0, 0.0])
        for (k, m), (sg, lo, hi, slope, c0) in zip(ends, combo):
            stamp(Gm, k, m, slope)
            if k >= 0:
                r[k] -= c0
            if m >= 0:
                r[m] += c0
        x = np.linalg.solve(Gm, r)
        ok = True
        for (k, m), (sg, lo, hi, slope, c0) in zip(ends, combo):
            u = (x[k] if k >= 0 else 0.0) - (x[m] if m >= 0 else 0.0)
            ok &= (sg * u >= -1e-9 * max(1.0, abs(u))) and lo * (1 - 1e-12) <= abs(u) <= hi * (1 + 1e-12)
        if ok:
            sols.append(x)
    return sols


def test_several_in_one_subsystem_match_brute_force():
    net, vp, ip = three_arrester_ladder()
    N = 300
    v = oracle.simulate(net, N)
    reached = set()
    for n in range(1, N + 1, 3):
        sols = brute_force_step(vsrc(n) * 3.0, vp, ip)
        assert sols, n
        for x in sols:   # any consistent assignment is the (unique) solution
            assert np.max(np.abs(x - v[n - 1])) <= 1e-9 * max(1.0, np.max(np.abs(x))), n
        reached.add(round(float(np.max(np.abs(v[n - 1]))), -2))
    assert max(reached) > 1000.0        # the elements were driven past their breakpoints


def test_several_in_one_subsystem_monolithic_equals_partitioned():
    base = g.multi_subsystem(43, [4, 5, 3], n_lines=4, n_sources=2, dt=DT)
    net, vp, ip = base, None, None
    b_nodes = net.meta["bus_nodes"]
    sub, _ = oracle.partition(net)
    # three arresters in the first source bus's subsystem, one in another
    first = b_nodes[net.meta["source_bus"][0]]
    others = [x for x in range(net.n_nodes) if sub[x] != sub[first[0]]]
    bb = g.NetworkBuilder()
    for x in list(first) + [others[0]]:
        bb.nonlinear_resistor(int(x), g.GROUND, [v * 0.6 for v in g.ARRESTER_V], g.ARRESTER_I)
    nl = bb.build(DT, 0)
    for f_ in ("nl_k", "nl_m", "nl_np", "nl_v", "nl_i"):
        setattr(net, f_, getattr(nl, f_))
    N = 2000
    a = oracle.simulate(net, N)
    m = oracle.simulate(net, N, monolithic=True)
    assert np.max(np.abs(a - m)) / np.max(np.abs(m)) <= 1e-12
