"""Facts about the generated inputs that the parity bound relies on: the
2-norm condition number of every subsystem's conductance matrix (the
rounding of an explicit inverse grows with it) stays below 1e6 for the
seeded workloads, and every subsystem reaches ground or a source."""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import netgen as g


def subsystem_matrices(net):
    """G of every subsystem from the trapezoidal companions (R: 1/R, L:
    dt/2L, C: 2C/dt) and the lines' 1/Z_c shunts, switches open."""
    sub, n_sub = oracle.partition(net)
    local = np.zeros(net.n_nodes, np.int64)
    sizes = np.bincount(sub, minlength=n_sub)
    for s in range(n_sub):
        local[sub == s] = np.arange(sizes[s])
    G = [np.zeros((k, k)) for k in sizes]
    dt = net.dt
    for k, m, kind, val in zip(net.br_k, net.br_m, net.br_kind, net.br_value):
        gg = 1.0 / val if kind == 0 else (dt / (2 * val) if kind == 1 else 2 * val / dt)
        a = k if k >= 0 else m
        M, s = G[sub[a]], sub[a]
        if k >= 0:
            M[local[k], local[k]] += gg
        if m >= 0:
            M[local[m], local[m]] += gg
        if k >= 0 and m >= 0:
            M[local[k], local[m]] -= gg
            M[local[m], local[k]] -= gg
    for k, m, zc in zip(net.ln_k, net.ln_m, net.ln_zc):
        for x in (k, m):
            G[sub[x]][local[x], local[x]] += 1.0 / zc
    return G


@pytest.mark.parametrize("make", [lambda: g.single_rlc(), lambda: g.large_scale(n_steps=10),
                                  lambda: g.n1_contingency(n_steps=10)[0]])
def test_condition_numbers_below_bound(make):
    net = make()
    conds = [np.linalg.cond(M) for M in subsystem_matrices(net)]
    assert max(conds) < 1e6, max(conds)


def test_converter_study_scenarios_set_only_the_set_points():
    """Scenario s of the control study, written out: the converters' CONST
    set points scaled by its factors in [0.2, 1], every other block as in
    the base network; a subset writes out the same scenarios."""
    net, sc = g.converter_study(n_scenarios=6, n_converters=5, n_steps=10)
    refs = sc.meta["set_point_blocks"]
    base = np.asarray(net.cb_p0)
    for s in range(6):
        x = np.asarray(sc.expand(net, s).cb_p0)
        f = x[refs] / base[refs]
        assert np.all((f >= 0.2) & (f <= 1.0))
        other = np.setdiff1d(np.arange(net.n_control_blocks), refs)
        assert np.array_equal(x[other], base[other])
    sub = sc.subset([4, 1])
    assert np.array_equal(sub.expand(net, 0).cb_p0, sc.expand(net, 4).cb_p0)
    assert np.array_equal(sub.expand(net, 1).cb_p0, sc.expand(net, 1).cb_p0)
    assert np.array_equal(np.asarray(net.cb_p0), base)   # the base network is untouched
