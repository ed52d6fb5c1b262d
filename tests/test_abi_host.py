"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/emt.h declares, and rejects invalid
network descriptions before touching the device."""
import dataclasses
import os
import re

import numpy as np
import pytest

from paper_1903_01081_b300 import emt, netgen as g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(emt_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = emt.load_library()
    names = declared_functions()
    assert "emt_build_network" in names and "emt_step_n" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(emt.EXPORTS) <= names


def bad(net, **changes):
    net = net.copy()
    for k, v in changes.items():
        setattr(net, k, v)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_build_network(net)
    assert ei.value.status == emt.EMT_EINVAL
    return str(ei.value)


def test_rejects_invalid_descriptions():
    net = g.single_rlc(n_steps=10)
    assert "value" in bad(net, br_value=np.where(np.arange(net.n_branches) == 3, -1.0, net.br_value))
    k = net.br_k.copy(); k[0] = net.n_nodes
    assert "out of range" in bad(net, br_k=k)
    kind = net.br_kind.copy(); kind[1] = 7
    assert "kind" in bad(net, br_kind=kind)
    m = net.br_m.copy(); m[2] = net.br_k[2]
    assert "one node" in bad(net, br_m=m)
    assert "dt" in bad(net, dt=0.0)
    b = g.NetworkBuilder(); b.source(1.0, 0.0); b.branch(g.source_node(0), g.GROUND, 0, 1.0)
    assert "unknown end" in bad(b.build(1e-5, 0))


def test_rejects_bad_lines_and_switches():
    net = g.multi_subsystem(3, [2, 2], n_lines=1, n_sources=1, dt=20e-6)
    assert "delay" in bad(net, ln_delay=np.zeros_like(net.ln_delay))
    assert "Z_c" in bad(net, ln_zc=-net.ln_zc)
    lk = net.ln_k.copy(); lk[0] = -1
    assert "unknown nodes" in bad(net, ln_k=lk)
    net2 = g.single_rlc(n_steps=10)
    assert "resistance" in bad(net2, sw_r=np.zeros_like(net2.sw_r))


def test_rejects_oversized_subsystem():
    b = g.NetworkBuilder()
    b.source(1.0, 0.0)
    n = 129
    b.branch(g.source_node(0), 0, 0, 1.0)
    for i in range(n - 1):
        b.branch(i, i + 1, 0, 1.0)
    assert "at most 128" in bad(b.build(1e-5, n))


def test_rejects_bad_runtime_switches():
    net = g.with_rectifier_loads(g.multi_subsystem(5, [6, 6], n_lines=2, n_sources=2, dt=20e-6),
                                 n_rectifiers=3, n_breakers=1)
    assert net.n_runtime_switches == 4
    kind = net.rs_kind.copy(); kind[0] = 2
    assert "diode" in bad(net, rs_kind=kind)
    assert "resistances" in bad(net, rs_ron=np.zeros_like(net.rs_ron))
    assert "resistances" in bad(net, rs_roff=np.full_like(net.rs_roff, np.inf))
    k = net.rs_k.copy(); m = net.rs_m.copy(); k[1] = -1; m[1] = -1
    assert "ground" in bad(net, rs_k=k, rs_m=m)
    # more two-state switches in one subsystem than the state word holds (30;
    # above 8 the states are factorised at run time)
    b = g.NetworkBuilder()
    b.source(1.0, 0.0)
    b.branch(g.source_node(0), 0, 0, 1.0)
    for i in range(31):
        b.branch(0, i + 1, 0, 2.0)
        b.diode(i + 1, g.GROUND, 0.01, 1e6)
    assert "more than 30 runtime switches" in str(pytest.raises(
        emt.EmtError, emt.emt_build_network, b.build(20e-6, 32)).value)


def test_rejects_bad_coupled_lines():
    net = g.with_coupled_lines(g.multi_subsystem(7, [6, 6], n_lines=1, n_sources=2, dt=20e-6))
    assert net.n_coupled_lines >= 1
    tau = net.cl_tau.copy(); tau.flat[0] = 0.5 * net.dt
    assert "at least dt" in bad(net, cl_tau=tau)
    z = net.cl_z.copy(); z.flat[1] = 0.0
    assert "Z_c" in bad(net, cl_z=z)
    tv = net.cl_tv.copy().reshape(-1, 3, 3); tv[0, 2] = tv[0, 0]
    assert "singular" in bad(net, cl_tv=tv.reshape(net.cl_tv.shape))
    k = net.cl_k.copy(); k.flat[0] = -1
    assert "unknown nodes" in bad(net, cl_k=k)


def test_rejects_bad_controls():
    net = g.with_converter_controls(g.multi_subsystem(11, [4, 5, 3, 6], n_lines=5, n_sources=3, dt=20e-6),
                                    n_converters=4)
    t = net.cb_type.copy(); t[3] = 9
    assert "type" in bad(net, cb_type=t)
    i0 = net.cb_in0.copy(); i0[4] = net.n_control_blocks
    assert "not a block" in bad(net, cb_in0=i0)
    p1 = net.cb_p1.copy(); p1[21] = 0.0
    assert "time constant" in bad(net, cb_p1=p1)
    p0 = net.cb_p0.copy(); p0[14] = 1e9
    assert "p0 <= p1" in bad(net, cb_p0=p0)
    p0 = net.cb_p0.copy(); p0[3] = np.nan
    assert "non-finite" in bad(net, cb_p0=p0)
    nd = net.cb_node.copy(); nd[0] = net.n_nodes
    assert "unknown" in bad(net, cb_node=nd)
    cb = net.ci_block.copy(); cb[0] = -1
    assert "needs a block" in bad(net, ci_block=cb)
    # one converter measuring a node of another subsystem
    from oracle import partition
    sub, _ = partition(net)
    other = int(np.nonzero(sub != sub[net.cb_node[0]])[0][0])
    nd = net.cb_node.copy(); nd[0] = other
    assert "spanning two subsystems" in bad(net, cb_node=nd)
    cn = net.ci_node.copy(); cn[0] = other
    assert "outside its block group" in bad(net, ci_node=cn)
    # per-scenario control parameters are validated before any device work
    sc_net, sc = g.n1_contingency(n_scenarios=2, n_buses=24, n_sub=4, n_steps=10)
    ctl = g.with_converter_controls(sc_net, n_converters=2)
    lim = int(np.flatnonzero(np.asarray(ctl.cb_type) == g.CB_LIMIT)[0])

    def bad_sc(blocks, values, match):
        x = dataclasses.replace(sc, cbo_ptr=np.array([0, len(blocks), len(blocks)], np.int64),
                                cbo_block=np.asarray(blocks, np.int32), cbo_p0=np.asarray(values, np.float64))
        with pytest.raises(emt.EmtError, match=match):
            emt.emt_build_network(ctl, x)
    bad_sc([ctl.n_control_blocks], [1.0], "out of range")
    bad_sc([3, 3], [1.0, 2.0], "twice")
    bad_sc([3], [np.nan], "not finite")
    bad_sc([lim], [float(ctl.cb_p1[lim]) + 1.0], "lower bound exceeds")


def test_rejects_bad_fd_lines():
    net = g.with_fd_lines(g.multi_subsystem(21, [4, 5, 3, 6], n_lines=6, n_sources=3, dt=20e-6))
    assert "at least dt" in bad(net, fl_tau=np.full_like(net.fl_tau, 0.5 * net.dt))
    ny = net.fl_ny.copy(); ny[0] = 5
    assert "at most 4" in bad(net, fl_ny=ny)
    q = net.fl_yq.copy(); q[0] = 1.0
    assert "< 0" in bad(net, fl_yq=q)
    ap = net.fl_ap.copy(); ap[1] = np.nan
    assert "< 0" in bad(net, fl_ap=ap)
    assert "y0" in bad(net, fl_y0=-net.fl_y0)
    m = net.fl_m.copy(); m[0] = net.fl_k[0]
    assert "one node" in bad(net, fl_m=m)
    k = net.fl_k.copy(); k[0] = -1
    assert "unknown nodes" in bad(net, fl_k=k)
    y0 = np.zeros_like(net.fl_y0); ny0 = np.zeros_like(net.fl_ny)
    assert "end conductance" in bad(net, fl_y0=y0, fl_ny=ny0)
    # scenario sets take frequency-dependent lines, but their removals name lossless lines only
    sc_net, sc = g.n1_contingency(n_scenarios=4, n_buses=24, n_sub=4, n_steps=10)
    x = dataclasses.replace(sc, rm_line_ptr=np.array([0, 1, 1, 1, 1], np.int64), rm_line=np.array([0], np.int32))
    with pytest.raises(emt.EmtError, match="removed line out of range"):
        emt.emt_build_network(g.with_fd_lines(sc_net), x)


def test_rejects_bad_nonlinear():
    base = g.multi_subsystem(41, [4, 5, 3], n_lines=4, n_sources=2, dt=20e-6)
    net = g.with_arresters(base, n_arresters=2)
    v = net.nl_v.copy(); v[1] = v[0]
    assert "breakpoints" in bad(net, nl_v=v)
    assert "1 to 8" in bad(net, nl_np=np.array([9, 6], np.int32))
    assert "ground" in bad(net, nl_k=np.array([-1, net.nl_k[1]], np.int32))
    # five in one subsystem (four are solved together; one in a scenario set)
    from oracle import partition
    sub, _ = partition(net)
    same = [x for x in range(net.n_nodes) if sub[x] == sub[net.nl_k[0]]][:5]
    assert len(same) == 5
    rep = lambda a: np.repeat(np.asarray(a).reshape(2, -1)[:1], 5, axis=0).reshape(-1)
    assert "more than 4 nonlinear resistors" in bad(
        net, nl_k=np.asarray(same, np.int32), nl_m=np.full(5, -1, np.int32), nl_np=np.repeat(net.nl_np[:1], 5),
        nl_v=rep(net.nl_v), nl_i=rep(net.nl_i))
    # the same checks hold with a scenario set (validated before any device work)
    sc_net, sc = g.n1_contingency(n_scenarios=4, n_buses=24, n_sub=4, n_steps=10)
    arr = g.with_arresters(sc_net, n_arresters=1)
    with pytest.raises(emt.EmtError, match="1 to 8"):
        emt.emt_build_network(dataclasses.replace(arr, nl_np=np.array([9], np.int32)), sc)


def test_out_of_range_indices_rejected_before_any_launch():
    """Every index in a description is checked on the host: a node, source,
    line end or switch end outside its range returns EINVAL from
    emt_build_network (nothing reaches the device; the checks build only
    guards indices the kernels compute)."""
    net = g.multi_subsystem(7, [4, 5], n_lines=2, n_sources=2, dt=20e-6)
    n = net.n_nodes
    k = net.br_k.copy(); k[0] = n
    assert "node" in bad(net, br_k=k)
    m = net.br_m.copy(); m[1] = -2 - net.n_sources                        # a source that does not exist
    assert "out of range" in bad(net, br_m=m)
    lk = net.ln_k.copy(); lk[0] = n + 5
    bad(net, ln_k=lk)
    lm = net.ln_m.copy(); lm[0] = -1                                      # a line end at ground
    bad(net, ln_m=lm)
    sw = g.NetworkBuilder()
    sw.source(1.0, 0.0)
    sw.branch(g.source_node(0), 0, 0, 1.0)
    sw.switch(0, 7, 0.1, 10)
    bad(sw.build(20e-6, 1, 20))
