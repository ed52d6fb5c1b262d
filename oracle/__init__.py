"""Plain FP64 CPU oracle of the EMTP-type time loop -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does; the C
library below shares no code with the CUDA library.

The oracle follows the four basic processes of the EMTP-type algorithm
listed in Sec. III-A of the CloudPSS paper (companion models, nodal
injections, factorisation, forward/backward substitution), with the
trapezoidal companion formulas of the paper's ref. [2] and lossless
Bergeron lines; see ``emt_oracle.cpp`` for every formula.

Pins (in ``tests/test_oracle_*.py``): Tustin/bilinear equivalence against
``scipy.signal``, discrete sinusoidal steady state against a complex phasor
solve, exact travel-time delay of a lossless line, KCL residuals from an
independent current recursion, LU against exact rational arithmetic,
monolithic vs partitioned solves, and the adjoint against complex-step and
central finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C++ source into ``oracle/liboracle.so``."""
    src = os.path.join(_HERE, "emt_oracle.cpp")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "emt_oracle.h"))):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", _LIB_PATH, src])
    return _LIB_PATH


class _Net(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("n_nodes", ctypes.c_int64),
        ("n_br", ctypes.c_int64), ("br_k", ctypes.c_void_p), ("br_m", ctypes.c_void_p),
        ("br_kind", ctypes.c_void_p), ("br_val", ctypes.c_void_p),
        ("n_src", ctypes.c_int64), ("src_amp", ctypes.c_void_p), ("src_phase", ctypes.c_void_p),
        ("src_freq", ctypes.c_void_p),
        ("n_ln", ctypes.c_int64), ("ln_k", ctypes.c_void_p), ("ln_m", ctypes.c_void_p),
        ("ln_zc", ctypes.c_void_p), ("ln_d", ctypes.c_void_p),
        ("n_sw", ctypes.c_int64), ("sw_k", ctypes.c_void_p), ("sw_m", ctypes.c_void_p),
        ("sw_r", ctypes.c_void_p), ("sw_on", ctypes.c_void_p), ("sw_off", ctypes.c_void_p),
        ("n_rs", ctypes.c_int64), ("rs_k", ctypes.c_void_p), ("rs_m", ctypes.c_void_p),
        ("rs_kind", ctypes.c_void_p), ("rs_ron", ctypes.c_void_p), ("rs_roff", ctypes.c_void_p),
        ("rs_on0", ctypes.c_void_p), ("rs_trip", ctypes.c_void_p),
        ("n_cl", ctypes.c_int64), ("cl_k", ctypes.c_void_p), ("cl_m", ctypes.c_void_p),
        ("cl_tv", ctypes.c_void_p), ("cl_z", ctypes.c_void_p), ("cl_tau", ctypes.c_void_p),
        ("n_fl", ctypes.c_int64), ("fl_k", ctypes.c_void_p), ("fl_m", ctypes.c_void_p),
        ("fl_tau", ctypes.c_void_p), ("fl_y0", ctypes.c_void_p), ("fl_ny", ctypes.c_void_p),
        ("fl_yq", ctypes.c_void_p), ("fl_yc", ctypes.c_void_p), ("fl_a0", ctypes.c_void_p),
        ("fl_na", ctypes.c_void_p), ("fl_ap", ctypes.c_void_p), ("fl_ar", ctypes.c_void_p),
        ("n_nl", ctypes.c_int64), ("nl_k", ctypes.c_void_p), ("nl_m", ctypes.c_void_p),
        ("nl_np", ctypes.c_void_p), ("nl_v", ctypes.c_void_p), ("nl_i", ctypes.c_void_p),
        ("n_cb", ctypes.c_int64), ("cb_type", ctypes.c_void_p), ("cb_in0", ctypes.c_void_p),
        ("cb_in1", ctypes.c_void_p), ("cb_node", ctypes.c_void_p), ("cb_p0", ctypes.c_void_p),
        ("cb_p1", ctypes.c_void_p),
        ("n_ci", ctypes.c_int64), ("ci_block", ctypes.c_void_p), ("ci_node", ctypes.c_void_p),
        ("n_fg", ctypes.c_int64), ("fg_line", ctypes.c_void_p), ("fg_tv", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.orc_run.argtypes = [P, ctypes.c_int, ctypes.c_int64, P, ctypes.c_int64, P, P, P]
        lib.orc_loss_cs.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_double, P, P]
        lib.orc_adjoint.argtypes = [P, ctypes.c_int64, P, P, P]
        lib.orc_partition.argtypes = [P, P, P]
        lib.orc_lu_solve.argtypes = [ctypes.c_int64, P, P, P]
        lib.orc_rs_states.argtypes = [P, ctypes.c_int64, P]
        lib.orc_controls.argtypes = [P, ctypes.c_int64, P]
        lib.orc_open.argtypes = [P]
        lib.orc_open.restype = P
        lib.orc_advance.argtypes = [P, ctypes.c_int64, P, P]
        lib.orc_line_ends.argtypes = [P, P, P, P]
        lib.orc_sent.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int]
        lib.orc_close.argtypes = [P]
        lib.orc_close.restype = None
        for f in (lib.orc_run, lib.orc_loss_cs, lib.orc_adjoint, lib.orc_partition, lib.orc_lu_solve,
                  lib.orc_rs_states, lib.orc_controls, lib.orc_advance, lib.orc_line_ends, lib.orc_sent):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _arr(x, dtype):
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


class _Pinned:
    """Holds the numpy arrays a ``_Net`` points into."""

    def __init__(self, net):
        self.keep = []

        def p(x, dt):
            a = _arr(x, dt)
            self.keep.append(a)
            return a.ctypes.data if a.size else None

        n = _Net()
        n.dt = float(net.dt)
        n.n_nodes = int(net.n_nodes)
        n.n_br = int(len(net.br_k))
        n.br_k, n.br_m = p(net.br_k, np.int32), p(net.br_m, np.int32)
        n.br_kind, n.br_val = p(net.br_kind, np.uint8), p(net.br_value, np.float64)
        n.n_src = int(len(net.src_amp))
        n.src_amp, n.src_phase, n.src_freq = (p(net.src_amp, np.float64), p(net.src_phase, np.float64),
                                              p(net.src_freq, np.float64))
        n.n_ln = int(len(net.ln_k))
        n.ln_k, n.ln_m = p(net.ln_k, np.int32), p(net.ln_m, np.int32)
        n.ln_zc, n.ln_d = p(net.ln_zc, np.float64), p(net.ln_delay, np.int32)
        n.n_sw = int(len(net.sw_k))
        n.sw_k, n.sw_m = p(net.sw_k, np.int32), p(net.sw_m, np.int32)
        n.sw_r = p(net.sw_r, np.float64)
        n.sw_on, n.sw_off = p(net.sw_close_step, np.int64), p(net.sw_open_step, np.int64)
        rs = lambda name, dt: getattr(net, name, np.zeros(0, dt))
        n.n_rs = int(len(rs("rs_k", np.int32)))
        n.rs_k, n.rs_m = p(rs("rs_k", np.int32), np.int32), p(rs("rs_m", np.int32), np.int32)
        n.rs_kind = p(rs("rs_kind", np.uint8), np.uint8)
        n.rs_ron, n.rs_roff = p(rs("rs_ron", np.float64), np.float64), p(rs("rs_roff", np.float64), np.float64)
        n.rs_on0, n.rs_trip = p(rs("rs_on0", np.uint8), np.uint8), p(rs("rs_trip", np.int64), np.int64)
        n.n_cl = int(len(rs("cl_z", np.float64))) // 3
        n.cl_k, n.cl_m = p(rs("cl_k", np.int32), np.int32), p(rs("cl_m", np.int32), np.int32)
        n.cl_tv, n.cl_z = p(rs("cl_tv", np.float64), np.float64), p(rs("cl_z", np.float64), np.float64)
        n.cl_tau = p(rs("cl_tau", np.float64), np.float64)
        n.n_fl = int(len(rs("fl_k", np.int32)))
        n.fl_k, n.fl_m = p(rs("fl_k", np.int32), np.int32), p(rs("fl_m", np.int32), np.int32)
        n.fl_tau, n.fl_y0 = p(rs("fl_tau", np.float64), np.float64), p(rs("fl_y0", np.float64), np.float64)
        n.fl_ny, n.fl_na = p(rs("fl_ny", np.int32), np.int32), p(rs("fl_na", np.int32), np.int32)
        n.fl_yq, n.fl_yc = p(rs("fl_yq", np.float64), np.float64), p(rs("fl_yc", np.float64), np.float64)
        n.fl_a0 = p(rs("fl_a0", np.float64), np.float64)
        n.fl_ap, n.fl_ar = p(rs("fl_ap", np.float64), np.float64), p(rs("fl_ar", np.float64), np.float64)
        n.n_nl = int(len(rs("nl_k", np.int32)))
        n.nl_k, n.nl_m = p(rs("nl_k", np.int32), np.int32), p(rs("nl_m", np.int32), np.int32)
        n.nl_np = p(rs("nl_np", np.int32), np.int32)
        n.nl_v, n.nl_i = p(rs("nl_v", np.float64), np.float64), p(rs("nl_i", np.float64), np.float64)
        n.n_cb = int(len(rs("cb_type", np.uint8)))
        n.cb_type = p(rs("cb_type", np.uint8), np.uint8)
        n.cb_in0, n.cb_in1 = p(rs("cb_in0", np.int32), np.int32), p(rs("cb_in1", np.int32), np.int32)
        n.cb_node = p(rs("cb_node", np.int32), np.int32)
        n.cb_p0, n.cb_p1 = p(rs("cb_p0", np.float64), np.float64), p(rs("cb_p1", np.float64), np.float64)
        n.n_ci = int(len(rs("ci_block", np.int32)))
        n.ci_block, n.ci_node = p(rs("ci_block", np.int32), np.int32), p(rs("ci_node", np.int32), np.int32)
        n.n_fg = int(len(rs("fg_line", np.int32))) // 3
        n.fg_line, n.fg_tv = p(rs("fg_line", np.int32), np.int32), p(rs("fg_tv", np.float64), np.float64)
        self.net = n

    @property
    def ref(self):
        return ctypes.byref(self.net)


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc} ({'invalid input' if rc == -1 else 'singular matrix'})")


def simulate(net, n_steps: int, monolithic: bool = False, rec=None, v_target=None):
    """Node voltages of steps 1..n_steps: array [n_steps, n_rec] (all nodes
    when ``rec`` is None).  With ``v_target`` also returns the loss."""
    lib = _load()
    pin = _Pinned(net)
    n_rec = int(net.n_nodes) if rec is None else len(rec)
    rec_a = None if rec is None else _arr(rec, np.int32)
    out = np.zeros((int(n_steps), n_rec), dtype=np.float64)
    J = ctypes.c_double(0.0)
    tg = None if v_target is None else _arr(v_target, np.float64)
    rc = lib.orc_run(pin.ref, int(bool(monolithic)), int(n_steps),
                     None if rec_a is None else rec_a.ctypes.data, n_rec,
                     out.ctypes.data if out.size else None,
                     None if tg is None else tg.ctypes.data,
                     None if tg is None else ctypes.addressof(J))
    _check(rc, "orc_run")
    return (out, J.value) if v_target is not None else out


def loss(net, n_steps: int, v_target) -> float:
    lib = _load()
    pin = _Pinned(net)
    tg = _arr(v_target, np.float64)
    J = ctypes.c_double(0.0)
    _check(lib.orc_run(pin.ref, 0, int(n_steps), None, 0, None, tg.ctypes.data, ctypes.addressof(J)), "orc_run")
    return J.value


def loss_complex_step(net, n_steps: int, v_target, param: int, h: float = 1e-30):
    """(J, dJ/dp) for parameter ``param`` by the complex-step method."""
    lib = _load()
    pin = _Pinned(net)
    tg = _arr(v_target, np.float64)
    J = ctypes.c_double(0.0)
    dJ = ctypes.c_double(0.0)
    _check(lib.orc_loss_cs(pin.ref, int(n_steps), tg.ctypes.data, int(param), float(h),
                           ctypes.addressof(J), ctypes.addressof(dJ)), "orc_loss_cs")
    return J.value, dJ.value


def adjoint(net, n_steps: int, v_target):
    """(grad [n_br + n_src], J) by the oracle's discrete adjoint."""
    lib = _load()
    pin = _Pinned(net)
    tg = _arr(v_target, np.float64)
    grad = np.zeros(len(net.br_k) + len(net.src_amp), dtype=np.float64)
    J = ctypes.c_double(0.0)
    _check(lib.orc_adjoint(pin.ref, int(n_steps), tg.ctypes.data, grad.ctypes.data, ctypes.addressof(J)),
           "orc_adjoint")
    return grad, J.value


def runtime_switch_states(net, n_steps: int):
    """States of the runtime switches in force at steps 1..n_steps: [n_steps, n_rs] uint8."""
    lib = _load()
    pin = _Pinned(net)
    out = np.zeros((int(n_steps), pin.net.n_rs), dtype=np.uint8)
    _check(lib.orc_rs_states(pin.ref, int(n_steps), out.ctypes.data if out.size else None), "orc_rs_states")
    return out


def controls(net, n_steps: int):
    """Control block outputs of steps 1..n_steps: [n_steps, n_cb]."""
    lib = _load()
    pin = _Pinned(net)
    out = np.zeros((int(n_steps), pin.net.n_cb), dtype=np.float64)
    _check(lib.orc_controls(pin.ref, int(n_steps), out.ctypes.data if out.size else None), "orc_controls")
    return out


def partition(net):
    """(subsystem id per unknown node, number of subsystems)."""
    lib = _load()
    pin = _Pinned(net)
    sub = np.zeros(int(net.n_nodes), dtype=np.int32)
    ns = ctypes.c_int64(0)
    _check(lib.orc_partition(pin.ref, sub.ctypes.data, ctypes.addressof(ns)), "orc_partition")
    return sub, ns.value


def lu_solve(A, b):
    lib = _load()
    A = _arr(A, np.float64)
    b = _arr(b, np.float64)
    x = np.zeros_like(b)
    _check(lib.orc_lu_solve(int(A.shape[0]), A.ctypes.data, b.ctypes.data, x.ctypes.data), "orc_lu_solve")
    return x


def line_ends(net):
    """(node, far end, d) of every line end: lines (k, m), coupled lines
    (end k's modes, end m's modes), frequency-dependent lines (k, m)."""
    lib = _load()
    pin = _Pinned(net)
    n = 2 * pin.net.n_ln + 6 * pin.net.n_cl + 2 * pin.net.n_fl
    node, far, d = (np.zeros(n, dtype=np.int32) for _ in range(3))
    if n:
        _check(lib.orc_line_ends(pin.ref, node.ctypes.data, far.ctypes.data, d.ctypes.data), "orc_line_ends")
    return node, far, d


class Session:
    """The loop run window by window on a chosen set of subsystems (see
    orc_advance in emt_oracle.h): the oracle side of a sharded run."""

    def __init__(self, net):
        lib = _load()
        self.n_nodes = int(net.n_nodes)
        self._pin = _Pinned(net)          # the C session points into these arrays
        self._h = lib.orc_open(self._pin.ref)
        if not self._h:
            raise OracleError("orc_open failed (invalid input)")
        self.step = 0

    def advance(self, n_steps: int, active=None):
        """Run n_steps more steps; ``active``: per subsystem (orc_partition), truthy = run it.
        Returns the node voltages [n_steps, n_nodes]."""
        out = np.zeros((int(n_steps), self.n_nodes), dtype=np.float64)
        act = None if active is None else _arr(active, np.uint8)
        _check(_load().orc_advance(self._h, int(n_steps), None if act is None else act.ctypes.data,
                                   out.ctypes.data if out.size else None), "orc_advance")
        self.step += int(n_steps)
        return out

    def sent(self, end: int, n0: int, w: int):
        vals = np.zeros(int(w), dtype=np.float64)
        _check(_load().orc_sent(self._h, int(end), int(n0), int(w), vals.ctypes.data if w else None, 0), "orc_sent")
        return vals

    def set_sent(self, end: int, n0: int, vals):
        v = _arr(vals, np.float64)
        _check(_load().orc_sent(self._h, int(end), int(n0), v.size, v.ctypes.data if v.size else None, 1),
               "orc_sent")

    def close(self):
        if self._h:
            _load().orc_close(self._h)
            self._h = None

    def __del__(self):
        self.close()
