"""Seeded synthetic network generator.

This module only draws inputs: topology, element values, sources, lines,
switches and per-scenario overrides.  It holds none of the simulation's
arithmetic (no companion conductances, no partitioning, no solves), so both
the CUDA path and the CPU oracle can take its output as their common input.

Node codes follow one convention everywhere:
  * ``k >= 0``   an unknown node,
  * ``k == -1``  ground,
  * ``k == -2-s`` the known-voltage node of source ``s``.

Element value ranges are those of the paper's test-case family as stated for
the synthetic workloads: R ~ U[0.1, 10] ohm, L ~ U[1, 100] mH,
C ~ U[1, 100] uF, sources of 1 kV peak at 60 Hz, lossless lines with
Z_c ~ U[200, 500] ohm and integer travel times of 1..20 steps.  The paper's
own test feeder (Sec. IV-A, Fig. 5) is not available, so these networks
stand in for its large-scale and multi-scenario cases (Sec. IV-B, IV-C).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

R_RANGE = (0.1, 10.0)          # ohm
L_RANGE = (1e-3, 100e-3)       # henry
C_RANGE = (1e-6, 100e-6)       # farad
ZC_RANGE = (200.0, 500.0)      # ohm
DELAY_RANGE = (1, 20)          # steps, inclusive
V_PEAK = 1000.0                # volt (1 kV peak = 1 p.u.)
F_HZ = 60.0
R_FAULT = 0.01                 # ohm

KIND_R, KIND_L, KIND_C = 0, 1, 2
GROUND = -1


def source_node(s: int) -> int:
    """Node code of the known-voltage node of source ``s``."""
    return -2 - s


@dataclass
class Network:
    """Plain arrays describing one network (all numpy, C-contiguous)."""
    dt: float
    n_nodes: int
    br_k: np.ndarray            # int32 [n_br]
    br_m: np.ndarray            # int32 [n_br]
    br_kind: np.ndarray         # uint8 [n_br]  0=R 1=L 2=C
    br_value: np.ndarray        # float64 [n_br] ohm / henry / farad
    src_amp: np.ndarray         # float64 [n_src] peak volts
    src_phase: np.ndarray       # float64 [n_src] rad
    src_freq: np.ndarray        # float64 [n_src] Hz
    ln_k: np.ndarray            # int32 [n_ln]
    ln_m: np.ndarray            # int32 [n_ln]
    ln_zc: np.ndarray           # float64 [n_ln] ohm
    ln_delay: np.ndarray        # int32 [n_ln] steps >= 1
    sw_k: np.ndarray            # int32 [n_sw]
    sw_m: np.ndarray            # int32 [n_sw]
    sw_r: np.ndarray            # float64 [n_sw] ohm (closed resistance)
    sw_close_step: np.ndarray   # int64 [n_sw]; closed for close <= n < open
    sw_open_step: np.ndarray    # int64 [n_sw]; -1 = never opens
    # runtime switches: two-state resistors whose state is decided from the
    # previous step's solution (kind 0 diode k->m, kind 1 current-zero breaker)
    rs_k: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    rs_m: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    rs_kind: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))
    rs_ron: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    rs_roff: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    rs_on0: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))
    rs_trip: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    # coupled three-phase lossless lines in modal form: phase nodes per end
    # [3 L], T_v [9 L] (phase voltages = T_v modal voltages), modal Z_c and
    # travel times in seconds [3 L]
    cl_k: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    cl_m: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    cl_tv: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    cl_z: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    cl_tau: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    # frequency-dependent lines (one conductor each): ends, travel time (s),
    # Y_c = y0 + sum c_i/(s - q_i) and A = e^{-s tau}(a0 + sum r_i/(s - p_i)),
    # up to 4 poles each in [4 l + i] slots (unused slots 0)
    fl_k: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    fl_m: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    fl_tau: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    fl_y0: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    fl_ny: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    fl_yq: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    fl_yc: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    fl_a0: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    fl_na: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    fl_ap: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    fl_ar: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    # nonlinear resistors (compensation method): ends, and an odd piecewise-
    # linear i(v) through (0, 0) and up to 8 points (v > 0 increasing, i
    # nondecreasing) in [8 e + j] slots; at most one per subsystem
    nl_k: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    nl_m: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    nl_np: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    nl_v: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    nl_i: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    # control blocks (CB_* types), evaluated after each step's solve; an input
    # of lower index reads its step-n output, of equal or higher index its
    # step-(n-1) output.  Controlled current injections: block output y(n)
    # enters node ci_node at step n + 1.
    cb_type: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))
    cb_in0: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    cb_in1: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    cb_node: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    cb_p0: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    cb_p1: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    ci_block: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    ci_node: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    # frequency-dependent line groups: fg_line[3 g + j] is the frequency-
    # dependent line carrying mode j of a three-phase line (its ends are
    # phase j's nodes), fg_tv[9 g + 3 p + j] the group's T_v (phase voltages
    # = T_v modal voltages; modal currents T_i = T_v^-T)
    fg_line: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    fg_tv: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    n_steps: int = 0            # suggested run length
    meta: dict = field(default_factory=dict)

    @property
    def n_branches(self) -> int:
        return int(self.br_k.shape[0])

    @property
    def n_sources(self) -> int:
        return int(self.src_amp.shape[0])

    @property
    def n_lines(self) -> int:
        return int(self.ln_k.shape[0])

    @property
    def n_switches(self) -> int:
        return int(self.sw_k.shape[0])

    @property
    def n_runtime_switches(self) -> int:
        return int(self.rs_k.shape[0])

    @property
    def n_coupled_lines(self) -> int:
        return int(self.cl_z.shape[0]) // 3

    @property
    def n_nonlinear(self) -> int:
        return int(self.nl_k.shape[0])

    @property
    def n_fd_lines(self) -> int:
        return int(self.fl_k.shape[0])

    @property
    def n_control_blocks(self) -> int:
        return int(self.cb_type.shape[0])

    @property
    def n_control_injections(self) -> int:
        return int(self.ci_block.shape[0])

    def copy(self) -> "Network":
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            kw[f.name] = v.copy() if isinstance(v, np.ndarray) else (dict(v) if isinstance(v, dict) else v)
        return Network(**kw)

    def with_params(self, br_value: Optional[np.ndarray] = None, src_amp: Optional[np.ndarray] = None) -> "Network":
        net = self.copy()
        if br_value is not None:
            net.br_value = np.ascontiguousarray(br_value, dtype=np.float64)
        if src_amp is not None:
            net.src_amp = np.ascontiguousarray(src_amp, dtype=np.float64)
        return net


@dataclass
class Scenarios:
    """Per-scenario overrides of a base network.

    * ``src_amp`` / ``src_phase``: [S, n_src] or None (base values).
    * removed branches / lines: CSR lists (``*_ptr`` has S+1 entries).
    * extra switches (faults): CSR over scenarios of (k, m, r, close, open).
    * control-block parameters: CSR over scenarios of (block, new p0).
    """
    n_scenarios: int
    src_amp: Optional[np.ndarray] = None
    src_phase: Optional[np.ndarray] = None
    rm_branch_ptr: Optional[np.ndarray] = None
    rm_branch: Optional[np.ndarray] = None
    rm_line_ptr: Optional[np.ndarray] = None
    rm_line: Optional[np.ndarray] = None
    sw_ptr: Optional[np.ndarray] = None
    sw_k: Optional[np.ndarray] = None
    sw_m: Optional[np.ndarray] = None
    sw_r: Optional[np.ndarray] = None
    sw_close_step: Optional[np.ndarray] = None
    sw_open_step: Optional[np.ndarray] = None
    cbo_ptr: Optional[np.ndarray] = None
    cbo_block: Optional[np.ndarray] = None
    cbo_p0: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    def subset(self, idx) -> "Scenarios":
        """The scenarios ``idx`` (a sequence of indices) as a new set."""
        idx = [int(i) for i in idx]
        out = Scenarios(n_scenarios=len(idx), meta=dict(self.meta))
        if self.src_amp is not None:
            out.src_amp = np.ascontiguousarray(self.src_amp[idx])
        if self.src_phase is not None:
            out.src_phase = np.ascontiguousarray(self.src_phase[idx])

        def sub_csr(ptr, *cols):
            if ptr is None:
                return (None,) * (len(cols) + 1)
            new_ptr = [0]
            parts = [[] for _ in cols]
            for i in idx:
                a, b = int(ptr[i]), int(ptr[i + 1])
                for p, c in zip(parts, cols):
                    p.append(c[a:b])
                new_ptr.append(new_ptr[-1] + (b - a))
            res = [np.asarray(new_ptr, dtype=np.int64)]
            for p, c in zip(parts, cols):
                res.append(np.ascontiguousarray(np.concatenate(p) if p else c[:0]).astype(c.dtype))
            return tuple(res)

        out.rm_branch_ptr, out.rm_branch = sub_csr(self.rm_branch_ptr, self.rm_branch) if self.rm_branch_ptr is not None else (None, None)
        out.rm_line_ptr, out.rm_line = sub_csr(self.rm_line_ptr, self.rm_line) if self.rm_line_ptr is not None else (None, None)
        if self.sw_ptr is not None:
            (out.sw_ptr, out.sw_k, out.sw_m, out.sw_r, out.sw_close_step, out.sw_open_step) = sub_csr(
                self.sw_ptr, self.sw_k, self.sw_m, self.sw_r, self.sw_close_step, self.sw_open_step)
        if self.cbo_ptr is not None:
            out.cbo_ptr, out.cbo_block, out.cbo_p0 = sub_csr(self.cbo_ptr, self.cbo_block, self.cbo_p0)
        return out

    def expand(self, base: Network, s: int) -> Network:
        """Scenario ``s`` written out as a plain network.

        Removed branches and lines are dropped, extra switches appended and
        source overrides substituted.  This is input bookkeeping only.
        """
        net = base.copy()
        if self.src_amp is not None:
            net.src_amp = np.ascontiguousarray(self.src_amp[s], dtype=np.float64)
        if self.src_phase is not None:
            net.src_phase = np.ascontiguousarray(self.src_phase[s], dtype=np.float64)
        if self.rm_branch_ptr is not None:
            rm = set(int(x) for x in self.rm_branch[self.rm_branch_ptr[s]:self.rm_branch_ptr[s + 1]])
            keep = np.array([i not in rm for i in range(base.n_branches)], dtype=bool)
            for f in ("br_k", "br_m", "br_kind", "br_value"):
                setattr(net, f, np.ascontiguousarray(getattr(net, f)[keep]))
            net.meta["kept_branches"] = np.nonzero(keep)[0]
        if self.rm_line_ptr is not None:
            rm = set(int(x) for x in self.rm_line[self.rm_line_ptr[s]:self.rm_line_ptr[s + 1]])
            keep = np.array([i not in rm for i in range(base.n_lines)], dtype=bool)
            for f in ("ln_k", "ln_m", "ln_zc", "ln_delay"):
                setattr(net, f, np.ascontiguousarray(getattr(net, f)[keep]))
        if self.sw_ptr is not None:
            a, b = int(self.sw_ptr[s]), int(self.sw_ptr[s + 1])
            net.sw_k = np.ascontiguousarray(np.concatenate([net.sw_k, self.sw_k[a:b]]).astype(np.int32))
            net.sw_m = np.ascontiguousarray(np.concatenate([net.sw_m, self.sw_m[a:b]]).astype(np.int32))
            net.sw_r = np.ascontiguousarray(np.concatenate([net.sw_r, self.sw_r[a:b]]).astype(np.float64))
            net.sw_close_step = np.ascontiguousarray(
                np.concatenate([net.sw_close_step, self.sw_close_step[a:b]]).astype(np.int64))
            net.sw_open_step = np.ascontiguousarray(
                np.concatenate([net.sw_open_step, self.sw_open_step[a:b]]).astype(np.int64))
        if self.cbo_ptr is not None:
            a, b = int(self.cbo_ptr[s]), int(self.cbo_ptr[s + 1])
            net.cb_p0 = np.array(net.cb_p0, dtype=np.float64)
            net.cb_p0[self.cbo_block[a:b]] = self.cbo_p0[a:b]
        return net


# ----------------------------------------------------------------------------
# helpers

def _value(rng: np.random.Generator, kind: int) -> float:
    lo, hi = (R_RANGE, L_RANGE, C_RANGE)[kind]
    return float(rng.uniform(lo, hi))


class NetworkBuilder:
    def __init__(self):
        self.br = []     # (k, m, kind, value)
        self.src = []    # (amp, phase, freq)
        self.ln = []     # (k, m, zc, d)
        self.sw = []     # (k, m, r, close, open)
        self.rs = []     # (k, m, kind, r_on, r_off, on0, trip)
        self.cl = []     # (k3, m3, tv9, z3, tau3)
        self.fl = []     # (k, m, tau, y0, yq4, yc4, ny, a0, ap4, ar4, na)
        self.nl = []     # (k, m, np, v8, i8)
        self.cb = []     # (type, in0, in1, node, p0, p1)
        self.ci = []     # (block, node)

    def branch(self, k, m, kind, value):
        self.br.append((int(k), int(m), int(kind), float(value)))
        return len(self.br) - 1

    def source(self, amp, phase, freq=F_HZ):
        self.src.append((float(amp), float(phase), float(freq)))
        return len(self.src) - 1

    def line(self, k, m, zc, d):
        self.ln.append((int(k), int(m), float(zc), int(d)))
        return len(self.ln) - 1

    def switch(self, k, m, r, close, open_=-1):
        self.sw.append((int(k), int(m), float(r), int(close), int(open_)))

    def diode(self, anode, cathode, r_on, r_off, on0=False):
        self.rs.append((int(anode), int(cathode), 0, float(r_on), float(r_off), int(bool(on0)), -1))

    def breaker(self, k, m, r_on, r_off, trip_step):
        self.rs.append((int(k), int(m), 1, float(r_on), float(r_off), 1, int(trip_step)))

    def coupled_line(self, k3, m3, tv, z3, tau3):
        """Three-phase lossless line in modal form (see ``Network.cl_*``)."""
        self.cl.append(([int(x) for x in k3], [int(x) for x in m3], np.asarray(tv, np.float64).reshape(9),
                        np.asarray(z3, np.float64).reshape(3), np.asarray(tau3, np.float64).reshape(3)))

    def fd_line(self, k, m, tau, y0, yq=(), yc=(), a0=0.0, ap=(), ar=()):
        """Frequency-dependent line (see ``Network.fl_*``): travel time ``tau``
        in seconds, Y_c's direct term and poles/residues, A's direct term and
        poles/residues (at most 4 each)."""
        pad = lambda x: list(map(float, x)) + [0.0] * (4 - len(x))
        assert len(yq) == len(yc) <= 4 and len(ap) == len(ar) <= 4
        self.fl.append((int(k), int(m), float(tau), float(y0), pad(yq), pad(yc), len(yq), float(a0), pad(ap), pad(ar),
                        len(ap)))
        return len(self.fl) - 1

    def nonlinear_resistor(self, k, m, v_points, i_points):
        """Odd piecewise-linear resistor i = f(v_k - v_m) through (0, 0) and the
        given points (see ``Network.nl_*``)."""
        assert 1 <= len(v_points) == len(i_points) <= 8
        pad = lambda x: list(map(float, x)) + [0.0] * (8 - len(x))
        self.nl.append((int(k), int(m), len(v_points), pad(v_points), pad(i_points)))
        return len(self.nl) - 1

    def block(self, kind, in0=-1, in1=-1, node=-1, p0=0.0, p1=0.0):
        """Control block of type ``kind`` (CB_*); returns its index."""
        self.cb.append((int(kind), int(in0), int(in1), int(node), float(p0), float(p1)))
        return len(self.cb) - 1

    def injection(self, block, node):
        """Controlled current: block output y(n) enters ``node`` at step n + 1."""
        self.ci.append((int(block), int(node)))

    def build(self, dt, n_nodes, n_steps=0, meta=None) -> Network:
        def col(lst, i, dt_):
            return np.ascontiguousarray(np.array([x[i] for x in lst], dtype=dt_))
        return Network(
            dt=float(dt), n_nodes=int(n_nodes),
            br_k=col(self.br, 0, np.int32), br_m=col(self.br, 1, np.int32),
            br_kind=col(self.br, 2, np.uint8), br_value=col(self.br, 3, np.float64),
            src_amp=col(self.src, 0, np.float64), src_phase=col(self.src, 1, np.float64),
            src_freq=col(self.src, 2, np.float64),
            ln_k=col(self.ln, 0, np.int32), ln_m=col(self.ln, 1, np.int32),
            ln_zc=col(self.ln, 2, np.float64), ln_delay=col(self.ln, 3, np.int32),
            sw_k=col(self.sw, 0, np.int32), sw_m=col(self.sw, 1, np.int32),
            sw_r=col(self.sw, 2, np.float64), sw_close_step=col(self.sw, 3, np.int64),
            sw_open_step=col(self.sw, 4, np.int64),
            rs_k=col(self.rs, 0, np.int32), rs_m=col(self.rs, 1, np.int32), rs_kind=col(self.rs, 2, np.uint8),
            rs_ron=col(self.rs, 3, np.float64), rs_roff=col(self.rs, 4, np.float64),
            rs_on0=col(self.rs, 5, np.uint8), rs_trip=col(self.rs, 6, np.int64),
            cl_k=np.ascontiguousarray(np.array([x for c in self.cl for x in c[0]], np.int32)),
            cl_m=np.ascontiguousarray(np.array([x for c in self.cl for x in c[1]], np.int32)),
            cl_tv=np.ascontiguousarray(np.concatenate([c[2] for c in self.cl]) if self.cl else np.zeros(0)),
            cl_z=np.ascontiguousarray(np.concatenate([c[3] for c in self.cl]) if self.cl else np.zeros(0)),
            cl_tau=np.ascontiguousarray(np.concatenate([c[4] for c in self.cl]) if self.cl else np.zeros(0)),
            fl_k=col(self.fl, 0, np.int32), fl_m=col(self.fl, 1, np.int32), fl_tau=col(self.fl, 2, np.float64),
            fl_y0=col(self.fl, 3, np.float64), fl_ny=col(self.fl, 6, np.int32), fl_a0=col(self.fl, 7, np.float64),
            fl_na=col(self.fl, 10, np.int32),
            fl_yq=np.ascontiguousarray(np.array([x for f in self.fl for x in f[4]], np.float64)),
            fl_yc=np.ascontiguousarray(np.array([x for f in self.fl for x in f[5]], np.float64)),
            fl_ap=np.ascontiguousarray(np.array([x for f in self.fl for x in f[8]], np.float64)),
            fl_ar=np.ascontiguousarray(np.array([x for f in self.fl for x in f[9]], np.float64)),
            nl_k=col(self.nl, 0, np.int32), nl_m=col(self.nl, 1, np.int32), nl_np=col(self.nl, 2, np.int32),
            nl_v=np.ascontiguousarray(np.array([x for e in self.nl for x in e[3]], np.float64)),
            nl_i=np.ascontiguousarray(np.array([x for e in self.nl for x in e[4]], np.float64)),
            cb_type=col(self.cb, 0, np.uint8), cb_in0=col(self.cb, 1, np.int32), cb_in1=col(self.cb, 2, np.int32),
            cb_node=col(self.cb, 3, np.int32), cb_p0=col(self.cb, 4, np.float64), cb_p1=col(self.cb, 5, np.float64),
            ci_block=col(self.ci, 0, np.int32), ci_node=col(self.ci, 1, np.int32),
            n_steps=int(n_steps), meta=dict(meta or {}))


# ----------------------------------------------------------------------------
# single-subsystem random RLC network (config 1 shape)

def single_rlc(seed: int = 1001, n_nodes: int = 12, n_branches: int = 20, dt: float = 50e-6,
               n_steps: int = 20000, fault_step: Optional[int] = 2000) -> Network:
    """Random single-phase RLC network with one 60 Hz source of 1 kV peak.

    Topology: a random spanning tree over {ground, source node, unknown
    nodes} plus random extra edges up to ``n_branches`` (never ground to
    source, never a self loop, no duplicate pair).  Each branch holds one
    element whose kind is uniform over {R, L, C}.  A 0.01 ohm fault switch to
    ground at a random unknown node closes at ``fault_step``.
    """
    rng = np.random.default_rng(seed)
    b = NetworkBuilder()
    b.source(V_PEAK, 0.0)
    # vertices: 0 = ground, 1 = source, 2.. = unknown nodes
    nv = n_nodes + 2
    code = lambda v: GROUND if v == 0 else (source_node(0) if v == 1 else v - 2)
    edges = []
    seen = set()

    def add(a, c):
        key = (min(a, c), max(a, c))
        if a == c or key == (0, 1) or key in seen:
            return False
        seen.add(key)
        edges.append(key)
        return True

    # spanning tree over {ground, unknown nodes} by random attachment,
    # then the source vertex hangs off a random unknown node
    order = [0] + [int(x) + 2 for x in rng.permutation(n_nodes)]
    for i in range(1, len(order)):
        add(order[i], order[int(rng.integers(0, i))])
    add(1, int(rng.integers(2, nv)))
    while len(edges) < n_branches:
        a, c = (int(x) for x in rng.integers(0, nv, size=2))
        add(a, c)
    for (a, c) in edges:
        kind = int(rng.integers(0, 3))
        k, m = code(c), code(a)   # c > a, so k is never ground
        if m >= 0 and rng.random() < 0.5:
            k, m = m, k
        b.branch(k, m, kind, _value(rng, kind))
    if fault_step is not None:
        node = int(rng.integers(0, n_nodes))
        b.switch(node, GROUND, R_FAULT, fault_step, -1)
    return b.build(dt, n_nodes, n_steps, meta={"kind": "single_rlc", "seed": seed})


# ----------------------------------------------------------------------------
# multi-subsystem three-phase networks cut by Bergeron lines (configs 2-5)

def multi_subsystem(seed: int, bus_counts, n_lines: int, n_sources: int, dt: float,
                    n_steps: int = 0, phases: int = 3, p2p_frac: float = 0.2,
                    n_series_extra: int = 0, source_phase_random: bool = True,
                    shunt_kinds=(KIND_R, KIND_L, KIND_C), shuffle_nodes: bool = True,
                    delay_range=DELAY_RANGE, zc_range=ZC_RANGE) -> Network:
    """Three-phase (or single-phase) network made of subsystems cut by lines.

    * ``bus_counts[j]`` buses in subsystem j; each bus has ``phases`` nodes.
    * inside a subsystem: a random spanning tree of series connections over
      its buses plus ``n_series_extra`` extra connections network-wide; a
      series connection is one branch per phase, kind uniform over {R, L, C}
      per connection, value drawn per phase.
    * every node has one shunt branch to ground (kind from ``shunt_kinds``).
    * every subsystem gets phase-to-phase branches (a-b, b-c) at one random
      bus, and ``p2p_frac`` of all buses get one more phase-to-phase branch.
    * ``n_lines`` lines: first a random spanning tree over the subsystems,
      then random pairs of distinct subsystems; a line joins a random bus of
      each side, one lossless conductor per phase, with one Z_c and one delay
      per line.
    * ``n_sources`` sources: one known node per phase at 1 kV peak, phase
      shifts 0, -2pi/3, +2pi/3 on top of a random (or zero) angle, each
      joined to its bus's phase node by an R or L branch.
    Unknown node numbers are randomly permuted when ``shuffle_nodes``.
    """
    rng = np.random.default_rng(seed)
    bus_counts = [int(x) for x in bus_counts]
    n_sub = len(bus_counts)
    n_bus = sum(bus_counts)
    n_nodes = n_bus * phases
    perm = rng.permutation(n_nodes) if shuffle_nodes else np.arange(n_nodes)
    node = lambda bus, p: int(perm[bus * phases + p])
    sub_of_bus = np.repeat(np.arange(n_sub), bus_counts)
    first_bus = np.concatenate([[0], np.cumsum(bus_counts)[:-1]]).astype(int)
    b = NetworkBuilder()

    def series(ba, bb, kind=None):
        kind = int(rng.integers(0, 3)) if kind is None else kind
        for p in range(phases):
            b.branch(node(ba, p), node(bb, p), kind, _value(rng, kind))

    conn = []  # inter-bus three-phase connections: ("br", [branch ids]) or ("ln", [line ids])
    for j in range(n_sub):
        f, nb = first_bus[j], bus_counts[j]
        for i in range(1, nb):
            a = f + i
            c = f + int(rng.integers(0, i))
            start = len(b.br)
            series(a, c)
            conn.append(("br", list(range(start, len(b.br)))))
    for _ in range(n_series_extra):
        j = int(rng.integers(0, n_sub))
        if bus_counts[j] < 2:
            continue
        a, c = rng.choice(bus_counts[j], size=2, replace=False) + first_bus[j]
        start = len(b.br)
        series(int(a), int(c))
        conn.append(("br", list(range(start, len(b.br)))))
    for bus in range(n_bus):
        for p in range(phases):
            kind = int(rng.choice(shunt_kinds))
            b.branch(node(bus, p), GROUND, kind, _value(rng, kind))
    if phases >= 2:
        # couple the phases of every subsystem at one random bus so that a
        # subsystem is one electrical component, not one per phase
        for j in range(n_sub):
            bus = first_bus[j] + int(rng.integers(0, bus_counts[j]))
            for p in range(phases - 1):
                kind = int(rng.integers(0, 3))
                b.branch(node(bus, p), node(bus, p + 1), kind, _value(rng, kind))
        for bus in range(n_bus):
            if rng.random() < p2p_frac:
                p, q = rng.choice(phases, size=2, replace=False)
                kind = int(rng.integers(0, 3))
                b.branch(node(bus, int(p)), node(bus, int(q)), kind, _value(rng, kind))
    # lines
    pairs = []
    order = rng.permutation(n_sub)
    for i in range(1, n_sub):
        pairs.append((int(order[i]), int(order[rng.integers(0, i)])))
    while len(pairs) < n_lines and n_sub >= 2:
        a, c = rng.choice(n_sub, size=2, replace=False)
        pairs.append((int(a), int(c)))
    for (sa, sb) in pairs[:n_lines]:
        ba = first_bus[sa] + int(rng.integers(0, bus_counts[sa]))
        bb = first_bus[sb] + int(rng.integers(0, bus_counts[sb]))
        zc = float(rng.uniform(*zc_range))
        d = int(rng.integers(delay_range[0], delay_range[1] + 1))
        start = len(b.ln)
        for p in range(phases):
            b.line(node(ba, p), node(bb, p), zc, d)
        conn.append(("ln", list(range(start, len(b.ln)))))
    # sources
    shifts = [0.0, -2.0 * np.pi / 3.0, 2.0 * np.pi / 3.0][:phases]
    src_bus = []
    for _ in range(n_sources):
        bus = int(rng.integers(0, n_bus))
        src_bus.append(bus)
        phi0 = float(rng.uniform(0.0, 2.0 * np.pi)) if source_phase_random else 0.0
        kind = int(rng.integers(0, 2))   # R or L source impedance
        for p in range(phases):
            s = b.source(V_PEAK, phi0 + shifts[p])
            b.branch(source_node(s), node(bus, p), kind, _value(rng, kind))
    meta = {"kind": "multi_subsystem", "seed": seed, "bus_counts": bus_counts, "phases": phases,
            "n_subsystems": n_sub, "connections": conn, "source_bus": src_bus,
            "bus_nodes": [[node(bus, p) for p in range(phases)] for bus in range(n_bus)]}
    return b.build(dt, n_nodes, n_steps, meta=meta)


def _sizes_uniform_to_total(rng, total, lo, hi):
    """Draw sizes ~ U{lo..hi} until they sum to ``total`` (last one clipped/merged)."""
    sizes = []
    left = total
    while left > 0:
        s = int(rng.integers(lo, hi + 1))
        if left - s < lo and left - s != 0:
            s = left if left <= hi else left - lo
        s = min(s, left)
        sizes.append(s)
        left -= s
    return sizes


def _sizes_fixed_count(rng, total, count, lo, hi):
    """``count`` sizes in [lo, hi] summing to ``total``: start at ``lo``, add units at random."""
    sizes = np.full(count, lo, dtype=int)
    left = total - lo * count
    assert 0 <= left <= (hi - lo) * count
    while left > 0:
        j = int(rng.integers(0, count))
        if sizes[j] < hi:
            sizes[j] += 1
            left -= 1
    return [int(x) for x in sizes]


def large_scale(seed: int = 1002, n_buses: int = 1000, n_lines: int = 700, n_sources: int = 50,
                dt: float = 20e-6, n_steps: int = 50000, target_branches: int = 6000,
                strict_500: bool = False, n_sub: Optional[int] = None) -> Network:
    """Large-scale three-phase network: 1,000 buses (3,000 nodes), ~6,000
    branches, 700 three-phase Bergeron lines, 50 three-phase sources.

    Subsystem sizes are 3*U{2..20} nodes drawn until the 1,000 buses are used
    (the subsystem count falls out, about a hundred).  ``strict_500`` instead
    makes 500 subsystems of 2 buses (6 nodes) each; ``n_sub`` makes exactly
    that many subsystems of 2..20 buses.
    """
    rng = np.random.default_rng(seed)
    if strict_500:
        bus_counts = [2] * (n_buses // 2)
    elif n_sub is not None:
        bus_counts = _sizes_fixed_count(rng, n_buses, n_sub, 2, 20)
    else:
        bus_counts = _sizes_uniform_to_total(rng, n_buses, 2, 20)
    tree = n_buses - len(bus_counts)
    p2p = int(round(0.2 * n_buses)) + 2 * len(bus_counts)
    extra = max(0, (target_branches - 3 * n_buses - p2p - 3 * n_sources - 3 * tree) // 3)
    sub_seed = int(rng.integers(0, 2**31))
    net = multi_subsystem(sub_seed, bus_counts, n_lines, n_sources, dt, n_steps=n_steps,
                          n_series_extra=extra)
    net.meta.update({"config": "large_scale_strict500" if strict_500 else "large_scale", "seed": seed})
    return net


def paper_scale(n_sub: int = 500, seed: int = 1011, dt: float = 20e-6, n_steps: int = 20000) -> Network:
    """The large-scale family grown towards the size of the paper's largest
    case (16,653 nodes): ``n_sub`` subsystems of 2..20 three-phase buses
    (11 on average), and lines, sources and branches scaled from the
    1,000-bus network by the bus count (500 subsystems: 16,500 nodes)."""
    n_buses = 11 * n_sub
    f = n_buses / 1000.0
    net = large_scale(seed=seed, n_buses=n_buses, n_lines=int(round(700 * f)), n_sources=int(round(50 * f)),
                      dt=dt, n_steps=n_steps, target_branches=int(round(6000 * f)), n_sub=n_sub)
    net.meta.update({"config": "paper_scale", "seed": seed})
    return net


def n1_contingency(seed: int = 1003, n_scenarios: int = 1024, n_buses: int = 200, n_sub: int = 40,
                   n_lines: int = 56, n_sources: int = 10, dt: float = 20e-6, n_steps: int = 10000,
                   fault_step: int = 2500, target_branches: int = 1200):
    """Multi-scenario N-1 workload: a 200-bus (600-node) network in 40
    subsystems of 2..15 buses; scenario s removes one random three-phase
    connection (series branch triplet or line) and applies a three-phase
    fault (three 0.01 ohm phase-to-ground resistors) at a random bus at
    ``fault_step``.  Scenario s draws from ``default_rng([seed, s])``.
    """
    rng = np.random.default_rng(seed)
    bus_counts = _sizes_fixed_count(rng, n_buses, n_sub, 2, 15)
    tree = n_buses - n_sub
    p2p = int(round(0.2 * n_buses)) + 2 * n_sub
    extra = max(0, (target_branches - 3 * n_buses - p2p - 3 * n_sources - 3 * tree) // 3)
    net = multi_subsystem(int(rng.integers(0, 2**31)), bus_counts, n_lines, n_sources, dt,
                          n_steps=n_steps, n_series_extra=extra)
    net.meta.update({"config": "n1_contingency", "seed": seed})
    conns = net.meta["connections"]
    n_bus = n_buses
    rm_b_ptr, rm_b, rm_l_ptr, rm_l = [0], [], [0], []
    sw_ptr, swk, swm, swr, swc, swo = [0], [], [], [], [], []
    removed = []
    for s in range(n_scenarios):
        srng = np.random.default_rng([seed, s])
        kind, ids = conns[int(srng.integers(0, len(conns)))]
        removed.append((kind, list(ids)))
        if kind == "br":
            rm_b.extend(ids)
        else:
            rm_l.extend(ids)
        rm_b_ptr.append(len(rm_b))
        rm_l_ptr.append(len(rm_l))
        bus = int(srng.integers(0, n_bus))
        for nd in net.meta["bus_nodes"][bus]:
            swk.append(nd); swm.append(GROUND); swr.append(R_FAULT); swc.append(fault_step); swo.append(-1)
        sw_ptr.append(len(swk))
    sc = Scenarios(
        n_scenarios=n_scenarios,
        rm_branch_ptr=np.asarray(rm_b_ptr, np.int64), rm_branch=np.asarray(rm_b, np.int32),
        rm_line_ptr=np.asarray(rm_l_ptr, np.int64), rm_line=np.asarray(rm_l, np.int32),
        sw_ptr=np.asarray(sw_ptr, np.int64), sw_k=np.asarray(swk, np.int32), sw_m=np.asarray(swm, np.int32),
        sw_r=np.asarray(swr, np.float64), sw_close_step=np.asarray(swc, np.int64),
        sw_open_step=np.asarray(swo, np.int64), meta={"removed": removed, "fault_step": fault_step})
    return net, sc


def shared_g(seed: int = 1004, n_scenarios: int = 4096, dt: float = 20e-6, n_steps: int = 10000,
             fault_step: int = 2500, base: Optional[Network] = None):
    """Shared-G multi-scenario workload on the large-scale topology.

    Scenario s: each three-phase source gets amplitude 1 kV * U[0.9, 1.1]
    and angle U[0, 2pi) (phases keep their -2pi/3, +2pi/3 shifts); a
    three-phase fault of resistance R_f ~ U[0.01, 10] ohm per phase to
    ground at one seeded bus (the same bus for all scenarios) closes at
    ``fault_step``.
    """
    if base is None:
        base = large_scale(n_steps=n_steps, dt=dt)
    net = base.copy()
    net.dt = dt
    net.n_steps = n_steps
    rng = np.random.default_rng(seed)
    n_bus = len(net.meta["bus_nodes"])
    phases = net.meta["phases"]
    fault_bus = int(rng.integers(0, n_bus))
    n_src = net.n_sources
    n3 = n_src // phases
    shifts = np.array([0.0, -2.0 * np.pi / 3.0, 2.0 * np.pi / 3.0][:phases])
    amp = np.empty((n_scenarios, n_src))
    ph = np.empty((n_scenarios, n_src))
    sw_ptr, swk, swm, swr, swc, swo = [0], [], [], [], [], []
    for s in range(n_scenarios):
        srng = np.random.default_rng([seed, s])
        a = srng.uniform(0.9, 1.1, size=n3) * V_PEAK
        phi = srng.uniform(0.0, 2.0 * np.pi, size=n3)
        amp[s] = np.repeat(a, phases)
        ph[s] = (phi[:, None] + shifts[None, :]).reshape(-1)
        rf = float(srng.uniform(0.01, 10.0))
        for nd in net.meta["bus_nodes"][fault_bus]:
            swk.append(nd); swm.append(GROUND); swr.append(rf); swc.append(fault_step); swo.append(-1)
        sw_ptr.append(len(swk))
    sc = Scenarios(n_scenarios=n_scenarios, src_amp=amp, src_phase=ph,
                   sw_ptr=np.asarray(sw_ptr, np.int64), sw_k=np.asarray(swk, np.int32),
                   sw_m=np.asarray(swm, np.int32), sw_r=np.asarray(swr, np.float64),
                   sw_close_step=np.asarray(swc, np.int64), sw_open_step=np.asarray(swo, np.int64),
                   meta={"fault_bus": fault_bus, "fault_step": fault_step})
    return net, sc


def converter_study(seed: int = 1012, n_scenarios: int = 1024, n_converters: int = 40, dt: float = 20e-6,
                    n_steps: int = 10000, fault_step: int = 2500):
    """Multi-scenario study with control blocks, after the paper's PV case
    (scenarios that differ in the PV units' irradiance): the 600-node
    network of the N-1 study with ``n_converters`` power-regulated converter
    loads (``with_converter_controls``, 24 blocks each).  Scenario s scales
    every converter's power set point (its CONST block) by U[0.2, 1.0], and a
    three-phase fault of R_f ~ U[0.01, 10] ohm at one seeded bus closes at
    ``fault_step``.  Scenario s draws from ``default_rng([seed, s])``."""
    base, _ = n1_contingency(n_scenarios=1, dt=dt, n_steps=n_steps)
    net = with_converter_controls(base, seed=seed, n_converters=n_converters)
    net.n_steps = n_steps
    rng = np.random.default_rng(seed)
    fault_bus = int(rng.integers(0, len(net.meta["bus_nodes"])))
    refs = np.arange(n_converters, dtype=np.int32) * 24 + 11     # each converter's set-point block
    assert np.all(np.asarray(net.cb_type)[refs] == CB_CONST)
    cbo_ptr, cbo_block, cbo_p0 = [0], [], []
    sw_ptr, swk, swm, swr, swc, swo = [0], [], [], [], [], []
    for s in range(n_scenarios):
        srng = np.random.default_rng([seed, s])
        f = srng.uniform(0.2, 1.0, size=n_converters)
        cbo_block += refs.tolist()
        cbo_p0 += (np.asarray(net.cb_p0)[refs] * f).tolist()
        cbo_ptr.append(len(cbo_block))
        rf = float(srng.uniform(0.01, 10.0))
        for nd in net.meta["bus_nodes"][fault_bus]:
            swk.append(nd); swm.append(GROUND); swr.append(rf); swc.append(fault_step); swo.append(-1)
        sw_ptr.append(len(swk))
    sc = Scenarios(n_scenarios=n_scenarios,
                   sw_ptr=np.asarray(sw_ptr, np.int64), sw_k=np.asarray(swk, np.int32),
                   sw_m=np.asarray(swm, np.int32), sw_r=np.asarray(swr, np.float64),
                   sw_close_step=np.asarray(swc, np.int64), sw_open_step=np.asarray(swo, np.int64),
                   cbo_ptr=np.asarray(cbo_ptr, np.int64), cbo_block=np.asarray(cbo_block, np.int32),
                   cbo_p0=np.asarray(cbo_p0, np.float64),
                   meta={"fault_bus": fault_bus, "fault_step": fault_step, "set_point_blocks": refs})
    return net, sc


def adjoint_target(net: Network, seed: int = 1005, rel: float = 0.05):
    """Perturbed parameters p* = p (1 + delta), delta ~ U[-rel, rel], for
    every branch value and every source amplitude (the target run)."""
    rng = np.random.default_rng(seed)
    br = net.br_value * (1.0 + rng.uniform(-rel, rel, size=net.n_branches))
    amp = net.src_amp * (1.0 + rng.uniform(-rel, rel, size=net.n_sources))
    return br, amp


# ----------------------------------------------------------------------------
# runtime switches: rectifier loads and breakers on an existing network

def with_rectifier_loads(base: Network, seed: int = 1006, n_rectifiers: int = 30, n_breakers: int = 10,
                         trip_range=(1000, 4000)) -> Network:
    """``base`` plus diode-rectifier loads and series breakers.

    Rectifier at a random unknown node a: diode a -> x (r_on 0.01 ohm,
    r_off 1 Mohm), then R ~ U[50, 500] ohm and C ~ U[10, 100] uF from the new
    node x to ground.  Breaker at a random node b: breaker b -> y (r_on 1
    mohm, r_off 1 Mohm, trip step ~ U[trip_range)), then R ~ U[5, 50] ohm to
    ground from the new node y.  New nodes join the subsystem of the node
    they hang from."""
    rng = np.random.default_rng(seed)
    net = base.copy()
    n = net.n_nodes
    br = [list(net.br_k), list(net.br_m), list(net.br_kind), list(net.br_value)]
    rs = {k: [] for k in ("k", "m", "kind", "ron", "roff", "on0", "trip")}
    picks = rng.choice(net.n_nodes, size=n_rectifiers + n_breakers, replace=False)
    for i, a in enumerate(picks):
        x = n
        n += 1
        if i < n_rectifiers:
            rs["k"].append(int(a)); rs["m"].append(x); rs["kind"].append(0)
            rs["ron"].append(0.01); rs["roff"].append(1e6); rs["on0"].append(0); rs["trip"].append(-1)
            for kind, val in ((KIND_R, rng.uniform(50.0, 500.0)), (KIND_C, rng.uniform(10e-6, 100e-6))):
                br[0].append(x); br[1].append(GROUND); br[2].append(kind); br[3].append(val)
        else:
            rs["k"].append(int(a)); rs["m"].append(x); rs["kind"].append(1)
            rs["ron"].append(1e-3); rs["roff"].append(1e6); rs["on0"].append(1)
            rs["trip"].append(int(rng.integers(*trip_range)))
            br[0].append(x); br[1].append(GROUND); br[2].append(KIND_R); br[3].append(rng.uniform(5.0, 50.0))
    net.n_nodes = n
    net.br_k = np.asarray(br[0], np.int32)
    net.br_m = np.asarray(br[1], np.int32)
    net.br_kind = np.asarray(br[2], np.uint8)
    net.br_value = np.asarray(br[3], np.float64)
    net.rs_k = np.asarray(rs["k"], np.int32)
    net.rs_m = np.asarray(rs["m"], np.int32)
    net.rs_kind = np.asarray(rs["kind"], np.uint8)
    net.rs_ron = np.asarray(rs["ron"], np.float64)
    net.rs_roff = np.asarray(rs["roff"], np.float64)
    net.rs_on0 = np.asarray(rs["on0"], np.uint8)
    net.rs_trip = np.asarray(rs["trip"], np.int64)
    net.meta = dict(net.meta, runtime_switches={"seed": seed, "rectifiers": n_rectifiers, "breakers": n_breakers})
    return net


def _subsystem_roots(net: Network):
    """Union-find roots of the subsystems (components over branches,
    switches and runtime switches; lines cut them)."""
    parent = list(range(net.n_nodes))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for k, m in list(zip(net.br_k, net.br_m)) + list(zip(net.rs_k, net.rs_m)) + list(zip(net.sw_k, net.sw_m)):
        if k >= 0 and m >= 0:
            a, b = find(int(k)), find(int(m))
            if a != b:
                parent[max(a, b)] = min(a, b)
    return find


def with_converter_stations(base: Network, seed: int = 1013, n_stations: int = 10, bridges: int = 2) -> Network:
    """``base`` plus diode converter stations, each ``bridges`` six-pulse
    bridges on one three-phase bus (two bridges: 12 diodes in one subsystem).

    Bridge on bus phase nodes (a, b, c): per phase a commutation inductance
    L ~ U[1, 5] mH from the phase node to a new AC terminal t_p, an upper
    diode t_p -> P and a lower diode ground -> t_p (r_on 0.01 ohm, r_off
    1 Mohm, off at the start), each valve with a 500 ohm snubber resistor
    across it (without one, a valve that opens on the inductance's current
    leaves a trapezoidal-rule oscillation that makes the valves chatter
    every step); the DC node P feeds R ~ U[50, 200] ohm and C ~ U[20, 100]
    uF to ground.  Stations go to the source buses first, then to random
    buses, one per subsystem."""
    rng = np.random.default_rng(seed)
    net = base.copy()
    find = _subsystem_roots(net)
    buses = list(net.meta.get("source_bus", [])) + rng.permutation(len(net.meta["bus_nodes"])).tolist()
    taken, picks = set(), []
    for bus in buses:
        r = find(int(net.meta["bus_nodes"][bus][0]))
        if r not in taken:
            taken.add(r)
            picks.append(int(bus))
        if len(picks) == n_stations:
            break
    n = net.n_nodes
    br = [list(net.br_k), list(net.br_m), list(net.br_kind), list(net.br_value)]
    rs = {k: list(getattr(net, "rs_" + k)) for k in ("k", "m", "kind", "ron", "roff", "on0", "trip")}

    def diode(a, c):
        for key, val in (("k", a), ("m", c), ("kind", 0), ("ron", 0.01), ("roff", 1e6), ("on0", 0), ("trip", -1)):
            rs[key].append(val)
        br[0].append(a); br[1].append(c); br[2].append(KIND_R); br[3].append(500.0)   # snubber
    for bus in picks:
        for _ in range(bridges):
            dc = n + 3
            for p, nd in enumerate(net.meta["bus_nodes"][bus]):
                t = n + p
                br[0].append(int(nd)); br[1].append(t); br[2].append(KIND_L); br[3].append(rng.uniform(1e-3, 5e-3))
                diode(t, dc)
                diode(GROUND, t)
            for kind, val in ((KIND_R, rng.uniform(50.0, 200.0)), (KIND_C, rng.uniform(20e-6, 100e-6))):
                br[0].append(dc); br[1].append(GROUND); br[2].append(kind); br[3].append(val)
            n += 4
    net.n_nodes = n
    net.br_k = np.asarray(br[0], np.int32)
    net.br_m = np.asarray(br[1], np.int32)
    net.br_kind = np.asarray(br[2], np.uint8)
    net.br_value = np.asarray(br[3], np.float64)
    for key, dt in (("k", np.int32), ("m", np.int32), ("kind", np.uint8), ("ron", np.float64), ("roff", np.float64),
                    ("on0", np.uint8), ("trip", np.int64)):
        setattr(net, "rs_" + key, np.asarray(rs[key], dt))
    net.meta = dict(net.meta, converter_stations={"seed": seed, "buses": picks, "bridges": bridges})
    return net


def with_fd_lines(base: Network, seed: int = 1009, fractional: bool = True) -> Network:
    """``base`` with every Bergeron line replaced by a lossy frequency-dependent
    line of the same surge impedance Z_c and travel time (plus U[0, 1) dt when
    ``fractional``): Y_c = 1/Z_c + c/(s - q), q ~ -U[1e3, 1e5] 1/s, c = -q
    delta / Z_c with delta ~ U[0.05, 0.3] (so Y_c(0) = (1 + delta) / Z_c,
    positive real); A = e^{-s tau} sum_{i=1,2} r_i / (s - p_i), p_1 ~ -U[2e3,
    2e4], p_2 ~ -U[2e4, 2e5] 1/s, r_i = -p_i w_i A_0 with weights w ~ U(0, 1),
    w_1 + w_2 = 1 and DC transmission A_0 = exp(-U[0.02, 0.2]), so |A(jw)| <=
    A_0 < 1: a passive line whose losses grow with frequency.  The fitted
    models of real lines are not available; these stand in for them."""
    rng = np.random.default_rng(seed)
    net = base.copy()
    L = base.n_lines
    yq = np.zeros((L, 4)); yc = np.zeros((L, 4)); ap = np.zeros((L, 4)); ar = np.zeros((L, 4))
    tau = (base.ln_delay.astype(np.float64) + (rng.uniform(0.0, 1.0, L) if fractional else 0.0)) * base.dt
    for l in range(L):
        z = float(base.ln_zc[l])
        q = -rng.uniform(1e3, 1e5)
        yq[l, 0], yc[l, 0] = q, -q * rng.uniform(0.05, 0.3) / z
        a0 = np.exp(-rng.uniform(0.02, 0.2))
        w1 = rng.uniform(0.0, 1.0)
        p1, p2 = -rng.uniform(2e3, 2e4), -rng.uniform(2e4, 2e5)
        ap[l, :2] = p1, p2
        ar[l, :2] = -p1 * w1 * a0, -p2 * (1.0 - w1) * a0
    net.fl_k, net.fl_m = base.ln_k.copy(), base.ln_m.copy()
    net.fl_tau = tau
    net.fl_y0 = 1.0 / base.ln_zc
    net.fl_ny = np.ones(L, np.int32)
    net.fl_yq, net.fl_yc = yq.reshape(-1), yc.reshape(-1)
    net.fl_a0 = np.zeros(L)
    net.fl_na = np.full(L, 2, np.int32)
    net.fl_ap, net.fl_ar = ap.reshape(-1), ar.reshape(-1)
    for f in ("ln_k", "ln_m", "ln_zc", "ln_delay"):
        setattr(net, f, getattr(base, f)[:0].copy())
    net.meta = dict(net.meta, fd_lines={"seed": seed, "lines": L, "fractional": fractional})
    return net


# a surge arrester's characteristic as an odd piecewise-linear resistor
# (volts, amperes): nearly open below ~0.8 kV (the 1 kV-peak system clips
# at its source buses), a few kA near 1.5 kV
ARRESTER_V = (800.0, 950.0, 1050.0, 1150.0, 1300.0, 1500.0)
ARRESTER_I = (1e-3, 1.0, 50.0, 300.0, 1500.0, 4000.0)


def with_arresters(base: Network, seed: int = 1010, n_arresters: int = 40, scale=(0.9, 1.1)) -> Network:
    """``base`` plus ``n_arresters`` phase-to-ground surge arresters (odd
    piecewise-linear resistors, characteristic ``ARRESTER_V/I`` with its
    voltages scaled by U[scale]): first at a phase node of each source bus
    (where the 1 kV peaks make them conduct), then at random nodes, at most
    one per subsystem (the compensation method solves one nonlinear element
    per subsystem)."""
    rng = np.random.default_rng(seed)
    net = base.copy()
    # subsystems: components over branches and switches (lines cut them)
    parent = list(range(net.n_nodes))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for k, m in list(zip(net.br_k, net.br_m)) + list(zip(net.rs_k, net.rs_m)) + list(zip(net.sw_k, net.sw_m)):
        if k >= 0 and m >= 0:
            a, b = find(int(k)), find(int(m))
            if a != b:
                parent[max(a, b)] = min(a, b)
    for x in range(0, len(net.cl_k), 3):
        for y in (net.cl_k, net.cl_m):
            for p in (1, 2):
                a, b = find(int(y[x])), find(int(y[x + p]))
                if a != b:
                    parent[max(a, b)] = min(a, b)
    taken, nodes = set(), []
    first = [int(net.meta["bus_nodes"][b_][0]) for b_ in net.meta.get("source_bus", [])]
    for x in first + rng.permutation(net.n_nodes).tolist():
        r = find(int(x))
        if r not in taken:
            taken.add(r)
            nodes.append(int(x))
        if len(nodes) == n_arresters:
            break
    b = NetworkBuilder()
    for x in nodes:
        s = rng.uniform(*scale)
        b.nonlinear_resistor(x, GROUND, [v * s for v in ARRESTER_V], ARRESTER_I)
    nl = b.build(base.dt, 0)
    for f in ("nl_k", "nl_m", "nl_np", "nl_v", "nl_i"):
        setattr(net, f, getattr(nl, f))
    net.meta = dict(net.meta, arresters={"seed": seed, "count": len(nodes)})
    return net


def with_bus_arresters(base: Network, seed: int = 1014, n_buses: int = 20, scale=(0.55, 0.7)) -> Network:
    """``base`` plus surge arresters on every phase of ``n_buses`` three-phase
    buses (several nonlinear resistors in one subsystem, solved together):
    the source buses first, then random buses, one bus per subsystem; the
    characteristic ``ARRESTER_V/I`` with its voltages scaled by U[scale], low
    enough that they conduct near the 1 kV peaks."""
    rng = np.random.default_rng(seed)
    net = base.copy()
    find = _subsystem_roots(net)
    buses = list(net.meta.get("source_bus", [])) + rng.permutation(len(net.meta["bus_nodes"])).tolist()
    taken, picks = set(), []
    for bus in buses:
        r = find(int(net.meta["bus_nodes"][bus][0]))
        if r not in taken:
            taken.add(r)
            picks.append(int(bus))
        if len(picks) == n_buses:
            break
    b = NetworkBuilder()
    for bus in picks:
        for x in net.meta["bus_nodes"][bus]:
            s_ = rng.uniform(*scale)
            b.nonlinear_resistor(int(x), GROUND, [v * s_ for v in ARRESTER_V], ARRESTER_I)
    nl = b.build(base.dt, 0)
    for f in ("nl_k", "nl_m", "nl_np", "nl_v", "nl_i"):
        setattr(net, f, getattr(nl, f))
    net.meta = dict(net.meta, bus_arresters={"seed": seed, "buses": picks})
    return net


# control block types (see Network.cb_*)
CB_CONST, CB_MEAS, CB_GAIN, CB_SUM, CB_MUL, CB_LIMIT, CB_INTEG, CB_LAG, CB_PI = range(9)


def add_converter_control(b: NetworkBuilder, phase_nodes, i_ref: float, t_filter: float,
                          kp: float = 0.05, ki: float = 5.0, m_max: float = 100.0, i_max: float = 40.0) -> int:
    """A three-phase converter drawing a regulated power, as 24 control
    blocks and three controlled current injections; returns its first block.
    Per phase p: u_p = v_p / V_PEAK; drawn power P = sum u_p c_p with the
    converter's own currents c_p of the previous step (the loop closes
    through blocks of higher index); m = limit(PI(1.5 i_ref - P), 0, m_max);
    c_p = lag(limit(m u_p, -i_max, i_max), t_filter), and -c_p is injected
    into the phase node, so the injected currents stay within i_max."""
    c0 = len(b.cb)
    meas = [b.block(CB_MEAS, node=x) for x in phase_nodes]
    u = [b.block(CB_GAIN, m, p0=1.0 / V_PEAK) for m in meas]
    out0 = c0 + 21                                  # first output block (lags, below)
    pw = [b.block(CB_MUL, u[p], out0 + p, p0=-1.0) for p in range(3)]
    s01 = b.block(CB_SUM, pw[0], pw[1], p0=1.0, p1=1.0)
    ptot = b.block(CB_SUM, s01, pw[2], p0=1.0, p1=1.0)
    ref = b.block(CB_CONST, p0=1.5 * i_ref)
    err = b.block(CB_SUM, ref, ptot, p0=1.0, p1=-1.0)
    m = b.block(CB_PI, err, p0=kp, p1=ki)
    mlim = b.block(CB_LIMIT, m, p0=0.0, p1=m_max)
    iraw = [b.block(CB_MUL, mlim, u[p], p0=1.0) for p in range(3)]
    iref = [b.block(CB_LIMIT, iraw[p], p0=-i_max, p1=i_max) for p in range(3)]
    outs = [b.block(CB_LAG, iref[p], p0=-1.0, p1=t_filter) for p in range(3)]
    assert outs[0] == out0
    for p in range(3):
        b.injection(outs[p], phase_nodes[p])
    return c0


def with_converter_controls(base: Network, seed: int = 1008, n_converters: int = 180,
                            r_damp: float = 20.0) -> Network:
    """``base`` (a three-phase network with ``meta['bus_nodes']``) plus
    ``n_converters`` power-regulated loads (``add_converter_control``) at distinct
    buses (the source buses, then random ones), i_ref ~ U[5, 20] A, current filter ~ U[0.5, 2] ms, and a damping
    resistor ``r_damp`` from each of their phase nodes to ground.  The block
    count per node is about that of the paper's largest PV case (990 PV
    units with their controls on 16,653 nodes); the PV models themselves are
    not available, so this synthetic control stands in for them."""
    rng = np.random.default_rng(seed)
    buses = base.meta["bus_nodes"]
    # the source buses first (stiff, near 1 p.u.: the power loop regulates),
    # then random others (weak: the loop mostly runs into its limits)
    first = list(dict.fromkeys(int(x) for x in base.meta.get("source_bus", [])))[:n_converters]
    rest = [x for x in rng.permutation(len(buses)).tolist() if x not in set(first)]
    picks = first + rest[:max(0, min(n_converters, len(buses)) - len(first))]
    b = NetworkBuilder()
    damp = []
    for bus in picks:
        add_converter_control(b, buses[int(bus)], float(rng.uniform(5.0, 20.0)), float(rng.uniform(0.5e-3, 2e-3)))
        damp += list(buses[int(bus)])
    net = base.copy()
    ctl = b.build(base.dt, 0)
    for f in ("cb_type", "cb_in0", "cb_in1", "cb_node", "cb_p0", "cb_p1", "ci_block", "ci_node"):
        setattr(net, f, getattr(ctl, f))
    # the converter's output filter: a damping resistor per phase to ground
    net.br_k = np.concatenate([net.br_k, np.asarray(damp, np.int32)])
    net.br_m = np.concatenate([net.br_m, np.full(len(damp), GROUND, np.int32)])
    net.br_kind = np.concatenate([net.br_kind, np.full(len(damp), KIND_R, np.uint8)])
    net.br_value = np.concatenate([net.br_value, np.full(len(damp), r_damp, np.float64)])
    net.meta = dict(net.meta, controls={"seed": seed, "converters": len(picks), "blocks": ctl.n_control_blocks})
    return net


# Power-invariant Clarke transformation (rows: phases a, b, c; columns:
# modes 0, alpha, beta); orthonormal, so T_i = T_v for a transposed line.
CLARKE = np.array([[1 / np.sqrt(3), 2 / np.sqrt(6), 0.0],
                   [1 / np.sqrt(3), -1 / np.sqrt(6), 1 / np.sqrt(2)],
                   [1 / np.sqrt(3), -1 / np.sqrt(6), -1 / np.sqrt(2)]])


def with_coupled_lines(base: Network, seed: int = 1007) -> Network:
    """``base`` with every three-phase line (a triplet of single-phase lines,
    phases 0, 1, 2) replaced by one transposed coupled line in Clarke modes:
    aerial modes Z_1 = Z_2 = the triplet's Z_c with travel time (d + U[0, 1))
    dt, zero-sequence mode Z_0 = Z_c U[1.4, 1.9] with travel time
    U[1.05, 1.25] times the aerial one (non-integer numbers of steps)."""
    if base.n_lines % 3:
        raise ValueError("lines must come in three-phase triplets")
    rng = np.random.default_rng(seed)
    net = base.copy()
    L = base.n_lines // 3
    cl_k, cl_m, cl_tv, cl_z, cl_tau = [], [], [], [], []
    for l in range(L):
        idx = slice(3 * l, 3 * l + 3)
        zc, d = float(base.ln_zc[3 * l]), int(base.ln_delay[3 * l])
        tau1 = (d + rng.uniform(0.0, 1.0)) * base.dt
        tau0 = tau1 * rng.uniform(1.05, 1.25)
        cl_k.extend(base.ln_k[idx].tolist())
        cl_m.extend(base.ln_m[idx].tolist())
        cl_tv.extend(CLARKE.reshape(9).tolist())
        cl_z.extend([zc * rng.uniform(1.4, 1.9), zc, zc])
        cl_tau.extend([tau0, tau1, tau1])
    net.ln_k = np.zeros(0, np.int32)
    net.ln_m = np.zeros(0, np.int32)
    net.ln_zc = np.zeros(0, np.float64)
    net.ln_delay = np.zeros(0, np.int32)
    net.cl_k = np.asarray(cl_k, np.int32)
    net.cl_m = np.asarray(cl_m, np.int32)
    net.cl_tv = np.asarray(cl_tv, np.float64)
    net.cl_z = np.asarray(cl_z, np.float64)
    net.cl_tau = np.asarray(cl_tau, np.float64)
    net.meta = dict(net.meta, coupled_lines={"seed": seed, "lines": L})
    return net


def fd_groups_from_coupled(cnet: Network, seed: int = 1011, lossless: bool = False,
                           same_modes: bool = False) -> Network:
    """The coupled lines of ``cnet`` as frequency-dependent line groups: mode j
    of each becomes a frequency-dependent line between phase j's nodes with
    the mode's Z_c and travel time, grouped with the line's T_v.  Lossless:
    Y_c = 1/Z_j, A = e^{-s tau_j} (the coupled Bergeron line itself);
    otherwise each mode gets poles drawn as in ``with_fd_lines`` (Y_c(0) =
    (1 + delta)/Z_j, DC transmission exp(-U[0.02, 0.2])).  ``same_modes``:
    every mode of a line takes mode 1's impedance, travel time and poles (with
    an orthogonal T_v the phases then decouple into three equal lines)."""
    rng = np.random.default_rng(seed)
    net = cnet.copy()
    L = len(cnet.cl_z) // 3
    n = 3 * L
    fl_k, fl_m = np.zeros(n, np.int32), np.zeros(n, np.int32)
    tau, y0, a0 = np.zeros(n), np.zeros(n), np.zeros(n)
    ny, na = np.zeros(n, np.int32), np.zeros(n, np.int32)
    yq, yc, ap, ar = np.zeros((n, 4)), np.zeros((n, 4)), np.zeros((n, 4)), np.zeros((n, 4))
    for l in range(L):
        for j in range(3):
            x, src = 3 * l + j, 3 * l + (1 if same_modes else j)
            fl_k[x], fl_m[x] = cnet.cl_k[x], cnet.cl_m[x]
            z = float(cnet.cl_z[src])
            tau[x], y0[x] = float(cnet.cl_tau[src]), 1.0 / z
            if lossless:
                a0[x] = 1.0
                continue
            if same_modes and j != 1:
                continue   # (copied from mode 1 below)
            q = -rng.uniform(1e3, 1e5)
            ny[x], yq[x, 0], yc[x, 0] = 1, q, -q * rng.uniform(0.05, 0.3) / z
            dc = np.exp(-rng.uniform(0.02, 0.2))
            w1 = rng.uniform(0.0, 1.0)
            p1, p2 = -rng.uniform(2e3, 2e4), -rng.uniform(2e4, 2e5)
            na[x], ap[x, :2] = 2, (p1, p2)
            ar[x, :2] = -p1 * w1 * dc, -p2 * (1.0 - w1) * dc
        if same_modes and not lossless:
            for j in (0, 2):
                x, src = 3 * l + j, 3 * l + 1
                ny[x], na[x], a0[x] = ny[src], na[src], a0[src]
                yq[x], yc[x], ap[x], ar[x] = yq[src], yc[src], ap[src], ar[src]
    net.fl_k, net.fl_m, net.fl_tau, net.fl_y0, net.fl_a0 = fl_k, fl_m, tau, y0, a0
    net.fl_ny, net.fl_na = ny, na
    net.fl_yq, net.fl_yc, net.fl_ap, net.fl_ar = yq.reshape(-1), yc.reshape(-1), ap.reshape(-1), ar.reshape(-1)
    net.fg_line = np.arange(n, dtype=np.int32)
    net.fg_tv = np.asarray(cnet.cl_tv, np.float64).copy()
    for f in ("cl_k", "cl_m", "cl_tv", "cl_z", "cl_tau"):
        setattr(net, f, np.zeros(0, getattr(cnet, f).dtype))
    net.meta = dict(net.meta, fd_line_groups={"seed": seed, "groups": L, "lossless": lossless,
                                              "same_modes": same_modes})
    return net


def with_fd_line_groups(base: Network, seed: int = 1011) -> Network:
    """``base`` with every three-phase line a frequency-dependent line group:
    Clarke modes with the impedances and travel times of ``with_coupled_lines``
    (zero-sequence mode slower and of higher impedance, fractional travel
    times), each mode lossy as in ``with_fd_lines``."""
    return fd_groups_from_coupled(with_coupled_lines(base, seed=seed), seed=seed + 1)
