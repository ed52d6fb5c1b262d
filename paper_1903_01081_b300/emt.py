"""Thin Python binding of libemt (include/emt.h).

Argument marshalling only: every step of the time loop runs in the CUDA
library.  Functions keep the C names; ``Simulator`` is a small convenience
wrapper around one context.  There is no CPU fallback: if the library
cannot be built or loaded, or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

EMT_OK, EMT_EINVAL, EMT_ESINGULAR, EMT_ENOMEM, EMT_ECUDA, EMT_ETIMEOUT, EMT_ERESOURCE, EMT_ESTATE = range(8)
_STATUS = {0: "EMT_OK", 1: "EMT_EINVAL", 2: "EMT_ESINGULAR", 3: "EMT_ENOMEM", 4: "EMT_ECUDA",
           5: "EMT_ETIMEOUT", 6: "EMT_ERESOURCE", 7: "EMT_ESTATE"}

# every function include/emt.h declares
EXPORTS = ("emt_build_network", "emt_prefactor", "emt_set_recording", "emt_step_n", "emt_read_waveforms",
           "emt_reset", "emt_sync", "emt_set_option", "emt_get_info", "emt_get_node_order", "emt_last_error",
           "emt_destroy", "emt_prefactor_noalloc", "emt_adjoint", "emt_autotune", "emt_read_controls",
           "emt_read_waveforms_async")


class EmtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class _NetworkDesc(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("n_nodes", ctypes.c_int64),
        ("n_branches", ctypes.c_int64), ("br_k", ctypes.c_void_p), ("br_m", ctypes.c_void_p),
        ("br_kind", ctypes.c_void_p), ("br_value", ctypes.c_void_p),
        ("n_sources", ctypes.c_int64), ("src_amp", ctypes.c_void_p), ("src_phase", ctypes.c_void_p),
        ("src_freq", ctypes.c_void_p),
        ("n_lines", ctypes.c_int64), ("ln_k", ctypes.c_void_p), ("ln_m", ctypes.c_void_p),
        ("ln_zc", ctypes.c_void_p), ("ln_delay", ctypes.c_void_p),
        ("n_switches", ctypes.c_int64), ("sw_k", ctypes.c_void_p), ("sw_m", ctypes.c_void_p),
        ("sw_r", ctypes.c_void_p), ("sw_close_step", ctypes.c_void_p), ("sw_open_step", ctypes.c_void_p),
        ("n_rswitches", ctypes.c_int64), ("rs_k", ctypes.c_void_p), ("rs_m", ctypes.c_void_p),
        ("rs_kind", ctypes.c_void_p), ("rs_ron", ctypes.c_void_p), ("rs_roff", ctypes.c_void_p),
        ("rs_on0", ctypes.c_void_p), ("rs_trip_step", ctypes.c_void_p),
        ("n_clines", ctypes.c_int64), ("cl_k", ctypes.c_void_p), ("cl_m", ctypes.c_void_p),
        ("cl_tv", ctypes.c_void_p), ("cl_z", ctypes.c_void_p), ("cl_tau", ctypes.c_void_p),
        ("n_cblocks", ctypes.c_int64), ("cb_type", ctypes.c_void_p), ("cb_in0", ctypes.c_void_p),
        ("cb_in1", ctypes.c_void_p), ("cb_node", ctypes.c_void_p), ("cb_p0", ctypes.c_void_p),
        ("cb_p1", ctypes.c_void_p),
        ("n_cinj", ctypes.c_int64), ("ci_block", ctypes.c_void_p), ("ci_node", ctypes.c_void_p),
        ("n_fdlines", ctypes.c_int64), ("fl_k", ctypes.c_void_p), ("fl_m", ctypes.c_void_p),
        ("fl_tau", ctypes.c_void_p), ("fl_y0", ctypes.c_void_p), ("fl_ny", ctypes.c_void_p),
        ("fl_yq", ctypes.c_void_p), ("fl_yc", ctypes.c_void_p), ("fl_a0", ctypes.c_void_p),
        ("fl_na", ctypes.c_void_p), ("fl_ap", ctypes.c_void_p), ("fl_ar", ctypes.c_void_p),
        ("n_nonlin", ctypes.c_int64), ("nl_k", ctypes.c_void_p), ("nl_m", ctypes.c_void_p),
        ("nl_np", ctypes.c_void_p), ("nl_v", ctypes.c_void_p), ("nl_i", ctypes.c_void_p),
        ("n_fdgroups", ctypes.c_int64), ("fg_line", ctypes.c_void_p), ("fg_tv", ctypes.c_void_p),
    ]


class _ScenarioDesc(ctypes.Structure):
    _fields_ = [
        ("n_scenarios", ctypes.c_int64),
        ("src_amp", ctypes.c_void_p), ("src_phase", ctypes.c_void_p),
        ("rm_branch_ptr", ctypes.c_void_p), ("rm_branch", ctypes.c_void_p),
        ("rm_line_ptr", ctypes.c_void_p), ("rm_line", ctypes.c_void_p),
        ("sw_ptr", ctypes.c_void_p), ("sw_k", ctypes.c_void_p), ("sw_m", ctypes.c_void_p),
        ("sw_r", ctypes.c_void_p), ("sw_close_step", ctypes.c_void_p), ("sw_open_step", ctypes.c_void_p),
        ("cbo_ptr", ctypes.c_void_p), ("cbo_block", ctypes.c_void_p), ("cbo_p0", ctypes.c_void_p),
    ]


_lib = None


def checks_build() -> bool:
    """EMT_CHECKS=1 in the environment selects the checks build of the library."""
    return os.environ.get("EMT_CHECKS", "0") == "1"


def phases_build() -> bool:
    """EMT_PHASES=1 in the environment selects the phase-clock build of the library."""
    return os.environ.get("EMT_PHASES", "0") == "1"


def library_path() -> str:
    if checks_build():
        return _build.CHECKS_LIB_PATH
    return _build.PHASES_LIB_PATH if phases_build() else _build.LIB_PATH


def load_library(build_if_needed: bool = True):
    """Load libemt.so, or libemt_checks.so under EMT_CHECKS=1 (building it
    with nvcc first if missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_needed and _build.needs_build(path):
        _build.build(checks=checks_build(), phases=phases_build() and not checks_build())
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not found at {path}; build it with "
                           "paper_1903_01081_b300.build.build()")
    lib = ctypes.CDLL(path)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    sig = {
        "emt_build_network": [P, P, P],
        "emt_prefactor": [P],
        "emt_prefactor_noalloc": [P, P],
        "emt_set_recording": [P, P, I64, I32, I64],
        "emt_step_n": [P, I64, P],
        "emt_read_waveforms": [P, P, I64, I64, I64, I64, I64, P, I32],
        "emt_read_waveforms_async": [P, P, I64, I64, I64, I64, I64, P, I32, P],
        "emt_reset": [P],
        "emt_sync": [P, P],
        "emt_set_option": [P, ctypes.c_char_p, I64],
        "emt_get_info": [P, ctypes.c_char_p, P],
        "emt_get_node_order": [P, P],
        "emt_adjoint": [P, P, I64, I32, P, P, I32, P],
        "emt_autotune": [P, I64, P],
        "emt_read_controls": [P, P, I64, I32],
        "emt_save_state": [P, P, I64, P],
        "emt_load_state": [P, P, I64],
        "emt_get_node_ctas": [P, P],
        "emt_get_line_ends": [P, P, P, P],
        "emt_set_shard": [P, P, I32],
        "emt_shard_pack": [P, I32, P, I64, P, P],
        "emt_shard_unpack": [P, I32, P, I64, P],
        "emt_phase_clocks": [P, P, I32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.emt_last_error.argtypes = [P]
    lib.emt_last_error.restype = ctypes.c_char_p
    lib.emt_destroy.argtypes = [P]
    lib.emt_destroy.restype = None
    _lib = lib
    return lib


def _arr(x, dtype):
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


class Ctx:
    """Owner of one ``emt_ctx*``."""

    def __init__(self, handle: int, n_nodes: int, n_scenarios: int):
        self.handle = ctypes.c_void_p(handle)
        self.n_nodes = n_nodes
        self.n_scenarios = n_scenarios

    def __del__(self):
        try:
            emt_destroy(self)
        except Exception:
            pass


def _check(ctx: Optional[Ctx], status: int):
    if status != EMT_OK:
        lib = load_library(False)
        msg = lib.emt_last_error(ctx.handle if ctx is not None else None)
        raise EmtError(status, msg.decode() if msg else "")


def network_desc(net, keep: list) -> _NetworkDesc:
    """ctypes ``emt_network_desc`` pointing into arrays appended to ``keep``."""
    def p(x, dt):
        a = _arr(x, dt)
        keep.append(a)
        return a.ctypes.data if a.size else None

    d = _NetworkDesc()
    d.dt = float(net.dt)
    d.n_nodes = int(net.n_nodes)
    d.n_branches = int(len(net.br_k))
    d.br_k, d.br_m = p(net.br_k, np.int32), p(net.br_m, np.int32)
    d.br_kind, d.br_value = p(net.br_kind, np.uint8), p(net.br_value, np.float64)
    d.n_sources = int(len(net.src_amp))
    d.src_amp, d.src_phase, d.src_freq = (p(net.src_amp, np.float64), p(net.src_phase, np.float64),
                                          p(net.src_freq, np.float64))
    d.n_lines = int(len(net.ln_k))
    d.ln_k, d.ln_m = p(net.ln_k, np.int32), p(net.ln_m, np.int32)
    d.ln_zc, d.ln_delay = p(net.ln_zc, np.float64), p(net.ln_delay, np.int32)
    d.n_switches = int(len(net.sw_k))
    d.sw_k, d.sw_m = p(net.sw_k, np.int32), p(net.sw_m, np.int32)
    d.sw_r = p(net.sw_r, np.float64)
    d.sw_close_step, d.sw_open_step = p(net.sw_close_step, np.int64), p(net.sw_open_step, np.int64)
    rs = lambda name, dt: getattr(net, name, np.zeros(0, dt))
    d.n_rswitches = int(len(rs("rs_k", np.int32)))
    d.rs_k, d.rs_m = p(rs("rs_k", np.int32), np.int32), p(rs("rs_m", np.int32), np.int32)
    d.rs_kind = p(rs("rs_kind", np.uint8), np.uint8)
    d.rs_ron, d.rs_roff = p(rs("rs_ron", np.float64), np.float64), p(rs("rs_roff", np.float64), np.float64)
    d.rs_on0, d.rs_trip_step = p(rs("rs_on0", np.uint8), np.uint8), p(rs("rs_trip", np.int64), np.int64)
    d.n_clines = int(len(rs("cl_z", np.float64))) // 3
    d.cl_k, d.cl_m = p(rs("cl_k", np.int32), np.int32), p(rs("cl_m", np.int32), np.int32)
    d.cl_tv, d.cl_z = p(rs("cl_tv", np.float64), np.float64), p(rs("cl_z", np.float64), np.float64)
    d.cl_tau = p(rs("cl_tau", np.float64), np.float64)
    d.n_cblocks = int(len(rs("cb_type", np.uint8)))
    d.cb_type = p(rs("cb_type", np.uint8), np.uint8)
    d.cb_in0, d.cb_in1 = p(rs("cb_in0", np.int32), np.int32), p(rs("cb_in1", np.int32), np.int32)
    d.cb_node = p(rs("cb_node", np.int32), np.int32)
    d.cb_p0, d.cb_p1 = p(rs("cb_p0", np.float64), np.float64), p(rs("cb_p1", np.float64), np.float64)
    d.n_cinj = int(len(rs("ci_block", np.int32)))
    d.ci_block, d.ci_node = p(rs("ci_block", np.int32), np.int32), p(rs("ci_node", np.int32), np.int32)
    d.n_fdlines = int(len(rs("fl_k", np.int32)))
    d.fl_k, d.fl_m = p(rs("fl_k", np.int32), np.int32), p(rs("fl_m", np.int32), np.int32)
    d.fl_tau, d.fl_y0 = p(rs("fl_tau", np.float64), np.float64), p(rs("fl_y0", np.float64), np.float64)
    d.fl_ny, d.fl_na = p(rs("fl_ny", np.int32), np.int32), p(rs("fl_na", np.int32), np.int32)
    d.fl_yq, d.fl_yc = p(rs("fl_yq", np.float64), np.float64), p(rs("fl_yc", np.float64), np.float64)
    d.fl_a0 = p(rs("fl_a0", np.float64), np.float64)
    d.fl_ap, d.fl_ar = p(rs("fl_ap", np.float64), np.float64), p(rs("fl_ar", np.float64), np.float64)
    d.n_nonlin = int(len(rs("nl_k", np.int32)))
    d.nl_k, d.nl_m = p(rs("nl_k", np.int32), np.int32), p(rs("nl_m", np.int32), np.int32)
    d.nl_np = p(rs("nl_np", np.int32), np.int32)
    d.nl_v, d.nl_i = p(rs("nl_v", np.float64), np.float64), p(rs("nl_i", np.float64), np.float64)
    d.n_fdgroups = int(len(rs("fg_line", np.int32))) // 3
    d.fg_line, d.fg_tv = p(rs("fg_line", np.int32), np.int32), p(rs("fg_tv", np.float64), np.float64)
    return d


def scenario_desc(sc, keep: list) -> _ScenarioDesc:
    def p(x, dt):
        if x is None:
            return None
        a = _arr(x, dt)
        keep.append(a)
        return a.ctypes.data if a.size else None

    d = _ScenarioDesc()
    d.n_scenarios = int(sc.n_scenarios)
    d.src_amp, d.src_phase = p(sc.src_amp, np.float64), p(sc.src_phase, np.float64)
    d.rm_branch_ptr, d.rm_branch = p(sc.rm_branch_ptr, np.int64), p(sc.rm_branch, np.int32)
    d.rm_line_ptr, d.rm_line = p(sc.rm_line_ptr, np.int64), p(sc.rm_line, np.int32)
    d.sw_ptr, d.sw_k, d.sw_m = p(sc.sw_ptr, np.int64), p(sc.sw_k, np.int32), p(sc.sw_m, np.int32)
    d.sw_r = p(sc.sw_r, np.float64)
    d.sw_close_step, d.sw_open_step = p(sc.sw_close_step, np.int64), p(sc.sw_open_step, np.int64)
    d.cbo_ptr, d.cbo_block = p(sc.cbo_ptr, np.int64), p(sc.cbo_block, np.int32)
    d.cbo_p0 = p(sc.cbo_p0, np.float64)
    return d


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


# ------------------------------------------------------------------ C names

def emt_build_network(net, scenarios=None) -> Ctx:
    lib = load_library()
    keep: list = []
    d = network_desc(net, keep)
    sd = scenario_desc(scenarios, keep) if scenarios is not None else None
    out = ctypes.c_void_p()
    st = lib.emt_build_network(ctypes.byref(d), ctypes.byref(sd) if sd is not None else None, ctypes.byref(out))
    _check(None, st)
    return Ctx(out.value, int(net.n_nodes), 1 if scenarios is None else int(scenarios.n_scenarios))


def emt_prefactor(ctx: Ctx) -> None:
    _check(ctx, load_library().emt_prefactor(ctx.handle))


def emt_prefactor_noalloc(ctx: Ctx, stream=None) -> None:
    """emt_prefactor without device allocation (fixed workspace; see include/emt.h)."""
    _check(ctx, load_library().emt_prefactor_noalloc(ctx.handle, _stream_handle(stream)))


def emt_set_recording(ctx: Ctx, channels: Optional[Sequence[int]] = None, decim: int = 1, max_rows: int = 0) -> None:
    lib = load_library()
    if channels is None:
        _check(ctx, lib.emt_set_recording(ctx.handle, None, ctx.n_nodes, int(decim), int(max_rows)))
    else:
        ch = _arr(channels, np.int32)
        _check(ctx, lib.emt_set_recording(ctx.handle, ch.ctypes.data if ch.size else None, int(ch.size),
                                          int(decim), int(max_rows)))


def emt_step_n(ctx: Ctx, n_steps: int, stream=None) -> None:
    _check(ctx, load_library().emt_step_n(ctx.handle, int(n_steps), _stream_handle(stream)))


def emt_read_waveforms(ctx: Ctx, channels, step0: int, n_rows: int, scen0: int = 0, n_scen: int = 1, out=None):
    """Recorded waveforms [n_rows][n_scen][n_ch].  ``out`` may be a CUDA
    torch tensor (filled on the device) or a numpy array; by default a new
    numpy array is returned."""
    lib = load_library()
    ch = _arr(channels, np.int32)
    shape = (int(n_rows), int(n_scen), int(ch.size))
    on_device = 0
    if out is None:
        out = np.zeros(shape, dtype=np.float64)
        ptr = out.ctypes.data
    elif isinstance(out, np.ndarray):
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != int(np.prod(shape)):
            raise ValueError("out must be a C-contiguous float64 array of shape " + str(shape))
        ptr = out.ctypes.data
    else:   # torch tensor
        if not out.is_contiguous() or out.numel() != int(np.prod(shape)) or str(out.dtype) != "torch.float64":
            raise ValueError("out must be a contiguous float64 tensor of shape " + str(shape))
        ptr = out.data_ptr()
        on_device = 1 if out.is_cuda else 0
    if int(np.prod(shape)) == 0:
        return out
    _check(ctx, lib.emt_read_waveforms(ctx.handle, ch.ctypes.data, int(ch.size), int(step0), int(n_rows),
                                       int(scen0), int(n_scen), ptr, on_device))
    return out


def emt_read_waveforms_async(ctx: Ctx, channels, step0: int, n_rows: int, scen0: int, n_scen: int, out, stream=None):
    """Stream-ordered read of recorded waveforms into ``out`` ([n_rows][n_scen][n_ch]
    float64: a CUDA tensor, or a pinned host tensor for an asynchronous
    copy), enqueued on ``stream``; returns at once (include/emt.h)."""
    lib = load_library()
    ch = _arr(channels, np.int32)
    shape = (int(n_rows), int(n_scen), int(ch.size))
    if not out.is_contiguous() or out.numel() != int(np.prod(shape)) or str(out.dtype) != "torch.float64":
        raise ValueError("out must be a contiguous float64 tensor of shape " + str(shape))
    if int(np.prod(shape)) == 0:
        return out
    _check(ctx, lib.emt_read_waveforms_async(ctx.handle, ch.ctypes.data, int(ch.size), int(step0), int(n_rows),
                                             int(scen0), int(n_scen), out.data_ptr(), 1 if out.is_cuda else 0,
                                             _stream_handle(stream)))
    return out


def step_and_read(ctx: Ctx, channels, decim: int, n_steps: int, out, chunk: int = 5000, stream=None):
    """Run ``n_steps`` steps and copy their recorded rows (channels
    ``channels``, every scenario) into ``out``, a pinned host tensor
    [rows][scenarios][channels] whose row 0 is the first row recorded after
    the current step.  The steps go to ``stream`` (default: torch's current
    stream) in chunks; each chunk's rows are read on a second stream, which
    waits for the chunk, while the next chunk runs (emt_step_n and
    emt_read_waveforms_async).  Returns ``out`` once both streams are done."""
    import torch
    compute = stream if stream is not None else torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    decim = int(decim)
    n_scen = ctx.n_scenarios
    base = emt_get_info(ctx, "step")
    row_base = base // decim + 1
    done = 0
    while done < n_steps:
        n = min(int(chunk), n_steps - done)
        emt_step_n(ctx, n, compute)
        first, last = (base + done) // decim + 1, (base + done + n) // decim   # rows completed by this chunk
        if last >= first:
            ev = torch.cuda.Event()
            ev.record(compute)
            copy.wait_event(ev)
            r0 = first - row_base
            emt_read_waveforms_async(ctx, channels, first * decim, last - first + 1, 0, n_scen,
                                     out[r0:r0 + last - first + 1], copy)
        done += n
    copy.synchronize()
    compute.synchronize()
    return out


def emt_read_controls(ctx: Ctx, out=None):
    """Control block outputs of the last completed step, caller's block
    order: a new numpy array, or written into ``out`` (numpy array or CUDA
    float64 tensor of n_control_blocks entries)."""
    lib = load_library()
    n = emt_get_info(ctx, "n_control_blocks")
    on_device = 0
    if out is None:
        out = np.zeros(n, dtype=np.float64)
        ptr = out.ctypes.data if n else None
    elif isinstance(out, np.ndarray):
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != n:
            raise ValueError(f"out must be a C-contiguous float64 array of {n} entries")
        ptr = out.ctypes.data if n else None
    else:   # torch tensor
        if not out.is_contiguous() or out.numel() != n or str(out.dtype) != "torch.float64":
            raise ValueError(f"out must be a contiguous float64 tensor of {n} entries")
        ptr = out.data_ptr() if n else None
        on_device = 1 if out.is_cuda else 0
    _check(ctx, lib.emt_read_controls(ctx.handle, ptr, int(n), on_device))
    return out


def emt_adjoint(ctx: Ctx, v_target, n_steps: int, ckpt_every: int = 256, stream=None, grad=None):
    """Loss J = sum_n ||v_n - v*_n||^2 over steps 1..n_steps and dJ/dp for
    p = [branch values..., source amplitudes...] (include/emt.h).

    ``v_target`` is [n_steps][n_nodes] float64: a numpy array (host path) or
    a CUDA torch tensor (device path; the gradient is then a CUDA tensor,
    written into ``grad`` if given).  Returns (loss, grad)."""
    lib = load_library()
    n_steps = int(n_steps)
    shape = (n_steps, ctx.n_nodes)
    if isinstance(v_target, np.ndarray):
        tg = _arr(v_target, np.float64)
        if tg.shape != shape:
            raise ValueError(f"v_target must have shape {shape}")
        n_par = _n_params(ctx)
        g = np.zeros(n_par, dtype=np.float64) if grad is None else grad
        if not isinstance(g, np.ndarray) or g.dtype != np.float64 or g.size != n_par or not g.flags.c_contiguous:
            raise ValueError(f"grad must be a C-contiguous float64 array of {n_par} entries")
        tptr, gptr, on_device = tg.ctypes.data, g.ctypes.data if g.size else None, 0
    else:   # torch tensor on the device
        import torch
        if not v_target.is_cuda or v_target.dtype != torch.float64 or tuple(v_target.shape) != shape:
            raise ValueError(f"v_target must be a CUDA float64 tensor of shape {shape}")
        tg = v_target.contiguous()
        n_par = _n_params(ctx)
        g = torch.empty(n_par, dtype=torch.float64, device=tg.device) if grad is None else grad
        if not g.is_cuda or g.dtype != torch.float64 or g.numel() != n_par or not g.is_contiguous():
            raise ValueError(f"grad must be a contiguous CUDA float64 tensor of {n_par} entries")
        tptr, gptr, on_device = tg.data_ptr(), g.data_ptr() if n_par else None, 1
    loss = ctypes.c_double(0.0)
    _check(ctx, lib.emt_adjoint(ctx.handle, tptr, n_steps, int(ckpt_every), gptr, ctypes.byref(loss), on_device,
                                _stream_handle(stream)))
    return loss.value, g


def _n_params(ctx: Ctx) -> int:
    return emt_get_info(ctx, "n_branches") + emt_get_info(ctx, "n_sources")


def emt_autotune(ctx: Ctx, trial_steps: int = 50, stream=None) -> None:
    """Measure the multi-scenario launch shapes and keep the fastest (include/emt.h)."""
    _check(ctx, load_library().emt_autotune(ctx.handle, int(trial_steps), _stream_handle(stream)))


def emt_reset(ctx: Ctx) -> None:
    _check(ctx, load_library().emt_reset(ctx.handle))


def emt_save_state(ctx: Ctx) -> np.ndarray:
    """The context's run state as bytes (include/emt.h)."""
    lib = load_library()
    size = ctypes.c_int64(0)
    _check(ctx, lib.emt_save_state(ctx.handle, None, 0, ctypes.byref(size)))
    buf = np.empty(size.value, np.uint8)
    _check(ctx, lib.emt_save_state(ctx.handle, buf.ctypes.data, size.value, ctypes.byref(size)))
    return buf


def emt_load_state(ctx: Ctx, state) -> None:
    """Restore a state from emt_save_state (include/emt.h)."""
    buf = np.ascontiguousarray(state, np.uint8)
    _check(ctx, load_library().emt_load_state(ctx.handle, buf.ctypes.data, buf.size))


def emt_sync(ctx: Ctx):
    info = (ctypes.c_int32 * 4)()
    _check(ctx, load_library().emt_sync(ctx.handle, info))
    return list(info)


def emt_set_option(ctx: Ctx, key: str, value: int) -> None:
    _check(ctx, load_library().emt_set_option(ctx.handle, key.encode(), int(value)))


def emt_get_info(ctx: Ctx, key: str) -> int:
    v = ctypes.c_int64(0)
    _check(ctx, load_library().emt_get_info(ctx.handle, key.encode(), ctypes.byref(v)))
    return v.value


def emt_get_node_order(ctx: Ctx) -> np.ndarray:
    perm = np.zeros(ctx.n_nodes, dtype=np.int32)
    _check(ctx, load_library().emt_get_node_order(ctx.handle, perm.ctypes.data if perm.size else None))
    return perm


def emt_get_node_ctas(ctx: Ctx) -> np.ndarray:
    """CTA of every node, in the caller's node order (include/emt.h)."""
    cta = np.zeros(ctx.n_nodes, dtype=np.int32)
    _check(ctx, load_library().emt_get_node_ctas(ctx.handle, cta.ctypes.data if cta.size else None))
    return cta


def emt_get_line_ends(ctx: Ctx):
    """(cta, far_end, d) of every line end, library order (include/emt.h)."""
    n = emt_get_info(ctx, "n_line_ends")
    cta, far, d = (np.zeros(n, dtype=np.int32) for _ in range(3))
    ptr = (lambda a: a.ctypes.data if a.size else None)
    _check(ctx, load_library().emt_get_line_ends(ctx.handle, ptr(cta), ptr(far), ptr(d)))
    return cta, far, d


def emt_set_shard(ctx: Ctx, owner, rank: int) -> None:
    """Run only the CTAs with owner[c] == rank (owner None: all of them)."""
    if owner is None:
        _check(ctx, load_library().emt_set_shard(ctx.handle, None, int(rank)))
        return
    own = _arr(owner, np.int32)
    if own.size != emt_get_info(ctx, "n_ctas"):
        raise ValueError("owner needs one rank per CTA")
    _check(ctx, load_library().emt_set_shard(ctx.handle, own.ctypes.data, int(rank)))


def emt_shard_pack(ctx: Ctx, peer: int, out=None, stream=None) -> int:
    """Pack the last window's slots for rank ``peer`` into ``out`` (a CUDA
    uint8 torch tensor of at least that many bytes); out None: the size only."""
    lib = load_library()
    size = ctypes.c_int64(0)
    if out is None:
        _check(ctx, lib.emt_shard_pack(ctx.handle, int(peer), None, 0, ctypes.byref(size), None))
        return size.value
    _check(ctx, lib.emt_shard_pack(ctx.handle, int(peer), out.data_ptr(), out.numel() * out.element_size(),
                                   ctypes.byref(size), _stream_handle(stream)))
    return size.value


def emt_shard_unpack(ctx: Ctx, peer: int, buf, n_bytes: int, stream=None) -> None:
    """Write rank ``peer``'s packed slots (a CUDA tensor, ``n_bytes`` bytes) into the rings."""
    _check(ctx, load_library().emt_shard_unpack(ctx.handle, int(peer), buf.data_ptr() if n_bytes else None,
                                                int(n_bytes), _stream_handle(stream)))


PHASES = ("injection", "solve", "node_voltages", "updates", "poll_wait_line_end0", "updates_polls_barrier",
          "steps", "cycles_last_launch")


SS_PHASES = ("product_rows_thread0", "collect_next_values", "rows_to_barrier_thread0", "", "", "", "steps",
             "cycles_last_launch")


def emt_phase_clocks(ctx: Ctx, reset: bool = False) -> np.ndarray:
    """Per-CTA phase cycle counts [n_ctas, 8] (phase-clock build only; see include/emt.h)."""
    out = np.zeros((emt_get_info(ctx, "n_ctas"), len(PHASES)), dtype=np.uint64)
    _check(ctx, load_library().emt_phase_clocks(ctx.handle, out.ctypes.data if out.size else None, int(reset)))
    return out


def emt_last_error(ctx: Optional[Ctx] = None) -> str:
    msg = load_library().emt_last_error(ctx.handle if ctx is not None else None)
    return msg.decode() if msg else ""


def emt_destroy(ctx: Ctx) -> None:
    if ctx is not None and ctx.handle:
        load_library(False).emt_destroy(ctx.handle)
        ctx.handle = ctypes.c_void_p(None)


# ------------------------------------------------------------------ wrapper

class Simulator:
    """One network (optionally with scenarios) on the current CUDA device."""

    def __init__(self, net, scenarios=None, record: bool = True, n_steps: Optional[int] = None,
                 channels=None, decim: int = 1, options: Optional[dict] = None):
        self.net = net
        self.ctx = emt_build_network(net, scenarios)
        for k, v in (options or {}).items():
            emt_set_option(self.ctx, k, v)
        emt_prefactor(self.ctx)
        self.channels = np.arange(net.n_nodes, dtype=np.int32) if channels is None else _arr(channels, np.int32)
        self.decim = int(decim)
        if record:
            rows = int(n_steps if n_steps is not None else net.n_steps) // self.decim
            emt_set_recording(self.ctx, None if channels is None else self.channels, self.decim, rows)

    def run(self, n_steps: int, stream=None):
        emt_step_n(self.ctx, n_steps, stream)

    def waveforms(self, n_rows: Optional[int] = None, step0: Optional[int] = None, scen0: int = 0,
                  n_scen: Optional[int] = None, out=None):
        step0 = self.decim if step0 is None else step0
        if n_rows is None:
            n_rows = emt_get_info(self.ctx, "step") // self.decim - (step0 // self.decim - 1)
        n_scen = self.ctx.n_scenarios if n_scen is None else n_scen
        return emt_read_waveforms(self.ctx, self.channels, step0, n_rows, scen0, n_scen, out)

    def run_to_host(self, n_steps: int, out, chunk: int = 5000, stream=None):
        """Run ``n_steps`` steps and copy their recorded rows into ``out``
        (see step_and_read)."""
        return step_and_read(self.ctx, self.channels, self.decim, n_steps, out, chunk, stream)

    def controls(self, out=None):
        """Control block outputs of the last completed step."""
        return emt_read_controls(self.ctx, out)

    def sync(self):
        return emt_sync(self.ctx)

    def reset(self):
        emt_reset(self.ctx)

    def info(self, key: str) -> int:
        return emt_get_info(self.ctx, key)

    def close(self):
        emt_destroy(self.ctx)
