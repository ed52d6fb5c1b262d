"""Benchmark of the EMT time loop on B300 (one JSON line on rank 0).

Workload: the large-scale case -- a synthetic three-phase network of 1,000
buses (3,000 nodes, ~6,000 R/L/C branches, 50 three-phase sources) cut by
700 three-phase lossless Bergeron lines into 95 subsystems of 6..60 nodes,
dt = 20 us, 50,000 steps, every node voltage recorded every step.  One
benchmark "step" is one full run of those 50,000 time steps from the
de-energised state (emt_step_n), i.e. one pass of the whole hot path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--time-steps T] [--skip-extras] [--leg all|single|n1|shared_g|adjoint]
                  [--leg-steps N] [--leg-warm N] [--shape S_t,threads]

--time-steps shortens each run (for profiling small cases); --skip-extras
leaves out the end-to-end leg, the CPU baseline, the parity check and the
two further legs the metric names, reported as extra keys of the line:
  "scenarios": multi-scenario throughput (scenario-steps/s) of the N-1 study
      (1,024 scenarios of a 600-node network, 10,000 steps, one launch), of
      the shared-G study (4,096 scenarios of the large-scale network, all
      10,000 steps across the fault at step 2,500, every node recorded
      every 100th step) and of a
      control study (1,024 scenarios of the 600-node network with 40
      converter loads, set points per scenario, 10,000 steps), of the N-1
      study with 20 surge arresters and of studies of the 600-node network
      with frequency-dependent and with coupled lines;
  "adjoint": emt_adjoint time over the forward time for the gradient of
      sum_n ||v_n - v*_n||^2 over 20,000 steps of the large-scale network
      with checkpoints every 256 steps (and with the whole tape kept);
  "small_network": the 12-node single-subsystem network (latency of one
      CTA's dependent chain), with parity over every step;
  "runtime_switches": the large-scale network with 30 diode-rectifier loads
      and 10 current-zero breakers, against the same network without them;
  "coupled_lines": the large-scale network with its three-phase lines as
      coupled modal lines with interpolated travel times, against the plain one;
  "fd_line_groups": the same with its three-phase lines as frequency-dependent
      line groups (Clarke modes, each a lossy frequency-dependent line);
  "fd_lines": the same with its line conductors as lossy frequency-dependent
      lines, against the plain one;
  "nonlinear": the same with 40 surge arresters solved by the compensation
      method, against the plain one;
  "controls": the same with 180 converter loads (4,320 layered control
      blocks driving controlled current injections), against the plain one;
  "converter_stations": the same with 10 two-bridge diode converter stations
      (12 valves per subsystem, states factorised on the device), against
      the plain one;
  "bus_arresters": the same with arresters on all phases of 20 buses (three
      nonlinear resistors per subsystem), against the plain one;
  "sizes": the same family as 500 subsystems of 6 nodes, and as 500
      subsystems of 6..60 nodes (16,500 nodes, packed several to a CTA).

N > 1 runs N independent replicas (the single-network path does not shard:
its subsystems exchange line values every few steps), launched by
torch.distributed.run.  `--impl reference`
times the plain CPU oracle (test infrastructure) on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-steps/s and scenario-steps/s at 1 B300 (FP64, rel err ≤1e-10); adjoint/forward time ratio"
UNIT = "node-steps/s"
N_STEPS = 50000
E2E_CHUNK = 5000      # time steps per launch of the end-to-end leg (its copies overlap the next chunk)
FP64_PEAK_GFLOPS = 148 * 4 * 2.032          # derived: 148 SMs x 2 DFMA/clk x 2 flop x 2.032 GHz (max SM clock)
PEAKS_SOURCE = os.path.join(ROOT, "bench_peaks.cu")
_PEAKS = {}


def build_peaks() -> str:
    """Compile bench_peaks.cu for sm_103a into _build/ (once per source
    version); return the executable's path."""
    src = open(PEAKS_SOURCE, "rb").read()
    exe = os.path.join(ROOT, "_build", "bench_peaks_" + hashlib.sha256(src).hexdigest()[:12])
    if not os.path.exists(exe):
        os.makedirs(os.path.dirname(exe), exist_ok=True)
        subprocess.check_call([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-o", exe + ".tmp", PEAKS_SOURCE])
        os.replace(exe + ".tmp", exe)
    return exe


def measure_peaks() -> dict:
    """FP64 (and bf16 mma.sync) peaks measured on this GPU by bench_peaks.cu,
    built with nvcc into _build/ on first use; {} if it cannot run."""
    if _PEAKS:
        return _PEAKS
    try:
        exe = build_peaks()
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120).stdout.strip().splitlines()
        _PEAKS.update(json.loads(out[-1]))
    except (OSError, subprocess.SubprocessError, ValueError, IndexError) as e:
        _PEAKS.update({"error": str(e)})
    return _PEAKS


def fp64_peak_gflops() -> float:
    """The roofline's FP64 denominator: the DFMA rate measured in this run,
    else the derived figure."""
    return float(measure_peaks().get("fp64_dfma_gflops") or FP64_PEAK_GFLOPS)
KERNEL_SOURCES = ["paper_1903_01081_b300/csrc/emt_kernels.cu", "paper_1903_01081_b300/csrc/emt_device.cuh",
                  "paper_1903_01081_b300/csrc/emt_internal.h"]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "fwd_kernel_large_scale.json")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float) -> float:
    """The largest value of x over the ranks (x itself without a process
    group); NCCL reduces a CUDA tensor, gloo a CPU one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling:
    every rank processes the same units)."""
    return world * units_per_rank / t_max


def run_rank_selftest():
    """CPU check of the multi-rank aggregation (gloo): each rank reports a
    rank-dependent time; rank 0 prints the aggregate as the bench would."""
    import torch.distributed as dist
    rank, world, _ = dist_env()
    dist.init_process_group("gloo")
    t_local = 1.0 + 0.5 * rank
    t_max = max_over_ranks(t_local)
    value = whole_job_rate(1000.0, world, t_max)
    dist.barrier()
    if rank == 0:
        print(json.dumps({"selftest": "ranks", "world": world, "t_max": t_max, "value": value}), flush=True)
    dist.destroy_process_group()
    return 0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def algorithmic_flops_per_step(net, sim) -> float:
    """FP64 operations the method needs per time step:
    dense solve 2 n_s^2 per subsystem, plus 1 add per injection term (two
    per L/C branch, one per source branch and line end), 3 per L/C branch
    history update, 2 per line-end output, 1 per source-branch injection."""
    from paper_1903_01081_b300 import emt
    sum_n2 = emt.emt_get_info(sim.ctx, "sum_n2_components")   # the subsystems' own blocks, not a packed CTA's zeros
    kinds = np.asarray(net.br_kind)
    n_lc = int(np.sum(kinds != 0))
    n_sb = int(np.sum((np.asarray(net.br_k) <= -2) | (np.asarray(net.br_m) <= -2)))
    n_le = 2 * net.n_lines
    return 2.0 * sum_n2 + (2 * n_lc + n_sb + n_le) + 3 * n_lc + 2 * n_le + n_sb


def sparse_solve_flops_per_step(net) -> dict:
    """The solve as the paper's own processes 3-4 do it (sparse LU once,
    forward and back substitution every step; Sec. III-A), counted for the
    same subsystems at the first step's switch state: 2 (nnz(L) + nnz(U))
    - 3 n flop per subsystem with SuperLU's COLAMD ordering, against the
    explicit inverse's 2 n^2.  Reported beside the roofline, not used as its
    work (the method here is the dense prefactored inverse)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    from scipy.sparse.linalg import splu
    n = int(net.n_nodes)
    gk, gm, gv = [], [], []
    dt = float(net.dt)
    for k, m, kind, val in zip(net.br_k, net.br_m, net.br_kind, net.br_value):
        g = 1.0 / val if kind == 0 else (dt / (2.0 * val) if kind == 1 else 2.0 * val / dt)
        gk.append(int(k)); gm.append(int(m)); gv.append(g)
    for k, m, r, c0, c1 in zip(net.sw_k, net.sw_m, net.sw_r, net.sw_close_step, net.sw_open_step):
        if c0 <= 1 and (c1 < 0 or 1 < c1):
            gk.append(int(k)); gm.append(int(m)); gv.append(1.0 / r)
    rows, cols, vals = [], [], []
    for k, m, g in zip(gk, gm, gv):
        for a in (k, m):
            if a >= 0:
                rows.append(a); cols.append(a); vals.append(g)
        if k >= 0 and m >= 0:
            rows += [k, m]; cols += [m, k]; vals += [-g, -g]
    for k, m, z in zip(net.ln_k, net.ln_m, net.ln_zc):
        for a in (int(k), int(m)):
            rows.append(a); cols.append(a); vals.append(1.0 / z)
    G = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    adj = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    n_comp, lab = connected_components(adj, directed=False)
    sparse = dense = 0
    for c in range(n_comp):
        idx = np.flatnonzero(lab == c)
        lu = splu(G[idx][:, idx].tocsc(), permc_spec="COLAMD")
        sparse += 2 * (lu.L.nnz + lu.U.nnz) - 3 * len(idx)
        dense += 2 * len(idx) ** 2
    return {"sparse_lu_substitution_flop_per_step": int(sparse), "dense_inverse_flop_per_step": int(dense),
            "note": "the paper's sparse LU solve would need this many flop per step for the same subsystems "
                    "(SuperLU, COLAMD); the explicit inverse does the dense count"}


def cpu_baseline(net, n_steps: int):
    """The CPU oracle as it stands, single thread, on `n_steps` steps."""
    import oracle
    t0 = time.perf_counter()
    oracle.simulate(net, n_steps)
    dt = time.perf_counter() - t0
    return {"value": net.n_nodes * n_steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"large-scale network, {n_steps} of the 50,000 steps, all nodes recorded, 1 thread",
            "seconds": round(dt, 3), "host_cores_available": os.cpu_count()}


def scenario_leg(name, net, sc, n_steps, n_check, rec_channels, decim, tune_steps, warm_steps=500, shape=None):
    """Throughput of one multi-scenario study: one emt_step_n launch over all
    scenarios, CUDA events on the launching stream, after a short warm-up
    run; parity of `n_check` sampled scenarios against the oracle on the
    recorded (decimated) rows."""
    import torch
    import oracle
    from paper_1903_01081_b300 import emt
    t0 = time.perf_counter()
    sim = emt.Simulator(net, sc, n_steps=n_steps, channels=rec_channels, decim=decim)
    build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    if shape:
        emt.emt_set_option(sim.ctx, "scenarios_per_cta", shape[0])
        emt.emt_set_option(sim.ctx, "batch_threads", shape[1])
    else:
        emt.emt_autotune(sim.ctx, tune_steps, stream)
    tune_s = time.perf_counter() - t0
    if warm_steps > 0:
        sim.run(warm_steps, stream)
        sim.sync()
        sim.reset()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.run(n_steps, stream)
    e1.record(stream)
    sim.sync()
    ms = e0.elapsed_time(e1)
    S = sc.n_scenarios
    flops_per_scen_step = 2.0 * sim.info("sum_n2")
    rng = np.random.default_rng(7)
    check = sorted(rng.choice(S, size=n_check, replace=False).tolist())
    worst = 0.0
    ch = np.arange(net.n_nodes) if rec_channels is None else np.asarray(rec_channels)
    for s_ in check:
        got = sim.waveforms(scen0=s_, n_scen=1)[:, 0, :]
        ref = oracle.simulate(sc.expand(net, s_), n_steps, rec=ch)[decim - 1::decim]
        worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    out = {"scenarios": S, "nodes": int(net.n_nodes), "time_steps": n_steps, "ms": ms,
           "scenario_steps_per_s": S * n_steps / (ms / 1e3),
           "node_steps_per_s": S * net.n_nodes * n_steps / (ms / 1e3),
           "solve_gflops": flops_per_scen_step * S * n_steps / (ms / 1e3) / 1e9,
           "solve_frac_of_fp64_peak": flops_per_scen_step * S * n_steps / (ms / 1e3) / 1e9 / fp64_peak_gflops(),
           "n_matrix_variants": sim.info("n_matrix_variants"), "scenarios_per_cta": sim.info("scenarios_per_cta"),
           "threads_per_cta": sim.info("batch_threads"), "subsystem_groups": sim.info("batch_groups"),
           "solve_form": ("tensor cores (tcgen05 digit form) for the shared matrices of at least "
                          f"{sim.info('digit_min_rows')} rows, FP64 for the rest" if sim.info("digit_solve")
                          else "FP64"),
           "build_prefactor_s": round(build_s, 3), "autotune_s": round(tune_s, 3),
           "autotune_trial_steps": tune_steps, "kernel_launches": 1, "launch": "one CUDA-graph launch",
           "parity_rel_err_sampled": worst, "parity_scenarios": check,
           "recorded": f"{len(ch)} nodes every {decim} steps"}
    sim.close()
    return out


def _oracle_scenario(args):
    """One scenario on the CPU oracle (a spawn-pool worker): seconds taken."""
    net, sc, s_, n = args
    import oracle
    t0 = time.perf_counter()
    oracle.simulate(sc.expand(net, s_), n, rec=np.zeros(1, np.int32))
    return time.perf_counter() - t0


def oracle_scenario_baseline(net, sc, n_scen, n_steps, seed=64):
    """The CPU oracle as it stands on a seeded subset of `n_scen` scenarios
    of a study, `n_steps` steps each, one scenario per process over the
    host's cores (a spawn pool: the parent already holds a CUDA context).
    The rate divides the scenario-steps by the busy time per core (pool
    start-up excluded), and extrapolates per scenario-step."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    picks = sorted(np.random.default_rng(seed).choice(sc.n_scenarios, size=n_scen, replace=False).tolist())
    workers = max(1, min(os.cpu_count() or 1, n_scen))
    # an executor, not a Pool: a worker that dies raises here instead of hanging
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        secs = list(ex.map(_oracle_scenario, [(net, sc, s_, n_steps) for s_ in picks], timeout=600))
    total = float(sum(secs))
    return {"value": n_scen * n_steps / (total / workers), "unit": "scenario-steps/s", "cores": workers,
            "kind": "oracle", "single_thread_value": n_scen * n_steps / total,
            "sample": f"{n_scen} seeded scenarios, {n_steps} steps each, one process per core"}


def scenario_legs(which=("n1", "shared_g", "controls", "arresters", "fd", "coupled"), steps=None, shape=None,
                  warm=500, cpu=False):
    from paper_1903_01081_b300 import netgen as g
    out = {}
    if "n1" in which:
        net, sc = g.n1_contingency()
        n1 = scenario_leg("n1", net, sc, steps or 10000, 4, None, 100, 100, warm, shape)
        out["n1_contingency"] = dict(workload="N-1: 600-node three-phase network, 40 subsystems, one connection "
                                              "removed + three-phase fault at step 2,500 per scenario", **n1)
        if cpu:
            out["n1_contingency"]["cpu_baseline"] = oracle_scenario_baseline(net, sc, 64, 3000)
    if "shared_g" in which:
        net, sc = g.shared_g()
        sg = scenario_leg("shared_g", net, sc, steps or 10000, 2, None, 100, 20, warm, shape)
        out["shared_g"] = dict(workload="large-scale network, per-scenario source amplitude/phase and fault "
                                        "resistance at step 2,500; all 10,000 steps timed, every node of every "
                                        "scenario recorded every 100th step", **sg)
        if cpu:
            out["shared_g"]["cpu_baseline"] = oracle_scenario_baseline(net, sc, 64, 1000)
    if "controls" in which:
        net, sc = g.converter_study()
        ct = scenario_leg("controls", net, sc, steps or 10000, 4, None, 100, 100, warm, shape)
        out["control_study"] = dict(workload="600-node network with 40 converter loads (960 control blocks in 11 "
                                             "layers, 120 controlled injections), per scenario the converters' power "
                                             "set points x U[0.2, 1] and a fault resistance at step 2,500 (after the "
                                             "paper's PV study across irradiances)", **ct)
        if cpu:
            out["control_study"]["cpu_baseline"] = oracle_scenario_baseline(net, sc, 64, 3000)
    if "arresters" in which:
        base, sc = g.n1_contingency()
        net = g.with_arresters(base, n_arresters=20)
        ar = scenario_leg("arresters", net, sc, steps or 10000, 4, None, 100, 100, warm, shape)
        out["arrester_study"] = dict(workload="the N-1 study (1,024 scenarios of the 600-node network, one connection "
                                              "removed + three-phase fault at step 2,500) with 20 surge arresters "
                                              "solved by the compensation method per scenario", **ar)
        if cpu:
            out["arrester_study"]["cpu_baseline"] = oracle_scenario_baseline(net, sc, 64, 3000)
    if "fd" in which:
        base, _ = g.n1_contingency(n_scenarios=1)
        net, sc = g.shared_g(n_scenarios=1024, base=g.with_fd_lines(base))
        fd = scenario_leg("fd", net, sc, steps or 10000, 4, None, 100, 100, warm, shape)
        out["fd_line_study"] = dict(workload="the 600-node network with its 168 line conductors frequency-dependent "
                                             "(one Y_c pole, two propagation poles, fractional travel times); per "
                                             "scenario source amplitudes and angles and a fault resistance at step "
                                             "2,500", **fd)
        if cpu:
            out["fd_line_study"]["cpu_baseline"] = oracle_scenario_baseline(net, sc, 64, 3000)
    if "coupled" in which:
        base, _ = g.n1_contingency(n_scenarios=1)
        net, sc = g.shared_g(n_scenarios=1024, base=g.with_coupled_lines(base))
        cl = scenario_leg("coupled", net, sc, steps or 10000, 4, None, 100, 100, warm, shape)
        out["coupled_line_study"] = dict(workload="the 600-node network with its 56 three-phase lines as coupled "
                                                  "Clarke-mode lines with interpolated travel times; per scenario "
                                                  "source amplitudes and angles and a fault resistance at step 2,500",
                                         **cl)
        if cpu:
            out["coupled_line_study"]["cpu_baseline"] = oracle_scenario_baseline(net, sc, 64, 3000)
    return out


def adjoint_leg(steps=None, reps=3):
    """emt_adjoint (loss + gradient for all branch values and source
    amplitudes) over the forward run, 20,000 steps of the large-scale
    network; wall time of the call (it allocates and synchronises)."""
    import torch
    from paper_1903_01081_b300 import emt, netgen as g
    net = g.large_scale()
    N = steps or 20000
    br, amp = g.adjoint_target(net, seed=1005)
    pert = net.copy()
    pert.br_value, pert.src_amp = br, amp
    tsim = emt.Simulator(pert, n_steps=N)
    tsim.run(N)
    tsim.sync()
    tgt = torch.empty((N, 1, net.n_nodes), dtype=torch.float64, device="cuda")
    tsim.waveforms(out=tgt)
    tsim.close()
    tgt = tgt.view(N, net.n_nodes)
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    stream = torch.cuda.current_stream()
    fwd = []
    for _ in range(reps):
        emt.emt_reset(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        emt.emt_step_n(ctx, N, stream)
        e1.record(stream)
        emt.emt_sync(ctx)
        fwd.append(e0.elapsed_time(e1))
    t_fwd = float(np.median(fwd))
    res = {}
    for K in (256, 0):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            J, _ = emt.emt_adjoint(ctx, tgt, N, K, stream)
            torch.cuda.synchronize()
            ts.append(1e3 * (time.perf_counter() - t0))
        res[K] = float(np.median(ts))
    emt.emt_destroy(ctx)
    return {"workload": "gradient of sum_n ||v_n - v*_n||^2 over all 3,000 nodes of the large-scale network, "
                        f"{N:,} steps, w.r.t. all branch values and source amplitudes",
            "n_params": int(net.n_branches + net.n_sources), "forward_ms": t_fwd,
            "adjoint_ms_ckpt256": res[256], "ratio_ckpt256": res[256] / t_fwd,
            "adjoint_ms_full_tape": res[0], "ratio_full_tape": res[0] / t_fwd,
            "timing": "wall time of the emt_adjoint call (allocations, forward with checkpoints, re-runs, reverse "
                      "sweep, gradient copy) over the CUDA-event time of emt_step_n for the same 20,000 steps",
            "loss": J, "cpu_baseline": oracle_adjoint_baseline(net, tgt, min(2000, N), N)}


def oracle_adjoint_baseline(net, tgt, n_sample, n_full):
    """The CPU oracle's full-tape adjoint (one thread) on the first n_sample
    steps of the same target, scaled to the leg's step count."""
    import oracle
    tg = tgt[:n_sample].cpu().numpy()
    t0 = time.perf_counter()
    oracle.adjoint(net, n_sample, tg)
    sec = time.perf_counter() - t0
    return {"seconds_for_sample": round(sec, 3), "sample_steps": n_sample, "cores": 1, "kind": "oracle",
            "estimated_ms_full": 1e3 * sec * n_full / n_sample,
            "sample": f"oracle adjoint (whole tape, 1 thread) over steps 1..{n_sample}, scaled to {n_full:,} steps"}


def small_network_leg(reps=3):
    """The 12-node single-subsystem RLC network with its fault at step 2,000:
    20,000 steps, one CTA (latency of the dependent chain), parity over all
    steps, and the CPU oracle on the same run."""
    import torch
    import oracle
    from paper_1903_01081_b300 import emt, netgen as g
    net = g.single_rlc()
    N = net.n_steps
    sim = emt.Simulator(net, n_steps=N)
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(reps):
        sim.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(N, stream)
        e1.record(stream)
        sim.sync()
        ms.append(e0.elapsed_time(e1))
    w = sim.waveforms()[:, 0, :]
    sim.close()
    t0 = time.perf_counter()
    ref = oracle.simulate(net, N)
    cpu = time.perf_counter() - t0
    t = float(np.median(ms))
    return {"workload": "12-node single-phase RLC network, 20 branches, 1 kV source, 0.01 ohm fault at step 2,000; "
                        "dt 50 us, 20,000 steps, all nodes recorded",
            "ms": t, "us_per_step": 1e3 * t / N, "node_steps_per_s": net.n_nodes * N / (t / 1e3),
            "parity_rel_err_all_steps": float(np.max(np.abs(w - ref)) / np.max(np.abs(ref))),
            "cpu_baseline": {"value": net.n_nodes * N / cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "the whole run, 1 thread"}}


def variant_leg(variant, workload, steps=None, reps=3, extra=None):
    """node-steps/s of a run from the de-energised state of ``variant`` (a
    variant of the large-scale network), beside the plain network, and
    sampled parity of the variant against the oracle."""
    import torch
    import oracle
    from paper_1903_01081_b300 import emt, netgen as g
    N = steps or N_STEPS
    out = {}
    for tag, net in (("variant", variant), ("plain", g.large_scale())):
        sim = emt.Simulator(net, n_steps=N)
        stream = torch.cuda.current_stream()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        ms = []
        for _ in range(reps):
            sim.reset()
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.run(N, stream)
            e1.record(stream)
            sim.sync()
            ms.append(e0.elapsed_time(e1))
        t = float(np.median(ms))
        d = {"nodes": int(net.n_nodes), "time_steps": N, "ms": t, "us_per_step": 1e3 * t / N,
             "node_steps_per_s": net.n_nodes * N / (t / 1e3)}
        if tag == "variant":
            n_chk = min(2000, N)
            w = sim.waveforms(n_rows=n_chk)[:, 0, :]
            ref = oracle.simulate(net, n_chk)
            d["parity_rel_err_first_steps"] = float(np.max(np.abs(w - ref)) / np.max(np.abs(ref)))
            if extra:
                d.update(extra(net, n_chk))
        sim.close()
        out[tag] = d
    out["workload"] = workload
    out["slowdown_vs_plain"] = out["variant"]["us_per_step"] / out["plain"]["us_per_step"]
    return out


def runtime_switch_leg(steps=None, reps=3):
    """The large-scale network with 30 diode-rectifier loads and 10
    current-zero breakers (runtime switches, 40 extra nodes)."""
    import oracle
    from paper_1903_01081_b300 import netgen as g

    def changes(net, n):
        st = oracle.runtime_switch_states(net, n)
        return {"runtime_switches": int(net.n_runtime_switches),
                "state_changes_in_checked_steps": int(np.sum(st[1:] != st[:-1]))}
    return variant_leg(g.with_rectifier_loads(g.large_scale(), seed=1006),
                       "large-scale network plus 30 diode-rectifier loads (diode, R, C) and 10 breakers that open "
                       "at the first current zero after a trip step; all nodes recorded", steps, reps, changes)


def coupled_line_leg(steps=None, reps=3):
    """The large-scale network with its 700 three-phase lines as coupled
    Clarke-mode lines with non-integer travel times."""
    from paper_1903_01081_b300 import netgen as g
    return variant_leg(g.with_coupled_lines(g.large_scale()),
                       "large-scale network with its 700 three-phase lines as transposed coupled lines in Clarke "
                       "modes (zero-sequence Z_c and travel time larger), travel times (d + U[0,1)) dt interpolated; "
                       "all nodes recorded", steps, reps)


def fd_line_leg(steps=None, reps=3):
    """The large-scale network with its 2,100 line conductors as lossy
    frequency-dependent lines (one Y_c pole, two propagation poles, travel
    times with a fractional part)."""
    from paper_1903_01081_b300 import netgen as g
    return variant_leg(g.with_fd_lines(g.large_scale()),
                       "large-scale network with its 2,100 line conductors as frequency-dependent lines: Y_c = 1/Z_c "
                       "+ one pole, A = e^{-s tau} x two poles (DC transmission 0.82-0.98), travel times (d + U[0,1)) "
                       "dt; all nodes recorded", steps, reps)


def fd_group_leg(steps=None, reps=3):
    """The large-scale network with its 700 three-phase lines as frequency-
    dependent line groups: Clarke modes, each mode a lossy frequency-dependent
    line with its own impedance, travel time and poles."""
    from paper_1903_01081_b300 import netgen as g
    return variant_leg(g.with_fd_line_groups(g.large_scale()),
                       "large-scale network with its 700 three-phase lines as frequency-dependent line groups: "
                       "Clarke modes (zero sequence slower, of higher impedance), each mode Y_c = 1/Z + one pole, "
                       "A = e^{-s tau} x two poles, fractional travel times; all nodes recorded", steps, reps)


def nonlinear_leg(steps=None, reps=3):
    """The large-scale network with 40 surge arresters (odd piecewise-linear
    resistors solved by the compensation method, one per subsystem)."""
    import oracle
    from paper_1903_01081_b300 import netgen as g

    def active(net, n):
        v = oracle.simulate(net, n, rec=net.nl_k)
        return {"nonlinear_resistors": int(net.n_nonlinear),
                "conducting_in_checked_steps": int(np.sum(np.max(np.abs(v), axis=0) > g.ARRESTER_V[0]))}
    return variant_leg(g.with_arresters(g.large_scale()),
                       "large-scale network plus 40 phase-to-ground surge arresters (odd piecewise-linear, knee "
                       "~0.8-1.5 kV, one per subsystem, at the source buses first) solved by the compensation "
                       "method; all nodes recorded", steps, reps, active)


def station_leg(steps=None, reps=3):
    """The large-scale network with 10 converter stations of two six-pulse
    diode bridges each (12 valves in one subsystem: switch states factorised
    on the device when first met)."""
    import oracle
    from paper_1903_01081_b300 import netgen as g

    def states(net, n):
        st = oracle.runtime_switch_states(net, n)
        return {"runtime_switches": int(net.n_runtime_switches),
                "state_changes_in_checked_steps": int(np.sum(st[1:] != st[:-1])),
                "distinct_network_states_in_checked_steps": len({tuple(r) for r in st})}
    return variant_leg(g.with_converter_stations(g.large_scale(), n_stations=10),
                       "large-scale network plus 10 converter stations (two six-pulse diode bridges each, 12 valves "
                       "with snubbers in one subsystem, commutation inductances, R-C DC loads); switch states "
                       "factorised on the device the first time they occur; all nodes recorded", steps, reps, states)


def bus_arrester_leg(steps=None, reps=3):
    """The large-scale network with three-phase arrester sets at 20 buses
    (three nonlinear resistors per subsystem, solved together)."""
    import oracle
    from paper_1903_01081_b300 import netgen as g

    def active(net, n):
        v = oracle.simulate(net, n, rec=net.nl_k)
        knee = np.asarray(net.nl_v).reshape(-1, 8)[:, 0]
        return {"nonlinear_resistors": int(net.n_nonlinear),
                "conducting_in_checked_steps": int(np.sum(np.max(np.abs(v), axis=0) > knee))}
    return variant_leg(g.with_bus_arresters(g.large_scale(), n_buses=20),
                       "large-scale network plus surge arresters on all three phases of 20 buses (3 per subsystem, "
                       "solved together through their Thevenin matrix); all nodes recorded", steps, reps, active)


def control_leg(steps=None, reps=3):
    """The large-scale network with 180 power-regulated converter loads, each
    24 layered control blocks driving three controlled current injections."""
    import oracle
    from paper_1903_01081_b300 import netgen as g

    def blocks(net, n):
        y = oracle.controls(net, n)
        return {"control_blocks": int(net.n_control_blocks), "control_injections": int(net.n_control_injections),
                "max_abs_injected_current_in_checked_steps": float(np.max(np.abs(y[:, 21::24])))}
    return variant_leg(g.with_converter_controls(g.large_scale()),
                       "large-scale network plus 180 converter loads (the 50 source buses, then random buses): "
                       "24 control blocks each in 11 layers (measure, per-unit, power, PI, limits, lag), drawing "
                       "a regulated power through controlled current injections, a 20 ohm damping resistor per "
                       "phase; all nodes recorded", steps, reps, blocks)


def size_leg(net, workload, steps, reps=3, n_check=1000, cpu_steps=1000):
    """node-steps/s of one network from the de-energised state (L2 flushed
    between runs), its whole-chip and critical-path FP64 fractions, parity
    on the first steps and the single-thread oracle on a sample."""
    import torch
    import oracle
    from paper_1903_01081_b300 import emt
    N = steps
    sim = emt.Simulator(net, n_steps=N)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ms = []
    for _ in range(reps):
        sim.reset()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(N, stream)
        e1.record(stream)
        sim.sync()
        ms.append(e0.elapsed_time(e1))
    t = float(np.median(ms)) / 1e3
    flops = algorithmic_flops_per_step(net, sim)
    n_max = sim.info("max_subsystem_nodes")
    out = {"workload": workload, "nodes": int(net.n_nodes), "subsystems": sim.info("n_components"),
           "ctas": sim.info("n_subsystems"), "largest_component": sim.info("max_component_nodes"),
           "largest_cta_nodes": n_max, "time_steps": N, "ms": 1e3 * t, "us_per_step": 1e6 * t / N,
           "node_steps_per_s": net.n_nodes * N / t,
           "fp64_frac_of_measured_peak": flops * N / t / 1e9 / fp64_peak_gflops(),
           # the largest CTA's dense solve (a packed CTA's zero blocks included: its SM runs them)
           "critical_path_sm_frac": (2.0 * n_max * n_max) / (t / N) / (fp64_peak_gflops() / 148 * 1e9),
           "smem_bytes_per_cta": sim.info("smem_bytes")}
    n_chk = min(n_check, N)
    w = sim.waveforms(n_rows=n_chk)[:, 0, :]
    sim.close()
    t0 = time.perf_counter()
    ref = oracle.simulate(net, n_chk)
    cpu = time.perf_counter() - t0
    out["parity_rel_err_first_steps"] = float(np.max(np.abs(w - ref)) / np.max(np.abs(ref)))
    out["parity_steps"] = n_chk
    out["cpu_baseline"] = {"value": net.n_nodes * n_chk / cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                           "sample": f"the first {n_chk} steps, all nodes recorded, 1 thread"}
    return out


def phases_leg(steps=None):
    """clock64 cycles per phase of every step of the single-network kernel
    (the phase-clock build, EMT_PHASES=1; this function re-runs bench.py
    under it when needed) for the 12-node RLC network, the strict 500 x 6
    reading and the large-scale network: per step, the mean over CTAs and
    the CTA with the most own work (injection + solve + node voltages +
    updates), beside the event-timed microseconds per step."""
    from paper_1903_01081_b300 import emt, netgen as g
    if not emt.phases_build():
        cmd = [sys.executable, os.path.abspath(__file__), "--leg", "phases"]
        if steps:
            cmd += ["--leg-steps", str(steps)]
        r = subprocess.run(cmd, capture_output=True, text=True, env=dict(os.environ, EMT_PHASES="1"))
        if r.returncode != 0:
            raise RuntimeError("phase-clock run failed: " + r.stderr[-2000:])
        return json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])["phases"]
    import torch
    N = steps or 20000
    cases = (("single_rlc_12_nodes", g.single_rlc()), ("strict_500x6", g.large_scale(strict_500=True)),
             ("large_scale_3000_nodes", g.large_scale()))
    out = {}
    runs = [(tag, net, 0) for tag, net in cases] + [(tag + "_state_space", net, 2) for tag, net in cases[:2]]
    for tag, net, ss in runs:
        names = emt.PHASES if ss == 0 else emt.SS_PHASES
        n = min(N, net.n_steps) if tag.startswith("single_rlc") else N
        sim = emt.Simulator(net, n_steps=n, options={"state_space": ss})
        stream = torch.cuda.current_stream()
        sim.run(min(n, 2000), stream)          # warm-up launch
        sim.sync()
        sim.reset()
        emt.emt_phase_clocks(sim.ctx, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(n, stream)
        e1.record(stream)
        sim.sync()
        ms = e0.elapsed_time(e1)
        ph = emt.emt_phase_clocks(sim.ctx).astype(np.float64)
        steps_run = ph[:, 6]
        per = ph[:, :6] / steps_run[:, None]
        own = per[:, 0] + per[:, 1] + per[:, 2] + per[:, 3] if ss == 0 else per[:, 0]
        crit = int(np.argmax(own))
        cyc_per_step = float(np.max(ph[:, 7] / steps_run))   # the slowest CTA's (independent subsystems end apart)
        out[tag] = {"ctas": int(ph.shape[0]), "largest_cta_nodes": sim.info("max_subsystem_nodes"),
                    "steps": n, "us_per_step_events": 1e3 * ms / n,
                    "cycles_per_step_span": cyc_per_step,
                    "sm_mhz_implied": cyc_per_step / (1e3 * ms / n),
                    "kernel": "fwd_kernel (CTA per subsystem)" if ss == 0 else "fwd_ss_kernel (state-space form)",
                    "mean_over_ctas": {k: round(float(v), 1) for k, v in zip(names[:6], per.mean(axis=0)) if k},
                    "critical_cta": {"cta": crit, **{k: round(float(v), 1) for k, v in zip(names[:6], per[crit]) if k}}}
        sim.close()
    return out


def shared_g_digit_leg(steps=None):
    """The shared-G study (4,096 scenarios, 3,000 nodes) at fixed launch
    shapes with the solve in FP64 and in digit form on the tensor cores
    (option digit_solve): scenario-steps/s of 100 steps each."""
    import torch
    from paper_1903_01081_b300 import emt, netgen as g
    net, sc = g.shared_g(n_scenarios=4096)
    N = steps or 100
    out = []
    for St, th in ((16, 1024), (28, 512), (28, 1024), (None, None)):
        for digit in (0, 1, 2):   # 2: the digit form for every shared matrix (digit_min_rows 1)
            ctx = emt.emt_build_network(net, sc)
            emt.emt_prefactor(ctx)
            emt.emt_set_option(ctx, "digit_solve", min(digit, 1))
            if digit == 2:
                emt.emt_set_option(ctx, "digit_min_rows", 1)
            tuned = St is None
            try:
                if tuned:   # the autotuner's pick for this form
                    emt.emt_autotune(ctx, 20)
                    St, th = emt.emt_get_info(ctx, "scenarios_per_cta"), emt.emt_get_info(ctx, "batch_threads")
                else:
                    emt.emt_set_option(ctx, "scenarios_per_cta", St)
                    emt.emt_set_option(ctx, "batch_threads", th)
            except emt.EmtError as e:   # (a shape whose tables do not fit in shared memory)
                out.append({"scenarios_per_cta": St, "threads": th, "digit_solve": digit, "error": str(e)})
                emt.emt_destroy(ctx)
                continue
            stream = torch.cuda.current_stream()
            emt.emt_step_n(ctx, 10, stream)
            emt.emt_sync(ctx)
            emt.emt_reset(ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            emt.emt_step_n(ctx, N, stream)
            e1.record(stream)
            emt.emt_sync(ctx)
            ms = e0.elapsed_time(e1)
            out.append({"scenarios_per_cta": St, "threads": th, "digit_solve": digit, "autotuned": tuned,
                        "groups": emt.emt_get_info(ctx, "batch_groups"),
                        "scenario_steps_per_s": 4096 * N / (ms / 1e3)})
            emt.emt_destroy(ctx)
            if tuned:
                St = th = None
    return {"workload": "shared-G study, 4,096 scenarios of the 3,000-node network, fixed launch shapes",
            "runs": out}


def scale_legs(steps=None, reps=3):
    """The large-scale family at two other sizes: the strict reading of
    500 subsystems of 6 nodes (3,000 nodes), and 500 subsystems of 6..60
    nodes (33 on average, 16,500 nodes, near the paper's 16,653-node case),
    more than one launch holds co-resident, so packed several to a CTA."""
    from paper_1903_01081_b300 import netgen as g
    N = steps or 20000
    n_sub = 500
    net = g.paper_scale(n_sub, n_steps=N)
    return {"strict_500x6": size_leg(g.large_scale(strict_500=True), "strict reading: 500 subsystems of 2 "
                                     "three-phase buses (3,000 nodes), 700 three-phase lines, 50 sources; dt 20 us",
                                     N, reps),
            "paper_scale": size_leg(net, f"{n_sub} subsystems of 2..20 three-phase buses ({net.n_nodes:,} nodes, "
                                    f"{net.n_branches:,} R/L/C branches, {net.n_lines // 3:,} three-phase lines, "
                                    f"{net.n_sources // 3} three-phase sources; lines, sources and branches scaled "
                                    "from the 1,000-bus network); dt 20 us", N, reps)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1903_01081_b300 import netgen as g
    net = g.large_scale()
    sample = 10000
    for _ in range(args.warmup):
        cpu_baseline(net, 2000)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        import oracle
        oracle.simulate(net, sample)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = net.n_nodes * sample * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "large-scale network (3,000 nodes, 95 subsystems, 700 three-phase lines)",
                       "sample_steps_per_bench_step": sample, "parallelism": "none (CPU oracle, 1 thread)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{sample} time steps per bench step, 1 thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_1903_01081_b300 import emt, netgen as g
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    net = g.large_scale()
    n = net.n_nodes
    N_STEPS = args.time_steps

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident timing
    sim = emt.Simulator(net, n_steps=N_STEPS)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 126 MB L2
    for _ in range(args.warmup):
        sim.reset()
        sim.run(N_STEPS, stream)
    sim.sync()
    launches0 = sim.info("kernel_launches")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clocks:
        for i in range(args.steps):
            sim.reset()
            flush.zero_()
            ev[i][0].record(stream)
            sim.run(N_STEPS, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    sim.sync()
    launches = sim.info("kernel_launches") - launches0
    ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(ms) / 1e3
    t_max = max_over_ranks(t_local)
    value = whole_job_rate(n * N_STEPS * args.steps, world, t_max)

    # parity of the timed configuration against the oracle on sampled steps
    w = sim.waveforms(n_rows=min(2000, N_STEPS))[:, 0, :]
    flops = algorithmic_flops_per_step(net, sim) * N_STEPS
    n_sub = sim.info("n_subsystems")
    n_max = sim.info("max_subsystem_nodes")
    sim.close()

    if args.skip_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "ms_per_step": 1e3 * t_max / args.steps, "time_steps": N_STEPS,
                              "note": "profiling run: extras skipped"}), flush=True)
        return 0

    # ---------------- end to end through the C ABI with host buffers
    e2e_times = []
    h2d = sum(np.asarray(getattr(net, f)).nbytes for f in
              ("br_k", "br_m", "br_kind", "br_value", "src_amp", "src_phase", "src_freq", "ln_k", "ln_m", "ln_zc",
               "ln_delay", "sw_k", "sw_m", "sw_r", "sw_close_step", "sw_open_step"))
    out = torch.empty((N_STEPS, 1, n), dtype=torch.float64, pin_memory=True)
    channels = np.arange(n, dtype=np.int32)
    for i in range(args.warmup + args.steps):
        barrier()
        t0 = time.perf_counter()
        ctx = emt.emt_build_network(net)
        emt.emt_prefactor(ctx)
        emt.emt_set_recording(ctx, None, 1, N_STEPS)
        # the steps in chunks of 5,000, each chunk's 120 MB of waveforms copied to
        # pinned host memory on a second stream while the next chunk runs
        emt.step_and_read(ctx, channels, 1, N_STEPS, out, E2E_CHUNK, stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        emt.emt_destroy(ctx)
        if i >= args.warmup:
            e2e_times.append(dt)
    e2e_value = whole_job_rate(n * N_STEPS * args.steps, world, max_over_ranks(sum(e2e_times)))

    if rank == 0:
        import oracle
        ref = oracle.simulate(net, min(2000, N_STEPS))
        parity = float(np.max(np.abs(w - ref)) / np.max(np.abs(ref)))
        per_launch_s = t_max / args.steps
        achieved = flops / per_launch_s / 1e9
        traffic = None
        if os.path.exists(PROFILE_SUMMARY):
            prof = json.load(open(PROFILE_SUMMARY))
            if prof.get("kernel_source_hash") == kernel_hash():
                traffic = prof.get("dram_bytes_full_run")
        peak = fp64_peak_gflops()
        peaks = measure_peaks()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "large-scale network: 3,000 nodes (1,000 three-phase buses), ~6,250 R/L/C "
                                   "branches, 700 three-phase lossless lines, 50 three-phase sources; "
                                   "dt 20 us, 50,000 steps per bench step, all nodes recorded",
                       "n_subsystems": n_sub, "time_steps_per_bench_step": N_STEPS,
                       "l2": "flushed between timed iterations (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "fwd_kernel (+ source_kernel, <0.5% of the time)",
                         "peak_source": ("measured in this run by bench_peaks.cu: FP64 DFMA, 8 independent chains "
                                         "per thread, best of 148 x {1,2,4,8} CTAs of 256 threads (of measured)"
                                         if "fp64_dfma_gflops" in peaks else
                                         "derived: 148 SMs x 2 DFMA/clk x 2 flop x 2.032 GHz (measurement failed)"),
                         "derived_peak": FP64_PEAK_GFLOPS, "frac_of_derived_peak": achieved / FP64_PEAK_GFLOPS,
                         "measured_peaks": peaks,
                         "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of the fwd_kernel and "
                                           "source_kernel launches of one full 50,000-step run (profiles/"
                                           "fwd_kernel_large_scale.json); null if the kernel sources changed since",
                         # the step cannot end before the largest subsystem's dense solve (2 n^2 flop) has run
                         # on its one SM: that SM's share of the FP64 peak against the measured step time
                         "critical_path_sm_frac": (2.0 * n_max * n_max) / (per_launch_s / N_STEPS)
                                                  / (peak / 148 * 1e9),
                         "critical_path": f"2 n^2 flop of the largest subsystem (n = {n_max}) per step on one SM",
                       "paper_sparse_solve": sparse_solve_flops_per_step(net)},
            "cpu_baseline": cpu_baseline(net, N_STEPS),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(N_STEPS * n * 8),
                    "path": f"emt_build_network, emt_prefactor, emt_set_recording, then {N_STEPS // E2E_CHUNK} x "
                            f"emt_step_n({E2E_CHUNK}) with each chunk's waveforms read by emt_read_waveforms_async "
                            "into pinned host memory on a second stream (step_and_read)"},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "parity_rel_err_first_2000_steps": parity,
            **({"scenarios": scenario_legs(cpu=True), "adjoint": adjoint_leg(), "small_network": small_network_leg(), "runtime_switches": runtime_switch_leg(),
                "coupled_lines": coupled_line_leg(), "fd_lines": fd_line_leg(),
                "fd_line_groups": fd_group_leg(), "nonlinear": nonlinear_leg(),
                "controls": control_leg(), "converter_stations": station_leg(),
                "bus_arresters": bus_arrester_leg(), "sizes": scale_legs()}
               if args.leg == "all" else {}),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--time-steps", type=int, default=N_STEPS)
    ap.add_argument("--skip-extras", action="store_true")
    ap.add_argument("--leg", choices=["all", "single", "n1", "shared_g", "adjoint", "runtime_switches", "coupled_lines",
                                      "fd_lines", "fd_line_groups", "nonlinear", "controls", "sizes", "control_study",
                                      "arrester_study", "fd_line_study", "coupled_line_study", "converter_stations",
                                      "bus_arresters", "phases", "shared_g_digit"],
                    default="all",
                    help="all: the JSON line with every leg; single: the single-network leg only; "
                         "n1 / shared_g / adjoint: that leg alone (profiling)")
    ap.add_argument("--leg-steps", type=int, default=None, help="time steps of a lone n1 / shared_g / adjoint leg")
    ap.add_argument("--leg-warm", type=int, default=500, help="warm-up steps of a lone scenario leg")
    ap.add_argument("--shape", default=None, help="S_t,threads for a lone scenario leg (no autotuning)")
    ap.add_argument("--selftest-ranks", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--peaks", action="store_true", help="print the peaks bench_peaks.cu measures and exit")
    args = ap.parse_args()
    if args.selftest_ranks:
        return run_rank_selftest()
    if args.peaks:
        print(json.dumps(measure_peaks()), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.leg in ("n1", "shared_g", "adjoint", "runtime_switches", "coupled_lines", "fd_lines", "fd_line_groups",
                    "nonlinear",
                    "controls", "sizes", "control_study", "arrester_study", "fd_line_study", "coupled_line_study",
                    "converter_stations", "bus_arresters", "phases", "shared_g_digit"):
        return run_leg(args)
    return run_ours(args)


def run_leg(args):
    """One leg alone, one JSON line (for profiling small cases)."""
    import torch
    torch.cuda.set_device(dist_env()[2])
    if args.leg == "adjoint":
        out = adjoint_leg(args.leg_steps, reps=1)
    elif args.leg == "runtime_switches":
        out = runtime_switch_leg(args.leg_steps, reps=1)
    elif args.leg == "coupled_lines":
        out = coupled_line_leg(args.leg_steps, reps=1)
    elif args.leg == "controls":
        out = control_leg(args.leg_steps, reps=1)
    elif args.leg == "fd_lines":
        out = fd_line_leg(args.leg_steps, reps=1)
    elif args.leg == "fd_line_groups":
        out = fd_group_leg(args.leg_steps, reps=1)
    elif args.leg == "nonlinear":
        out = nonlinear_leg(args.leg_steps, reps=1)
    elif args.leg == "converter_stations":
        out = station_leg(args.leg_steps, reps=1)
    elif args.leg == "bus_arresters":
        out = bus_arrester_leg(args.leg_steps, reps=1)
    elif args.leg == "sizes":
        out = scale_legs(args.leg_steps, reps=1)
    elif args.leg == "phases":
        out = {"phases": phases_leg(args.leg_steps)}
    elif args.leg == "shared_g_digit":
        out = shared_g_digit_leg(args.leg_steps)
    elif args.leg in ("control_study", "arrester_study", "fd_line_study", "coupled_line_study"):
        shape = tuple(int(x) for x in args.shape.split(",")) if args.shape else None
        which = {"control_study": "controls", "arrester_study": "arresters", "fd_line_study": "fd",
                 "coupled_line_study": "coupled"}[args.leg]
        out = scenario_legs((which,), args.leg_steps, shape, args.leg_warm)
    else:
        shape = tuple(int(x) for x in args.shape.split(",")) if args.shape else None
        out = scenario_legs((args.leg,), args.leg_steps, shape, args.leg_warm)
    print(json.dumps({"leg": args.leg, **out}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
