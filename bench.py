"""Benchmark: atom-steps/s of NVE molecular dynamics driven by the PaiNN-form potential.

One step = velocity-Verlet half kick + drift, per-step prune of the Verlet list (rebuild when
an atom moved more than skin/2), energy + forces + virial (forward and adjoint kernels), second
half kick.  Workload (default): single-species fcc crystal, a = 4.05 A, 63x63x63 cells
(1,000,188 atoms), Gaussian jitter 0.05 A, cutoff 5 A, skin 1 A, F = 128, 3 layers, 20 radial
basis functions, Xavier-uniform weights from seed 0; synthetic inputs (no datasets/weights).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s (E+F) at 1M atoms, BF16 vs FP32 at stated force RMSE; p50/p99"
FCC_CELLS = 63
F, K, T, S = 128, 20, 3, 1
RC, SKIN, DT, TEMP = 5.0, 1.0, 1.0, 300.0

# Algorithmic work (the per-unit figures of the roofline):
#   per active edge and layer, the message step is (6K + 22) F FLOP: the filter contraction
#   2 x 3F x K (the K x 3F filter times the basis), bias and cutoff, and the s / v message terms
#   (22 F); its adjoint is counted as the same again (input gradients only);
#   per atom and step, 2 T (30 F^2 + n_e (6K + 22) F) + F^2 FLOP (node MLPs 30 F^2 per layer,
#   forward and adjoint, plus the readout) and 42 F T stored values (read and written node
#   features and saved activations) plus 2 T n_e 8 B of edge indices.
def edge_flop_per_edge():
    return (6 * K + 22) * F


def step_flop_per_atom(n_e):
    return 2 * T * (30 * F * F + n_e * (6 * K + 22) * F) + F * F


def step_bytes_per_atom(n_e, value_bytes):
    return 42 * F * T * value_bytes + 2 * T * n_e * 8


# FMA-pipe FLOPs per (active edge, feature channel) the edge kernels execute on CUDA cores
# (reported beside the roofline): FP32 message 6K + 18, FP32 adjoint 12K + 45; with the filter
# on the tensor pipe (BF16, F = 128, the cutoff and bias folded into the basis so the MMA yields
# the filter and its derivative) the adjoint keeps 35 (the tensor-core message kernel's CUDA-core
# work is per receiver, counted where it is reported).
EDGE_FWD_FLOP_PER_EF = 6 * K + 18
EDGE_BWD_FLOP_PER_EF = 12 * K + 45
EDGE_BWD_TC_ALU_FLOP_PER_EF = 35
FP32_LANES_PER_SM, N_SM = 128, 152


def workload_desc(cells):
    n = 4 * cells ** 3
    return (f"fcc {cells}x{cells}x{cells} cells ({n:,} atoms), a=4.05 A, jitter 0.05 A, 1 species; "
            f"PaiNN F={F}, T={T}, K={K} Gaussians, rc={RC} A, skin={SKIN} A; NVE velocity Verlet "
            f"dt={DT} fs from {TEMP:.0f} K")


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


def kernel_traffic(name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(name)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2506_04055_gb300", "csrc", rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return rec.get("bytes_per_launch") if h == rec.get("source_sha") else None


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_eval(job):
    """One oracle E+F+W evaluation of an fcc sub-cell (run in a spawned worker process);
    returns (atoms, wall-clock start, wall-clock end)."""
    cells, reps = job
    import oracle
    import synthetic as syn
    sy = syn.fcc(cells, cells, cells, a=4.05, jitter=0.05, seed=0)
    vals = syn.xavier_params(F, K, T, S, seed=0)
    t0 = time.time()
    for _ in range(reps):
        oracle.painn(vals, F, K, T, S, sy.species, sy.positions, sy.cell)
    return sy.n * reps, t0, time.time()


def _oracle_all_cores(cells, reps, cores):
    """The oracle as it stands, one single-threaded process per host core, each evaluating the
    same sub-cell `reps` times; throughput = all atoms evaluated / wall span of the evaluations."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_eval, [(cells, reps)] * cores)
    atoms = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    per_core = min(r[2] - r[1] for r in res)
    return atoms / span, span, res[0][0] / per_core


def cpu_baseline():
    """The FP64 oracle as it stands: one E+F+W evaluation (its own linked-cell pair search
    included) of the 4,000-atom 10x10x10 fcc sub-cell per host core, all cores at once."""
    cores = _host_cores()
    value, span, single = _oracle_all_cores(10, 1, cores)
    return {"value": value, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
            "single_core": single,
            "sample": f"one E+F+W evaluation of the 4000-atom 10x10x10 fcc sub-cell (F=128, T=3) in each of "
                      f"{cores} single-threaded processes, one per host core ({span:.1f} s wall), pair search "
                      f"included, no integration"}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same metric; each step is one round in
    which every host core evaluates E+F+W of the 500-atom 5x5x5 fcc sub-cell of the same crystal
    and model (one single-threaded oracle process per core)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = _host_cores()
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_eval, [(5, 1)] * cores)
        times, atoms = [], 0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            res = pool.map(_oracle_eval, [(5, 1)] * cores)
            times.append(time.perf_counter() - t0)
            atoms += sum(r[0] for r in res)
    total = sum(times)
    value = atoms / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "atom-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(FCC_CELLS),
                       "sample": f"5x5x5 fcc sub-cell (500 atoms) per host core per step, {cores} cores",
                       "parallelism": f"{cores} single-threaded oracle processes on the host cores"},
            "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"E+F+W of the 500-atom 5x5x5 fcc sub-cell on each of {cores} cores per "
                                       f"step, {args.steps} steps"},
            "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself without a process group): every rank's
    timed region ends at the slowest rank, so whole-job throughput uses the maximum time."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, world, steps, max_ms):
    """Aggregate throughput of `world` ranks that each processed units_per_rank units per step
    for `steps` steps, over the slowest rank's time (ms): units/s for the whole job."""
    return units_per_rank * world * steps / (max_ms / 1e3)


def run_ours(args):
    import torch

    import paper_2506_04055_gb300 as eng
    import synthetic as syn

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        eng.build()
    if dist:
        dist.barrier()
    eng.load()

    cells = args.cells
    sy = syn.fcc(cells, cells, cells, a=4.05, jitter=0.05, seed=rank)
    v0 = syn.maxwell_boltzmann(sy.masses, TEMP, seed=rank)
    blob = syn.params_blob(F, K, T, S, rc=RC, seed=0)
    stream = torch.cuda.current_stream()
    results = {}
    precisions = ["fp32"] if args.precision == "fp32" else (["bf16"] if args.precision == "bf16" else ["fp32", "bf16"])
    for prec in precisions:
        try:
            pot = eng.Potential(F, K=K, T=T, n_species=S, rc=RC, precision=prec, params=blob,
                                stream=stream.cuda_stream)
        except eng.CtdError as e:
            results[prec] = {"error": str(e)}
            continue
        from paper_2506_04055_gb300 import _lib as L
        if args.tc_adjoint is not None and prec == "bf16":
            pot.set_option(L.CTD_OPT_TC_ADJOINT, args.tc_adjoint)
        if args.tc_message is not None and prec == "bf16":
            pot.set_option(L.CTD_OPT_TC_MESSAGE, args.tc_message)
        if args.chunk_rows is not None:
            pot.set_option(L.CTD_OPT_EDGE_CHUNK_ROWS, args.chunk_rows)
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=SKIN)
        for _ in range(args.warmup):
            pot.md_run(1, DT)
        torch.cuda.synchronize()
        pot.profile(True)
        pot.profile_read(reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        rebuilds = 0
        with ClockSampler(local) as clk:
            t_start = torch.cuda.Event(enable_timing=True)
            t_end = torch.cuda.Event(enable_timing=True)
            t_start.record(stream)
            for k in range(args.steps):
                ev[k][0].record(stream)
                _, _, nreb = pot.md_run(1, DT)
                rebuilds += nreb
                ev[k][1].record(stream)
            t_end.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        total_ms = t_start.elapsed_time(t_end)
        step_ms = sorted(a.elapsed_time(b) for a, b in ev)
        prof = pot.profile_read(reset=True)
        pot.profile(False)
        ep, ek, _ = pot.md_run(0, DT)
        # e2e: the public C-ABI call with host (pinned) buffers, copies inside the timed region
        n = sy.n
        x_pin = torch.from_numpy(sy.positions.copy()).pin_memory()
        z_pin = torch.from_numpy(sy.species.copy()).pin_memory()
        f_pin = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        e_pin = torch.empty(1, dtype=torch.float64).pin_memory()
        w_pin = torch.empty(9, dtype=torch.float64).pin_memory()
        H = np.ascontiguousarray(sy.cell)
        import ctypes
        from paper_2506_04055_gb300 import _lib
        flags = _lib.CTD_NEED_FORCES | _lib.CTD_NEED_VIRIAL
        P = lambda t: ctypes.c_void_p(t.data_ptr())
        for _ in range(max(1, args.warmup // 2)):
            _lib.ctd_compute(pot.ctx, n, P(z_pin), P(x_pin), H.ctypes.data_as(ctypes.c_void_p), flags,
                             P(e_pin), P(f_pin), P(w_pin))
        e2e_steps = max(3, args.steps // 2)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            _lib.ctd_compute(pot.ctx, n, P(z_pin), P(x_pin), H.ctypes.data_as(ctypes.c_void_p), flags,
                             P(e_pin), P(f_pin), P(w_pin))
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if dist:
            dist.barrier()
        # device memory the context holds for this system (all buffers, after the runs above)
        mst = pot.compute(sy.species, sy.positions, sy.cell, stats=True)["stats"]
        held, in_use = mst["bytes_allocated"], mst["bytes_in_use"]
        pot.close()
        results[prec] = {"total_ms": total_ms, "step_ms": step_ms, "prof": prof, "rebuilds": rebuilds,
                         "device_bytes_per_atom": held / sy.n, "device_bytes_in_use_per_atom": in_use / sy.n,
                         "clocks": clk.summary(), "e2e_s": e2e_s, "e2e_steps": e2e_steps,
                         "h2d": n * 3 * 8 + n * 4 + 72, "d2h": n * 3 * 8 + 8 + 72,
                         "epot": [float(ep[0])], "ekin": [float(ek[0])]}

    def maxall(x):
        return max_over_ranks(x, dist, "cuda")

    head = "bf16" if "bf16" in results and "error" not in results["bf16"] else "fp32"
    summary = {}
    for prec, r in results.items():
        if "error" in r:
            summary[prec] = r
            continue
        tot = maxall(r["total_ms"])
        e2e = maxall(r["e2e_s"])
        summary[prec] = {"value": whole_job_value(sy.n, world, args.steps, tot), "ms_per_step": tot / args.steps,
                         "p50_ms": r["step_ms"][len(r["step_ms"]) // 2],
                         "p99_ms": r["step_ms"][min(len(r["step_ms"]) - 1, int(0.99 * len(r["step_ms"])))],
                         "e2e": whole_job_value(sy.n, world, r["e2e_steps"], 1e3 * e2e), "rebuilds": r["rebuilds"],
                         "device_bytes_per_atom": round(r["device_bytes_per_atom"]),
                         "device_bytes_in_use_per_atom": round(r["device_bytes_in_use_per_atom"])}
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    r = results[head]
    s = summary[head]
    peaks, peak_kind = read_peaks()
    prof = r["prof"]
    # dominant kernel stage by device time in the timed region
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    active_edges_per_launch = r.get("active_edges")
    roofline = None
    # active edges per launch and n_e from the stats of one compute call on the same system
    import paper_2506_04055_gb300 as eng2
    with eng2.Potential(F, K=K, T=T, n_species=S, rc=RC, params=blob) as p2:
        st = p2.compute(sy.species, sy.positions, sy.cell, stats=True)["stats"]
    ea = st["n_active_edges"]
    n_e = ea / sy.n
    if dom in ("edge_bwd", "edge_fwd") and dom_launches:
        launch_s = dom_ms / dom_launches / 1e3
        tc = head == "bf16" and F == 128 and ((dom == "edge_fwd" and args.tc_message != 0) or
                                              (dom == "edge_bwd" and args.tc_adjoint != 0))
        kname = ("k_edge_bwd_tcg" if dom == "edge_bwd" else "k_edge_msg_mma") if tc else f"k_{dom}"
        flop = ea * edge_flop_per_edge()
        achieved = flop / launch_s / 1e12
        if tc:
            # the contraction runs on tcgen05 in BF16: the sustained BF16 peak (timed in a long step)
            peak, bound = peaks.get("bf16_tflops_sustained", 1700.0), "tensor"
            peak_source = f"bf16_tflops_sustained ({peak_kind})"
        else:
            peak = N_SM * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            bound = "alu"
            peak_source = (f"FP32 FMA: {N_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                           f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peak_kind} max clock)")
        traffic = kernel_traffic(kname)
        roofline = {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic, "peak_source": peak_source,
                    "algorithmic_flop_per_launch": flop, "flop_per_active_edge": edge_flop_per_edge(),
                    "launch_ms": dom_ms / dom_launches, "active_edges": ea}
        if traffic:
            roofline["hbm_gbs"] = traffic / launch_s / 1e9
            roofline["hbm_frac"] = traffic / launch_s / 1e9 / peaks.get("hbm_gbs", 6800.0)
        if tc and dom == "edge_fwd":
            # the contraction kernel's CUDA-core work is per receiver: the FP32 filter weights
            # applied to 7 accumulator groups of K + 1 columns, 2 x 7 (K + 1) FLOP per channel
            alu_flop = sy.n * F * 2 * 7 * (K + 1)
        else:
            alu_flop = ea * F * ((EDGE_BWD_TC_ALU_FLOP_PER_EF if tc else EDGE_BWD_FLOP_PER_EF) if dom == "edge_bwd"
                                 else EDGE_FWD_FLOP_PER_EF)
        fma_peak = N_SM * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roofline["fma_pipe"] = {"flop_per_launch": alu_flop, "tflops": alu_flop / launch_s / 1e12,
                                "frac_of_fp32_fma_peak": alu_flop / launch_s / 1e12 / fma_peak}
    # the whole step against both roofs (algorithmic FLOPs and bytes per atom-step)
    step_s = s["ms_per_step"] / 1e3
    vb = 2 if head == "bf16" else 4
    step_flop = sy.n * step_flop_per_atom(n_e)
    step_bytes = sy.n * step_bytes_per_atom(n_e, vb)
    tpk = peaks.get("bf16_tflops_sustained", 1700.0) if head == "bf16" else \
        N_SM * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    step_roof = {"flop": step_flop, "bytes": step_bytes, "tflops": step_flop / step_s / 1e12,
                 "flop_frac": step_flop / step_s / 1e12 / tpk,
                 "gbs": step_bytes / step_s / 1e9, "bytes_frac": step_bytes / step_s / 1e9 / peaks.get("hbm_gbs", 6800.0),
                 "bound_ms": 1e3 * max(step_flop / (tpk * 1e12), step_bytes / (peaks.get("hbm_gbs", 6800.0) * 1e9)),
                 "n_e": n_e}
    if roofline is not None:
        roofline["step"] = step_roof
    launches = int(sum(v[1] for v in prof.values()))
    line = {
        "metric": METRIC, "value": s["value"], "unit": "atom-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": s["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if head == "bf16" else "f32", "data": "synthetic",
        "config": {"workload": workload_desc(cells), "atoms_per_gpu": sy.n,
                   "precision": head, "parallelism": f"replicas x{world} (independent systems)",
                   "l2": "inputs larger than L2 (tens of GB resident per GPU)"},
        "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"], "rebuilds": s["rebuilds"],
        "roofline": roofline,
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": launches,
        "e2e": {"value": s["e2e"], "unit": "atom-steps/s", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "clocks": r["clocks"],
    }
    for prec in summary:
        line[prec] = summary[prec]
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ supplementary workloads
# The default run above is the 1M-atom fcc line.  --workload selects one of the other
# configurations of the method's evaluation (each prints its own JSON line):
#   water192   192-atom water, F=64, T=3: E+F+W call latency, 100-step NVE drift vs the oracle
#   water96k   96,000-atom water, F=64, T=3, skin 1 A: 1,000 NVE steps, p50/p99, drift
#   mixture90k 90,300-atom triclinic 4-species mixture, F=64, T=2: stored vs recomputed edge filters
#   serve      512 replicas (log-uniform 64..20,000 atoms, water / fcc), Poisson arrivals swept
#              around the saturation rate; p50/p99 latency vs serial per-system FP32 launches
#   nvt_al     the paper's aluminium NVT protocol on 1,000,188 atoms: fcc a=4.065 A, 1000 K,
#              dt=3 fs, skin 2 A, Nose-Hoover chain (3 thermostats, tau=1.1 ps), 100 equilibration
#              and 250 production steps; conserved extended energy and mean temperature
#   domains    the 1M-atom fcc system evaluated through a spatial domain decomposition with copied
#              atoms (grids 1x1x1 ... 2x2x2, T-hop pruning on and off) against the periodic system:
#              copies, edges, time, and the parallel efficiency of Results "Parallelization cost"


def _init_engine():
    import torch

    import paper_2506_04055_gb300 as eng
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    eng.build()
    eng.load()
    return eng, torch


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))] if xs else None


def _timed_md(pot, torch, steps, warmup, dt):
    """steps x md_run(1) with CUDA events per step on the context's (torch's) stream; returns
    per-step ms, total ms, energy series (steps + 1), rebuilds, stage profile, clocks."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        pot.md_run(1, dt)
    torch.cuda.synchronize()
    pot.profile(True)
    pot.profile_read(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    ep_s, ek_s, reb = [], [], 0
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(steps):
            ev[k][0].record(stream)
            ep, ek, nreb = pot.md_run(1, dt)
            ev[k][1].record(stream)
            if k == 0:
                ep_s.append(ep[0]); ek_s.append(ek[0])
            ep_s.append(ep[1]); ek_s.append(ek[1])
            reb += nreb
        t1.record(stream)
        torch.cuda.synchronize()
    prof = pot.profile_read(reset=True)
    pot.profile(False)
    return {"step_ms": [a.elapsed_time(b) for a, b in ev], "total_ms": t0.elapsed_time(t1),
            "ep": np.array(ep_s), "ek": np.array(ek_s), "rebuilds": reb,
            "stage_ms_per_step": {k: v[0] / steps for k, v in prof.items()},
            "launches": int(sum(v[1] for v in prof.values())), "clocks": clk.summary()}


def _md_line(metric, n, steps, warmup, r, dtype, config, extra):
    e = r["ep"] + r["ek"]
    line = {"metric": metric, "value": n * steps / (r["total_ms"] / 1e3), "unit": "atom-steps/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": r["total_ms"] / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config,
            "p50_ms": _pct(r["step_ms"], 0.5), "p99_ms": _pct(r["step_ms"], 0.99), "rebuilds": r["rebuilds"],
            "drift_ev_per_atom": float((e[-1] - e[0]) / n), "max_abs_dE_ev_per_atom": float(np.abs(e - e[0]).max() / n),
            "stage_ms_per_step": r["stage_ms_per_step"], "gpu_launches": r["launches"], "clocks": r["clocks"]}
    line.update(extra)
    return line


def run_water192(args):
    """192-atom water (64 H2O, L = 12.42 A), F=64, T=3, 2 species, Xavier weights (seed 0):
    E+F+W call latency through the C ABI with host buffers, and 100 NVE steps at dt 0.5 fs from
    300 K compared with the FP64 oracle's own trajectory."""
    import oracle
    import synthetic as syn
    eng, torch = _init_engine()
    Fw, Tw, Sw, dtw = 64, 3, 2, 0.5
    sy = syn.water_box(64, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=0)
    vals = syn.xavier_params(Fw, K, Tw, Sw, seed=0)
    blob = syn.params_blob(Fw, K, Tw, Sw, rc=RC, values=vals)
    oracle.build()
    t0 = time.perf_counter()
    ref = oracle.painn(vals, Fw, K, Tw, Sw, sy.species, sy.positions, sy.cell)
    t_orc = time.perf_counter() - t0
    _, _, ep_o, ek_o = oracle.nve(vals, Fw, K, Tw, Sw, sy.species, sy.masses, sy.positions, v0, sy.cell, dtw, 100)
    eo = ep_o + ek_o
    out = {}
    for prec in ("fp32", "bf16"):
        with eng.Potential(Fw, K=K, T=Tw, n_species=Sw, rc=RC, precision=prec, params=blob,
                           stream=torch.cuda.current_stream().cuda_stream) as pot:
            for _ in range(max(3, args.warmup)):
                pot.compute(sy.species, sy.positions, sy.cell)
            lat = []
            for _ in range(max(args.steps, 200)):
                t0 = time.perf_counter()
                o = pot.compute(sy.species, sy.positions, sy.cell)
                lat.append((time.perf_counter() - t0) * 1e3)
            fr = float(np.sqrt(((o["forces"] - ref["forces"]) ** 2).sum() / (ref["forces"] ** 2).sum()))
            pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
            r = _timed_md(pot, torch, 100, 0, dtw)
            e = r["ep"] + r["ek"]
            out[prec] = {"call_ms_p50": _pct(lat, 0.5), "call_ms_p99": _pct(lat, 0.99),
                         "calls_per_s": 1e3 / statistics.mean(lat), "rel_force_rmse_vs_oracle": fr,
                         "abs_dE_per_atom_vs_oracle": abs(float(o["energy"]) - ref["energy"]) / sy.n,
                         "nve_100x0.5fs_drift_ev_per_atom": float((e[-1] - e[0]) / sy.n),
                         "nve_max_dev_from_oracle_etot_ev_per_atom": float(np.abs(e - eo).max() / sy.n),
                         "md_ms_per_step": r["total_ms"] / 100}
    line = {"metric": "E+F+W call latency (host buffers) and 100-step NVE drift, 192-atom water",
            "value": out["fp32"]["call_ms_p50"], "unit": "ms/call (p50, FP32)", "n_gpus": 1,
            "steps": max(args.steps, 200), "warmup": max(3, args.warmup), "higher_is_better": False,
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "water 64 H2O (192 atoms), L=12.42 A; PaiNN F=64, T=3, K=20, rc=5 A; "
                                   "NVE dt=0.5 fs, 300 K"},
            "fp32": out["fp32"], "bf16": out["bf16"],
            "oracle_nve_100x0.5fs_drift_ev_per_atom": float((eo[-1] - eo[0]) / sy.n),
            "cpu_baseline": {"value": t_orc * 1e3, "unit": "ms/call", "cores": 1, "kind": "oracle",
                             "sample": "one E+F+W evaluation of the same 192 atoms (single thread)"}}
    print(json.dumps(line), flush=True)


def run_water96k(args):
    """96,000-atom water (32,000 H2O, L = 98.6 A), F=64, T=3, skin 1 A, rebuild at skin/2,
    1,000 velocity-Verlet steps at dt 0.5 fs from 300 K (FP32, then BF16)."""
    import synthetic as syn
    eng, torch = _init_engine()
    Fw, Tw, Sw, dtw = 64, 3, 2, 0.5
    steps = args.steps if args.steps_given else 1000
    sy = syn.water_box(32000, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=0)
    blob = syn.params_blob(Fw, K, Tw, Sw, rc=RC, seed=0)
    res = {}
    for prec in ("fp32", "bf16"):
        with eng.Potential(Fw, K=K, T=Tw, n_species=Sw, rc=RC, precision=prec, params=blob,
                           stream=torch.cuda.current_stream().cuda_stream) as pot:
            pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
            res[prec] = _timed_md(pot, torch, steps, max(3, args.warmup), dtw)
    cfg = {"workload": f"water 32,000 H2O ({sy.n:,} atoms), L={sy.cell[0, 0]:.2f} A; PaiNN F=64, T=3, K=20, "
                       f"rc=5 A, skin=1 A; NVE dt=0.5 fs, 300 K", "precision": "fp32",
           "l2": "inputs larger than L2"}
    line = _md_line("atom-steps/s, 96k-atom water NVE (FP32), p50/p99, energy drift", sy.n, steps, max(3, args.warmup),
                    res["fp32"], "f32", cfg, {})
    b = res["bf16"]
    eb = b["ep"] + b["ek"]
    line["bf16"] = {"value": sy.n * steps / (b["total_ms"] / 1e3), "ms_per_step": b["total_ms"] / steps,
                    "p50_ms": _pct(b["step_ms"], 0.5), "p99_ms": _pct(b["step_ms"], 0.99),
                    "drift_ev_per_atom": float((eb[-1] - eb[0]) / sy.n), "rebuilds": b["rebuilds"]}
    print(json.dumps(line), flush=True)


def _local_cpu_baseline():
    """The local model's FP64 oracle as it stands (PyTorch CPU, its own threads): one E+F+W
    evaluation of a 1,536-atom box of the same water (512 H2O, same density), brute-force pairs
    included."""
    import torch
    import oracle.local as ol
    import synthetic as syn
    sy = syn.water_box(512, seed=0)
    vals = syn.local_xavier_params(64, K, 2, 2, 16, seed=0)
    t0 = time.perf_counter()
    ol.local_model(vals, 64, K, 2, 2, 16, sy.species, sy.positions, sy.cell, rc=RC)
    dt = time.perf_counter() - t0
    return {"value": sy.n / dt, "unit": "atom-steps/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"one E+F+W evaluation of 512 H2O ({sy.n} atoms) at the same density, {dt:.1f} s, "
                      f"brute-force pair search included"}


def run_local96k(args):
    """96,000-atom water (32,000 H2O) with the strictly local equivariant edge model (Allegro
    form, l <= 1): F=64 latent, C=16 channels, L=2 layers; NVE dt 0.5 fs from 300 K.  The BF16
    path (dense edge GEMMs on tcgen05) is the headline, the FP32 path beside it, with the BF16
    forces' relative RMSE against the FP32 path's on the first frame."""
    import synthetic as syn
    eng, torch = _init_engine()
    Fl, Ll, Sl, Cl = 64, 2, 2, 16
    steps = args.steps if args.steps_given else 50
    sy = syn.water_box(args.local_waters, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=0)
    blob = syn.local_params_blob(Fl, K, Ll, Sl, Cl, rc=RC, seed=0)
    res, st, frames = {}, {}, {}
    precs = ("fp32", "bf16") if args.local_precision == "both" else (args.local_precision,)
    for prec in precs:
        with eng.Potential(Fl, K=K, T=Ll, n_species=Sl, rc=RC, params=blob, family="local", channels=Cl,
                           precision=prec, stream=torch.cuda.current_stream().cuda_stream) as pot:
            out = pot.compute(sy.species, sy.positions, sy.cell, stats=True)
            st[prec], frames[prec] = out["stats"], out["forces"]
            pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
            res[prec] = _timed_md(pot, torch, steps, max(3, args.warmup), 0.5)
    if len(precs) == 1:   # one precision only (profiling runs): its own line
        r = res[precs[0]]
        cfg = {"workload": f"water {args.local_waters:,} H2O ({sy.n:,} atoms); strictly local edge model F=64, C=16, L=2",
               "precision": precs[0], "active_edges": st[precs[0]]["n_active_edges"]}
        print(json.dumps(_md_line("atom-steps/s, 96k-atom water NVE, strictly local model", sy.n, steps,
                                  max(3, args.warmup), r, "bf16" if precs[0] == "bf16" else "f32", cfg, {})),
              flush=True)
        return
    d = frames["bf16"] - frames["fp32"]
    f_rmse = float(np.sqrt((d ** 2).sum() / (frames["fp32"] ** 2).sum()))
    cfg = {"workload": f"water {args.local_waters:,} H2O ({sy.n:,} atoms), L={sy.cell[0, 0]:.2f} A; strictly local edge model "
                       f"F=64, C=16, L=2, K=20, rc=5 A, skin=1 A; NVE dt=0.5 fs, 300 K",
           "precision": "bf16", "l2": "inputs larger than L2", "active_edges": st["bf16"]["n_active_edges"],
           "bytes_held": st["bf16"]["bytes_allocated"]}
    line = _md_line("atom-steps/s, 96k-atom water NVE, strictly local model (BF16 tensor-core GEMMs vs FP32), p50/p99",
                    sy.n, steps, max(3, args.warmup), res["bf16"], "bf16", cfg, {})
    r = res["fp32"]
    line["fp32"] = {"value": sy.n * steps / (r["total_ms"] / 1e3), "ms_per_step": r["total_ms"] / steps,
                    "p50_ms": _pct(r["step_ms"], 0.5), "p99_ms": _pct(r["step_ms"], 0.99),
                    "stage_ms_per_step": r["stage_ms_per_step"], "bytes_held": st["fp32"]["bytes_allocated"]}
    line["bf16_vs_fp32_force_rmse"] = f_rmse
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _local_cpu_baseline()
    print(json.dumps(line), flush=True)


def run_mixture90k(args):
    """Triclinic 4-species mixture (300-atom chain in 30,000 triatomics, 90,300 atoms), F=64,
    T=2: NVE steps with the adjoint recomputing the edge filters versus reading them stored."""
    import synthetic as syn
    eng, torch = _init_engine()
    from paper_2506_04055_gb300 import _lib as L
    Fm, Tm, Sm = 64, 2, 4
    steps = args.steps if args.steps_given else 100
    sy = syn.mixture(n_chain=300, n_water=30000, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, 300.0, seed=0)
    blob = syn.params_blob(Fm, K, Tm, Sm, rc=RC, seed=0)
    res, held, stored = {}, {}, {}
    for mode in ("recompute", "store"):
        with eng.Potential(Fm, K=K, T=Tm, n_species=Sm, rc=RC, precision="fp32", params=blob,
                           stream=torch.cuda.current_stream().cuda_stream) as pot:
            pot.set_option(L.CTD_OPT_EDGE_STORE, 1 if mode == "store" else 0)
            st = pot.compute(sy.species, sy.positions, sy.cell, stats=True)["stats"]
            held[mode], stored[mode] = st["bytes_allocated"], st["edges_stored"]
            pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=1.0)
            res[mode] = _timed_md(pot, torch, steps, max(3, args.warmup), 0.5)
    cfg = {"workload": f"mixture: 300-atom chain in 30,000 triatomics ({sy.n:,} atoms), triclinic tilts <= 10%, "
                       f"4 species; PaiNN F=64, T=2, K=20, rc=5 A, skin=1 A; NVE dt=0.5 fs, 300 K",
           "precision": "fp32", "l2": "inputs larger than L2"}
    r = res["recompute"]
    line = _md_line("atom-steps/s, 90k-atom mixture, recomputed vs stored edge filters", sy.n, steps,
                    max(3, args.warmup), r, "f32", cfg, {})
    s_ = res["store"]
    line["store"] = {"value": sy.n * steps / (s_["total_ms"] / 1e3), "ms_per_step": s_["total_ms"] / steps,
                     "p50_ms": _pct(s_["step_ms"], 0.5), "p99_ms": _pct(s_["step_ms"], 0.99),
                     "stage_ms_per_step": s_["stage_ms_per_step"], "bytes_held": held["store"],
                     "edges_stored": stored["store"]}
    line["recompute"] = {"bytes_held": held["recompute"], "edges_stored": stored["recompute"]}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Continuous-batching server: R replicas (atom counts log-uniform in [64, 20,000], water and
    fcc alternating), each S steps; closed loop (all at t=0) to find the saturation rate, then
    Poisson arrivals at 0.1, 0.5, 1 and 2 times it.  Baseline: the same replicas one after
    another through the single-system FP32 MD loop (a subset, scaled)."""
    import synthetic as syn
    eng, torch = _init_engine()
    Fs, Ts, Ss = 64, 3, 2
    R, S_ = args.replicas, args.serve_steps
    dts = 0.5
    sizes = syn.request_sizes(R, seed=0)
    reps = []
    for k, nt in enumerate(sizes):
        sy = syn.system_near(int(nt), "water" if k % 2 == 0 else "fcc", seed=k)
        reps.append((sy, syn.maxwell_boltzmann(sy.masses, 300.0, seed=1000 + k)))
    natoms = np.array([sy.n for sy, _ in reps])
    blob = syn.params_blob(Fs, K, Ts, Ss, rc=RC, seed=0)
    stream = torch.cuda.current_stream()
    budget = int(args.serve_budget_gib * (1 << 30))

    def session(rate, precision):
        srv = eng.Server(Fs, blob, K=K, T=Ts, n_species=Ss, rc=RC, precision=precision, dt=dts,
                         hbm_budget_bytes=budget, max_replicas=R, stream=stream.cuda_stream)
        rng = np.random.Generator(np.random.PCG64(7))
        arrive = np.zeros(R) if rate is None else np.cumsum(rng.exponential(1.0 / rate, size=R))
        sub_t, fin_t, lat, res_atoms = [], [], [], []
        nsub = nfin = 0
        t0 = time.perf_counter()
        while nfin < R:
            now = time.perf_counter() - t0
            while nsub < R and arrive[nsub] <= now:
                sy, v = reps[nsub]
                srv.submit(sy.species, sy.masses, sy.positions, v, sy.cell, S_, skin=1.0)
                sub_t.append(now)
                nsub += 1
            st = srv.stats()
            if st["resident_replicas"] == 0 and st["queued"] == 0 and nsub < R:
                time.sleep(max(0.0, min(0.01, arrive[nsub] - now)))
                continue
            a = time.perf_counter()
            _, _, nf = srv.step()
            stream.synchronize()
            b = time.perf_counter()
            lat.append((b - a) * 1e3)
            res_atoms.append(st["resident_atoms"])
            for _ in range(nf):
                fin_t.append(b - t0)
            nfin += nf
        wall = time.perf_counter() - t0
        gstats = srv.graph_stats()
        srv.close()
        req = np.array(fin_t) - np.array(sub_t)
        busy = sum(lat) / 1e3
        return {"rate_per_s": rate, "wall_s": wall, "atom_steps_per_s": float(natoms.sum()) * S_ / wall,
                "atom_steps_per_busy_s": float(natoms.sum()) * S_ / busy,
                "step_ms_p50": _pct(lat, 0.5), "step_ms_p99": _pct(lat, 0.99), "server_steps": len(lat),
                "request_s_p50": float(np.percentile(req, 50)), "request_s_p99": float(np.percentile(req, 99)),
                "mean_resident_atoms": float(np.mean(res_atoms)),
                # steps whose device work after the rebuild decisions ran as one CUDA-graph launch
                "graph_steps": gstats["graph_steps"], "eager_steps": gstats["eager_steps"],
                "kernels_per_graph_launch": gstats["kernels_per_replay"]}

    # warm-up session (kernels, allocations)
    session(None, args.serve_precision)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        sat = session(None, args.serve_precision)
        rate_sat = R / sat["wall_s"]
        sweep = [session(f * rate_sat, args.serve_precision) for f in (0.1, 0.5, 1.0, 2.0)]
    # serial baseline: single-system FP32 MD loop, replicas one after another (first few)
    nser = min(R, args.serial_replicas)
    with eng.Potential(Fs, K=K, T=Ts, n_species=Ss, rc=RC, precision="fp32", params=blob,
                       stream=stream.cuda_stream) as pot:
        sy, v = reps[0]
        pot.md_set_state(sy.species, sy.masses, sy.positions, v, sy.cell, skin=1.0)
        pot.md_run(S_, dts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(nser):
            sy, v = reps[k]
            pot.md_set_state(sy.species, sy.masses, sy.positions, v, sy.cell, skin=1.0)
            pot.md_run(S_, dts)
        torch.cuda.synchronize()
        ser_s = time.perf_counter() - t0
    serial = float(natoms[:nser].sum()) * S_ / ser_s
    line = {"metric": "serving: aggregate atom-steps/s at saturation, p50/p99 step and request latency vs arrival rate",
            "value": sat["atom_steps_per_s"], "unit": "atom-steps/s", "n_gpus": 1, "steps": S_, "warmup": 1,
            "ms_per_step": sat["step_ms_p50"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.serve_precision == "bf16" else "f32", "data": "synthetic",
            "config": {"workload": f"{R} MD replicas, atoms log-uniform in [64, 20000] (water / fcc alternating, "
                                   f"{int(natoms.sum()):,} atoms in all, mean {natoms.mean():.0f}); PaiNN F=64, "
                                   f"T=3, K=20, rc=5 A, skin 1 A; {S_} NVE steps each at dt 0.5 fs; HBM budget "
                                   f"{args.serve_budget_gib} GiB", "precision": args.serve_precision},
            "saturation": sat, "saturation_rate_per_s": rate_sat, "sweep": sweep,
            "serial_fp32": {"value": serial, "unit": "atom-steps/s", "replicas": nser,
                            "sample": f"first {nser} replicas, set_state + {S_} steps each, one after another"},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_domains(args):
    """E+F+W of the 1M-atom fcc system through ctd_domains_compute for several domain grids,
    next to the periodic single-system call on the same positions (no neighbour rebuild inside
    the timed calls).  For each grid: owned atoms + copies, copies before T-hop pruning, active
    edges, ms per call, and the parallel efficiency eps = S / P with
    S = prod_a (L_a + 2 T R) / (L_a / p_a + 2 T R) (the paper's speed-up estimate for P domains,
    R = rc) beside the measured eps = t(1x1x1 with copies) / t(grid) (all domains of a grid run
    on this one GPU, so the grid's time is the work P processors would share)."""
    import synthetic as syn
    eng, torch = _init_engine()
    prec = "fp32" if args.precision == "fp32" else "bf16"
    n_cells = args.cells
    sy = syn.fcc(n_cells, n_cells, n_cells, seed=0)
    n = sy.n
    blob = syn.params_blob(F, K, T, 1, rc=RC, seed=0)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    x = torch.tensor(sy.positions, device=dev)
    z = torch.tensor(sy.species, device=dev, dtype=torch.int32)
    reps = args.steps if args.steps_given else 5
    warm = max(3, args.warmup)

    def timed(obj):
        for _ in range(warm):
            out = obj.compute(z, x, sy.cell, stats=True)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = obj.compute(z, x, sy.cell, stats=True)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        assert out["stats"]["rebuilt"] == 0
        return out, float(np.median(ms))

    L = [float(np.linalg.norm(sy.cell[a])) for a in range(3)]
    TR = T * RC
    rows = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        with eng.Potential(F, K=K, T=T, n_species=1, rc=RC, precision=prec, params=blob,
                           stream=stream.cuda_stream) as pot:
            ref, t_ref = timed(pot)
            f_ref = ref["forces"].double()
            e_ref = float(ref["energy"].cpu()[0])
            ref_edges = ref["stats"]["n_active_edges"]
        for grid in [(1, 1, 1), (2, 1, 1), (2, 2, 1), (2, 2, 2)]:
            for hop in ([True, False] if grid == (2, 2, 2) else [True]):
                with eng.Domains(F, blob, grid=grid, K=K, T=T, n_species=1, rc=RC, precision=prec, hop_prune=hop,
                                 skin=1.0, stream=stream.cuda_stream) as dom:
                    out, t = timed(dom)
                    info = dom.info()
                    held = out["stats"]["bytes_allocated"]
                P = grid[0] * grid[1] * grid[2]
                S = float(np.prod([(L[a] + 2 * TR) / (L[a] / grid[a] + 2 * TR) for a in range(3)]))
                df = (out["forces"].double() - f_ref)
                rows.append({
                    "grid": list(grid), "hop_prune": hop, "ms": t,
                    "owned_plus_copies": int(sum(d["n_owned"] + d["n_copies"] for d in info)),
                    "copies": int(sum(d["n_copies"] for d in info)),
                    "copies_before_pruning": int(sum(d["n_candidates"] for d in info)),
                    "active_edges": int(sum(d["n_active_edges"] for d in info)),
                    "max_domain_atoms": int(max(d["n_owned"] + d["n_copies"] for d in info)),
                    "bytes_held": int(held),
                    "rel_dE_vs_periodic": abs(float(out["energy"].cpu()[0]) - e_ref) / abs(e_ref),
                    "rel_force_rmse_vs_periodic": float(torch.sqrt((df ** 2).sum() / (f_ref ** 2).sum())),
                    "paper_S": S, "paper_eps": S / P})
    t1 = next(r["ms"] for r in rows if r["grid"] == [1, 1, 1])
    for r in rows:
        r["measured_eps"] = t1 / r["ms"]
        r["work_vs_periodic"] = r["ms"] / t_ref
    best = next(r for r in rows if r["grid"] == [2, 2, 2] and r["hop_prune"])
    line = {"metric": "atom-steps/s of E+F+W through a 2x2x2 domain decomposition (1M fcc), grids and parallel "
                      "efficiency", "value": n / (best["ms"] / 1e3), "unit": "atom-steps/s", "n_gpus": 1,
            "steps": reps, "warmup": warm, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if prec == "bf16" else "f32", "data": "synthetic",
            "config": {"workload": workload_desc(n_cells) + "; E+F+W calls at fixed positions",
                       "precision": prec, "halo": f"R_comm = T rc + skin = {T * RC + 1.0:g} A",
                       "l2": "inputs larger than L2"},
            "periodic": {"ms": t_ref, "atoms": n, "active_edges": int(ref_edges)},
            "grids": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_nvt_al(args):
    """Methods, "MD simulations" (aluminium): NVT with a Nose-Hoover thermostat of damping
    1.1 ps at 1000 K, 3 fs steps, 2.0 A skin, lattice constant 4.065 A, 100 equilibration and 250
    production steps.  The chain length is not stated; 3 thermostats.  Random weights: the
    dynamics is not aluminium's, the cost per step is the method's."""
    import synthetic as syn
    eng, torch = _init_engine()
    prec = "fp32" if args.precision == "fp32" else "bf16"
    n_cells = args.cells
    sy = syn.fcc(n_cells, n_cells, n_cells, a=4.065, seed=0)
    n = sy.n
    blob = syn.params_blob(F, K, T, 1, rc=RC, seed=0)
    v0 = syn.maxwell_boltzmann(sy.masses, 1000.0, seed=0)
    equil = 100
    prod = args.steps if args.steps_given else 250
    stream = torch.cuda.current_stream()
    with eng.Potential(F, K=K, T=T, n_species=1, rc=RC, precision=prec, params=blob,
                       stream=stream.cuda_stream) as pot:
        pot.md_set_state(sy.species, sy.masses, sy.positions, v0, sy.cell, skin=2.0)
        pot.md_set_thermostat(1000.0, 1100.0, 3)
        _, _, reb_eq = pot.md_run(equil, 3.0)
        torch.cuda.synchronize()
        pot.profile(True)
        pot.profile_read(reset=True)
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ep, ek, reb = pot.md_run(prod, 3.0)
            b.record(stream)
            torch.cuda.synchronize()
        prof = pot.profile_read(reset=True)
        pot.profile(False)
        ms = a.elapsed_time(b)
        xi, vxi, eth = pot.md_get_thermostat(prod)
    kb = 8.617333262e-5
    temp = 2.0 * ek / ((3 * n - 3) * kb)
    h = ep + ek + eth
    line = {"metric": "atom-steps/s, NVT (Nose-Hoover chain) at the paper's aluminium settings, 1M atoms",
            "value": n * prod / (ms / 1e3), "unit": "atom-steps/s", "n_gpus": 1, "steps": prod, "warmup": equil,
            "ms_per_step": ms / prod, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec == "bf16" else "f32", "data": "synthetic",
            "config": {"workload": f"fcc {n_cells}^3 cells ({n:,} atoms), a=4.065 A, 1000 K Maxwell-Boltzmann start; "
                                   f"PaiNN F={F}, T={T}, K={K}, rc={RC} A, random weights; NVT Nose-Hoover chain "
                                   f"(3 thermostats, tau=1.1 ps), dt=3 fs, skin 2.0 A; {equil} equilibration + "
                                   f"{prod} production steps", "precision": prec, "l2": "inputs larger than L2"},
            "temperature_K": {"mean": float(temp.mean()), "first": float(temp[0]), "last": float(temp[-1]),
                              "min": float(temp.min()), "max": float(temp.max())},
            "conserved_drift_ev_per_atom": float((h[-1] - h[0]) / n),
            "conserved_max_dev_ev_per_atom": float(np.abs(h - h[0]).max() / n),
            "thermostat_xi": xi.tolist(), "thermostat_vxi": vxi.tolist(),
            "rebuilds": {"equilibration": int(reb_eq), "production": int(reb)},
            "stage_ms_per_step": {k: v[0] / prod for k, v in prof.items()},
            "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["fp32", "bf16", "both"])
    ap.add_argument("--cells", type=int, default=FCC_CELLS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tc-adjoint", type=int, default=None,
                    help="BF16 edge adjoint: 0 CUDA cores, 1 tcgen05 filter with FP16 operands (the library's default)")
    ap.add_argument("--tc-message", type=int, default=None,
                    help="BF16 message step: 0 CUDA cores, 1 tensor-core contraction (the library's default)")
    ap.add_argument("--chunk-rows", type=int, default=None,
                    help="rows per block-cyclic chunk of the tensor-core adjoint (0: contiguous)")
    ap.add_argument("--workload", default="fcc1m",
                    choices=["fcc1m", "water192", "water96k", "mixture90k", "serve", "domains", "nvt_al",
                             "local96k"])
    ap.add_argument("--replicas", type=int, default=512)
    ap.add_argument("--serve-steps", type=int, default=20)
    ap.add_argument("--serve-precision", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--local-precision", default="both", choices=["both", "fp32", "bf16"],
                    help="local96k: both precisions (BF16 headline) or one of them")
    ap.add_argument("--local-waters", type=int, default=32000,
                    help="local96k: water molecules in the box (32,000 = 96,000 atoms; fewer for profiling)")
    ap.add_argument("--serve-budget-gib", type=float, default=16.0)
    ap.add_argument("--serial-replicas", type=int, default=64)
    args = ap.parse_args()
    args.steps_given = any(a == "--steps" or a.startswith("--steps=") for a in sys.argv[1:])
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "fcc1m":
        run_ours(args)
    else:
        {"water192": run_water192, "water96k": run_water96k, "mixture90k": run_mixture90k,
         "serve": run_serve, "domains": run_domains, "nvt_al": run_nvt_al, "local96k": run_local96k}[args.workload](args)


if __name__ == "__main__":
    main()
