#!/usr/bin/env python3
"""Throughput benchmark of the fused Lagrangian-LBM step on GB300.

Workload (one "step" = one time step of the whole body: one launch of the
interior kernel and one of the edge-band kernel): a 4096 x 2048-node
plane-strain neo-Hooke body, left edge clamped, other edges traction-free,
initial transverse velocity v_y = v_max x / L, FP32 populations and
arithmetic.

Prints ONE JSON line (rank 0) with MLUPS (million lattice-node updates per
second), the HBM roofline fraction of the interior kernel (the dominant
launch) and of the whole step, the end-to-end number
through the C ABI with host buffers, the CPU oracle as a reported baseline,
and the SM clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own replica of the body
(independent problems, no collective on the data path; weak scaling).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FALLBACK_HBM_GBS = 6800.0
METRIC = "MLUPS and % HBM roofline, plain vs batched/low-precision; p50/p99 solve latency"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--storage", default="f32", choices=["f64", "f32", "f16", "bf16"])
    ap.add_argument("--ucarry", default="lo16", choices=["pair", "lo16", "native"],
                    help="FP32 displacement carry: compensated, its low word in 16 bits (default: 112 B per "
                         "node update, the FP32 parity bounds hold), the compensated FP32 pair (120 B), or "
                         "plain FP32")
    ap.add_argument("--native-ucarry", dest="ucarry", action="store_const", const="native",
                    help="plain FP32 displacement carry (same as --ucarry native)")
    ap.add_argument("--scheme", default="explicit", choices=["explicit", "predictor", "extrapolated"],
                    help="time level of 1S in the moment: Algorithm 1 (explicit), the footnote's "
                         "predictor-corrector, or the extrapolated j of Sec. 5")
    ap.add_argument("--nu", type=float, default=0.25)
    ap.add_argument("--vmax", type=float, default=0.01)
    ap.add_argument("--forms", default="f32c,f32n,f16,bf16",
                    help="extra population formats timed on the same body ('' to skip)")
    ap.add_argument("--form-steps", type=int, default=500)
    ap.add_argument("--schemes", default="predictor,extrapolated",
                    help="other schemes timed on the same body, FP32 + compensated carry ('' to skip)")
    ap.add_argument("--c3-steps", type=int, default=5000,
                    help="steps of the 8192 x 8192 16-bit storage run (0 to skip)")
    ap.add_argument("--hole-steps", type=int, default=500,
                    help="steps of the 4096 x 4096 plate with a hole (0 to skip)")
    ap.add_argument("--batch", type=int, default=256,
                    help="bodies of the batched workload (seeded, sides 64..1024; 0 to skip)")
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--solves", type=int, default=20,
                    help="repeated solves of the C1 and C2 workloads for p50 / p99 latency (0 to skip)")
    ap.add_argument("--serve", type=int, default=120,
                    help="requests of the serving trace replayed at 200/s (0 to skip)")
    ap.add_argument("--serve-window", type=float, default=12.0,
                    help="arrival window (s) of the sub-capacity serving run")
    ap.add_argument("--serve-long", type=int, default=2000,
                    help="requests of the long sub-capacity run (stable materials, steps log-U[50, 2000]; 0 to skip)")
    ap.add_argument("--cpu-steps", type=int, default=0, help="oracle sample steps (0 = auto, ~10-20 s)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the autotuner (library default decomposition)")
    return ap.parse_args()


def workload(a):
    from paper_2208_13769_gb300 import workloads as W

    return W.clamped_body(nx=a.nx, ny=a.ny, mu=0.3, nu=a.nu, vmax=a.vmax)


SCHEME_LABEL = {"explicit": "explicit (Algorithm 1: the time-t source in collision and moment)",
                "predictor": "predictor-corrector (the footnote to Sec. 5)",
                "extrapolated": "extrapolated j (Sec. 5, O(dt^3))"}


def scheme_id(name):
    from paper_2208_13769_gb300 import lbm

    return {"explicit": lbm.LBM_SCHEME_EXPLICIT, "predictor": lbm.LBM_SCHEME_PREDICTOR,
            "extrapolated": lbm.LBM_SCHEME_EXTRAPOLATED}[name]


def algorithmic_bytes(storage):
    """Bytes per node update that must cross HBM (9 populations and 4 carry
    values, each read and written once): FP64 208, FP32 104; 16-bit
    populations with an FP64-wide displacement carry and an FP32 source carry
    84.  A form that moves more (the compensated FP32 carry: 120, with its
    low word in 16 bits: 112) is charged these bytes, not its own."""
    return {"f64": 208, "f32": 104, "f16": 84, "bf16": 84}[storage]


def config_of(a, prob):
    return {
        "workload": f"clamped neo-Hooke body {a.nx}x{a.ny} nodes, FP32 populations/arithmetic",
        "nx": a.nx, "ny": a.ny, "mu": prob.mu, "lambda": prob.lam, "nu": a.nu, "rho0": prob.rho0,
        "omega": prob.omega, "v_max": a.vmax, "edges": "x- clamped (Dirichlet), x+/y-/y+ traction-free",
        "storage": a.storage, "u_carry": UCARRY_LABEL[a.ucarry],
        "scheme": SCHEME_LABEL[a.scheme],
        "l2": "no flush: the state (two ping-pong copies, ~1 GB) is 8x the 129 MB L2",
    }


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the interior kernel's sources: the committed DRAM-traffic profile is valid
# while these are unchanged
KERNEL_SOURCES = ("lbm_interior.cu", "lbm_device.cuh", "lbm_pipeline.cuh", "lbm_params.h", "lbm_kernels.h")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2208_13769_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


UCARRY_LABEL = {"pair": "compensated", "lo16": "compensated, 16-bit low word", "native": "native"}


def comp_arg(ucarry):
    """Body's `compensated` argument for a --ucarry choice."""
    return {"pair": True, "lo16": "lo16", "native": False}[ucarry]


def ncu_traffic(storage, ucarry, nodes):
    """DRAM bytes of one interior launch over `nodes` nodes, from the DRAM
    bytes per node of the committed ncu summary; None if absent or taken on
    other kernel sources."""
    path = os.path.join(ROOT, "profiles", "interior_step_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    key = storage + ({"pair": "c", "lo16": "h"}.get(ucarry, "") if storage == "f32" else "")
    e = d.get("formats", {}).get(key)
    # a format captured at other sources than the file's carries their hash
    if not e or e.get("source_hash", d.get("source_hash")) != kernel_source_hash():
        return None
    return e["dram_bytes_per_node"] * nodes


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, by ctypes) every millisecond from a host thread, so that a
    timed region of a few milliseconds still holds samples.  Reads only."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device):
        import ctypes
        import threading

        self.ct = ctypes
        self.threading = threading
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.handle = ctypes.c_void_p()
        bus = None
        try:
            import torch

            pr = torch.cuda.get_device_properties(device)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
        except Exception:
            bus = None
        rc = 1
        if bus is not None:
            rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(self.handle))
        if rc != 0:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device), ctypes.byref(self.handle))
        if rc != 0:
            raise OSError("no NVML handle for the device")
        self.reason_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        self.max_mhz = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.handle, 1, ctypes.byref(mx)) == 0 \
            and mx.value else None
        self.samples = []
        self.stop_flag = False
        self.thread = None

    def sample(self):
        ct = self.ct
        clk, rs = ct.c_uint(0), ct.c_ulonglong(0)
        if self.lib.nvmlDeviceGetClockInfo(self.handle, 1, ct.byref(clk)) != 0:  # NVML_CLOCK_SM
            return
        if self.reason_fn(self.handle, ct.byref(rs)) != 0:
            return
        self.samples.append((float(clk.value), int(rs.value)))

    def start(self):
        def run():
            while not self.stop_flag:
                self.sample()
                time.sleep(0.001)

        self.sample()
        self.thread = self.threading.Thread(target=run, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag = True
        if self.thread is not None:
            self.thread.join(timeout=5)
        self.sample()
        if not self.samples:
            return None
        reasons = sorted({nm for _, r in self.samples for bit, nm in self.REASONS.items() if r & bit})
        sm = [c for c, _ in self.samples]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz or max(sm), "reasons": reasons,
                "samples": len(sm), "source": "NVML, every 1 ms during the timed region"}


def clock_sampler(device):
    """NVML where the driver's library loads, else nvidia-smi."""
    try:
        return NvmlClockSampler(device)
    except Exception:
        return ClockSampler(device)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        try:
            os.unlink(self.file.name)
        except OSError:
            pass
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle (CPU)

ORACLE_SCHEME = {"explicit": "EXPLICIT", "predictor": "PREDICTOR", "extrapolated": "EXTRAPOLATED"}


def oracle_solver(prob, scheme):
    """The FP64 CPU oracle on prob with the benchmark's scheme."""
    import oracle

    return oracle.solver_from(prob, getattr(oracle, ORACLE_SCHEME[scheme]))


def oracle_sample(prob, steps, scheme="explicit", solver=None):
    """Times the FP64 CPU oracle as it stands on `steps` steps of prob: on
    `solver`, which goes on from its current state, or on a new one."""
    import oracle

    s = solver if solver is not None else oracle_solver(prob, scheme)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    if solver is None:
        s.close()
    return prob.nodes * steps / dt / 1e6, dt, oracle.threads()


def oracle_single_thread(a, steps):
    """The oracle on one core: the reference arm in a child process with
    OMP_NUM_THREADS=1 (the OpenMP runtime reads it at start-up), on `steps`
    steps of the same body."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--cpu-steps", str(steps), "--nx", str(a.nx), "--ny", str(a.ny), "--nu", str(a.nu),
           "--vmax", str(a.vmax), "--scheme", a.scheme]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600, check=True)
        line = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": line["value"], "unit": "MLUPS", "cores": line["cpu_baseline"]["cores"],
                "sample": line["cpu_baseline"]["sample"]}
    except Exception as exc:  # reported, not fatal: the all-core figure stands
        return {"value": None, "error": str(exc)[:200]}


def auto_cpu_steps(prob, budget_s=12.0, scheme="explicit", solver=None):
    mlups, dt, _ = oracle_sample(prob, 1, scheme, solver)
    per = prob.nodes / (mlups * 1e6)
    return max(1, min(200, int(budget_s / max(per, 1e-9))))


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob = workload(a)
    # one oracle body, timed over W untimed and then K timed samples of the
    # same number of time steps, the whole run held to about two minutes of
    # oracle time (the body stays well inside its stable horizon)
    k = max(1, a.steps)
    warm = max(0, a.warmup)
    solver = oracle_solver(prob, a.scheme)
    steps = a.cpu_steps or auto_cpu_steps(prob, min(12.0, max(0.5, 120.0 / (k + warm))), a.scheme, solver)
    vals = []
    for _ in range(warm):
        oracle_sample(prob, steps, a.scheme, solver)
    t_all = 0.0
    cores = 1
    for _ in range(k):
        v, dt, cores = oracle_sample(prob, steps, a.scheme, solver)
        vals.append(v)
        t_all += dt
    solver.close()
    value = statistics.median(vals)
    sample = f"{steps} time steps of the full {a.nx}x{a.ny} body per timed repetition, {len(vals)} repetitions"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": a.gpus,
        "steps": k, "warmup": warm, "ms_per_step": 1e3 * prob.nodes / (value * 1e6),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(a, prob),
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- ranks

class Ranks:
    """One process per GPU under torchrun (RANK / WORLD_SIZE / LOCAL_RANK /
    MASTER_* from the environment): barrier and max over ranks.  Each rank
    advances its own replica of the workload (independent bodies), so no
    collective touches the solver's data; these reductions serve the timing
    only.  backend "nccl" on GPUs, "gloo" on host cores (tests)."""

    def __init__(self, backend: str = "nccl"):
        import torch

        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.dist = None
        self.device = "cpu"
        if backend == "nccl":
            torch.cuda.set_device(self.local)
            self.device = "cuda"
        if self.world > 1:
            import torch.distributed as dist

            if backend == "nccl":
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        import torch

        if self.dist is not None:
            self.dist.barrier()
        if self.device == "cuda":
            torch.cuda.synchronize()

    def max(self, x: float) -> float:
        import torch

        if self.dist is None:
            return float(x)
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def weak_scaling_value(world: int, units_per_rank: float, steps: int, max_secs: float) -> float:
    """Whole-job throughput in millions of units per second: every rank
    advanced units_per_rank units `steps` times; the job took the slowest
    rank's time."""
    return world * units_per_rank * steps / max_secs / 1e6


# ---------------------------------------------------------------- native (GPU)

def time_steps(body, stream, steps):
    """Seconds of body.step(steps) (anything with a step(n) method), by CUDA
    events on the stream the library launches on."""
    import torch

    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    body.step(steps)
    end.record(stream)
    end.synchronize()
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3


def run_native(a):
    import torch

    from paper_2208_13769_gb300 import lbm

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    ranks = Ranks("nccl")
    rank, world, local = ranks.rank, ranks.world, ranks.local
    if world > 1:  # the extra sections run on single-GPU invocations only
        a.forms, a.schemes, a.batch, a.serve, a.solves = "", "", 0, 0, 0

    def barrier():
        ranks.barrier()

    def max_over_ranks(x):
        return ranks.max(x)

    prob = workload(a)
    nodes = prob.nodes
    stream = torch.cuda.Stream()
    # the library's autotuner picks the interior decomposition for this body
    # shape (timed on scratch contexts; it never changes the results)
    tuning, tuning_info = None, None
    if a.tune:
        d = lbm.lbm_desc()
        d.nx, d.ny, d.dX = prob.nx, prob.ny, prob.dX
        d.storage = lbm.STORAGE[a.storage]
        d.u_carry = lbm.ucarry_of(comp_arg(a.ucarry))
        d.scheme = scheme_id(a.scheme)
        d.cuda_stream = stream.cuda_stream
        d.device = local
        t0 = time.perf_counter()
        tuning, tms = lbm.lbm_autotune(d, [e.kind for e in prob.edges], 129)
        tuning_info = dict(tuning.as_dict(), candidate_ms_per_step=tms, seconds=time.perf_counter() - t0)
    body = lbm.Body(prob, storage=a.storage, compensated=comp_arg(a.ucarry), scheme=scheme_id(a.scheme),
                    stream=stream.cuda_stream, device=local, tuning=tuning)
    _, moved_per_node = lbm.lbm_memory_info(body.ctx)
    bytes_per_node = algorithmic_bytes(a.storage)
    body.step(a.warmup)
    body.read(lbm.LBM_FIELD_U, allow_unstable=True)
    clocks = clock_sampler(local)
    barrier()
    clocks.start()
    secs = time_steps(body, stream, a.steps)
    clk = clocks.stop()
    barrier()
    secs = max_over_ranks(secs)
    # the dominant kernel's duration: 200 interior launches back to back
    # between CUDA events on the library's stream (the state is saved and
    # restored around them); and each of a step's two launches timed by
    # events around it (the shares of the step)
    # a body under the size-based plan's threshold runs as edge tiles only:
    # its roofline is the edge kernel's
    has_interior = lbm.lbm_get_tuning(body.ctx).plan == 2
    iprof = lbm.lbm_profile_interior(body.ctx, 200, allow_unstable=True)[1] if has_interior else None
    _, prof = lbm.lbm_profile_steps(body.ctx, min(a.steps, 300), allow_unstable=True)
    status = body.read(lbm.LBM_FIELD_U, allow_unstable=True)["status"]
    body.close()

    ms_per_step = 1e3 * secs / a.steps
    value = weak_scaling_value(world, nodes, a.steps, secs)
    peak, peak_kind = measured_peak()
    interior_step_ms, band_ms, serial_ms, interior_nodes = (float(x) for x in prof)
    step_gbs = bytes_per_node * nodes / (secs / a.steps) / 1e9
    if has_interior:
        interior_ms = float(iprof[0])
        achieved = bytes_per_node * interior_nodes / (interior_ms * 1e-3) / 1e9
        traffic = ncu_traffic(a.storage, a.ucarry, interior_nodes)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": "interior_step_kernel",
                "algorithmic_bytes_per_node": bytes_per_node, "units_per_launch": interior_nodes,
                "moved_bytes_per_node": moved_per_node,
                "frac_at_moved_bytes": moved_per_node * interior_nodes / (interior_ms * 1e-3) / 1e9 / peak,
                "launch_ms": interior_ms,
                "launch_timing": "200 launches back to back between CUDA events on the library's stream",
                "launch_ms_in_step": interior_step_ms,
                "step": {"achieved": step_gbs, "frac": step_gbs / peak,
                         "note": "whole time step (interior + edge-band launch) at the same bytes per node"},
                "edge_band_kernel": {"launch_ms": band_ms, "nodes": nodes - interior_nodes}}
    else:
        achieved = bytes_per_node * nodes / (band_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_kind": peak_kind, "kernel": "edge_tile_kernel",
                "algorithmic_bytes_per_node": bytes_per_node, "units_per_launch": nodes,
                "moved_bytes_per_node": moved_per_node,
                "launch_ms": band_ms,
                "launch_timing": "CUDA events around each launch of lbm_profile_steps (the body runs as edge "
                                 "tiles only: fewer than 2^17 nodes)",
                "step": {"achieved": step_gbs, "frac": step_gbs / peak,
                         "note": "whole time step at the same bytes per node"}}

    # extra population formats on the same body, each with its displacement
    # error against the FP64 path (validated against the oracle) after
    # --form-steps steps
    forms = {}
    ref_u = None
    if a.forms:
        with lbm.Body(prob, storage="f64", scheme=scheme_id(a.scheme), stream=stream.cuda_stream,
                      device=local) as b64:
            b64.step(a.warmup + a.form_steps)
            ref_u = b64.read(lbm.LBM_FIELD_U, allow_unstable=True)["u"]
    for f in [x for x in a.forms.split(",") if x]:
        st, comp = {"f32c": ("f32", True), "f32n": ("f32", False), "f32h": ("f32", "lo16")}.get(f, (f, False))
        b = lbm.Body(prob, storage=st, compensated=comp, scheme=scheme_id(a.scheme), stream=stream.cuda_stream,
                     device=local)
        _, bpn = lbm.lbm_memory_info(b.ctx)
        b.step(a.warmup)
        torch.cuda.synchronize()
        s = time_steps(b, stream, a.form_steps)
        out = b.read(lbm.LBM_FIELD_U, allow_unstable=True)
        ok = out["status"] == lbm.LBM_OK
        uerr = float(np.linalg.norm(out["u"] - ref_u) / np.linalg.norm(ref_u))
        b.close()
        alg = algorithmic_bytes(st)
        ach = alg * nodes / (s / a.form_steps) / 1e9
        forms[f] = {"mlups": nodes * a.form_steps / s / 1e6, "algorithmic_bytes_per_node": alg,
                    "moved_bytes_per_node": bpn, "achieved_gbs": ach, "frac": ach / peak,
                    "frac_at_moved_bytes": bpn * nodes / (s / a.form_steps) / 1e9 / peak,
                    "steps": a.form_steps, "stable": ok, "u_rel_err_vs_f64": uerr}

    # the other time levels of the moment's source (Sec. 5) on the same body,
    # FP32 with the compensated carry, each with its displacement difference
    # from the FP64 predictor path after --form-steps steps (the schemes
    # differ by O(dt^2) in the moment, so this measures how much the choice
    # matters on this workload, not an error)
    schemes = {}
    scheme_ids = {"explicit": lbm.LBM_SCHEME_EXPLICIT, "predictor": lbm.LBM_SCHEME_PREDICTOR,
                  "extrapolated": lbm.LBM_SCHEME_EXTRAPOLATED}
    for name in [x for x in a.schemes.split(",") if x]:
        if ref_u is None:
            with lbm.Body(prob, storage="f64", scheme=scheme_id(a.scheme), stream=stream.cuda_stream,
                          device=local) as b64:
                b64.step(a.warmup + a.form_steps)
                ref_u = b64.read(lbm.LBM_FIELD_U, allow_unstable=True)["u"]
        b = lbm.Body(prob, storage="f32", compensated=True, scheme=scheme_ids[name], stream=stream.cuda_stream,
                     device=local)
        _, bpn = lbm.lbm_memory_info(b.ctx)
        b.step(a.warmup)
        torch.cuda.synchronize()
        s = time_steps(b, stream, a.form_steps)
        out = b.read(lbm.LBM_FIELD_U, allow_unstable=True)
        b.close()
        ach = bpn * nodes / (s / a.form_steps) / 1e9
        schemes[name] = {"mlups": nodes * a.form_steps / s / 1e6, "bytes_per_node_update": bpn,
                         "achieved_gbs": ach, "frac": ach / peak, "steps": a.form_steps,
                         "stable": out["status"] == lbm.LBM_OK,
                         "u_rel_diff_vs_f64_" + a.scheme: float(np.linalg.norm(out["u"] - ref_u)
                                                              / np.linalg.norm(ref_u))}

    # the 8192 x 8192 clamped body with 16-bit population storage, timed, and
    # its displacement error against the FP64 path on the same inputs (the
    # full field and the stride-16 downsample, 512 x 512 points); the FP64
    # path stands in for the oracle, which this size would keep busy for an
    # hour; at the default 5000 steps the body stays inside the method's
    # stable horizon (at the planned 20 000 it does not: the runs report
    # LBM_E_UNSTABLE and the errors are not finite)
    c3 = None
    if a.c3_steps > 0 and world == 1:
        from paper_2208_13769_gb300 import workloads as W

        big = W.clamped_body(nx=8192, ny=8192, mu=0.3, nu=a.nu, vmax=a.vmax)
        with lbm.Body(big, storage="f64", stream=stream.cuda_stream, device=local) as b64:
            b64.step(a.c3_steps)
            u64 = b64.read(lbm.LBM_FIELD_U, allow_unstable=True)["u"]
        c3 = {"workload": f"clamped neo-Hooke body 8192x8192, {a.c3_steps} steps, nu {a.nu}, v_max {a.vmax}",
              "reference": "FP64 GPU path (oracle-validated), same inputs"}
        for st in ("f16", "bf16"):
            b = lbm.Body(big, storage=st, stream=stream.cuda_stream, device=local)
            _, bpn = lbm.lbm_memory_info(b.ctx)
            b.step(a.warmup)
            s = time_steps(b, stream, a.c3_steps - a.warmup)
            out = b.read(lbm.LBM_FIELD_U, allow_unstable=True)
            b.close()
            du = out["u"] - u64
            ds = du[::16, ::16]
            ach = bpn * big.nodes / (s / (a.c3_steps - a.warmup)) / 1e9
            c3[st] = {"mlups": big.nodes * (a.c3_steps - a.warmup) / s / 1e6, "bytes_per_node_update": bpn,
                      "achieved_gbs": ach, "frac": ach / peak, "stable": out["status"] == lbm.LBM_OK,
                      "u_rel_err_vs_f64": float(np.linalg.norm(du) / np.linalg.norm(u64)),
                      "u_rel_err_vs_f64_512x512": float(np.linalg.norm(ds) / np.linalg.norm(u64[::16, ::16]))}
        del u64

    # the plate with a square hole of Sec. 7 (hole 0.4 l, traction along x2 on
    # top and bottom) at 4096 x 4096 nodes: four interior rectangles around
    # the hole and the bands of the edges and of the hole per step
    hole = None
    if a.hole_steps > 0 and world == 1:
        from paper_2208_13769_gb300 import workloads as W

        plate = W.plate_with_hole(4096, T=0.02, t_off=math.inf)
        b = lbm.Body(plate, storage=a.storage, compensated=comp_arg(a.ucarry), stream=stream.cuda_stream, device=local)
        _, pbpn = lbm.lbm_memory_info(b.ctx)
        b.step(a.warmup)
        s = time_steps(b, stream, a.hole_steps)
        st = b.read(lbm.LBM_FIELD_U, allow_unstable=True)["status"]
        b.close()
        ach = pbpn * plate.nodes / (s / a.hole_steps) / 1e9
        hole = {"workload": "plate with a centred square hole (0.4 l), 4096 x 4096 nodes, traction 0.02 mu along x2",
                "nodes": plate.nodes, "steps": a.hole_steps, "mlups": plate.nodes * a.hole_steps / s / 1e6,
                "achieved_gbs": ach, "frac": ach / peak, "stable": st == lbm.LBM_OK}

    # batched workload: many uneven bodies advanced by shared launches, and
    # the same bodies stepped one after another; the footnote's predictor,
    # stable over more of the workload's materials than Algorithm 1's
    # explicit moment (the cost per node is the same)
    batched = None
    if a.batch > 0:
        from paper_2208_13769_gb300 import workloads as W

        spec = W.body_batch(a.batch)
        bnodes = sum(p.nx * p.ny for p in spec.problems)
        pred = lbm.LBM_SCHEME_PREDICTOR
        bodies = [lbm.Body(p, storage=a.storage, compensated=comp_arg(a.ucarry), scheme=pred,
                           stream=stream.cuda_stream, device=local) for p in spec.problems]
        # the batch autotuner picks ring depth and rows per interior tile on
        # scratch copies of the members
        btune, bt_ms, bt_s = None, None, None
        if a.tune:
            t0 = time.perf_counter()
            btune, bt_ms = lbm.lbm_batch_autotune([b.ctx for b in bodies], 128)
            bt_s = time.perf_counter() - t0
        bt = lbm.Batch(bodies, stream=stream.cuda_stream, tuning=btune)
        bt.step(a.warmup)
        bsec = time_steps(bt, stream, a.batch_steps)
        info = bt.info()
        statuses = bt.sync()
        bt.close()

        class _OneByOne:
            @staticmethod
            def step(n):
                for b in bodies:
                    b.step(n)

        osteps = max(2, a.batch_steps // 2)
        osec = time_steps(_OneByOne, stream, osteps)
        for b in bodies:
            b.close()
        # the reduced-storage batched form: the same bodies with FP16
        # populations, the same decomposition
        hbodies = [lbm.Body(p, storage="f16", scheme=pred, stream=stream.cuda_stream, device=local)
                   for p in spec.problems]
        htune, ht_ms = None, None
        if a.tune:  # its own decomposition: the strip grid that suits 2-byte planes differs
            htune, ht_ms = lbm.lbm_batch_autotune([b.ctx for b in hbodies], 128)
        hb = lbm.Batch(hbodies, stream=stream.cuda_stream, tuning=htune)
        hb.step(a.warmup)
        hsec = time_steps(hb, stream, a.batch_steps)
        _, hbpn = lbm.lbm_memory_info(hbodies[0].ctx)
        hb.close()
        for b in hbodies:
            b.close()
        hach = hbpn * bnodes / (hsec / a.batch_steps) / 1e9
        bach = bytes_per_node * bnodes / (bsec / a.batch_steps) / 1e9
        batched = {
            "workload": f"{a.batch} bodies, sides U{{64..1024}}, mu log-U[0.05, 0.4], nu U[0.2, 0.45], "
                        "half periodic / half clamped, seed 20220825",
            "scheme": "the footnote's predictor-corrector",
            "nodes": bnodes, "steps": a.batch_steps, "mlups": bnodes * a.batch_steps / bsec / 1e6,
            "ms_per_step": 1e3 * bsec / a.batch_steps, "achieved_gbs": bach, "frac": bach / peak,
            "one_by_one_mlups": bnodes * osteps / osec / 1e6, "one_by_one_steps": osteps,
            "f16_storage": {"mlups": bnodes * a.batch_steps / hsec / 1e6, "ms_per_step": 1e3 * hsec / a.batch_steps,
                            "bytes_per_node_update": hbpn, "achieved_gbs": hach, "frac": hach / peak,
                            "tuning": (dict(htune.as_dict(), candidate_ms_per_step=ht_ms) if htune is not None
                                       else "library defaults")},
            "interior_ctas": info["interior_ctas"], "edge_ctas": info["edge_ctas"],
            "tuning": (dict(btune.as_dict(), candidate_ms_per_step=bt_ms, seconds=bt_s) if btune is not None
                       else "library defaults"),
            "unstable_members": int(sum(1 for x in statuses if x != lbm.LBM_OK)),
            "note": "members outside the method's stable range (nu > 0.25 with traction-free edges, "
                    "nu > 0.40 periodic) report LBM_E_UNSTABLE; their cost is the same"}

    # serving: Poisson arrivals of uneven requests, continuous batching, FCFS
    # admission under a 150 GB budget; first at the trace's 200 requests/s
    # (far above capacity), then at 0.7 x the capacity that run measured
    serving = None
    if a.serve > 0:
        from paper_2208_13769_gb300 import serve
        from paper_2208_13769_gb300 import workloads as W

        def strip(st):
            return {k: v for k, v in st.items() if k != "records"}

        be = serve.GpuBackend(storage="f16", stream=stream.cuda_stream, device=local)
        trace = W.serving_trace(max_requests=a.serve + 4000)
        over = strip(serve.Server(be, hbm_budget=150e9).run(trace[:a.serve]))
        mean_work = float(np.mean([q.problem.nx * q.problem.ny * q.steps for q in trace[:a.serve]]))
        capacity = over["served_mlups"] * 1e6 / mean_work  # requests per second
        rate = 0.7 * capacity
        nsub = max(4, int(rate * a.serve_window))
        sub_trace = serve.trace_at_rate(trace[a.serve:a.serve + nsub], rate)
        sub = strip(serve.Server(be, hbm_budget=150e9).run(sub_trace))
        serving = {"storage": "f16", "scheme": "the footnote's predictor-corrector", "trace": "Poisson 200/s, sides U{128..2048}, steps log-U[500, 20000], seed 7",
                   "overload": dict(over, rate_per_s=200.0), "capacity_requests_per_s": capacity,
                   "sub_capacity": dict(sub, rate_per_s=rate)}
        # a long sub-capacity run: the literal trace's sizes, arrival process
        # and initial fields, with Poisson ratios drawn where the method is
        # stable (0.25 for clamped bodies, U[0.2, 0.4] for periodic ones) and
        # step counts log-U[50, 2000] (a tenth of the literal trace's, whose
        # 2000 requests would take over 5 minutes of GPU time).  Its shorter
        # solves weigh the per-request host work (body creation, upload,
        # read-back) more, so its capacity is measured on its own mix: its
        # first 300 requests all at once; the run then offers 0.7 x that
        if a.serve_long > 0:
            ltrace = W.serving_trace(rate=200.0, duration=1e9, seed=8, steps_lo=50, steps_hi=2000,
                                     max_requests=a.serve_long, stable_materials=True)
            head = [dataclasses.replace(q, arrival=0.0) for q in ltrace[:300]]
            lover = strip(serve.Server(be, hbm_budget=150e9).run(head))
            hwork = float(np.mean([q.problem.nx * q.problem.ny * q.steps for q in head]))
            lcap = lover["served_mlups"] * 1e6 / hwork
            lrate = 0.7 * lcap
            lrun = strip(serve.Server(be, hbm_budget=150e9).run(serve.trace_at_rate(ltrace, lrate)))
            serving["long_capacity"] = dict(lover, capacity_requests_per_s=lcap,
                                            trace="the long run's first 300 requests, all arriving at t = 0")
            serving["long_sub_capacity"] = dict(
                lrun, rate_per_s=lrate,
                trace="Poisson at 0.7 x its mix's capacity, sides U{128..2048}, steps log-U[50, 2000], Poisson "
                      "ratio 0.25 (clamped) / U[0.2, 0.4] (periodic), seed 8")

    # end to end through the C ABI from host buffers: create (H2D of u0, v0),
    # K steps, read u (D2H)
    # solve latency: a solve creates the body from host arrays, initialises
    # it, runs its steps and reads u back to the host (host clock around
    # all of it); p50 / p99 over repeated solves of the 64 x 64 FP64 shear
    # wave (1000 steps), the benchmark's clamped body in its format (5000
    # steps) and the 256-body batch (2000 steps; its members complete
    # together)
    solves = None
    if a.solves > 0 and world == 1:
        from paper_2208_13769_gb300 import workloads as W

        def one_solve(make, steps):
            t0 = time.perf_counter()
            bodies = make()
            if len(bodies) == 1:
                bodies[0].step(steps)
            else:
                with lbm.Batch(bodies, stream=stream.cuda_stream) as bt:
                    bt.step(steps)
            for b in bodies:
                b.read(lbm.LBM_FIELD_U, allow_unstable=True)
            t1 = time.perf_counter()
            for b in bodies:
                b.close()
            return t1 - t0

        def stats(times, nodes_per_solve, steps):
            times = sorted(times)
            q = lambda f: times[min(len(times) - 1, int(round(f * (len(times) - 1))))]
            return {"solves": len(times), "steps": steps, "p50_s": q(0.5), "p99_s": q(0.99),
                    "mlups_at_p50": nodes_per_solve * steps / q(0.5) / 1e6}

        c1 = W.shear_wave(64, amp=0.01, lam=0.5, mu=0.3)
        c2 = W.clamped_body(a.nx, a.ny, mu=0.3, nu=a.nu, vmax=a.vmax)
        c4 = W.body_batch(256)
        solves = {}
        for name, make, steps, n_solves, nodes_per in (
                ("c1_64x64_f64", lambda: [lbm.Body(c1, storage="f64", scheme=lbm.LBM_SCHEME_PREDICTOR,
                                                   stream=stream.cuda_stream, device=local)],
                 1000, a.solves, 64 * 64),
                ("c2_%dx%d_%s" % (a.nx, a.ny, a.storage),
                 lambda: [lbm.Body(c2, storage=a.storage, compensated=comp_arg(a.ucarry), scheme=scheme_id(a.scheme),
                                   stream=stream.cuda_stream, device=local, tuning=tuning)], 5000, a.solves,
                 a.nx * a.ny),
                ("c4_256_bodies_f32", lambda: [lbm.Body(p, storage="f32", scheme=lbm.LBM_SCHEME_PREDICTOR,
                                                        stream=stream.cuda_stream, device=local)
                                               for p in c4.problems], 2000, max(1, a.solves // 4),
                 sum(p.nx * p.ny for p in c4.problems))):
            one_solve(make, 8)  # warm: kernels loaded, graphs of this shape built once
            solves[name] = stats([one_solve(make, steps) for _ in range(n_solves)], nodes_per, steps)

    e2e = None
    if not a.no_e2e:

        # inputs in pinned host memory before the clock starts; the upload,
        # the whole solve and the read-back of u into pinned memory inside it
        u0_h = torch.empty((prob.ny, prob.nx, 2), dtype=torch.float64, pin_memory=True)
        v0_h = torch.empty((prob.ny, prob.nx, 2), dtype=torch.float64, pin_memory=True)
        u_h = torch.empty((prob.ny, prob.nx, 2), dtype=torch.float64, pin_memory=True)
        u0, v0 = prob.initial()
        u0_h.numpy()[...] = u0
        v0_h.numpy()[...] = v0
        pprob = dataclasses.replace(prob, u0=u0_h.numpy(), v0=v0_h.numpy(), make_initial=None)
        barrier()
        t0 = time.perf_counter()
        b = lbm.Body(pprob, storage=a.storage, compensated=comp_arg(a.ucarry), scheme=scheme_id(a.scheme),
                     stream=stream.cuda_stream, device=local, tuning=tuning)
        b.step(a.steps)
        st, _ = lbm.lbm_read_fields(b.ctx, lbm.LBM_FIELD_U, u_h.numpy().reshape(-1), allow_unstable=True)
        t1 = time.perf_counter()
        b.close()
        e_secs = max_over_ranks(t1 - t0)
        h2d = u0_h.numel() * 8 + v0_h.numel() * 8
        d2h = u_h.numel() * 8
        e2e = {"value": world * nodes * a.steps / e_secs / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / a.steps, "d2h_bytes_per_step": d2h / a.steps,
               "h2d_bytes_total": h2d, "d2h_bytes_total": d2h, "seconds": e_secs,
               "includes": "context creation, u0/v0 upload from pinned memory, initialisation, K steps, "
                           "u read-back into pinned memory"}

    cpu = None
    if rank == 0 and not a.no_cpu:
        steps = a.cpu_steps or auto_cpu_steps(prob, scheme=a.scheme)
        v, dt, cores = oracle_sample(prob, steps, a.scheme)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{steps} time steps of the full {a.nx}x{a.ny} body ({dt:.1f} s, FP64 oracle)",
               "single_thread": oracle_single_thread(a, max(1, steps // max(1, cores)))}

    ranks.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "f16": "f16", "bf16": "bf16"}[a.storage],
        "data": "synthetic", "config": config_of(a, prob), "roofline": roof, "cpu_baseline": cpu,
        "e2e": e2e, "gpu_launches": 2 * a.steps, "clocks": clk,
        # the plain-carry FP32 form (104 bytes moved per node, like the survey's count)
        "plain_carry_f32": ({k: forms["f32n"][k] for k in ("mlups", "frac", "u_rel_err_vs_f64")}
                            if "f32n" in forms else None),
        "forms": forms, "schemes": schemes, "solves": solves, "c3_8192": c3, "plate_hole": hole, "batched": batched,
        "serving": serving, "tuning": tuning_info,
        "status": lbm.status_string(status),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_native(a)


if __name__ == "__main__":
    sys.exit(main())
