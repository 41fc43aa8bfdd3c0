#!/usr/bin/env python3
"""Throughput of the BP1.0 / BP3.5 / BP3.0 hot path on GB300.

One step = one pass of the whole path over the synthetic 32^3 jittered
hex mesh (E = 32768, degree N = 7, lambda = 1):
  geometric factors for BP1.0 (wJ at Gauss points), BP3.5 (7 planes at GLL
  nodes) and BP3.0 (7 planes at Gauss points) from the element vertices,
  then the BP1.0, BP3.5 and BP3.0 matvecs of one field q, BP1.0 and BP3.0
  in one pass that interpolates q to the Gauss points once for both
  (fem_bp1_bp30_apply; the step with separate BP1.0 and BP3.0 launches is
  timed as well and reported beside it).
The degree-N basis (a few KB of tables) is built once before timing.
value = 3 E (N+1)^3 DOFs per step (one field through each operator) / time.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.  Under torchrun every rank runs its own
replica of the workload (the operators are block diagonal: no data-path
collective); rank 0 reports the aggregate over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import fem_synth  # noqa: E402

WORKLOAD = "BP1.0+BP3.5+BP3.0 FP64 with geometric factors, 32x32x32 jittered hex mesh (E=32768), N=7, lambda=1"
METRIC = "GDOF/s (BP1.0+BP3.5+BP3.0 step, FP64, N=7, E=32768)"
KERNELS = ["geofacs_bp35", "geofacs_bp30_bp1", "bp35", "bp1_bp30"]

# Measured DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) per
# element at N = 7, with the sha256 of the kernel source it was taken from;
# a kernel whose source changed since reports traffic null.
NCU_TRAFFIC = {
    # ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on E = 4096:
    # (184.09 + 19.69) MB over 4096 elements, ncu capture of the one-pass kernel at N = 7
    "bp1_bp30": {"N": 7, "bytes_per_elem": 49750, "sha": "63b3cce49d1ad5cd",
                 "files": ["bp30.cu", "bp30_body.cuh", "eo.cuh", "kernels_common.cuh"]},
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d
    return 6800.0, "fallback", {}


# FP64 issue rate of the GB300 SM: 2 FP64 instructions per clock per SM
# (ncu: dfma peak_sustained 2 per SM per cycle; the nominal 1.25 TFLOP/s
# over 152 SMs at 2.07 GHz), an FMA counting 2 flops.
SMS = 152
FP64_INST_PER_CLK_SM = 2


def fp64_peak_tflops(sm_mhz: float) -> float:
    return SMS * FP64_INST_PER_CLK_SM * 2 * sm_mhz * 1e6 / 1e12


def fp64_peak_ginst(sm_mhz: float) -> float:
    return SMS * FP64_INST_PER_CLK_SM * sm_mhz * 1e6 / 1e9


def eo_cost(P: int, Q: int, sig: int):
    """(FP64 instructions, flops) of one even-odd folded line y(P) = A x(Q)
    as the kernels execute it: Q/2 fold pairs (2 adds each), per output pair
    2(Q/2) + Q%2 FMAs and 2 adds, a middle output row of Q/2 (+1) FMAs."""
    hp, hq = P // 2, Q // 2
    fma = hp * (2 * hq + Q % 2) + (P % 2) * (hq + (1 if (Q % 2 and sig > 0) else 0))
    add = 2 * hq + 2 * hp
    return fma + add, 2 * fma + add


def alg_counts(N: int):
    """Per element of each kernel:
    std   -- algorithmic FP64 flops of the direct sum factorisation (every
             multiply-add = 2 flops): BP1.0 4(mn^3+m^2n^2+m^3n)+m^3, BP3.5
             12n^4+18n^3, BP3.0 4(mn^3+m^2n^2+m^3n)+12m^4+18m^3; for the
             geometric factors the flops the kernel executes;
    inst  -- FP64 instructions the kernels execute (even-odd lines);
    bytes -- algorithmic HBM bytes (Table 1 of the paper for the operators;
             24 vertex doubles in and the planes out for the factors)."""
    n, m = N + 1, N + 2
    n3, m3, mm, nn = n ** 3, m ** 3, m * m, n * n
    interp = 2 * (m * n3 + m * m * n * n + m3 * n)
    i_mn, f_mn = eo_cost(m, n, 1)      # interpolation line
    i_nm, f_nm = eo_cost(n, m, 1)      # projection line
    i_dd, f_dd = eo_cost(n, n, -1)     # GLL derivative line
    i_gg, f_gg = eo_cost(m, m, -1)     # Gauss derivative line
    lam_i, lam_f = 2, 3                # wJ q, then one FMA with lambda into the sum
    fma_pts = 2 * (m * n3 + m * m * n * n + m3 * n) + 6 * m ** 4  # direct contractions of the point layout
    inst = {
        "bp30_points": fma_pts + m3 * (9 + 3 + 2),  # (lambda wJ) q as two products
        # one thread per node: 3 derivatives and 3 transposed derivatives of
        # length n per node, the 3x3 product and (lambda wJ) q
        "bp35_points": 6 * n ** 4 + n3 * (9 + 2),
        "bp1": (nn + m * n + mm) * (i_mn + i_nm) + m3,
        "bp35": 6 * nn * i_dd + n3 * (9 + lam_i + 2),
        "bp30": (nn + m * n + mm) * (i_mn + i_nm) + 6 * mm * i_gg + m3 * (9 + lam_i + 2),
        # BP3.0 plus BP1.0's three projections (the interpolation and the
        # wJ scaling are shared)
        "bp1_bp30": (nn + m * n + mm) * (i_mn + 2 * i_nm) + 6 * mm * i_gg + m3 * (9 + lam_i + 2),
        "geofacs_bp30_bp1": 52 * m3 + 27 * mm,
        "geofacs_bp35": 52 * n3 + 27 * nn,
    }
    std = {
        "bp30_points": 2 * interp + 12 * m ** 4 + 18 * m3,
        "bp35_points": 12 * n ** 4 + 18 * n3,
        "bp1": 2 * interp + m3,
        "bp35": 12 * n ** 4 + 18 * n3,
        "bp30": 2 * interp + 12 * m ** 4 + 18 * m3,
        "bp1_bp30": 3 * interp + 12 * m ** 4 + 18 * m3 + m3,
        "geofacs_bp30_bp1": 79 * m3 + 54 * mm,
        "geofacs_bp35": 79 * n3 + 54 * nn,
    }
    byts = {
        "bp30_points": 8 * (2 * n3 + 7 * m3),
        "bp35_points": 8 * (9 * n3),
        "geofacs_bp30_bp1": 8 * (24 + 8 * m3),
        "geofacs_bp35": 8 * (24 + 7 * n3),
        "bp1": 8 * (2 * n3 + m3),
        "bp35": 8 * (9 * n3),
        "bp30": 8 * (2 * n3 + 7 * m3),
        "bp1_bp30": 8 * (3 * n3 + 7 * m3),  # q and the factors once, Mq and Aq
    }
    return std, inst, byts


def smem_counts(N: int, word: int = 8):
    """Shared-memory bytes per element that the operator kernels load and
    store, counted from their phases (the quantity of the paper's
    shared-memory roofline, Section 5):
    BP1.0  2n^3 + 3mn^2 + 4m^2n words (staging, five line phases);
    BP3.5  17n^3 words (staging, three derivative lines, chain rule with the
           mass term, two in-place transposes, final sum);
    BP3.0  2n^3 + 3mn^2 + 4m^2n + 16m^3 words (BP1.0's interpolation and
           projection phases plus the Gauss-point derivative, chain-rule and
           transpose phases);
    BP3.0, point layout: two words per multiply-add (operand and operator
           entry) plus every phase output;
    BP3.5, point layout: likewise, 6 n^4 multiply-adds and 5 n^3 stores
           and loads of whole boxes."""
    n, m = N + 1, N + 2
    # point layout: every multiply-add reads an operand and an operator entry
    # from shared memory; every phase output is stored once
    fma_pts = 2 * (m * n ** 3 + m * m * n * n + m ** 3 * n) + 6 * m ** 4
    outs_pts = n ** 3 + 2 * (m * n * n + m * m * n) + 5 * m ** 3 + n ** 3
    return {
        "bp30_points": word * (2 * fma_pts + outs_pts + m ** 3),
        # one thread per node: operand and operator entry per multiply-add,
        # the staged field, the three products stored and q read for the mass term
        "bp35_points": word * (2 * 6 * n ** 4 + 5 * n ** 3),
        "bp1": word * (2 * n ** 3 + 3 * m * n * n + 4 * m * m * n),
        "bp35": word * 17 * n ** 3,
        "bp30": word * (2 * n ** 3 + 3 * m * n * n + 4 * m * m * n + 16 * m ** 3),
        # plus BP1.0's t-projection (stored, read back) and s-projection
        # (stored, read back)
        "bp1_bp30": word * (2 * n ** 3 + 5 * m * n * n + 6 * m * m * n + 16 * m ** 3),
    }


# Shared-memory bandwidth of the SM: 32 banks x 4 bytes per clock.
SMEM_BYTES_PER_CLK_SM = 128


def smem_peak_gbs(sm_mhz: float) -> float:
    return SMS * SMEM_BYTES_PER_CLK_SM * sm_mhz * 1e6 / 1e9


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during timing."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (a timing reduction only)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def workload_arrays(N: int, E_side: int, rank: int):
    verts = fem_synth.box_mesh(E_side)
    E = verts.shape[0]
    # each rank draws its own field (offset stream), same mesh recipe
    q = fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3, offset=rank * E * (N + 1) ** 3)
    return verts, q


def _src_hash(names) -> str:
    """Hash of the kernel's source files (a name or a list of names under csrc/)."""
    h = hashlib.sha256()
    for name in ([names] if isinstance(names, str) else names):
        with open(os.path.join(ROOT, "paper_1711_00903_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------- CPU oracle

def cpu_model() -> str:
    """The host CPU's architecture and model name, as lscpu reports them."""
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                name = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{platform.machine()}, {name or 'model not reported'}"


def cpu_oracle_rate(N: int, verts, q, lam: float, target_s: float, cores: int):
    """Times the oracle's step (geometric factors + the three operators) on a
    sample of about target_s seconds: a prefix of the elements, or whole-mesh
    passes repeated when one pass is shorter than that.  Returns
    (GDOF/s, elements per pass, passes, seconds, threads)."""
    import oracle
    threads = oracle.set_threads(cores)
    E = verts.shape[0]
    Es = min(64, E)
    t0 = time.perf_counter()
    cpu_oracle_step(N, verts[:Es], q[:Es], lam)
    dt = time.perf_counter() - t0
    Es = int(min(E, max(Es, Es * target_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    cpu_oracle_step(N, verts[:Es], q[:Es], lam)
    dt = time.perf_counter() - t0
    reps = max(1, int(round(target_s / max(dt, 1e-6)))) if Es == E else 1
    for _ in range(reps - 1):
        cpu_oracle_step(N, verts[:Es], q[:Es], lam)
    dt = time.perf_counter() - t0
    return 3 * Es * reps * (N + 1) ** 3 / dt / 1e9, Es, reps, dt, threads


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    N, lam = args.degree, 1.0
    verts, q = workload_arrays(N, 32, 0)
    cores = len(os.sched_getaffinity(0))
    import oracle
    oracle.set_threads(cores)
    # size one step for about 1 s of CPU work so the whole run stays short
    rate, Es, reps, dt, threads = cpu_oracle_rate(N, verts, q, lam, 1.0, cores)
    for _ in range(args.warmup):
        cpu_oracle_step(N, verts[:Es], q[:Es], lam)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_step(N, verts[:Es], q[:Es], lam)
    T = time.perf_counter() - t0
    value = args.steps * 3 * Es * (N + 1) ** 3 / T / 1e9
    sample = f"first {Es} of 32768 elements per step (geometric factors + BP1.0 + BP3.5 + BP3.0, N={N})"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": step_config(32768, N, lam, 1),
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": threads, "kind": "oracle",
                          "sample": sample},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def step_config(E, N, lam, world):
    """The workload description of the step, the same for both arms."""
    return {"workload": WORKLOAD if E == 32768 else f"{WORKLOAD} [profiling size E={E}]",
            "E": E, "N": N, "lambda": lam,
            "mesh": "32^3 unit cube, interior vertices jittered U[-0.1h,0.1h], trilinear",
            "l2": "inputs larger than L2 (no flush)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def cpu_oracle_step(N, v, qq, lam):
    import oracle
    wJ, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    G35, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    G30, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    oracle.bp1(N, wJ, qq)
    oracle.bp35(N, G35, lam, qq)
    oracle.bp30(N, G30, lam, qq)


# ---------------------------------------------------------------- GPU path

def run_ours(args):
    import torch
    import paper_1711_00903_gb300 as fem

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    N, lam = args.degree, 1.0
    n, m = N + 1, N + 2
    verts_h, q_h = workload_arrays(N, args.mesh_side, rank)
    E = verts_h.shape[0]
    b = fem.fem_basis_setup(N)
    stream = torch.cuda.current_stream(device)

    verts = torch.from_numpy(verts_h).to(device)
    q = torch.from_numpy(q_h).to(device)
    wJ = torch.empty(fem.geo_shape(b, 1, E), dtype=torch.float64, device=device)
    G35 = torch.empty(fem.geo_shape(b, 2, E), dtype=torch.float64, device=device)
    G30 = torch.empty(fem.geo_shape(b, 3, E), dtype=torch.float64, device=device)
    o1, o35, o30 = (torch.empty_like(q) for _ in range(3))

    def step(ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        # the factors of the three operators: BP3.5 at the GLL nodes, then
        # BP3.0 and BP1.0's wJ (its seventh plane) at the Gauss points
        mark(0)
        fem.fem_mesh_geofacs_set(b, verts, G35=G35, stream=stream)
        mark(1)
        fem.fem_mesh_geofacs_set(b, verts, wJ=wJ, G30=G30, stream=stream)
        mark(2)
        fem.fem_bp35_apply(b, G35, lam, q, out=o35, stream=stream)
        mark(3)
        fem.fem_bp1_bp30_apply(b, G30, lam, q, out_m=o1, out_a=o30, stream=stream)
        mark(4)

    def step_unfused():
        # the same step with BP1.0 and BP3.0 as separate launches
        fem.fem_mesh_geofacs_set(b, verts, G35=G35, stream=stream)
        fem.fem_mesh_geofacs_set(b, verts, wJ=wJ, G30=G30, stream=stream)
        fem.fem_bp1_apply(b, wJ, q, out=o1, stream=stream)
        fem.fem_bp35_apply(b, G35, lam, q, out=o35, stream=stream)
        fem.fem_bp30_apply(b, G30, lam, q, out=o30, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(len(KERNELS) + 1)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world, device)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(events[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world, device)
    clocks = sampler.stop()
    ms_local = t_start.elapsed_time(t_end)
    ms = reduce_max(ms_local, world, device)
    per_kernel = {name: statistics.fmean(events[k][i].elapsed_time(events[k][i + 1]) for k in range(args.steps))
                  for i, name in enumerate(KERNELS)}

    # the same step with separate BP1.0 and BP3.0 launches, for comparison
    uf_steps = max(3, min(args.steps, 20))
    for _ in range(3):
        step_unfused()
    torch.cuda.synchronize()
    barrier(world, device)
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u0.record(stream)
    for _ in range(uf_steps):
        step_unfused()
    u1.record(stream)
    torch.cuda.synchronize()
    ms_unfused = reduce_max(u0.elapsed_time(u1) / uf_steps, world, device)

    # end to end through the same calls: pinned host input -> device ->
    # step -> host output, every step.  Three streams: the host-to-device
    # copies, the kernels (in order on the step's stream, as in the device
    # step) and the device-to-host copies, over two sets of device buffers,
    # so that step k+1's inputs arrive and step k-1's outputs leave while
    # step k's kernels run; events order each set's reuse.  Every step still
    # copies its inputs in and its three outputs out inside the timed region.
    verts_p = torch.from_numpy(verts_h).pin_memory()
    q_p = torch.from_numpy(q_h).pin_memory()
    e2e_steps = max(4, min(args.steps, 20))
    h2d_s, d2h_s = torch.cuda.Stream(device), torch.cuda.Stream(device)
    sets = []
    for k in range(2):
        d = {"verts": torch.empty_like(verts), "q": torch.empty_like(q),
             "wJ": torch.empty_like(wJ), "G35": torch.empty_like(G35), "G30": torch.empty_like(G30),
             "o": [torch.empty_like(q) for _ in range(3)],
             "out": [torch.empty(q_h.shape, dtype=torch.float64).pin_memory() for _ in range(3)],
             "in_ready": torch.cuda.Event(), "computed": torch.cuda.Event(), "out_done": torch.cuda.Event(),
             "used": False}
        sets.append(d)

    def e2e_step(k):
        d = sets[k % 2]
        if d["used"]:
            h2d_s.wait_event(d["computed"])  # the kernels of step k-2 have read this set's inputs
        with torch.cuda.stream(h2d_s):
            d["verts"].copy_(verts_p, non_blocking=True)
            d["q"].copy_(q_p, non_blocking=True)
        d["in_ready"].record(h2d_s)
        stream.wait_event(d["in_ready"])
        if d["used"]:
            stream.wait_event(d["out_done"])  # the outputs of step k-2 have left
        fem.fem_mesh_geofacs_set(b, d["verts"], G35=d["G35"], stream=stream)
        fem.fem_mesh_geofacs_set(b, d["verts"], wJ=d["wJ"], G30=d["G30"], stream=stream)
        fem.fem_bp35_apply(b, d["G35"], lam, d["q"], out=d["o"][1], stream=stream)
        fem.fem_bp1_bp30_apply(b, d["G30"], lam, d["q"], out_m=d["o"][0], out_a=d["o"][2], stream=stream)
        d["computed"].record(stream)
        d2h_s.wait_event(d["computed"])
        with torch.cuda.stream(d2h_s):
            for dst, src in zip(d["out"], d["o"]):
                dst.copy_(src, non_blocking=True)
        d["out_done"].record(d2h_s)
        d["used"] = True

    for k in range(max(2, args.warmup)):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier(world, device)
    # five windows of e2e_steps steps each; the host copies share the host's
    # memory system with other work on the machine and now and then stall
    # for a few ms, so the median window is reported (all five are listed)
    windows = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h2d_s.wait_event(e0)
        d2h_s.wait_event(e0)
        for k in range(e2e_steps):
            e2e_step(k)
        stream.wait_event(sets[(e2e_steps - 1) % 2]["out_done"])
        e1.record(stream)
        torch.cuda.synchronize()
        windows.append(reduce_max(e0.elapsed_time(e1) / e2e_steps, world, device))
    e2e_ms = statistics.median(windows)
    # the step's output agrees with the single-stream step (same kernels)
    e2e_ok = all(torch.equal(a.to(device), c) for a, c in zip(sets[(e2e_steps - 1) % 2]["out"], (o1, o35, o30)))
    del sets

    dofs = 3 * E * n ** 3
    value = world * dofs * args.steps / (ms / 1e3) / 1e9
    std, inst, byts = alg_counts(N)
    smem = smem_counts(N)
    hbm, hbm_src, _ = _peaks()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    kern = {}
    for name in KERNELS:
        t = per_kernel[name] / 1e3
        ops = {"bp1": 1, "bp35": 1, "bp30": 1, "bp1_bp30": 2}.get(name)
        kern[name] = {
            "ms": per_kernel[name],
            "gdofs": ops * E * n ** 3 / t / 1e9 if ops else None,
            "alg_gbs": E * byts[name] / t / 1e9,
            "hbm_frac": E * byts[name] / t / 1e9 / hbm,
            "fp64_tflops": E * std[name] / t / 1e12,
            "fp64_frac": E * std[name] / t / 1e12 / fp64_peak_tflops(2070.0),
            "fp64_issue_frac": E * inst[name] / t / 1e9 / fp64_peak_ginst(sm_mhz),
            "smem_frac": E * smem[name] / t / 1e9 / smem_peak_gbs(sm_mhz) if name in smem else None,
        }
    dom = max(KERNELS, key=lambda k: per_kernel[k])
    tr = NCU_TRAFFIC.get(dom)
    traffic = tr["bytes_per_elem"] * E if tr and tr["sha"] == _src_hash(tr["files"]) and tr["N"] == N else None
    peak_alu = fp64_peak_tflops(2070.0)
    # the FP64 ceiling measured on this GPU: independent FMA chains on every SM
    probe_out, probe_flops = fem.fem_fma_probe(10000)
    fem.fem_fma_probe(10000, out=probe_out)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(3):
        fem.fem_fma_probe(10000, out=probe_out)
    pe1.record(stream)
    torch.cuda.synchronize()
    probe_tflops = 3 * probe_flops / (pe0.elapsed_time(pe1) / 1e3) / 1e12
    del probe_out
    roofline = {
        "kernel": dom, "bound": "alu", "unit": "TFLOP/s",
        "achieved": kern[dom]["fp64_tflops"], "peak": peak_alu,
        "frac": kern[dom]["fp64_tflops"] / peak_alu,
        "peak_source": "FP64 issue rate derived from unit counts: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz",
        "flop_count": "direct sum factorisation (multiply-add = 2); the even-odd folded kernels execute "
                      "about 0.65x of these at N=7, so frac can exceed 1",
        "fp64_issue_frac": kern[dom]["fp64_issue_frac"],
        "fp64_probe_tflops": probe_tflops,
        # FP64 instructions per second of the kernel over those of the probe
        # (2 flops per probe instruction): the fraction of the FP64 rate this
        # GPU sustains
        "fp64_issue_frac_of_probe": kern[dom]["fp64_issue_frac"] * fp64_peak_ginst(sm_mhz) / (probe_tflops * 1e3 / 2),
        "fp64_probe": "measured FP64 FMA rate of this GPU (fem_fma_probe: 8 independent FMA chains per thread, "
                      "8 x 256 threads per SM)",
        "traffic": traffic,
        "hbm": {"achieved_gbs": kern[dom]["alg_gbs"], "peak_gbs": hbm, "peak_source": hbm_src,
                "frac": kern[dom]["hbm_frac"]},
        "smem": None if dom not in smem else {
            "bytes_per_elem": smem[dom], "achieved_gbs": E * smem[dom] / (per_kernel[dom] / 1e3) / 1e9,
            "peak_gbs": smem_peak_gbs(sm_mhz), "frac": kern[dom]["smem_frac"],
            "peak_source": "152 SMs x 128 B/clk x median SM clock (the paper's Section 5 model)"},
    }

    sweep = None if (args.no_sweep or rank != 0) else run_sweep(fem, torch, device, verts, args, sm_mhz)
    pcg = None if args.no_pcg else run_pcg(fem, torch, device, verts_h, args)
    batch = None if args.no_batch else run_batch(fem, torch, device, args)
    if batch and sweep:
        # the batch's lower bound at the stand-alone operators' full-GPU rates
        # (the per-N sweep on the 32^3 mesh): every mesh's DOFs at its
        # degree's GDOF/s, summed over the two operators
        rates = {r["N"]: (r["bp35"]["gdofs"], r["bp30"]["gdofs"]) for r in sweep["rows"]}
        w = fem_synth.batch_workload()
        if all(s_["N"] in rates for s_ in w):
            ms_ideal = sum(s_["E"] * (s_["N"] + 1) ** 3 * (1 / rates[s_["N"]][0] + 1 / rates[s_["N"]][1])
                           for s_ in w) / 1e6
            batch["at_standalone_full_gpu_rates"] = {
                "ms": ms_ideal, "tuned_frac": ms_ideal / batch["persistent_tuned"]["ms"],
                "note": "every mesh at the sweep's GDOF/s for its degree and operator; the tuned "
                        "persistent launch's time against it"}
    serve = None if args.serve_requests <= 0 else run_serve(fem, torch, args)
    small = None if (args.no_sweep or rank != 0) else run_small_case(fem, torch, device)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        rate, Es, reps, dt, threads = cpu_oracle_rate(N, verts_h, q_h, lam, args.cpu_seconds, cores)
        cpu = {"value": rate, "unit": "GDOF/s", "cores": threads, "kind": "oracle",
               "sample": f"{reps} pass(es) over the first {Es} of {E} elements (geometric factors + "
                         f"BP1.0 + BP3.5 + BP3.0, N={N}), {dt:.1f} s"}
        r1, Es1, reps1, dt1, _ = cpu_oracle_rate(N, verts_h, q_h, lam, args.cpu_seconds / 4, 1)
        cpu["single_thread"] = {"value": r1, "unit": "GDOF/s", "cores": 1,
                                "sample": f"{reps1} pass(es) over the first {Es1} of {E} elements, {dt1:.1f} s"}
        cpu["host"] = cpu_model()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": step_config(E, N, lam, world),
            "e2e": {"value": world * dofs / (e2e_ms / 1e3) / 1e9, "unit": "GDOF/s",
                    "h2d_bytes_per_step": int(verts_h.nbytes + q_h.nbytes),
                    "d2h_bytes_per_step": int(3 * q_h.nbytes),
                    "ms_per_step": e2e_ms, "steps": e2e_steps,
                    "windows_ms_per_step": windows, "reported": "median of the five windows",
                    "pipelining": "host-to-device copies, kernels and device-to-host copies on three streams "
                                  "over two buffer sets: step k+1's inputs and step k-1's outputs move "
                                  "while step k's kernels run", "outputs_match_device_step": e2e_ok},
            "gpu_launches": len(KERNELS) * args.steps,
            "step_unfused": {"ms_per_step": ms_unfused, "value": world * dofs / (ms_unfused / 1e3) / 1e9,
                             "unit": "GDOF/s", "steps": uf_steps,
                             "kernels": "the two factor sets, then BP1.0, BP3.5 and BP3.0 as separate launches"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "kernels": kern,
        }
        sections = {"sweep": sweep, "small_case": small, "pcg": pcg, "batch": batch, "serve": serve}
        emit(line, sections, args.sections_out)
    b.free()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


HEADLINE_MAX_BYTES = 4096


def _r(x, digits=4):
    """x rounded to `digits` significant figures (floats only; containers
    recursively), to keep the headline line short."""
    if isinstance(x, float):
        return float(f"{x:.{digits}g}")
    if isinstance(x, dict):
        return {k: _r(v, digits) for k, v in x.items()}
    if isinstance(x, list):
        return [_r(v, digits) for v in x]
    return x


def headline_summary(sections):
    """A few figures of the side sections for the headline: the Helmholtz
    solves at 1e-13 (where the mixed solves reach the FP64 solution to
    1e-10), the batch and the serving measurement."""
    out = {}
    pcg = sections.get("pcg")
    if pcg:
        t = pcg.get("tight", {})
        out["pcg_tol_1e-13"] = {k: {"solves_per_s": v.get("solves_per_s"),
                                    "rel_diff_vs_fp64_solve": v.get("rel_diff_vs_fp64_solve"),
                                    "rel_err_vs_u_I": v.get("rel_err_vs_u_I")}
                                for k, v in t.items() if isinstance(v, dict)}
        for k, v in t.items():
            if k.endswith("_speedup"):
                out["pcg_tol_1e-13"][k] = v
        t30 = (pcg.get("bp30") or {}).get("tight", {})
        if t30:
            out["pcg_bp30_tol_5e-13"] = {k: (v.get("solves_per_s") if isinstance(v, dict) else v)
                                         for k, v in t30.items() if k != "tol"}
    b = sections.get("batch")
    if b:
        out["batch_gdofs"] = {"separate": b["separate_launches"]["gdofs"],
                              "persistent_tuned": b["persistent_tuned"]["gdofs"], "graph": b["graph"]["gdofs"]}
    sv = sections.get("serve")
    if sv:
        st = sv.get("steady_state") or {}
        cf = (sv.get("config_arrivals_200_per_s") or {}).get("fifo") or {}
        out["serve"] = {"steady": {k: st.get(k) for k in ("arrival_rate_per_s", "served_per_s", "p50_s", "p99_s")
                                   if k in st},
                        "config": {k: cf.get(k) for k in ("offered_per_s", "served_per_s", "p50_s", "p99_s")
                                   if k in cf}}
    return out


def compact_headline(line, sections):
    """The last stdout line: the contract's keys and the roofline, rounded,
    with the side sections reduced to a few figures."""
    keep_kern = ("ms", "gdofs", "alg_gbs", "hbm_frac", "fp64_tflops", "fp64_issue_frac", "smem_frac")
    head = dict(line)
    head["kernels"] = {k: {f: v.get(f) for f in keep_kern} for k, v in line.get("kernels", {}).items()}
    rf = dict(line.get("roofline") or {})
    for long_key in ("fp64_probe", "flop_count"):
        rf.pop(long_key, None)
    if isinstance(rf.get("smem"), dict):
        rf["smem"] = {k: rf["smem"][k] for k in ("achieved_gbs", "peak_gbs", "frac") if k in rf["smem"]}
    head["roofline"] = rf
    e2e = dict(line.get("e2e") or {})
    e2e.pop("pipelining", None)
    head["e2e"] = e2e
    head["summary"] = headline_summary(sections)
    head["sections"] = [k for k, v in sections.items() if v is not None]
    head = _r(head)
    if len(json.dumps(head)) > HEADLINE_MAX_BYTES:  # drop detail, never the contract's keys
        head.pop("kernels", None)
        head.pop("summary", None)
    return head


def emit(line, sections, sections_out=None):
    """Prints every side section as its own JSON line ({"section": name,
    ...}), then the compact headline as the last line.  With sections_out,
    the sections and the full headline also go to that file as one JSON
    document."""
    for name, data in sections.items():
        if data is not None:
            print(json.dumps({"section": name, **data}))
    head = compact_headline(line, sections)
    if sections_out:
        os.makedirs(os.path.dirname(os.path.abspath(sections_out)), exist_ok=True)
        with open(sections_out, "w") as f:
            json.dump({"headline": line, "sections": sections}, f, indent=1)
    sys.stdout.flush()
    print(json.dumps(head))
    sys.stdout.flush()
    return head


def parse_degrees(spec: str):
    out = []
    for part in spec.split(","):
        part = part.strip()
        if not part:
            continue
        if "-" in part:
            lo, hi = part.split("-")
            out.extend(range(int(lo), int(hi) + 1))
        else:
            out.append(int(part))
    return out


def run_sweep(fem, torch, device, verts, args, sm_mhz):
    """GDOF/s and roofline fractions of the three FP64 operators (and the
    FP32 BP3.5/BP3.0 operators of the mixed-precision solver) against N on
    the benchmark mesh, with the copy roofline recalibrated at every size as
    the paper does (Section 5): a device-to-device copy of half the
    operator's algorithmic bytes (a copy of T/2 bytes moves T), and the
    library's calibration stream with the operator's read:write ratio (k
    planes read, their sum written).  Each figure is the median of `reps`
    launches timed with CUDA events after two warm-up launches, each launch
    preceded (outside its events) by a 258 MB write that evicts L2, so that
    the low degrees, whose arrays would fit in L2, are timed cold too."""
    stream = torch.cuda.current_stream(device)
    E = verts.shape[0]
    lam, reps = 1.0, args.sweep_reps
    hbm, _, _ = _peaks()
    rows = []

    # a write of twice the L2 size before every timed launch, outside its
    # events: each launch starts from a cold L2, also at the low degrees
    # whose arrays would otherwise stay resident between launches
    flush = torch.empty(2 * 129 * 2 ** 20, dtype=torch.uint8, device=device)

    def timed(fn, count):
        for _ in range(2):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(count)]
        for a, b_ in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b_.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b_) for a, b_ in ev)

    degrees = parse_degrees(args.sweep)
    if not degrees:
        return None
    # one seeded U[-1,1] field of the largest size; smaller N take a prefix
    q_all = torch.from_numpy(fem_synth.field(fem_synth.SEED_Q, E, (max(degrees) + 1) ** 3)).to(device).view(-1)
    for N in degrees:
        n = N + 1
        b = fem.fem_basis_setup(N)
        q = q_all[:E * n ** 3].view(E, n ** 3)
        out = torch.empty_like(q)
        std, inst, byts = alg_counts(N)
        smem = smem_counts(N)
        row = {"N": N, "dofs": E * n ** 3}
        for name, kind in (("bp1", 1), ("bp35", 2), ("bp30", 3), ("bp1_bp30", 3), ("bp30_points", 3), ("bp35_points", 2),
                           ("bp35_f32", 2), ("bp30_f32", 3), ("bp35_f16", 2), ("bp30_f16", 3),
                           ("bp30_f32_block", 3), ("bp30_f32_warp", 3), ("bp30_tc", 3), ("bp35_tc", 2)):
            f16 = name.endswith("_f16")
            f32 = name.endswith("_f32") or f16 or name in ("bp30_f32_block", "bp30_f32_warp", "bp30_tc", "bp35_tc")
            base = ("bp30" if name in ("bp30_f32_block", "bp30_f32_warp", "bp30_tc")
                    else "bp35" if name == "bp35_tc" else (name[:-4] if f32 else name))
            ratio_base = "bp30" if base in ("bp30_points", "bp1_bp30") else ("bp35" if base == "bp35_points" else base)
            geo = torch.empty(fem.geo_shape(b, kind, E), dtype=torch.float64, device=device)
            fem.fem_mesh_geofacs(b, kind, verts, geo=geo, stream=stream)
            if f16:
                # binary16 factors scaled by 2^(14 - e), max|G| < 2^e, as the solver stores them
                ex = int(np.frexp(geo.abs().max().item())[1])
                gi = torch.tensor([2.0 ** (ex - 14)], dtype=torch.float64, device=device)
                geo, qx = (geo * 2.0 ** (14 - ex)).half(), q.float()
                o = torch.empty_like(qx)
                fn = fem.fem_bp35_apply_f16g if base == "bp35" else fem.fem_bp30_apply_f16g
                ms = timed(lambda: fn(b, geo, gi, lam, qx, out=o, stream=stream), reps)
                del qx, o, gi
            elif f32:
                geo, qx = geo.float(), q.float()
                o = torch.empty_like(qx)
                if name == "bp30_tc":
                    fn = fem.fem_bp30_apply_tc
                elif name == "bp35_tc":
                    fn = fem.fem_bp35_apply_tc
                elif name in ("bp30_f32_warp", "bp30_f32_block"):
                    lay = fem.FEM_LAYOUT_WARP if name == "bp30_f32_warp" else fem.FEM_LAYOUT_LINES

                    def fn(b_, g_, l_, q_, out, stream, lay=lay):
                        return fem.fem_bp30_apply_f32_layout(b_, g_, l_, q_, lay, out=out, stream=stream)
                else:
                    fn = fem.fem_bp35_apply_f32 if base == "bp35" else fem.fem_bp30_apply_f32
                ms = timed(lambda: fn(b, geo, lam, qx, out=o, stream=stream), reps)
                del qx, o
            elif name == "bp1_bp30":
                out2 = torch.empty_like(q)
                ms = timed(lambda: fem.fem_bp1_bp30_apply(b, geo, lam, q, out_m=out2, out_a=out, stream=stream),
                           reps)
                del out2
            elif name == "bp30_points":
                ms = timed(lambda: fem.fem_bp30_apply_layout(b, geo, lam, q, fem.FEM_LAYOUT_POINTS, out=out,
                                                             stream=stream), reps)
            elif name == "bp35_points":
                ms = timed(lambda: fem.fem_bp35_apply_layout(b, geo, lam, q, fem.FEM_LAYOUT_POINTS, out=out,
                                                             stream=stream), reps)
            elif name == "bp1":
                ms = timed(lambda: fem.fem_bp1_apply(b, geo, q, out=out, stream=stream), reps)
            elif name == "bp35":
                ms = timed(lambda: fem.fem_bp35_apply(b, geo, lam, q, out=out, stream=stream), reps)
            else:
                ms = timed(lambda: fem.fem_bp30_apply(b, geo, lam, q, out=out, stream=stream), reps)
            del geo
            word = 4 if f32 else 8
            per_elem = byts[base] * word // 8
            if f16:  # the factor planes move in two bytes per value
                per_elem = 4 * (2 * n ** 3) + 2 * 7 * (n ** 3 if base == "bp35" else (N + 2) ** 3)
            T = E * per_elem
            # recalibrated copy roofline at this byte count
            half = torch.empty(T // 2 // 8, dtype=torch.float64, device=device)
            dst = torch.empty_like(half)
            copy_ms = timed(lambda: dst.copy_(half), 10)
            del half, dst
            # read:write ratio of the operator (planes read per plane written)
            k = round((byts[ratio_base] - 8 * n ** 3) / (8 * n ** 3))
            src = torch.empty((k, E * n ** 3), dtype=torch.float32 if f32 else torch.float64, device=device)
            src.fill_(1.0)
            red = torch.empty(E * n ** 3, dtype=src.dtype, device=device)
            ratio_ms = timed(lambda: fem.fem_stream_sum(src, out=red, stream=stream), 10)
            ratio_gbs = word * (k + 1) * E * n ** 3 / (ratio_ms / 1e3) / 1e9
            del src, red
            t = ms / 1e3
            gbs = T / t / 1e9
            copy_gbs = T / (copy_ms / 1e3) / 1e9
            ops = 2 if name == "bp1_bp30" else 1  # the fused pass applies two operators
            row[name] = {
                "ms": ms, "gdofs": ops * E * n ** 3 / t / 1e9, "alg_gbs": gbs,
                "hbm_frac": gbs / hbm, "copy_gbs_at_size": copy_gbs, "copy_frac_at_size": gbs / copy_gbs,
                "ratio_stream_gbs": ratio_gbs, "ratio_read_planes": k,
                "hbm_bound_gdofs": ops * copy_gbs / (per_elem / n ** 3),
                "smem_frac": E * smem[base] * word // 8 / t / 1e9 / smem_peak_gbs(sm_mhz),
            }
            if not f32:
                row[name]["fp64_tflops"] = E * std[name] / t / 1e12
                row[name]["fp64_issue_frac"] = E * inst[name] / t / 1e9 / fp64_peak_ginst(sm_mhz)
        rows.append(row)
        del q, out
        b.free()
    del q_all
    torch.cuda.empty_cache()
    return {"workload": f"BP1.0/BP3.5/BP3.0 FP64 (BP3.0 also in the point-per-thread layout, and BP1.0 + BP3.0 "
                        f"in one pass, whose GDOF/s count both operators' DOFs; BP3.5/BP3.0 FP32 "
                        f"with FP32 and FP16 factors, the mixed solvers' inner operators; FP32 BP3.0 with one "
                        f"warp per element and with its contractions on the tensor cores, split f16 mma.sync) "
                        f"sweep, E={E} jittered "
                        f"hexes, lambda=1, median of {reps} launches per point, L2 evicted before each",
            "copy_roofline": "device-to-device copy of T/2 bytes moving T = the operator's algorithmic "
                             "bytes, recalibrated at every N (Section 5 of the paper)",
            "rows": rows}


def run_small_case(fem, torch, device):
    """The small configuration: BP1.0 at N = 3 on the 8^3 jittered mesh (E =
    512, 32768 DOFs, 1.04 MB of algorithmic traffic, resident in L2).  It is
    bound by launch latency, so the figure is microseconds per launch: back
    to back on one stream, and replayed from a CUDA graph of 100 launches."""
    N, reps = 3, 100
    b = fem.fem_basis_setup(N)
    v = torch.from_numpy(fem_synth.box_mesh(8)).to(device)
    E = v.shape[0]
    wJ = fem.fem_mesh_geofacs(b, fem.FEM_GEO_BP1, v)
    q = torch.from_numpy(fem_synth.field(fem_synth.SEED_Q, E, (N + 1) ** 3)).to(device)
    out = torch.empty_like(q)
    st = torch.cuda.Stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        for _ in range(10):
            fem.fem_bp1_apply(b, wJ, q, out=out, stream=st)
        st.synchronize()
        e0.record(st)
        for _ in range(reps):
            fem.fem_bp1_apply(b, wJ, q, out=out, stream=st)
        e1.record(st)
        st.synchronize()
        us_stream = e0.elapsed_time(e1) * 1e3 / reps
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for _ in range(reps):
                fem.fem_bp1_apply(b, wJ, q, out=out, stream=st)
        g.replay()
        st.synchronize()
        e0.record(st)
        g.replay()
        e1.record(st)
        st.synchronize()
        us_graph = e0.elapsed_time(e1) * 1e3 / reps
    dofs = E * (N + 1) ** 3
    b.free()
    return {"workload": "BP1.0 FP64, N=3, E=512 (8^3 jittered mesh), inputs resident in L2",
            "us_per_launch_stream": us_stream, "us_per_launch_graph": us_graph,
            "gdofs_graph": dofs / (us_graph * 1e-6) / 1e9}


def manufactured_u(fem, basis, verts_h):
    """u_I = sin(pi x) sin(pi y) sin(pi z) at every element's GLL nodes
    (physical coordinates through the trilinear map, GLL nodes from the
    library's basis tables)."""
    N = basis.N
    r = fem.fem_basis_tables(basis)["r"]
    n = N + 1
    R, S, T = np.meshgrid(r, r, r, indexing="ij")
    R, S, T = (a.transpose(2, 1, 0).reshape(-1) for a in (R, S, T))
    phi = np.stack([(1 + (1 if c & 1 else -1) * R) * (1 + (1 if c & 2 else -1) * S) *
                    (1 + (1 if c & 4 else -1) * T) / 8 for c in range(8)], axis=1)
    X = np.einsum("pc,ecd->epd", phi, verts_h)
    return np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])


def run_pcg(fem, torch, device, verts_h, args):
    """Jacobi-PCG of the BP3.5 Helmholtz system (lambda = 1; the precision
    configuration) and of the BP3.0 one, with the manufactured right-hand
    side b = A u_I: all-FP64 against FP64 defect correction with FP32 inner
    solves (FP32 factors; FP16 factors; the tensor-core
    contractions).  Each mode is solved to a tight residual (1e-13 for
    BP3.5, 5e-13 for BP3.0, whose FP64 residual stagnates near 2e-13), where
    every mode reaches the FP64 solution to 1e-10 and the distance to it is
    reported, and to 1e-10, the configuration's residual, where the solves
    differ by up to the FP64 solve's own distance to u_I (about 2e-8: the
    error is the residual times up to the condition number)."""
    N, lam = args.degree, 1.0
    basis = fem.fem_basis_setup(N)
    vd = torch.from_numpy(verts_h).to(device)
    u = torch.from_numpy(manufactured_u(fem, basis, verts_h)).to(device)
    out = {"workload": f"Helmholtz PCG (Jacobi), N={N}, E={verts_h.shape[0]}, lambda=1, b = A u_I with "
                       f"u = sin(pi x) sin(pi y) sin(pi z)",
           "error_reference": "u_I, the exact discrete solution; rel_diff_vs_fp64_solve against the FP64 "
                              "GPU solve of the same tolerance (the oracle PCG agrees with the GPU solvers to "
                              "1e-8 on the smaller meshes of tests/test_pcg_gpu.py)",
           "modes": {"fp64": "all-FP64 Jacobi-PCG",
                     "mixed": "FP64 defect correction, FP32 inner PCG with FP32 factors",
                     "mixed16": "FP64 defect correction, FP32 inner PCG with binary16 factors (power-of-two "
                                "scaled) widened to FP32 in the kernel",
                     "mixed_tc": "FP64 defect correction, FP32 inner PCG whose matvec runs its 1D "
                                 "contractions on the tensor cores (split f16 mma.sync, FP32 accumulate)"}}
    wanted = args.pcg_modes.split(",")
    for opname, op, kind in (("bp35", fem.FEM_OP_BP35, fem.FEM_GEO_BP35), ("bp30", fem.FEM_OP_BP30, fem.FEM_GEO_BP30)):
        G = fem.fem_mesh_geofacs(basis, kind, vd)
        apply = fem.fem_bp35_apply if op == fem.FEM_OP_BP35 else fem.fem_bp30_apply
        b = apply(basis, G, lam, u)
        modes = [(nm, md, it) for nm, md, it in (("fp64", fem.FEM_PCG_FP64, 0.0), ("mixed", fem.FEM_PCG_MIXED, 1e-3),
                                                 ("mixed16", fem.FEM_PCG_MIXED16, 1e-3),
                                                 ("mixed_tc", fem.FEM_PCG_MIXED_TC, 1e-3))
                 if nm in wanted]
        res = {}
        # the tight solve: 1e-13 for BP3.5; the FP64 BP3.0 residual stagnates
        # near 2e-13 on this mesh, so 5e-13 for BP3.0
        tight = 1e-13 if op == fem.FEM_OP_BP35 else 5e-13
        for tol, reps in ((tight, 1), (1e-10, max(1, args.pcg_solves))):
            blk, xs = {"tol": tol}, {}
            for name, mode, itol in modes:
                s = fem.fem_pcg_create(basis, G, lam, mode, op=op)
                x, info, code = s.solve(b, tol=tol, inner_tol=itol, raise_on_error=False)  # warm-up
                times = []
                for _ in range(reps):
                    x.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    x, info, code = s.solve(b, x=x, tol=tol, inner_tol=itol, raise_on_error=False)
                    torch.cuda.synchronize()
                    times.append(time.perf_counter() - t0)
                med = statistics.median(times)
                blk[name] = {"solves_per_s": 1.0 / med, "ms_per_solve": 1e3 * med, "iters": info["iters"],
                             "outer": info["outer"], "relres": info["relres"], "status": code,
                             "rel_err_vs_u_I": (torch.linalg.norm(x - u) / torch.linalg.norm(u)).item()}
                xs[name] = x.clone()
                s.free()
            for name in xs:
                if name != "fp64" and "fp64" in xs:
                    blk[name]["rel_diff_vs_fp64_solve"] = (torch.linalg.norm(xs[name] - xs["fp64"]) /
                                                           torch.linalg.norm(xs["fp64"])).item()
                    blk[name + "_speedup"] = blk[name]["solves_per_s"] / blk["fp64"]["solves_per_s"]
            res["tight" if tol == tight else "tol_1e-10"] = blk
            del xs
        out[opname] = res
        del G, b
        torch.cuda.empty_cache()
    # the precision configuration (BP3.5) at the top level, tight solve first
    out["tight"] = out["bp35"]["tight"]
    basis.free()
    return out


def run_batch(fem, torch, device, args):
    """64 independent jittered meshes, N uniform in 2..10, E log-uniform in
    64..8192, BP3.5 and BP3.0 (FP64, lambda = 1) on each: 128 separate launches
    against one persistent launch (default and autotuned configuration) and
    its CUDA-graph replay."""
    w = fem_synth.batch_workload()
    bases = {N: fem.fem_basis_setup(N) for N in sorted({s["N"] for s in w})}
    items, dofs = [], 0
    for s in w:
        b = bases[s["N"]]
        v = torch.from_numpy(fem_synth.box_mesh(s["nx"], s["ny"], s["nz"], jitter=0.1,
                                                seed=s["mesh_seed"])).to(device)
        q = torch.from_numpy(fem_synth.field(s["mesh_seed"] + 7, s["E"], (s["N"] + 1) ** 3)).to(device)
        for op, kind in ((fem.FEM_OP_BP35, fem.FEM_GEO_BP35), (fem.FEM_OP_BP30, fem.FEM_GEO_BP30)):
            g = fem.fem_mesh_geofacs(b, kind, v)
            items.append((op, b, g, 1.0, q, torch.empty_like(q)))
            dofs += q.numel()
    batch = fem.Batch(items)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def separate():
        for op, b, g, lam, q, out in items:
            (fem.fem_bp35_apply if op == fem.FEM_OP_BP35 else fem.fem_bp30_apply)(b, g, lam, q, out=out)

    ms_sep = timed(separate)
    ms_default = timed(batch.apply)
    results = batch.tune(reps=5)
    ms_tuned = timed(batch.apply)
    ms_graph = timed(batch.graph_launch)
    out = {"workload": "64 jittered meshes, N uniform 2..10, E log-uniform 64..8192 (108835 elements), "
                       "BP3.5 and BP3.0 FP64 lambda=1 on each (128 matvecs)",
           "dofs_per_pass": dofs,
           "separate_launches": {"ms": ms_sep, "gdofs": dofs / ms_sep / 1e6},
           "persistent_default": {"ms": ms_default, "gdofs": dofs / ms_default / 1e6},
           "persistent_tuned": {"ms": ms_tuned, "gdofs": dofs / ms_tuned / 1e6, "config": batch.config},
           "graph": {"ms": ms_graph, "gdofs": dofs / ms_graph / 1e6},
           "tuner_candidates": len(results)}
    batch.free()
    return out


def run_serve(fem, torch, args):
    """Serving configuration: Poisson arrivals (mean 200 requests/s) of
    Helmholtz PCG solves, BP3.0 or BP3.5 at random, N uniform in 3..9, E
    log-uniform in 512..32768, rhs uniform in [-1, 1], tolerance 1e-8, FP64
    or mixed precision (FP16 factors) at random, 120 GiB HBM budget,
    continuous batching in 8 slots.

    The requests cycle a pool of 32 distinct problems drawn from that
    distribution (each request is tens of MB of host data; the arrival times
    are the configuration's own).  Three runs:
      config   the configuration's arrival process, first come first served:
               the offered load is far above what one GPU serves, so the
               queue grows while requests arrive and drains after;
      steady   the same request stream arriving at 0.8 x the measured
               service rate (the Poisson process rescaled in time) for
               serve_window seconds: a steady state, first come first served
               and least estimated work first with aging;
      alone    the first 24 problems one at a time, for the check that each
               result is the same bits alone and in the mix.
    Latency percentiles exclude the first 10 % of requests (warm-up); the
    queue depth is sampled every 0.1 s of the server clock."""
    n_req = max(24, args.serve_requests)
    reqs = fem_synth.serve_workload(n_req)
    pool_n = min(32, n_req)
    pool = []
    for r in reqs[:pool_n]:
        v = fem_synth.box_mesh(r["nx"], r["ny"], r["nz"], jitter=0.1, seed=r["mesh_seed"])
        rhs = fem_synth.field(r["rhs_seed"], r["E"], (r["N"] + 1) ** 3)
        pool.append((r, v, rhs))
    arrivals = [r["t"] for r in reqs]

    def submit(srv, k):
        r, v, rhs = pool[k % pool_n]
        mode = fem.FEM_PCG_MIXED16 if r["mixed"] else fem.FEM_PCG_FP64
        return srv.submit(r["op"], r["N"], v, rhs, lam=1.0, mode=mode, tol=1e-8)

    def play(times, policy=fem.FEM_SERVE_FIFO, keep=24):
        srv = fem.Server(hbm_budget=120 << 30, max_active=8, policy=policy)
        t0 = srv.clock()
        k, depth, nxt = 0, [], 0.0
        xs, pending, done = {}, {}, {}

        def collect():
            # finished requests: keep their results, let go of their host arrays
            for kk, rid in list(pending.items()):
                p = srv.poll(rid)
                if p["state"] in (fem.FEM_REQ_DONE, fem.FEM_REQ_FAILED):
                    done[kk] = p
                    del pending[kk]
                    srv.forget(rid)

        while True:
            now = srv.clock() - t0
            while k < len(times) and times[k] <= now:
                rid, x = submit(srv, k)
                pending[k] = rid
                if k < keep:
                    xs[k] = x
                k += 1
            a, q = srv.progress()
            if now >= nxt:
                depth.append((round(now, 2), a, q))
                nxt += 0.1
                collect()
            if k == len(times) and a == 0 and q == 0:
                break
        collect()
        res = [done[kk] for kk in range(len(times))]
        srv.free()
        lat = np.array([p["t_done"] - p["t_submit"] for p in res])
        warm = len(res) // 10
        span = max(p["t_done"] for p in res) - min(p["t_submit"] for p in res)
        qd = np.array([d[2] for d in depth]) if depth else np.zeros(1)
        out = {"requests": len(res),
               "offered_per_s": (len(times) - 1) / max(times[-1] - times[0], 1e-9),
               "served_per_s": len(res) / span, "makespan_s": span,
               "p50_s": float(np.percentile(lat[warm:], 50)), "p99_s": float(np.percentile(lat[warm:], 99)),
               "warmup_excluded": warm,
               "failed": int(sum(p["state"] != fem.FEM_REQ_DONE for p in res)),
               "max_relres": float(max(p["relres"] for p in res)),
               "queue_depth": {"max": int(qd.max()), "mean": float(qd.mean()),
                               "every_0.5s": [d[2] for d in depth[::5]]}}
        for name, flag in (("mixed", True), ("fp64", False)):
            sel = np.array([pool[i % pool_n][0]["mixed"] == flag for i in range(len(res))])
            if sel[warm:].any():
                out[name] = {"count": int(sel.sum()), "p50_s": float(np.percentile(lat[warm:][sel[warm:]], 50)),
                             "p99_s": float(np.percentile(lat[warm:][sel[warm:]], 99))}
        return out, xs

    cfg_fifo, xs_mix = play(arrivals)
    rate = 0.8 * cfg_fifo["served_per_s"]
    # the same Poisson process slowed to `rate`, over a window of
    # args.serve_window seconds of arrivals
    steady_times = [t * 200.0 / rate for t in arrivals]
    steady_times = [t for t in steady_times if t <= args.serve_window] or steady_times[:2]
    steady, _ = play(steady_times, keep=0)
    steady["arrival_rate_per_s"] = rate
    steady_sjf, _ = play(steady_times, fem.FEM_SERVE_SHORTEST, keep=0)
    steady_sjf["arrival_rate_per_s"] = rate
    srv = fem.Server(max_active=1)
    same = True
    for k in range(min(24, n_req)):
        rid, x = submit(srv, k)
        srv.drain()
        same = same and srv.poll(rid)["state"] == fem.FEM_REQ_DONE and np.array_equal(x, xs_mix[k])
    srv.free()
    return {"workload": f"{n_req} requests cycling {pool_n} problems: BP3.0|BP3.5, N 3..9, E 512..32768 "
                        "log-uniform, rhs U[-1,1], tol 1e-8, FP64|mixed (FP16 factors), 120 GiB budget, 8 slots",
            "config_arrivals_200_per_s": {"fifo": cfg_fifo},
            "steady_state": steady,
            "steady_state_shortest_first_aging": steady_sjf,
            "results_identical_alone_and_in_mix": bool(same),
            "identical_check": "the first 24 requests of the config run against the same problems solved one "
                               "at a time"}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--degree", type=int, default=7)
    ap.add_argument("--mesh-side", type=int, default=32,
                    help="elements per side of the cube mesh (32 is the benchmark workload; "
                         "smaller sides are for profiling captures)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", default="1-15",
                    help="degrees of the per-N operator sweep (e.g. 1-15 or 3,7,11)")
    ap.add_argument("--sweep-reps", type=int, default=20)
    ap.add_argument("--no-sweep", action="store_true", help="skip the per-N operator sweep")
    ap.add_argument("--no-pcg", action="store_true", help="skip the Helmholtz solve measurement")
    ap.add_argument("--pcg-solves", type=int, default=3)
    ap.add_argument("--pcg-modes", default="fp64,mixed,mixed16,mixed_tc",
                    help="solver modes of the Helmholtz measurement (comma list of fp64, mixed, mixed16, "
                         "mixed_tc)")
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed-order batch measurement")
    ap.add_argument("--sections-out", default=None,
                    help="also write the side sections and the full headline to this JSON file")
    ap.add_argument("--serve-window", type=float, default=30.0,
                    help="seconds of arrivals of the steady-state serving runs")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests of the Poisson-arrival serving measurement (0 skips it)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
