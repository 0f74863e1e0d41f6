#!/usr/bin/env python
"""Benchmark of the GB300 MOT step: RHS*steps/s of the batched qHP TD-PMCHWT
march on one GPU (or N independent replicas under torchrun).

Workload (default): multiply-connected torus R = 1, r = 0.3, 64 x 24 quad grid
split into 3072 triangles (4608 edges, 9216 unknowns), eps_r = 4, c dt = 0.1
(k_max = 52, 53 history lags), 64 Gaussian plane waves with Fibonacci
directions and seeded polarisations, batched in one march.

One bench step = one MOT step for the whole batch: right-hand side, full-depth
history contraction over all lags (tensor cores on the mixed path), left
preconditioner factors, the Q_0 solve (mixed: right-preconditioned GMRES on
the FP32 dense Q_0 with one FP64 refinement sweep; fp64: GMRES with product-
form matvecs), ring update, current recovery. Before timing, the march is
advanced K+1 steps so every timed step contracts the full history (plus the
W warm-up steps given on the command line).

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MOT RHS·steps/s, batched mixed vs FP64 plain on one GB300, at ≤1e-6 rel err"

WORKLOADS = {
    # name: (mesh builder, eps_r, c dt, B, assembly options)
    "torus64x24": (lambda MS: MS.torus(1.0, 0.3, 64, 24), 4.0, 0.1, 64, dict(nq=3, ntheta=3, nrad=3, far_plain=6)),
    "torus32x12": (lambda MS: MS.torus(1.0, 0.3, 32, 12), 4.0, 0.1, 64, dict(nq=3, ntheta=3, nrad=3, far_plain=6)),
    # the non-smooth cube of side 2, 24 cells per edge: 6912 tris, 10368 edges, eps_r = 6, c dt = 0.25 (35 lags)
    "cube24": (lambda MS: MS.cube(2.0, 24), 6.0, 0.25, 32, dict(nq=3, ntheta=3, nrad=3, far_plain=6)),
    "icosphere3": (lambda MS: MS.icosphere(3), 2.0, 0.5, 1, dict(nq=3, ntheta=3, nrad=3, far_plain=6)),
    "pr1": (lambda MS: MS.icosphere(1), 2.0, 0.2, 1, dict()),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="torus64x24", choices=sorted(WORKLOADS) + ["uneven24"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tc-form", default="default", choices=["default", "gathered", "bulk"],
                    help="form of the tensor-core history kernel (default: the library's)")
    ap.add_argument("--fp64-steps", type=int, default=8,
                    help="timed steps of the FP64 plain arm measured beside the mixed one (0: skip it)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(values, world):
    """Max over ranks of a list of floats (identity for one rank)."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def throughput(world, B, steps, ms):
    """Whole-job RHS*steps/s: every rank marches its own B plane waves (weak
    scaling, no data-path collective), timed by the slowest rank."""
    return world * B * steps / (ms / 1e3)


def make_waves(name, rank=0, t0_steps=240.0):
    """The workload's plane waves (the paper's width w = 120 c dt) with the
    pulse peak at the origin at t0 = t0_steps dt; rank r draws its
    polarisations from seed 20251007 + r."""
    from paper_2510_07989_gb300.inputs import meshes as MS
    build_mesh, eps_r, dt, B, aopt = WORKLOADS[name]
    r_obj = float(np.linalg.norm(build_mesh(MS).verts, axis=1).max())
    if B == 1:
        return MS.single_wave(dt, t0_steps=t0_steps, r_obj=r_obj)
    return MS.fibonacci_batch(B, dt, seed=20251007 + rank, t0_steps=t0_steps, r_obj=r_obj)


def make_workload(name, rank=0):
    from paper_2510_07989_gb300.inputs import meshes as MS
    from paper_2510_07989_gb300.inputs.assemble import assemble
    build_mesh, eps_r, dt, B, aopt = WORKLOADS[name]
    mesh = build_mesh(MS)
    t = time.time()
    ops = assemble(mesh, eps_r, 1.0, dt, **aopt)
    t_asm = time.time() - t
    return ops, make_waves(name, rank), t_asm


CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def parse_clock_csv(lines, t_begin=None, t_end=None, slack=0.25):
    """Clock record of a region from nvidia-smi CSV lines (timestamp, index,
    clocks.sm, clocks.max.sm, power.draw, clocks_event_reasons.active and the
    four reasons of CLOCK_REASONS): median SM clock and the active reasons of
    the samples stamped within [t_begin - slack, t_end + slack] (host epoch
    seconds). With no window, or no sample stamped inside it (e.g. a timestamp
    format this parser does not read), every sample counts and
    "in_region_only" is false."""
    rows = []
    for line in lines:
        p = [x.strip() for x in line.split(",")]
        if len(p) < 10:
            continue
        try:
            f_sm, f_max = float(p[2]), float(p[3])
        except ValueError:
            continue
        try:
            ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        act = {nm for nm, v in zip(CLOCK_REASONS, p[6:10]) if v.lower().startswith("active")}
        rows.append((ts, f_sm, f_max, act))
    inside = [r for r in rows if t_begin is not None and r[0] is not None and
              t_begin - slack <= r[0] <= t_end + slack]
    use = inside if inside else rows
    return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
            "sm_max_mhz": max(r[2] for r in use) if use else None,
            "samples": len(use), "samples_outside_region": len(rows) - len(use),
            "in_region_only": bool(inside), "reasons": sorted(set().union(*[r[3] for r in use])) if use else []}


class Clocks:
    """nvidia-smi sampling (every 200 ms) of SM clocks and throttle reasons;
    the record keeps the samples taken between begin() and end()."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None
        self.t_begin = self.t_end = None

    def start(self):
        """Start the sampler and wait (up to 5 s) for its first sample."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t = time.time()
        while time.time() - t < 5.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.05)

    def begin(self):
        self.t_begin = time.time()

    def end(self):
        self.t_end = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            rec = parse_clock_csv(f.readlines(), self.t_begin, self.t_end)
        os.unlink(self.path)
        if self.t_begin is not None:
            rec["region_s"] = round(self.t_end - self.t_begin, 3)
        return rec


# DRAM bytes (read + write) of one full-depth history launch, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by kernel and
# workload, with the SHA-1 of the device code of the kernel source they were
# taken on (kernel_source_sha: comments and the host launch code excluded): a
# changed kernel reports null until the counters are taken again. The third
# item is the chunking the tuner chose in that capture (tasks per chunk, lag
# fraction of L2), reported beside the figure: DRAM reads depend on it.
TRAFFIC = {
    # ncu --profile-from-start off --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
    #     --clock-control none -k regex:k_hist_tc -c 1
    #     python bench.py --steps 2 --warmup 1 --no-cpu-baseline --fp64-steps 0
    ("k_hist_tc", "torus64x24"): (44900189440 + 417015296, "dcee7d90171b04be6fe27a79c864af694c7fbf2c",
                                  {"chunk_cap": 512, "lag_frac": 0.4, "stages": 3, "tasks_per_stage": 2,
                                   "epilogue_warps": 4}),
}


def kernel_source_sha(name):
    """SHA-1 of the device code of a kernel source file: its text before the
    host launch code (the first line that opens `namespace mot {`), with
    comments removed and whitespace collapsed, so that edits of the host side
    or of comments alone keep the measured counters."""
    import hashlib
    import re
    p = os.path.join(ROOT, "paper_2510_07989_gb300", "csrc", name)
    if not os.path.exists(p):
        return None
    src = open(p, encoding="utf-8").read()
    cut = src.find("\nnamespace mot {")
    code = src if cut < 0 else src[:cut]
    code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
    code = re.sub(r"//[^\n]*", " ", code)
    return hashlib.sha1(" ".join(code.split()).encode()).hexdigest()


def traffic_of(kernel, workload, source):
    """(bytes per launch, configuration of the capture) or (None, None)."""
    t = TRAFFIC.get((kernel, workload))
    if t and t[1] == kernel_source_sha(source):
        return t[0], t[2]
    return None, None


# issued tensor-core work of one history task: two K-halves of
# 128 x (192 + 128 + 64) x 16 bf16 multiply-adds
TC_FLOPS_PER_TASK = 2 * 2 * 128 * (192 + 128 + 64) * 16


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def oracle_one_step(ops, exc, b, hist, i):
    """The product-form FP64 oracle, as it stands, computes MOT step i of wave b
    from the GPU's own previous steps hist[j] = w_j (canonical [u; v], j < i);
    returns (w_i, seconds of the step, seconds of the oracle set-up)."""
    from oracle import product as P
    t = time.time()
    sysP = P.ProductSystem(ops)
    t_setup = time.time() - t
    ne = ops.ne
    L = np.zeros((i + 1, 2 * ne))
    S = np.zeros((i + 1, 2 * ne))
    for j, w in hist.items():
        if j < i:
            L[j], S[j] = sysP.split(w)
    t0 = time.time()
    w = sysP.step(exc, b, i, L, S)
    return w, time.time() - t0, t_setup


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    if args.workload == "uneven24":  # the oracle on the batch's largest scatterer
        from paper_2510_07989_gb300.inputs import meshes as MS
        from paper_2510_07989_gb300.inputs.assemble import assemble
        specs = MS.uneven_batch(24)
        i = max(range(len(specs)), key=lambda k: specs[k][0].ne)
        mesh, eps = specs[i]
        ops = assemble(mesh, eps, 1.0, UNEVEN_DT, nq=3, ntheta=3, nrad=3, far_plain=6)
        exc = MS.fibonacci_batch(UNEVEN_B, UNEVEN_DT, seed=20251007 + i,
                                 r_obj=float(np.linalg.norm(mesh.verts, axis=1).max()))
    else:
        ops, exc, _ = make_workload(args.workload)
    from oracle import product as P
    sysP = P.ProductSystem(ops)
    ne = ops.ne
    K = ops.kmax + 1
    rng = np.random.default_rng(7)
    L = np.zeros((K + 4, 2 * ne))
    S = np.zeros((K + 4, 2 * ne))
    for j in range(1, K + 2):
        L[j], S[j] = sysP.split(rng.standard_normal(2 * ne) * 1e-3)
    i = K + 2
    # The K bench steps of this arm are together ONE full-depth product-form
    # MOT step for one right-hand side (each bench step 1/K of it): an oracle
    # step takes about a minute on the host cores, so K whole steps would not
    # end within minutes. Warm-up: one Q_0 application (the code paths of the
    # step's solve).
    if args.warmup > 0:
        sysP.q0(L[K + 1] + S[K + 1])
    t0 = time.time()
    w = sysP.step(exc, 0, i, L, S)
    el = time.time() - t0
    assert np.all(np.isfinite(w))
    v = 1.0 / el  # one RHS-step
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "RHS·steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "rhs_per_step": 1},
            "cpu_baseline": {"value": v, "unit": "RHS·steps/s", "cores": cores, "kind": "oracle",
                             "sample": "one full-depth MOT step x 1 RHS of the same workload (product-form FP64 "
                                       "oracle, seeded history), timed as the K bench steps (each 1/K of it); "
                                       "warm-up: one Q_0 application; setup excluded"},
            "e2e": {"value": v, "unit": "RHS·steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def march_arm(M, torch, ops, exc, args, local, world, precision, steps, warmup, clocks=None, keep_waves=(),
              state_in=None, hand_over=False):
    """One measured arm: K + 1 + warmup untimed steps (full-depth history) --
    or, with state_in, the march state another arm handed over (mot_save_state)
    and one untimed step from it, whose w_i is returned; then `steps` steps
    through the public call with host buffers (waves in, w_i out every step),
    timed end to end; then `steps` steps timed with CUDA events on the
    launching stream (barrier + synchronize on both sides). The caller centres
    the waves' pulse in the device-timed window. The steps of keep_waves up to
    the end of the host-buffer window are returned for an oracle check of its
    last step. With hand_over, the state at the end of the host-buffer window
    is saved and one more untimed step taken before the device-timed window:
    the pair lets the next arm's first step be compared with this one's from
    the same state."""
    B = exc.B
    K = ops.kmax + 1
    kw = dict(device=local, timing=1, precision=precision)
    if precision == M.MOT_PREC_FP64:
        kw["fp64_precond"] = 1
    elif args.tc_form == "bulk":
        kw["mixed_flags"] = M.MOT_MIX_DEFAULT | M.MOT_MIX_TCBULK
    elif args.tc_form == "gathered":
        kw["mixed_flags"] = M.MOT_MIX_DEFAULT & ~M.MOT_MIX_TCBULK
    t = time.time()
    s = M.Solver(ops, **kw)
    t_load = time.time() - t
    waves = M.mot_waves(exc)
    stream = torch.cuda.current_stream()
    host_out = torch.empty((B, 2, ops.ne), dtype=torch.float64).pin_memory()
    hist = {b: {} for b in keep_waves}

    def keep(i):
        for b in keep_waves:
            hist[b][i] = host_out.numpy()[b].reshape(-1).copy()

    first = None
    if state_in is not None:
        M.mot_load_state(s.h, state_in)
        M.mot_step(s.h, waves, B, host_out.numpy(), stream)
        first = host_out.numpy().copy()
        n_pre = M.mot_get_info(s.h)["step"]
    else:
        n_pre = K + 1 + warmup
        for i in range(1, n_pre + 1):
            M.mot_step(s.h, waves, B, host_out.numpy() if keep_waves else None, stream)
            keep(i)
            if i == K + 1 and precision == M.MOT_PREC_MIXED and M.mot_get_info(s.h)["hist_kernel"] == 2:
                M.mot_tune([s.h], stream)  # the history kernel's configuration, chosen at full depth

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # end to end through the public API with host buffers: waves in (H2D) and
    # w_i out (D2H) every step, inside the timed region
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    peak = np.zeros(B)  # largest step norm of every wave in the host-buffer window
    for i in range(n_pre + 1, n_pre + steps + 1):
        M.mot_step(s.h, waves, B, host_out.numpy(), stream)
        keep(i)
        peak = np.maximum(peak, np.linalg.norm(host_out.numpy(), axis=(1, 2)))
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    state, after = None, None
    if hand_over:  # on the rising pulse, at the largest step norm so far
        state = M.mot_save_state(s.h)
        M.mot_step(s.h, waves, B, host_out.numpy(), stream)
        after = host_out.numpy().copy()
    info0 = M.mot_get_info(s.h)
    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.begin()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # the device-timed window is the profiler's range (ncu --profile-from-start off)
    if clocks:
        torch.cuda.profiler.start()
    ev0.record(stream)
    for _ in range(steps):
        M.mot_step(s.h, waves, B, None, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if clocks:
        torch.cuda.profiler.stop()
        clocks.end()
    barrier()
    ms = ev0.elapsed_time(ev1)
    info1 = M.mot_get_info(s.h)
    return dict(s=s, ms=ms, e2e_ms=e2e_s * 1e3, info0=info0, info1=info1, t_load=t_load, check_step=n_pre + steps,
                hist=hist, noconv=s.noconv, state=state, after=after, first=first, peak=peak)


def roofline_of(info0, info1, ms_step, steps, workload, peaks, how):
    hist_launches = info1["hist_timed_launches"] - info0["hist_timed_launches"]
    hist_ms = info1["hist_timed_ms"] - info0["hist_timed_ms"]
    flops = info1["hist_flops_per_step"]
    hbytes = info1["hist_bytes_per_step"]
    ms_l = hist_ms / hist_launches if hist_launches else None
    kern = info1["hist_kernel"]
    if kern == 2:
        # tensor-core kernel: a sparse contraction streaming its tiles once per
        # step; the roofline is HBM with the path's algorithmic bytes (FP32
        # nonzeros of the lag matrices + the FP32 coefficients of every lag)
        hbm = peaks.get("hbm_gbs")
        achieved = hbytes / (ms_l / 1e3) / 1e9 if ms_l else None
        tc_flops = info1["hist_tc_tasks"] * TC_FLOPS_PER_TASK
        bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        traffic, traffic_cfg = traffic_of("k_hist_tc", workload, "k_tc_hist.cu")
        roof = {"kernel": "k_hist_tc", "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm if achieved else None,
                "traffic": traffic, "traffic_config": traffic_cfg,
                "peak_source": f"measured copy bandwidth ({how})",
                "algorithmic_bytes_per_launch": hbytes, "algorithmic_flops_per_launch": flops,
                "tensor_issued_tflops": tc_flops / (ms_l / 1e3) / 1e12 if ms_l else None,
                "tensor_frac_of_bf16_sustained": tc_flops / (ms_l / 1e3) / 1e12 / bf16 if ms_l and bf16 else None}
    else:
        if kern == 1:
            peak, kname = 70.0, "k_hist_f32"  # FP32 FMA microbenchmark on this pool: 69.8-70.0 TFLOP/s
            psrc = "FP32 CUDA-core FMA rate measured on this pool (152 SMs x 128 lanes x 2 x clock)"
        else:
            peak, kname = 1.25, "k_hist_f64"  # GB300 FP64 nominal; FMA microbenchmark on this pool: 1.198
            psrc = "nominal FP64 rate of the profiling recipe (fp64 ALU bound)"
        achieved = flops / (ms_l / 1e3) / 1e12 if ms_l else None
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None, "peak_source": psrc,
                "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": hbytes}
    roof.update({"launches_timed": hist_launches, "ms_per_launch": ms_l,
                 "share_of_step": ms_l / ms_step if ms_l else None})
    return roof


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    from paper_2510_07989_gb300 import mot as M
    from paper_2510_07989_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    M.load_library()
    ops, _, t_asm = make_workload(args.workload, rank)
    K = ops.kmax + 1
    primary = M.MOT_PREC_MIXED if args.precision == "mixed" else M.MOT_PREC_FP64
    # the pulse (the paper's width, w = 120 c dt) peaks at the scatterer's
    # centre in the middle of the timed window
    n_pre = K + 1 + args.warmup
    # pulse peak at the middle of the device-timed window (after the host-buffer window)
    exc = make_waves(args.workload, rank, n_pre + 1.5 * args.steps)
    B = exc.B
    clocks = Clocks(local)
    clocks.start()  # running before the warm-up, so that it samples the whole timed region
    A = march_arm(M, torch, ops, exc, args, local, world, primary, args.steps, args.warmup, clocks,
                  keep_waves=(0,) if world == 1 and not args.no_cpu_baseline else (),
                  hand_over=primary == M.MOT_PREC_MIXED and args.fp64_steps > 0)
    ck = clocks.stop()
    ms_max, e2e_ms_max = reduce_max([A["ms"], A["e2e_ms"]], world)
    value = throughput(world, B, args.steps, ms_max)
    e2e_value = throughput(world, B, args.steps, e2e_ms_max)
    info0, info1 = A["info0"], A["info1"]
    A.pop("s")  # the mixed handle's device memory is released before the FP64 arm
    # the FP64 plain arm on the same workload and GPU, with the same dense
    # Q_0^{-1} right preconditioner (formed in FP64): the ratio isolates precision
    fp64 = None
    if primary == M.MOT_PREC_MIXED and args.fp64_steps > 0:
        n64 = args.fp64_steps
        # the FP64 arm continues the same march from the mixed arm's state (no
        # prefill of its own); its first step, from that common state, against
        # the mixed arm's step gives the accuracy of one mixed step on the pulse
        F = march_arm(M, torch, ops, exc, args, local, world, M.MOT_PREC_FP64, n64, args.warmup,
                      state_in=A["state"])
        f_ms, f_e2e = reduce_max([F["ms"], F["e2e_ms"]], world)
        fi0, fi1 = F["info0"], F["info1"]
        F.pop("s")
        wm, wf = A["after"], F["first"]
        step_rel = np.linalg.norm(wm - wf, axis=(1, 2)) / np.linalg.norm(wf, axis=(1, 2))
        peak_rel = np.linalg.norm(wm - wf, axis=(1, 2)) / np.maximum(A["peak"], 1e-300)
        fp64 = {"value": throughput(world, B, n64, f_ms), "unit": "RHS·steps/s", "steps": n64,
                "ms_per_step": f_ms / n64, "dtype": "f64",
                "solver": "right-preconditioned GMRES, Q_0 in FP64 product form, M = FP64 dense Q_0^-1",
                "gmres_iters_per_step": (fi1["gmres_iters_total"] - fi0["gmres_iters_total"]) / n64,
                "e2e": {"value": throughput(world, B, n64, f_e2e), "unit": "RHS·steps/s",
                        "h2d_bytes_per_step": 80 * B, "d2h_bytes_per_step": 8 * 2 * ops.ne * B},
                "load_s": round(F["t_load"], 1), "steps_not_converged": F["noconv"],
                "prefill": "none: the mixed arm's march state (mot_save_state / mot_load_state)",
                "mixed_vs_fp64_one_step": {"step": F["info0"]["step"] - n64, "waves": int(wm.shape[0]),
                                           "max_rel_err_2norm": float(step_rel.max()),
                                           "median_rel_err_2norm": float(np.median(step_rel)),
                                           "max_rel_err_vs_wave_peak": float(peak_rel.max()),
                                           "wave_peak": "largest step norm of the wave in the mixed arm's "
                                                        "host-buffer window, which ends at the common state "
                                                        "(on the rising pulse)"},
                "roofline": roofline_of(fi0, fi1, f_ms / n64, n64, args.workload, *measured_peaks())}
        del F
    if rank != 0:
        return
    peaks, how = measured_peaks()
    kern = info1["hist_kernel"]
    roof = roofline_of(info0, info1, ms_max / args.steps, args.steps, args.workload, peaks, how)
    line = {"metric": METRIC, "value": value, "unit": "RHS·steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "ne": ops.ne, "unknowns": 2 * ops.ne, "eps_r": ops.eps_r,
                       "c_dt": ops.dt, "k_max": ops.kmax, "history_lags": K, "rhs_per_step": B,
                       "precision": ("mixed (history on tensor cores: FP32 tiles and coefficients as bf16 x 3, "
                                     "compensated FP32 sums; FP32 dense Q_0 and Q_0^-1, FP64 left factor, "
                                     "FP64 refinement, FP64 CG projector)" if kern == 2 else
                                     "mixed (FP32 history tiles, dense FP32 Q_0 and left factors, FP64 sums, "
                                     "FP64 CG projector)") if args.precision == "mixed" else "fp64 plain",
                       "history_prefill_steps": K + 1,
                       "tc_form": args.tc_form,
                       "tuner": {"chunk_cap": info1["tc_chunk_cap"], "lag_frac": info1["tc_lag_frac"],
                                 "stages": info1["tc_stages"], "tasks_per_stage": info1["tc_tasks_per_stage"],
                                 "epilogue_warps": info1["tc_epilogue_warps"],
                                 "tuned": bool(info1["tc_tuned"]),
                                 "tuned_launch_ms": info1["tc_tune_ms"]},
                       "history_launches_before_timed": info0["tc_launches"],
                       "launches_before_timed": info0["gpu_launches"],
                       "pulse": "paper's Gaussian (w = 120 c dt), peak at the scatterer centre at the middle of "
                                "the device-timed window (t0 = (K + 1 + warmup + 1.5 steps) dt; the host-buffer "
                                "window precedes it)",
                       "load_s": round(A["t_load"], 1),
                       "l2": "inputs larger than L2 (history tiles read per step %.1f GB)" % (
                           info1["tile_count"] * {2: 6144, 1: 4096, 0: 8192}[kern] / 1e9),
                       "assembly_s": round(t_asm, 1), "parallelism": f"replicas{world}",
                       "gmres_iters_per_step": (info1["gmres_iters_total"] - info0["gmres_iters_total"]) / args.steps,
                       "steps_not_converged": A["noconv"],
                       "tile_fill": round(info1["tile_fill"], 3)},
            "clocks": ck,
            "e2e": {"value": e2e_value, "unit": "RHS·steps/s", "h2d_bytes_per_step": 80 * B,
                    "d2h_bytes_per_step": 8 * 2 * ops.ne * B},
            "gpu_launches": (info1["gpu_launches"] - info0["gpu_launches"]),
            "phase_ms_per_step": {name: round((info1["phase_ms"][k] - info0["phase_ms"][k]) / args.steps, 3)
                                  for k, name in enumerate(["rhs", "history", "left_factor", "gmres", "refine",
                                                            "projector_ring", "recover"])},
            "roofline": roof,
            "peaks": {"source": how, "hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops"),
                      "bf16_tflops_sustained": peaks.get("bf16_tflops_sustained")}}
    if fp64 is not None:
        line["fp64"] = fp64
        line["mixed_over_fp64"] = value / fp64["value"]
    if world == 1 and not args.no_cpu_baseline:
        # one oracle step of wave 0 from the GPU's own history: the CPU baseline
        # (timed) and the accuracy of the GPU's last step of the host-buffer window
        hist = A["hist"][0]
        i = A["check_step"]
        w_ref, el, t_setup = oracle_one_step(ops, exc, 0, hist, i)
        w_gpu = hist[i]
        peak = max(np.linalg.norm(w) for w in hist.values())
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        line["cpu_baseline"] = {"value": 1.0 / el, "unit": "RHS·steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"one full-depth MOT step (step {i}) x 1 RHS (wave 0) of the same "
                                          f"workload from the GPU's own history (product-form FP64 oracle; "
                                          f"set-up {t_setup:.0f} s excluded)"}
        line["accuracy"] = {"step": i, "wave": 0, "vs": "product-form FP64 oracle, one step from the GPU history",
                            "rel_err_2norm": float(np.linalg.norm(w_gpu - w_ref) / np.linalg.norm(w_ref)),
                            "rel_err_vs_run_peak": float(np.linalg.norm(w_gpu - w_ref) / peak),
                            "rel_err_max_element": float(np.abs(w_gpu - w_ref).max() / np.abs(w_ref).max()),
                            "step_norm_over_run_peak": float(np.linalg.norm(w_ref) / peak)}
    print(json.dumps(line), flush=True)


UNEVEN_DT = 0.2   # c dt of the uneven batch
UNEVEN_B = 16     # plane waves per scatterer


def run_uneven(args):
    """The uneven batch: 24 scatterers (icospheres L1-L3 and 21 seeded
    ellipsoids of 540-7260 unknowns, eps_r in [1.5, 8]), c dt = 0.2, 16 plane
    waves each, marched together by mot_run_many: one history launch for all
    of them per step (tuned once at full depth), the rest of every step on a
    stream per scatterer. Timing as for one scatterer (host-buffer window,
    then the device-timed window with the pulse at its middle)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    from paper_2510_07989_gb300 import mot as M
    from paper_2510_07989_gb300.build import build
    from paper_2510_07989_gb300.inputs import meshes as MS
    from paper_2510_07989_gb300.inputs.assemble import assemble
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    M.load_library()
    specs = MS.uneven_batch(24, seed=20251007 + 1000 * rank)
    flags = M.MOT_MIX_DEFAULT
    if args.tc_form == "bulk":
        flags |= M.MOT_MIX_TCBULK
    elif args.tc_form == "gathered":
        flags &= ~M.MOT_MIX_TCBULK
    solvers, ops_keep, t_asm, t_load, kmax = [], {}, 0.0, 0.0, 0
    check = (0, max(range(len(specs)), key=lambda i: specs[i][0].ne))  # smallest and largest scatterer
    for i, (mesh, eps) in enumerate(specs):
        t = time.time()
        ops = assemble(mesh, eps, 1.0, UNEVEN_DT, nq=3, ntheta=3, nrad=3, far_plain=6)
        t_asm += time.time() - t
        t = time.time()
        sv = M.Solver(ops, device=local, timing=1, precision=M.MOT_PREC_MIXED, mixed_flags=flags)
        t_load += time.time() - t
        kmax = max(kmax, ops.kmax)
        if i in check:
            ops_keep[i] = ops
        sv.ops = None  # host operators not kept
        solvers.append(sv)
        del ops
    n = len(solvers)
    K = kmax + 1
    n_pre = K + 1 + args.warmup
    excs = []
    for i, (mesh, _) in enumerate(specs):
        r_obj = float(np.linalg.norm(mesh.verts, axis=1).max())
        excs.append(MS.fibonacci_batch(UNEVEN_B, UNEVEN_DT, seed=20251007 + 1000 * rank + i,
                                       t0_steps=n_pre + 1.5 * args.steps, r_obj=r_obj))
    waves = [M.mot_waves(e) for e in excs]
    Bs = [UNEVEN_B] * n
    hs = [s_.h for s_ in solvers]
    stream = torch.cuda.current_stream()
    clocks = Clocks(local)
    clocks.start()
    keep_pre = {i: np.zeros((n_pre, UNEVEN_B, 2, solvers[i].ne)) for i in check}
    M.mot_run_many(hs, n_pre, waves, Bs, [keep_pre.get(i) for i in range(n)], stream)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    outs = [torch.empty((args.steps, UNEVEN_B, 2, sv.ne), dtype=torch.float64).pin_memory() for sv in solvers]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    M.mot_run_many(hs, args.steps, waves, Bs, [o.numpy() for o in outs], stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    info0 = [M.mot_get_info(h) for h in hs]
    barrier()
    torch.cuda.synchronize()
    clocks.begin()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()  # the device-timed window is the profiler's range
    ev0.record(stream)
    M.mot_run_many(hs, args.steps, waves, Bs, None, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clocks.end()
    barrier()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    info1 = [M.mot_get_info(h) for h in hs]
    ms_max, e2e_max = reduce_max([ms, e2e_ms], world)
    units = n * UNEVEN_B
    value = throughput(world, units, args.steps, ms_max)
    if rank != 0:
        return
    peaks, how = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    hl = info1[0]["hist_timed_launches"] - info0[0]["hist_timed_launches"]
    hms = info1[0]["hist_timed_ms"] - info0[0]["hist_timed_ms"]
    ms_l = hms / hl if hl else None
    hbytes = sum(x["hist_bytes_per_step"] for x in info1)
    achieved = hbytes / (ms_l / 1e3) / 1e9 if ms_l else None
    roof = {"kernel": "k_hist_tc (one launch for the 24 scatterers)", "bound": "hbm", "achieved": achieved,
            "peak": hbm, "unit": "GB/s", "frac": achieved / hbm if achieved else None, "traffic": None,
            "peak_source": f"measured copy bandwidth ({how})", "algorithmic_bytes_per_launch": hbytes,
            "launches_timed": hl, "ms_per_launch": ms_l,
            "share_of_step": ms_l / (ms_max / args.steps) if ms_l else None}
    line = {"metric": METRIC, "value": value, "unit": "RHS·steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "uneven24", "scatterers": n, "unknowns": [2 * sv.ne for sv in solvers],
                       "eps_r": [round(e, 3) for _, e in specs], "c_dt": UNEVEN_DT, "rhs_per_scatterer": UNEVEN_B,
                       "history_lags_max": K, "tc_form": args.tc_form,
                       "tuner": {"chunk_cap": info1[0]["tc_chunk_cap"], "lag_frac": info1[0]["tc_lag_frac"],
                                 "stages": info1[0]["tc_stages"], "tasks_per_stage": info1[0]["tc_tasks_per_stage"],
                                 "epilogue_warps": info1[0]["tc_epilogue_warps"],
                                 "tuned": bool(info1[0]["tc_tuned"]),
                                 "tuned_launch_ms": info1[0]["tc_tune_ms"]},
                       "assembly_s": round(t_asm, 1), "load_s": round(t_load, 1),
                       "gmres_iters_per_step": sum(b["gmres_iters_total"] - a["gmres_iters_total"]
                                                   for a, b in zip(info0, info1)) / (n * args.steps),
                       "l2": "inputs larger than L2 (history tiles read per step %.1f GB)" % (
                           sum(x["tile_count"] for x in info1) * 6144 / 1e9),
                       "parallelism": f"replicas{world}"},
            "clocks": ck,
            "e2e": {"value": throughput(world, units, args.steps, e2e_max), "unit": "RHS·steps/s",
                    "h2d_bytes_per_step": 80 * units, "d2h_bytes_per_step": sum(8 * 2 * sv.ne * UNEVEN_B
                                                                                 for sv in solvers)},
            "gpu_launches": sum(b["gpu_launches"] - a["gpu_launches"] for a, b in zip(info0, info1)),
            "roofline": roof,
            "peaks": {"source": how, "hbm_gbs": peaks.get("hbm_gbs")}}
    if world == 1 and not args.no_cpu_baseline:
        acc = []
        el_tot = 0.0
        for i in check:
            hist = {j + 1: keep_pre[i][j, 0].reshape(-1) for j in range(n_pre)}
            hist.update({n_pre + 1 + j: outs[i].numpy()[j, 0].reshape(-1).copy() for j in range(args.steps)})
            c = n_pre + args.steps
            w_ref, el, _ = oracle_one_step(ops_keep[i], excs[i], 0, hist, c)
            el_tot += el
            peak = max(np.linalg.norm(w) for w in hist.values())
            acc.append({"scatterer": i, "unknowns": 2 * solvers[i].ne, "step": c, "wave": 0,
                        "rel_err_2norm": float(np.linalg.norm(hist[c] - w_ref) / np.linalg.norm(w_ref)),
                        "rel_err_vs_run_peak": float(np.linalg.norm(hist[c] - w_ref) / peak)})
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        line["cpu_baseline"] = {"value": len(check) / el_tot, "unit": "RHS·steps/s", "cores": cores,
                                "kind": "oracle", "sample": "one full-depth MOT step x 1 RHS of the smallest and "
                                                            "of the largest scatterer (product-form FP64 oracle, "
                                                            "from the GPU's own history; set-up excluded)"}
        line["accuracy"] = acc
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven24":
        run_uneven(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
