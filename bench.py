"""Benchmark of the fast direct Poisson solver on one GB300 (or N replicas).

Workload: duct Poisson problem 1536 x 512 x 512 (periodic x with Lx = 6,
Neumann y walls with Ly = 2 -> DCT-II, Neumann z walls with Lz = 2 stretched
by tanh(beta = 1.5)); seeded Gaussian right-hand side with its dzf-weighted
mean removed.  One step = one Poisson solve in FP32 with double-float
refinement (the default 2 sweeps; by default the fast mode, whose second
residual is updated in FP32 from the first correction, ``--mode exact`` for
double-float residuals in every sweep) of a resident 3.2 GB FP64 right-hand
side into a resident FP64 solution; the other refinement mode and the plain
FP64 GPU solve are timed beside it, each with its error against the FP64 solve.

Prints one JSON line (rank 0).  Besides the headline it carries the FP64 CPU
oracle timed on a bounded sample of the workload (the 1536 x 512 cross-section
on 16 z cells) with the GPU's error against the oracle's solution of that
sample (``rel_err_vs_oracle``), and the timings of the other workloads
(``configs``: the 64x32x32 and 512x256x192 channels, the 16-domain RK3
substep graph, the differentiable 256x128x128 solve).  ``--impl reference``
times the FP64 CPU oracle on the same sample instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth_inputs as S  # noqa: E402

WORKLOAD = dict(name="duct_poisson_1536x512x512", nx=1536, ny=512, nz=512, bc=(0, 0, 1, 1, 1, 1),
                lx=6.0, ly=2.0, lz=2.0, beta=1.5, seed=3000)
# oracle sample of the same workload for the CPU baseline / reference arm: the
# full 1536 x 512 cross-section (the benchmark's own x and y transform
# kernels) on a thin stretched z; its oracle solution also pins the GPU error
SAMPLE = dict(nx=1536, ny=512, nz=16)
METRIC = "Gpoints/s per Poisson solve (FP32 + double-float refinement, rel err <= 1e-10 vs FP64)"
MODE_TEXT = {
    "fast": "FP32 solves + {s} refinement sweeps: first residual in double-float, later ones updated in FP32 "
            "from the correction (CALES_FP32_REFINE_FAST)",
    "exact": "FP32 solves + {s} refinement sweeps, every residual in double-float (CALES_FP32_REFINE)",
}
UNIT = "Gpoints/s"
# algorithmic bytes per grid point and launch of each kernel (FP32 mode space)
KERNEL_BYTES_PER_POINT = {
    "x_fwd": 12.0,            # read f (FP64 8 B), write 4 B
    "x_fwd_sweep": 8.0,       # read r 4 B, write 4 B
    "y_fwd": 8.0, "y_inv": 8.0, "z_solve": 8.0,
    "x_inv": 12.0,            # read 4 B, write the (hi, lo) pair 8 B
    "x_inv_acc": 20.0,        # read 4 B + pair 8 B, write 8 B (pair update / final FP64)
    "x_inv_acc_d": 24.0,      # the same, and the FP32 correction written (4 B): fast mode
    "residual": 20.0,         # read f 8 B + pair 8 B, write r 4 B
    "residual_update": 12.0,  # read r 4 B + correction 4 B, write r 4 B: fast mode
    "x_fwd_ru": 12.0,         # the last update fused into the x transform: read r 4 B + correction 4 B, write 4 B
}


def kernel_keys(prof):
    """Launch names of one profile, told apart by position: a forward x pass
    after a residual reads the FP32 residual; a pair update followed by a
    residual update also writes the correction."""
    keys = []
    for i, (name, _) in enumerate(prof):
        prev = prof[i - 1][0] if i > 0 else None
        nxt = prof[i + 1][0] if i + 1 < len(prof) else None
        if name == "x_fwd" and prev in ("residual", "residual_update"):
            keys.append("x_fwd_sweep")
        elif name == "x_inv_acc" and nxt in ("residual_update", "x_fwd_ru"):
            keys.append("x_inv_acc_d")
        else:
            keys.append(name)
    return keys


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def grid_arrays(w=WORKLOAD, nx=None, ny=None, nz=None):
    nx, ny, nz = nx or w["nx"], ny or w["ny"], nz or w["nz"]
    zf = S.tanh_faces(nz, w["beta"], w["lz"])
    return nx, ny, nz, zf


def make_rhs(nx, ny, nz, zf, seed):
    f = S.gaussian(seed, (nz, ny, nx))
    return S.remove_mean(f, np.diff(zf))


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a bounded sample per step."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle as O
    nx, ny, nz = SAMPLE["nx"], SAMPLE["ny"], SAMPLE["nz"]
    w = WORKLOAD
    zf = S.tanh_faces(nz, w["beta"], w["lz"])
    dzc, dzf = O.cell_spacings(zf)
    g = O.Grid(nx, ny, nz, w["lx"] / nx, w["ly"] / ny, dzc, dzf, w["bc"])
    f = make_rhs(nx, ny, nz, zf, w["seed"])
    for _ in range(args.warmup):
        O.solve(f, g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.solve(f, g)
    dt = time.perf_counter() - t0
    npts = nx * ny * nz
    val = npts * args.steps / dt / 1e9
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "sample": f"{nx}x{ny}x{nz}"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"FP64 oracle solve of the same duct family at {nx}x{ny}x{nz} per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg():
    """The oracle as it stands, timed on a bounded sample (about 10-30 s of CPU
    work).  Returns the timing record, the sample's right-hand side and the
    oracle's solution of it."""
    import oracle as O
    nx, ny, nz = SAMPLE["nx"], SAMPLE["ny"], SAMPLE["nz"]
    w = WORKLOAD
    zf = S.tanh_faces(nz, w["beta"], w["lz"])
    dzc, dzf = O.cell_spacings(zf)
    g = O.Grid(nx, ny, nz, w["lx"] / nx, w["ly"] / ny, dzc, dzf, w["bc"])
    f = make_rhs(nx, ny, nz, zf, w["seed"])
    p = O.solve(f, g)
    reps, t0 = 0, time.perf_counter()
    while True:
        O.solve(f, g)
        reps += 1
        if time.perf_counter() - t0 > 12.0 or reps >= 200:
            break
    dt = (time.perf_counter() - t0) / reps
    rec = {"value": nx * ny * nz / dt / 1e9, "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
           "kind": "oracle", "sample": f"FP64 oracle solve of the benchmark workload's {nx}x{ny} cross-section "
                                       f"on {nz} stretched z cells, {reps} repetitions ({dt:.2f} s each)"}
    return rec, f, p


def oracle_error(cs, dev, f_s, p_s):
    """Error of the GPU solves of the oracle's sample (the benchmark workload's
    1536 x 512 cross-section on a thin z: the benchmark's x and y kernels)
    against the oracle's solution, relative L2 over all points and the largest
    point error relative to max |p|."""
    import torch
    nx, ny, nz = SAMPLE["nx"], SAMPLE["ny"], SAMPLE["nz"]
    w = WORKLOAD
    zf = S.tanh_faces(nz, w["beta"], w["lz"])
    dzc, dzf = cs.cell_spacings(zf)
    plan = cs.Plan(nx, ny, nz, w["bc"], w["lx"] / nx, w["ly"] / ny, dzc, dzf, cs.FP32_REFINE, 2)
    ref = torch.from_numpy(p_s).to(dev)
    fd = torch.from_numpy(f_s).to(dev)
    out = {"sample": f"{nx}x{ny}x{nz} of the benchmark workload (oracle solution of the cpu_baseline leg)"}
    for mode, name in ((cs.FP32_REFINE, "fp32_refine"), (cs.FP32_REFINE_FAST, "fp32_refine_fast"), (cs.FP64, "fp64"),
                       (cs.FP32, "fp32")):
        plan.set_precision(mode, 2)
        x = fd if mode != cs.FP32 else fd.float()
        p = plan.poisson(x).double()
        d = p - ref
        out[name] = {"rel_l2": float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(ref)),
                     "max_abs_rel": float(d.abs().max() / ref.abs().max())}
    out["device_status"] = plan.status()
    return out


def _event_ms(fn, reps, flush=None):
    """Mean device time of fn over reps calls (CUDA events on the current
    stream, 3 warm-up calls first); with flush, an L2-sized buffer is
    rewritten before every timed call, outside the timed interval."""
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    if flush is None:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in evs:
        flush.add_(1.0)
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / reps


def other_configs(dev):
    """The other workloads of the solver, timed inside the default run (about
    20 s): the 64x32x32 channel (FP64; warm L2 and L2 flushed), the
    512x256x192 channel (FP64, FP32, FP32 + refinement; right-hand side = the
    discrete divergence of a seeded Gaussian velocity), the RK3 substep of 16
    uneven channel domains in one CUDA graph (FP32 + refinement; warm and
    flushed) and the differentiable 256x128x128 solve (FP32 forward +
    backward)."""
    import torch
    from paper_2411_09364_gb300 import autograd as AG
    from paper_2411_09364_gb300 import batch as B
    from paper_2411_09364_gb300 import solver as cs
    hbm = peaks()[0]
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)      # 256 MB > L2 (129 MB)
    res = {}
    # channel 64x32x32, P,P,N, uniform z, FP64 (fits L2: latency-bound)
    plan = cs.channel_plan(64, 32, 32, beta=0.0)
    f = torch.from_numpy(S.remove_mean(S.uniform(1000, (32, 32, 64)))).to(dev)
    p = torch.empty_like(f)
    warm = _event_ms(lambda: plan.poisson(f, p), 200)
    cold = _event_ms(lambda: plan.poisson(f, p), 50, flush)
    res["channel_poisson_64x32x32"] = {"mode": "fp64", "ms_warm_l2": warm, "ms_l2_flushed": cold,
                                       "solves_per_s_warm_l2": 1e3 / warm,
                                       "gpoints_per_s_warm_l2": f.numel() / warm / 1e6,
                                       "gpoints_per_s_l2_flushed": f.numel() / cold / 1e6}
    del plan
    # channel 512x256x192, P,P,N, tanh 1.8, f = div of a Gaussian staggered velocity (walls w = 0)
    nx, ny, nz = 512, 256, 192
    plan = cs.channel_plan(nx, ny, nz, beta=1.8)
    u, v, w = (torch.from_numpy(a).to(dev) for a in S.velocity_field(2000, nx, ny, nz))
    f64 = AG.divergence(plan, u, v, w)
    del u, v, w
    ch = {"rhs": "discrete divergence of a seeded Gaussian staggered velocity (sigma 1, w = 0 on the walls)",
          "l2": "f and p 201 MB (FP64) each, larger than L2"}
    p64 = None
    for mode, name in ((cs.FP64, "fp64"), (cs.FP32, "fp32"), (cs.FP32_REFINE, "fp32_refine")):
        plan.set_precision(mode, 2)
        fi = f64 if mode != cs.FP32 else f64.float()
        po = torch.empty_like(fi)
        ms = _event_ms(lambda: plan.poisson(fi, po), 20)
        if mode == cs.FP64:
            p64 = po.clone()
        rel = float(torch.linalg.vector_norm(po.double() - p64) / torch.linalg.vector_norm(p64))
        ch[name] = {"ms": ms, "gpoints_per_s": fi.numel() / ms / 1e6, "solves_per_s": 1e3 / ms,
                    "rel_err_vs_fp64_gpu": rel,
                    "min_traffic_roofline_frac": (fi.numel() * 2 * fi.element_size() / (ms * 1e-3) / 1e9) / hbm}
    res["channel_poisson_512x256x192"] = ch
    del plan, f64, p64, fi, po
    # 16 channel domains x {u, v, w Helmholtz, p Poisson}, FP32 + refinement, one CUDA graph
    alphas = [1e-4 if d % 2 == 0 else 1e-3 for d in range(len(S.BATCH_DOMAINS))]
    batch, plans, tags = B.rk3_substep_batch(S.BATCH_DOMAINS, alphas)
    fs = [torch.from_numpy(S.gaussian(4000 + i, pl.shape)).to(dev) for i, pl in enumerate(plans)]
    us = [torch.empty_like(x) for x in fs]
    st = batch.capture(fs, us)
    with torch.cuda.stream(st):
        warm = _event_ms(lambda: batch.launch(st), 10)
        cold = _event_ms(lambda: batch.launch(st), 10, flush)
    pts = sum(pl.numel for pl in plans)
    res["rk3_substep_16_channel_domains"] = {
        "mode": "fp32_refine", "solves": len(plans), "graph_nodes": batch.graph_nodes(),
        "ms_warm_l2": warm, "ms_l2_flushed": cold, "gpoint_solves_per_s_warm_l2": pts / warm / 1e6,
        "gpoint_solves_per_s_l2_flushed": pts / cold / 1e6,
        "l2": "inputs 1.76 GB in total (the small domains fit L2)"}
    del batch, plans, fs, us
    # differentiable 256x128x128 solve, FP32, forward + backward through the adjoint kernel
    plan = cs.channel_plan(256, 128, 128, beta=1.8, precision=cs.FP32)
    fd = torch.from_numpy(S.gaussian(5000, (128, 128, 256))).to(dev, torch.float32).requires_grad_(True)
    wd = torch.from_numpy(S.gaussian(5001, (128, 128, 256))).to(dev, torch.float32)

    def fwd_bwd():
        fd.grad = None
        (wd * AG.poisson_solve(fd, plan)).sum().backward()
    ms = _event_ms(fwd_bwd, 20)
    res["differentiable_poisson_256x128x128"] = {"mode": "fp32 forward+backward", "ms": ms,
                                                 "gpoints_per_s": fd.numel() / ms / 1e6}
    del plan, fd, wd, flush
    torch.cuda.empty_cache()
    return res


def run_configs(args):
    """Timings of the other workloads of the solver (one JSON line each): the
    small channel (L2-resident), the 512x256x192 channel in FP64 / FP32 /
    FP32 + refinement, the 16-domain RK3 substep graph and the differentiable
    256x128x128 solve (forward + backward).  Not the headline line."""
    import torch
    from paper_2411_09364_gb300 import autograd as AG
    from paper_2411_09364_gb300 import batch as B
    from paper_2411_09364_gb300 import solver as cs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def emit(d):
        print(json.dumps(d), flush=True)

    def want(tag):
        return args.only is None or args.only in tag

    # the bench grid (or --shape) for the line solves and the eddy viscosity
    wl = dict(WORKLOAD)
    if args.shape:
        sx, sy, sz = (int(v) for v in args.shape.split(","))
        wl.update(nx=sx, ny=sy, nz=sz, lx=wl["lx"] * sx / wl["nx"], ly=wl["ly"] * sy / wl["ny"])

    if want("channel_poisson_64x32x32"):
        # channel 64x32x32, P,P,N, uniform z, FP64: fits L2, latency-bound
        plan = cs.channel_plan(64, 32, 32, beta=0.0)
        f = torch.from_numpy(S.gaussian(1000, (32, 32, 64))).to(dev)
        p = torch.empty_like(f)
        ms = timed(lambda: plan.poisson(f, p), 200)
        emit({"workload": "channel_poisson_64x32x32", "mode": "fp64", "ms": ms, "solves_per_s": 1e3 / ms,
              "gpoints_per_s": f.numel() / ms / 1e6, "l2": "fits L2 (warm)"})
    if want("channel_poisson_512x256x192"):
        # channel 512x256x192, P,P,N, tanh beta = 1.8
        plan = cs.channel_plan(512, 256, 192, beta=1.8)
        f64 = torch.from_numpy(S.gaussian(2000, (192, 256, 512))).to(dev)
        out = {}
        for mode, name in ((cs.FP64, "fp64"), (cs.FP32, "fp32"), (cs.FP32_REFINE, "fp32_refine")):
            plan.set_precision(mode, 2)
            fi = f64 if mode != cs.FP32 else f64.float()
            po = torch.empty_like(fi)
            ms = timed(lambda: plan.poisson(fi, po), 20)
            out[name] = po.double()
            rel = (float(torch.linalg.vector_norm(out[name] - out["fp64"]) / torch.linalg.vector_norm(out["fp64"]))
                   if name != "fp64" else 0.0)
            emit({"workload": "channel_poisson_512x256x192", "mode": name, "ms": ms,
                  "gpoints_per_s": fi.numel() / ms / 1e6, "rel_err_vs_fp64_gpu": rel,
                  "min_traffic_roofline_frac": (fi.numel() * 2 * fi.element_size() / (ms * 1e-3) / 1e9) / peaks()[0]})
    if want("rk3_substep"):
        # 16 channel domains x {u, v, w Helmholtz, p Poisson}, FP32 + refinement, one CUDA graph
        # (--no-autotune keeps the default schedules; --warmup / --steps graph replays)
        alphas = [1e-4 if d % 2 == 0 else 1e-3 for d in range(len(S.BATCH_DOMAINS))]
        batch, plans, tags = B.rk3_substep_batch(S.BATCH_DOMAINS, alphas, autotune=not args.no_autotune)
        fs = [torch.from_numpy(S.gaussian(4000 + i, pl.shape)).to(dev) for i, pl in enumerate(plans)]
        us = [torch.empty_like(x) for x in fs]
        st = batch.capture(fs, us)
        for _ in range(args.warmup):
            batch.launch(st)
        st.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(args.steps):
            batch.launch(st)
        b.record(st)
        st.synchronize()
        ms = a.elapsed_time(b) / args.steps
        pts = sum(pl.numel for pl in plans)
        emit({"workload": "rk3_substep_16_channel_domains", "mode": "fp32_refine", "ms": ms,
              "gpoint_solves_per_s": pts / ms / 1e6, "solves": len(plans), "graph_nodes": batch.graph_nodes(),
              "grouped": batch.grouped(), "autotuned": not args.no_autotune})
    if want("z_line_helmholtz"):
        # wall-normal implicit line solves (Eq. 21) on the bench grid, Dirichlet walls
        w = wl
        zf = S.tanh_faces(w["nz"], w["beta"], w["lz"])
        dzc, dzf = cs.cell_spacings(zf)
        plan = cs.Plan(w["nx"], w["ny"], w["nz"], (0, 0, 1, 1, 2, 2), w["lx"] / w["nx"], w["ly"] / w["ny"], dzc, dzf,
                       cs.FP64)
        fz = torch.from_numpy(make_rhs(w["nx"], w["ny"], w["nz"], zf, w["seed"])).to(dev)
        for mode, name in ((cs.FP64, "fp64"), (cs.FP32, "fp32")):
            plan.set_precision(mode)
            fi = fz if mode == cs.FP64 else fz.float()
            uo = torch.empty_like(fi)
            ms = timed(lambda: plan.helmholtz_z(1e-4, fi, uo), 10)
            emit({"workload": f"z_line_helmholtz_{w['nx']}x{w['ny']}x{w['nz']}", "mode": name, "ms": ms,
                  "gpoints_per_s": fi.numel() / ms / 1e6,
                  "hbm_frac": (fi.numel() * 2 * fi.element_size() / (ms * 1e-3) / 1e9) / peaks()[0]})
        del fz, plan
        torch.cuda.empty_cache()
    if want("eddy_viscosity"):
        # Smagorinsky / van Driest eddy viscosity (Eq. 4) on a channel of the bench size
        w = wl
        zf = S.tanh_faces(w["nz"], w["beta"], w["lz"])
        dzc, dzf = cs.cell_spacings(zf)
        plan = cs.Plan(w["nx"], w["ny"], w["nz"], (0, 0, 0, 0, 1, 1), w["lx"] / w["nx"], w["ly"] / w["ny"], dzc, dzf,
                       cs.FP64)
        shp = (w["nz"], w["ny"], w["nx"])
        for mode, name in ((cs.FP32, "fp32"), (cs.FP64, "fp64")):
            plan.set_precision(mode)
            dt = torch.float32 if mode == cs.FP32 else torch.float64
            uu = torch.from_numpy(S.gaussian(6000, shp)).to(dev, dt)
            vv = torch.from_numpy(S.gaussian(6001, shp)).to(dev, dt)
            ww = torch.from_numpy(S.gaussian(6002, (w["nz"] + 1, w["ny"], w["nx"]))).to(dev, dt)
            ww[0].zero_()
            ww[-1].zero_()
            nt = torch.empty_like(uu)
            ms = timed(lambda: plan.eddy_viscosity(0.1, 1e-4, 0.05, uu, vv, ww, nt), 10)
            emit({"workload": f"eddy_viscosity_{w['nx']}x{w['ny']}x{w['nz']}", "mode": name, "ms": ms,
                  "gpoints_per_s": uu.numel() / ms / 1e6,
                  "hbm_frac": (uu.numel() * 4 * uu.element_size() / (ms * 1e-3) / 1e9) / peaks()[0]})
            del uu, vv, ww, nt
        del plan
        torch.cuda.empty_cache()
    if want("rk3_step_channel"):
        # one explicit RK3 time step (three substeps of Eqs. 11-14, each with the
        # eddy viscosity of Eq. 4) on the bench grid as a channel; seeded
        # Gaussian velocity and pressure drawn on the device
        w = wl
        zf = S.tanh_faces(w["nz"], w["beta"], w["lz"])
        dzc, dzf = cs.cell_spacings(zf)
        plan = cs.Plan(w["nx"], w["ny"], w["nz"], (0, 0, 0, 0, 1, 1), w["lx"] / w["nx"], w["ly"] / w["ny"], dzc,
                       dzf, cs.FP32)
        shp, shw = (w["nz"], w["ny"], w["nx"]), (w["nz"] + 1, w["ny"], w["nx"])
        vel = {}
        for mode, implicit, name in ((cs.FP32, 0, "fp32"), (cs.FP32_REFINE, 0, "fp32_refine"),
                                     (cs.FP32, 1, "fp32 cn-3d (Eqs. 17-19)"), (cs.FP32, 2, "fp32 cn-z (Eqs. 20-22)")):
            plan.set_precision(mode, 2)
            if implicit and not vel:
                vel["uv"], vel["w"] = cs.channel_velocity_plans(w["nx"], w["ny"], zf, w["lx"] / w["nx"],
                                                                w["ly"] / w["ny"], cs.FP32)
            dt = torch.float32 if mode == cs.FP32 else torch.float64
            gen = torch.Generator(device=dev)
            gen.manual_seed(7000)
            uu, vv, pp = (torch.randn(shp, generator=gen, device=dev, dtype=dt) for _ in range(3))
            ww = torch.randn(shw, generator=gen, device=dev, dtype=dt)
            ww[0].zero_()
            ww[-1].zero_()
            nut = plan.eddy_viscosity(0.1, 1e-4, 0.05, uu, vv, ww)
            ru, rv, rw = torch.zeros_like(uu), torch.zeros_like(uu), torch.zeros_like(ww)
            work = plan.rk3_work(dev)

            def rk3_step():
                for s in range(3):
                    if implicit:
                        plan.rk3_substep_cn(vel["uv"], vel["w"], implicit, s, 2e-4, 1e-4, 0.1, 0.05, uu, vv, ww, pp,
                                            nut, ru, rv, rw, work)
                    else:
                        plan.rk3_substep(s, 2e-4, 1e-4, 0.1, 0.05, uu, vv, ww, pp, nut, ru, rv, rw, work)
            ms = timed(rk3_step, 3)
            emit({"workload": f"rk3_step_channel_{w['nx']}x{w['ny']}x{w['nz']}", "mode": name, "ms": ms,
                  "ms_per_substep": ms / 3, "gpoints_per_s": uu.numel() / ms / 1e6,
                  "finite": bool(torch.isfinite(uu).all().item())})
            del uu, vv, ww, pp, nut, ru, rv, rw, work
        del plan, vel
        torch.cuda.empty_cache()
    if want("periodic_z_poisson"):
        # fully periodic box (x, y, z periodic; cyclic tridiagonal per mode), 512x256x256,
        # stretched z with the wrap distance joining the last and the first cell centre
        nx_, ny_, nz_ = 512, 256, 256
        zf = S.tanh_faces(nz_, 1.5, 2.0)
        dzc, dzf = cs.cell_spacings(zf)
        dzc = np.array(dzc)
        dzc[0] = dzc[-1] = 0.5 * (dzf[0] + dzf[-1])
        plan = cs.Plan(nx_, ny_, nz_, (0, 0, 0, 0, 0, 0), 2 * math.pi / nx_, math.pi / ny_, dzc, dzf, cs.FP64)
        fp = torch.from_numpy(S.gaussian(8000, (nz_, ny_, nx_))).to(dev)
        for mode, name in ((cs.FP64, "fp64"), (cs.FP32, "fp32")):
            plan.set_precision(mode)
            fi = fp if mode == cs.FP64 else fp.float()
            po = torch.empty_like(fi)
            ms = timed(lambda: plan.poisson(fi, po), 10)
            emit({"workload": f"periodic_z_poisson_{nx_}x{ny_}x{nz_}", "mode": name, "ms": ms,
                  "gpoints_per_s": fi.numel() / ms / 1e6})
        del plan, fp
        torch.cuda.empty_cache()
    if want("differentiable_poisson"):
        # differentiable 256x128x128 solve, FP32, forward + backward through the adjoint kernel
        plan = cs.channel_plan(256, 128, 128, beta=1.8, precision=cs.FP32)
        fd = torch.from_numpy(S.gaussian(5000, (128, 128, 256))).to(dev, torch.float32).requires_grad_(True)
        wd = torch.from_numpy(S.gaussian(5001, (128, 128, 256))).to(dev, torch.float32)

        def fwd_bwd():
            fd.grad = None
            (wd * AG.poisson_solve(fd, plan)).sum().backward()
        ms = timed(fwd_bwd, 20)
        emit({"workload": "differentiable_poisson_256x128x128", "mode": "fp32 forward+backward", "ms": ms,
              "gpoints_per_s": fd.numel() / ms / 1e6})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cales", choices=["cales", "reference"])
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--mode", default="fast", choices=["fast", "exact"],
                    help="refinement mode of the headline: fast = first residual double-float, later ones "
                         "updated in FP32; exact = every residual double-float")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the timings of the other workloads")
    ap.add_argument("--small", action="store_true", help="512x256x192 channel variant (profiling)")
    ap.add_argument("--shape", default=None, help="NX,NY,NZ: the duct at another size (profiling case)")
    ap.add_argument("--configs", action="store_true", help="time the other workloads (one JSON line each)")
    ap.add_argument("--only", default=None, help="with --configs: only the workloads whose name contains this")
    ap.add_argument("--no-autotune", action="store_true", help="with --configs: default schedules for the batch")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.configs:
        return run_configs(args)

    import torch
    import torch.distributed as dist

    from paper_2411_09364_gb300.replicas import dist_env
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo",
                                init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2411_09364_gb300 import solver as cs

    w = dict(WORKLOAD)
    if args.small:
        w.update(name="channel_poisson_512x256x192", nx=512, ny=256, nz=192, bc=(0, 0, 0, 0, 1, 1),
                 lx=2 * math.pi, ly=math.pi, beta=1.8)
    if args.shape:
        sx, sy, sz = (int(v) for v in args.shape.split(","))
        w.update(name=f"duct_poisson_{sx}x{sy}x{sz}", nx=sx, ny=sy, nz=sz,
                 lx=w["lx"] * sx / w["nx"], ly=w["ly"] * sy / w["ny"])
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    npts = nx * ny * nz
    zf = S.tanh_faces(nz, w["beta"], w["lz"])
    dzc, dzf = cs.cell_spacings(zf)
    head_mode = cs.FP32_REFINE_FAST if args.mode == "fast" else cs.FP32_REFINE
    other_mode = cs.FP32_REFINE if args.mode == "fast" else cs.FP32_REFINE_FAST
    plan = cs.Plan(nx, ny, nz, w["bc"], w["lx"] / nx, w["ly"] / ny, dzc, dzf, head_mode, args.sweeps)
    f_host = torch.from_numpy(make_rhs(nx, ny, nz, zf, w["seed"] + rank))
    f = f_host.to(dev)
    p = torch.empty_like(f)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # --- device-resident timing (FP32 + refinement) --------------------------
    for _ in range(args.warmup):
        plan.poisson(f, p)
    plan.profile(True)
    barrier()
    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.poisson(f, p)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    prof = plan.profile_read()
    plan.profile(False)
    p_ref = p.clone()

    # --- per-kernel breakdown and roofline of the dominant kernel ------------
    tot, cnt = {}, {}
    for key, (name, t) in zip(kernel_keys(prof), prof):
        tot[key] = tot.get(key, 0.0) + t
        cnt[key] = cnt.get(key, 0) + 1
    launches_per_step = len(prof) / args.steps if prof else 0
    dom = max(tot, key=tot.get) if tot else None
    hbm, src = peaks()
    roof = None
    if dom:
        avg_ms = tot[dom] / cnt[dom]
        bytes_per_launch = KERNEL_BYTES_PER_POINT.get(dom, 8.0) * npts
        ach = bytes_per_launch / (avg_ms * 1e-3) / 1e9
        traffic = None
        try:
            with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
                traffic = json.load(fh).get(w["name"], {}).get(dom)
        except Exception:
            traffic = None
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "peak_source": src,
                "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
                "bytes_per_launch": bytes_per_launch, "avg_ms": avg_ms}
    per_kernel = {k: {"ms_per_step": tot[k] / args.steps, "launches_per_step": cnt[k] / args.steps,
                      "GB/s": KERNEL_BYTES_PER_POINT.get(k, 8.0) * npts / (tot[k] / cnt[k] * 1e-3) / 1e9}
                  for k in tot}

    # --- plain FP64 GPU solve beside it --------------------------------------
    plan.set_precision(cs.FP64)
    p64 = torch.empty_like(f)
    plan.poisson(f, p64)
    barrier()
    ev0.record(stream)
    for _ in range(args.fp64_steps):
        plan.poisson(f, p64)
    ev1.record(stream)
    barrier()
    ms64 = max_over_ranks(ev0.elapsed_time(ev1) / args.fp64_steps)
    rel = float(torch.linalg.vector_norm(p_ref - p64) / torch.linalg.vector_norm(p64))

    # --- the other refinement mode beside it ---------------------------------
    plan.set_precision(other_mode, args.sweeps)
    pf = torch.empty_like(f)
    for _ in range(args.warmup):
        plan.poisson(f, pf)
    plan.profile(True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        plan.poisson(f, pf)
    ev1.record(stream)
    barrier()
    ms_fast = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    prof_fast = plan.profile_read()
    plan.profile(False)
    per_kernel_fast = {}
    for name, t in prof_fast:
        per_kernel_fast[name] = per_kernel_fast.get(name, 0.0) + t / args.steps
    rel_fast = float(torch.linalg.vector_norm(pf - p64) / torch.linalg.vector_norm(p64))
    del pf
    plan.set_precision(head_mode, args.sweeps)

    # --- end to end through the C ABI with host buffers ----------------------
    # Every step copies its right-hand side from pinned host memory, solves and
    # copies the solution back.  NB device buffer sets rotate so the copies of
    # one step overlap the solves of the others (copy engines vs SMs); with
    # three sets the device-to-host copy of step i and the host-to-device copy
    # of step i + NB need not finish before the next solve starts.
    NB = 3
    f_pin = f_host.pin_memory()
    p_pins = [torch.empty_like(f_pin).pin_memory() for _ in range(NB)]
    fds = [torch.empty_like(f) for _ in range(NB)]
    pds = [torch.empty_like(f) for _ in range(NB)]
    h2d = torch.cuda.Stream(dev)
    d2h = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(NB)]
    solved = [torch.cuda.Event() for _ in range(NB)]
    freed = [torch.cuda.Event() for _ in range(NB)]
    for b in range(NB):
        freed[b].record(d2h)

    def e2e_step(i):
        b = i % NB
        h2d.wait_event(freed[b])
        with torch.cuda.stream(h2d):
            fds[b].copy_(f_pin, non_blocking=True)
        copied[b].record(h2d)
        stream.wait_event(copied[b])
        plan.poisson(fds[b], pds[b], stream=stream)
        solved[b].record(stream)
        d2h.wait_event(solved[b])
        with torch.cuda.stream(d2h):
            p_pins[b].copy_(pds[b], non_blocking=True)
        freed[b].record(d2h)

    for i in range(NB):
        e2e_step(i)
    barrier()
    torch.cuda.synchronize(dev)
    e2e_steps = max(NB, min(args.steps, 9))
    ev0.record(stream)
    h2d.wait_event(ev0)
    for i in range(e2e_steps):
        e2e_step(i)
    stream.wait_stream(d2h)
    ev1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(ev0.elapsed_time(ev1) / e2e_steps)
    status = plan.status()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": npts * world / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "nx": nx, "ny": ny, "nz": nz, "bc": "P x, N y (DCT-II), N z tanh",
                   "precision": MODE_TEXT[args.mode].format(s=args.sweeps),
                   "l2": f"inputs larger than L2 (f and p {npts * 8 / 1e9:.1f} GB each), no flush needed",
                   "parallelism": f"replicas x{world}"},
        "fp64": {"value": npts * world / (ms64 * 1e-3) / 1e9, "ms_per_step": ms64, "unit": UNIT},
        ("fp32_refine_exact_residuals" if args.mode == "fast" else "fp32_refine_fast"): {
            "value": npts * world / (ms_fast * 1e-3) / 1e9, "ms_per_step": ms_fast, "unit": UNIT,
            "rel_err_vs_fp64_gpu": rel_fast, "per_kernel_ms_per_step": per_kernel_fast,
            "mode": MODE_TEXT["exact" if args.mode == "fast" else "fast"].format(s=args.sweeps)},
        "rel_err_refine_vs_fp64_gpu": rel,
        "device_status": status,
        "e2e": {"value": npts * world / (ms_e2e * 1e-3) / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": f.numel() * 8, "d2h_bytes_per_step": p.numel() * 8},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "roofline": roof,
        "per_kernel": per_kernel,
        "min_traffic_roofline_frac": (16.0 * npts / (ms * 1e-3) / 1e9) / hbm,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        rec, f_s, p_s = cpu_baseline_leg()
        line["cpu_baseline"] = rec
        line["rel_err_vs_oracle"] = oracle_error(cs, dev, f_s, p_s)
    if not args.no_configs:
        line["configs"] = other_configs(dev)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
