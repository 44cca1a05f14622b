#!/usr/bin/env python
"""Benchmark: SAP-preconditioned FGMRES time-to-solution for the
Wilson-clover Dirac equation on one GB300 (arXiv:1502.04025, Sec. 3).

Workload (one step = one complete solve to a true FP64 relative residual of
1e-10): 16^3x32 lattice, seeded SU(3) links U = exp(i 0.5 H), c_sw 1.0,
kappa 0.125, 8x4x4x4 domains, FP32 Schwarz preconditioner (nmr 4, ncy 4) on
FP32 storage, FP64 FGMRES(16), one Gaussian source.  Inputs are resident in
HBM when the timed region starts; L2 is flushed (256 MB write) before every
step.  The same solve through the C ABI with host buffers gives "e2e".

--impl reference times the FP64 CPU reference checker (oracle/) on a bounded
sample of the same workload (one FGMRES iteration per step) and scales it to
a time-to-solution with the iteration count the checker needs on this
workload (oracle/iterations_16c32.json, written by oracle/measure_iterations.py).

Under torchrun (--gpus N) every rank solves its own copy of the workload
(replicas; the solver has no multi-GPU path), the timed region is bracketed
by barriers, and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WL = dict(L=(16, 16, 16, 32), dom=(8, 4, 4, 4), eps=0.5, csw=1.0, kappa=0.125, gauge_seed=1002, source_seed=2002,
          nmr=4, ncy=4, m=16, tol=1e-10, sap_prec="f32", arnoldi_prec="f64")
# full-lattice operator throughput: a lattice larger than L2 (32^3x64, eps 0.7, c_sw 1.5, kappa 0.1355)
DSL = dict(L=(32, 32, 32, 64), dom=(4, 4, 4, 4), eps=0.7, csw=1.5, kappa=0.1355, gauge_seed=1003, source_seed=2003)
METRIC = "SAP-FGMRES time-to-1e-10 residual"
WORKLOAD_NAME = ("16^3x32 Wilson-clover, c_sw 1.0, kappa 0.125, eps 0.5 links; SAP-FGMRES(16), 8x4x4x4 domains, "
                 "nmr 4, ncy 4, FP32 preconditioner, FP64 outer, tol 1e-10, 1 Gaussian source")
SAP_FLOP = {"hop": 1320, "clover": 504, "combine": 24, "mr_blas": 336, "boundary_hop": 168}
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["qdd", "reference"], default="qdd")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dslash", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def crossing_hops_per_site(dom):
    """Average number of hops per site that leave a domain: 2 faces per
    direction, each holding Vd/dom[mu] sites."""
    vd = float(np.prod(dom))
    return sum(2 * vd / d for d in dom) / vd


def sap_flop_per_site(dom, nmr):
    """Algorithmic FP32 flop per site of one domain visit of the Schwarz
    kernel, counted as for the operator (1848 per full site apply):
      setup   t_o = A^-1 rho_o (504 per odd site), bhat_e (hops + combine per even site)
      MR      per step: odd site t = A^-1(-k H r) 1848, even site p = A r + k H t 1848,
              dots and updates 336 per even site
      recon   odd site x_o = A^-1(rho_o + k H x_e) 1848
      inflow  168 per hop entering from a neighbouring domain."""
    f = SAP_FLOP
    full = f["hop"] + f["clover"] + f["combine"]
    per_pair = (f["clover"] + f["hop"] + f["combine"]) + nmr * (2 * full + f["mr_blas"]) + full
    return per_pair / 2 + crossing_hops_per_site(dom) * f["boundary_hop"]


# ------------------------------------------------------------------ clocks

class Clocks:
    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- oracle leg

def oracle_sample(w, U=None):
    """Time a bounded sample of the FP64 oracle on the workload: FGMRES with
    one and with two Arnoldi steps, giving the cost per step and the fixed
    cost; scaled to a solve with the oracle's own iteration count."""
    from oracle import pyoracle as ora
    from paper_1502_04025_gb300 import inputs

    with open(os.path.join(ROOT, "oracle", "iterations_16c32.json")) as f:
        it = json.load(f)
    if U is None:
        U = inputs.gauge_field(w["L"], w["eps"], w["gauge_seed"])
    b = inputs.gaussian_source(w["L"], w["source_seed"])
    A = ora.clover(w["L"], U, w["csw"], w["kappa"])
    Ainv = ora.invert_clover(w["L"], A)
    times = []
    for m in (1, 2):
        t0 = time.perf_counter()
        ora.fgmres(w["L"], w["dom"], U, A, Ainv, w["kappa"], b, 1e-30, m=m, max_restarts=0, use_sap=True,
                   nmr=w["nmr"], ncy=w["ncy"])
        times.append(time.perf_counter() - t0)
    per_iter = max(times[1] - times[0], 0.0)
    fixed = max(times[0] - per_iter, 0.0)  # initial and final residual (two operator applies)
    est_s = fixed * (1 + it["restarts"]) + per_iter * it["iterations"]
    return {"value": est_s * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle FGMRES with 1 and 2 Arnoldi steps on the full 16^3x32 workload "
                       f"({times[0]:.1f} s, {times[1]:.1f} s), scaled to its {it['iterations']} iterations and "
                       f"{it['restarts']} restarts to 1e-10")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1502_04025_gb300 import inputs

    U = inputs.gauge_field(WL["L"], WL["eps"], WL["gauge_seed"])
    vals = []
    samples = []
    for k in range(args.warmup + args.steps):
        s = oracle_sample(WL, U)
        if k >= args.warmup:
            vals.append(s["value"])
            samples.append(s)
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "lattice": list(WL["L"]), "domain": list(WL["dom"])},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle", "sample": samples[-1]["sample"]},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg

def run_qdd(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1502_04025_gb300 import build, inputs

    build.build()
    from paper_1502_04025_gb300 import qdd

    pk, pk_kind = peaks()
    ctx = qdd.qdd_create(local, 0)
    U = inputs.gauge_field(WL["L"], WL["eps"], WL["gauge_seed"])
    b = inputs.gaussian_source(WL["L"], WL["source_seed"])
    g = qdd.qdd_create_gauge_field(ctx, WL["L"], WL["dom"], U)
    qdd.qdd_set_clover(g, WL["csw"], WL["kappa"])
    params = qdd.qdd_default_params(tol=WL["tol"], restart_m=WL["m"], nmr=WL["nmr"], ncy=WL["ncy"],
                                    sap_prec=WL["sap_prec"], arnoldi_prec=WL["arnoldi_prec"], max_restarts=50)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    rep = None
    # per-launch CUDA events on the Schwarz kernel (the dominant class); the
    # event pool is created here, before the timed region
    qdd.qdd_set_profiling(ctx, qdd.QDD_PROF_SAP)
    clocks = Clocks(local)
    clocks.start()  # the clock sampler starts during warm-up, before the timed region
    for _ in range(args.warmup):
        flush.fill_(1.0)
        _, rep = qdd.qdd_solve(g, bd, params, x=xd)
    torch.cuda.synchronize()

    # ---- timed region: K solves, inputs resident, L2 flushed before each
    qdd.qdd_get_kernel_times(ctx, reset=True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        _, rep = qdd.qdd_solve(g, bd, params, x=xd)
        reps.append(rep)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    kt = qdd.qdd_get_kernel_times(ctx, reset=True)
    qdd.qdd_set_profiling(ctx, 0)
    ms_step = ms_total / args.steps
    if dist is not None:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    launches = int(sum(r["kernel_launches"] for r in reps))

    # ---- kernel-class shares from one extra solve with every class event-timed
    qdd.qdd_set_profiling(ctx, qdd.QDD_PROF_ALL)
    qdd.qdd_get_kernel_times(ctx, reset=True)
    flush.fill_(1.0)
    qdd.qdd_solve(g, bd, params, x=xd)
    shares = qdd.qdd_get_kernel_times(ctx, reset=True)
    qdd.qdd_set_profiling(ctx, 0)

    # ---- roofline of the dominant kernel class (timed inside the timed region)
    classes = {k: v for k, v in shares.items() if v[1] > 0}
    dom_cls = max(classes, key=lambda k: classes[k][0])
    V = int(np.prod(WL["L"]))
    Vd = int(np.prod(WL["dom"]))
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = sm_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # TFLOP/s
    # per-launch time from the timed region when that class was event-timed there
    kt = kt if kt[dom_cls][0] > 0 else shares
    if dom_cls == "sap":
        ms_launch = kt["sap"][0] / kt["sap"][1]
        flop = (V // 2) * sap_flop_per_site(WL["dom"], WL["nmr"])
        achieved = flop / (ms_launch * 1e-3) / 1e12
        roof = {"kernel": "k_sap (Schwarz colour half-sweep, FP32)", "bound": "alu", "achieved": achieved,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                "ms_per_launch": ms_launch, "launches": kt["sap"][1],
                "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 flop x {pk.get('sm_max_mhz', 2070.0):.0f} MHz"}
    elif dom_cls == "dslash":
        ms_launch = kt["dslash"][0] / kt["dslash"][1]
        bytes_site = 576 + 576 + 96 + 192  # FP64 links + clover, FP32 input, FP64 output
        achieved = V * bytes_site / (ms_launch * 1e-3) / 1e9
        roof = {"kernel": "k_dslash (FP64 operator in the Arnoldi step)", "bound": "hbm", "achieved": achieved,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": None,
                "ms_per_launch": ms_launch, "launches": kt["dslash"][1]}
    else:
        ms_launch = kt["blas"][0] / kt["blas"][1]
        roof = {"kernel": "FP64 vector kernels", "bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": None, "traffic": None, "ms_per_launch": ms_launch,
                "launches": kt["blas"][1]}
    roof["peak_kind"] = "of measured" if pk_kind == "measured" else "of fallback"
    roof["class_ms_one_solve"] = {k: round(v[0], 4) for k, v in shares.items()}

    # ---- end to end through the C ABI with host buffers
    e2e_ms = []
    xh = np.empty_like(b)
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, r2 = qdd.qdd_solve(g, b, params, x=xh)
        t1 = time.perf_counter()
        if k > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e = {"value": statistics.mean(e2e_ms) if e2e_ms else None, "unit": "ms",
           "h2d_bytes_per_step": int(b.nbytes), "d2h_bytes_per_step": int(xh.nbytes)}

    # ---- full-lattice operator throughput (FP32 and FP16 storage) on a lattice > L2
    dslash = None
    if not args.no_dslash and rank == 0:
        Ud = inputs.gauge_field(DSL["L"], DSL["eps"], DSL["gauge_seed"])
        gd = qdd.qdd_create_gauge_field(ctx, DSL["L"], DSL["dom"], Ud)
        del Ud
        qdd.qdd_set_clover(gd, DSL["csw"], DSL["kappa"])
        xs = torch.from_numpy(inputs.gaussian_source(DSL["L"], DSL["source_seed"])).cuda()
        ys = torch.empty_like(xs)
        Vl = int(np.prod(DSL["L"]))
        dslash = {"lattice": list(DSL["L"]), "flop_per_site": 1848}
        for prec, bps in (("f32", 768), ("f16", 392), ("f64", 1536)):
            for _ in range(3):
                qdd.qdd_apply_D(gd, xs, prec, out=ys)
            qdd.qdd_set_profiling(ctx, qdd.QDD_PROF_DSLASH)
            qdd.qdd_get_kernel_times(ctx, reset=True)
            for _ in range(20):
                qdd.qdd_apply_D(gd, xs, prec, out=ys)
            kd = qdd.qdd_get_kernel_times(ctx, reset=True)
            qdd.qdd_set_profiling(ctx, 0)
            ms = kd["dslash"][0] / kd["dslash"][1]
            dslash[prec] = {"ms": ms, "gflops": 1848 * Vl / (ms * 1e-3) / 1e9,
                            "gbs": bps * Vl / (ms * 1e-3) / 1e9,
                            "frac_hbm": bps * Vl / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                            "bytes_per_site": bps}
        qdd.qdd_destroy_gauge(gd)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = oracle_sample(WL, U)
        except Exception as e:  # the GPU number stands without it
            cpu = {"value": None, "unit": "ms", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    if rank == 0:
        last = reps[-1]
        line = {"metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 outer / f32 preconditioner", "data": "synthetic",
                "config": {"workload": WORKLOAD_NAME, "lattice": list(WL["L"]), "domain": list(WL["dom"]),
                           "kappa": WL["kappa"], "c_sw": WL["csw"], "eps": WL["eps"], "nmr": WL["nmr"],
                           "ncy": WL["ncy"], "restart_m": WL["m"], "tol": WL["tol"],
                           "l2": "256 MB buffer written before every step; Krylov working set 0.7 GB",
                           "parallelism": f"{world} replica(s)"},
                "iters": last["iters"], "restarts": last["restarts"], "true_rel_res": last["true_rel_res"],
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "dslash": dslash}
        print(json.dumps(line), flush=True)
    qdd.qdd_destroy_gauge(g)
    qdd.qdd_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_qdd(args)


if __name__ == "__main__":
    main()
