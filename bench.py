#!/usr/bin/env python
"""Benchmark: SAP-preconditioned FGMRES time-to-solution for the
Wilson-clover Dirac equation on one GB300 (arXiv:1502.04025, Sec. 3).

Default workload (one step = one complete solve to a true FP64 relative
residual of 1e-10): the largest single-GPU configuration, 48^3x96 lattice
(10.6 million sites), seeded SU(3) links U = exp(i 0.7 H), c_sw 1.5,
kappa 0.1355, 4^4 domains, Schwarz preconditioner (nmr 4, ncy 4) in FP32
arithmetic on BF16 storage, FP64 FGMRES(16) (the Krylov basis alone is
34 GB), one Z2 noise source.  Inputs are resident in HBM when the timed
region starts; the working set is far larger than L2 and a 256 MB buffer is
written before every step as well.  The same solve through the C ABI with
host buffers gives "e2e".  --config 1..3 select the other configurations.

--impl reference times the FP64 CPU reference checker (oracle/) on a bounded
sample of the same workload: the oracle's operator at sampled sites of the
same gauge field and source, one sample per step; the line's value is that
measured time.  Time-to-solution estimates scaled from the sample are in
separately named keys.

Under torchrun (--gpus N) the lattice is sharded in t over the ranks (slabs
of whole domains; face slots and boundary planes exchanged, dot products
summed over the ranks: strong scaling) when it splits into equal slabs of an
even number of domain blocks, else (or with --replicas) every rank solves its
own copy of the workload (weak scaling).  The timed region is bracketed by
barriers, and the slowest rank's time is reported.
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
          nmr=4, ncy=4, m=16, tol=1e-10, sap_prec="f32", arnoldi_prec="df64", relax_eta=1e-6, reorth=0)
# full-lattice operator throughput: a lattice larger than L2 (32^3x64, eps 0.7, c_sw 1.5, kappa 0.1355)
DSL = dict(L=(32, 32, 32, 64), dom=(4, 4, 4, 4), eps=0.7, csw=1.5, kappa=0.1355, gauge_seed=1003, source_seed=2003)
METRIC = "SAP-FGMRES time-to-1e-10 residual"
# flop of the operator's parts: all eight hops of a site (1320 = 8 hops of 144, summed with 7 spinor adds of
# 24), two Hermitian 6x6 clover blocks, the final combination; MR vector algebra per even site; one hop entering
# a domain across its boundary (hop and its add)
SAP_FLOP = {"hop": 1320, "hop_one": 144, "spinor_add": 24, "clover": 504, "combine": 24, "mr_blas": 336,
            "boundary_hop": 168}
L2_FLUSH_BYTES = 256 << 20
DEFAULT_CONFIG = 4


# the workload configurations (--config N; the default line is the largest single-GPU one, 4)
CONFIGS = {
    1: dict(L=(8, 8, 8, 8), dom=(4, 4, 4, 4), eps=0.5, csw=1.0, kappa=0.12, gauge_seed=1001, source_seed=2001,
            nmr=4, ncy=4, m=16, tol=1e-10, sap_prec="f64", arnoldi_prec="f64", source="gaussian", nrhs=1,
            name="8^4 plain FP64 SAP-FGMRES(16), 4^4 domains, c_sw 1.0, kappa 0.12, eps 0.5"),
    2: dict(WL, source="gaussian", nrhs=1,
            name=("16^3x32 Wilson-clover, c_sw 1.0, kappa 0.125, eps 0.5 links; SAP-FGMRES(16), 8x4x4x4 domains, "
                  "nmr 4, ncy 4, FP32 preconditioner, FP64 outer (Gram-Schmidt, least squares, solution, true "
                  "residual; double-float Arnoldi operator relaxed to FP32 below est 1e-5), tol 1e-10, "
                  "1 Gaussian source")),
    3: dict(L=(32, 32, 32, 64), dom=(4, 4, 4, 4), eps=0.7, csw=1.5, kappa=0.1355, gauge_seed=1003, source_seed=2003,
            nmr=4, ncy=4, m=16, tol=1e-10, sap_prec="f16", arnoldi_prec="df64", relax_eta=1e-6, reorth=0,
            source="point12", nrhs=12,
            name="32^3x64, eps 0.7, c_sw 1.5, kappa 0.1355, FP16-stored SAP, FP64 outer, 12 point sources batched"),
    4: dict(L=(48, 48, 48, 96), dom=(4, 4, 4, 4), eps=0.7, csw=1.5, kappa=0.1355, gauge_seed=1004, source_seed=2004,
            nmr=4, ncy=4, m=16, tol=1e-10, sap_prec="bf16", arnoldi_prec="df64", relax_eta=1e-6, reorth=0,
            source="z2", nrhs=1,
            name=("48^3x96 (10,616,832 sites), eps 0.7, c_sw 1.5, kappa 0.1355, 4^4 domains, nmr 4, ncy 4, "
                  "BF16-stored Schwarz preconditioner with FP32 arithmetic, FP64 FGMRES(16) (Gram-Schmidt, least "
                  "squares, solution, true residual; double-float Arnoldi operator relaxed to FP32 below est "
                  "1e-5), tol 1e-10, one Z2 noise source")),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--config", type=int, default=DEFAULT_CONFIG, choices=[1, 2, 3, 4],
                    help="workload configuration (4, the largest single-GPU one, is the default line)")
    ap.add_argument("--serve", action="store_true", help="run the serving mix instead of single solves")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-in-line", type=int, default=100,
                    help="requests of the serving mix reported in the solve line (0 = none)")
    ap.add_argument("--op-bench", action="store_true", help="time only the full-lattice operator")
    ap.add_argument("--sap-bench", action="store_true",
                    help="time only the Schwarz preconditioner (nmr 4, 8 half-sweeps per application)")
    ap.add_argument("--sap-lattice", default="24,24,24,48")
    ap.add_argument("--sap-precs", default="bf16")
    ap.add_argument("--sap-iters", type=int, default=5)
    ap.add_argument("--sap-form", type=int, default=0, help="qdd_set_schwarz_variant form (0: the default)")
    ap.add_argument("--mg", action="store_true",
                    help="time-to-solution near the critical kappa: Schwarz-only against the two-level multigrid")
    ap.add_argument("--op-lattice", default="32,32,32,64")
    ap.add_argument("--op-precs", default="f32,h16,f16,df64,f64")
    ap.add_argument("--op-iters", type=int, default=20)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["qdd", "reference"], default="qdd")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dslash", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the plain FP64 path on the same system")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--dist-backend", choices=["nccl", "gloo"], default="gloo",
                    help=("torch.distributed backend of a multi-GPU run (gloo, the default: face slots and "
                          "boundary planes exchanged through host tensors, the path run end to end; nccl: "
                          "through CUDA tensors)"))
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs, solve one copy of the workload per GPU instead of sharding it")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def op_bytes_per_site(prec, three_rows=True):
    """Algorithmic bytes of one full-lattice operator apply per site: links
    (4 per site, whole or their first two rows), the two clover blocks, the
    input spinor and the output, each read or written once; 16-bit fields
    carry one FP32 scale per site."""
    rows = 3 if three_rows or prec in ("f64", "df64") else 2
    if prec in ("f64", "df64"):
        return 4 * 9 * 16 + 36 * 16 + 2 * 12 * 16  # df64 splits FP64 values into FP32 pairs: the same bytes
    link = 4 * rows * 3 * (8 if prec == "f32" else 4)
    clover = 36 * 8 if prec == "f32" else 36 * 4 + 4
    spinor = 12 * 8 if prec in ("f32", "h16") else 12 * 4 + 4
    return link + clover + 2 * spinor


def crossing_hops_per_site(dom):
    """Average number of hops per site that leave a domain: 2 faces per
    direction, each holding Vd/dom[mu] sites."""
    vd = float(np.prod(dom))
    return sum(2 * vd / d for d in dom) / vd


def sap_flop_per_site(dom, nmr):
    """Algorithmic FP32 flop per site of one domain visit of the Schwarz
    kernel.  Inside the domain the operator has only the hops that stay in
    it (Dirichlet boundary): 8 - c per site on average, c the hops that leave
    (crossing_hops_per_site), each 144 flop, summed with 7 - c spinor adds:
      setup   t_o = A^-1 rho_o (504 per odd site), bhat_e (inner hops + combine per even site)
      MR      per step: odd site t = A^-1(-k H r), even site p = A r + k H t (inner hops + clover +
              combine each), dots and updates 336 per even site
      recon   odd site x_o = A^-1(rho_o + k H x_e)
      inflow  168 per hop entering from a neighbouring domain (c per site)."""
    f = SAP_FLOP
    c = crossing_hops_per_site(dom)
    hops = (8 - c) * f["hop_one"] + (7 - c) * f["spinor_add"]
    full = hops + f["clover"] + f["combine"]
    per_pair = (f["clover"] + hops + f["combine"]) + nmr * (2 * full + f["mr_blas"]) + full
    return per_pair / 2 + c * f["boundary_hop"]


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
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu",
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
        sm, mx, util, reasons = [], [], [], set()
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
            try:
                util.append(float(parts[9]))  # % of the sample period with a kernel running
            except (IndexError, ValueError):
                pass
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                # meaningful only over several sample periods (the serving run)
                "gpu_busy_fraction": statistics.mean(util) / 100 if len(util) >= 5 else None}


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` on the default workload from one ncu
    capture (profiles/traffic.json), or None once the kernel's sources have
    changed since the capture (the record holds their SHA-256)."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, KeyError, ValueError):
        return None
    return rec["dram_bytes_per_launch"] if h.hexdigest() == rec["sha256"] else None


# --------------------------------------------------------------- oracle leg

def host_info():
    """Host cores and CPU model of the machine the oracle runs on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and model is None:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return {"nproc": os.cpu_count(), "cpu": model, "machine": platform.machine()}


def oracle_cost_units(W):
    """The oracle's cost of one FGMRES iteration and of the fixed part of a
    solve (two true residuals), in units of its operator evaluated at every
    site through apply_D_sites, measured on a small lattice (two domains per
    direction) with the workload's parameters."""
    from oracle import pyoracle as ora
    from paper_1502_04025_gb300 import inputs

    Ls = tuple(2 * d for d in W["dom"])
    Us = inputs.gauge_field(Ls, W["eps"], W["gauge_seed"])
    bs = inputs.gaussian_source(Ls, W["source_seed"])
    As = ora.clover(Ls, Us, W["csw"], W["kappa"])
    Ais = ora.invert_clover(Ls, As)
    Vs = int(np.prod(Ls))

    def best(fn, k=2):
        t = []
        for _ in range(k):
            t0 = time.perf_counter()
            fn()
            t.append(time.perf_counter() - t0)
        return min(t)

    t_op = best(lambda: ora.apply_D_sites(Ls, Us, W["csw"], W["kappa"], bs, np.arange(Vs)))
    t1, t2 = (best(lambda m=m: ora.fgmres(Ls, W["dom"], Us, As, Ais, W["kappa"], bs, 1e-30, m=m, max_restarts=0,
                                           use_sap=W["sap_prec"] is not None, nmr=W["nmr"], ncy=W["ncy"]))
              for m in (1, 2))
    per_it = max(t2 - t1, 0.0)
    return {"lattice": list(Ls), "per_iteration": per_it / t_op, "fixed": max(t1 - per_it, 0.0) / t_op}


def oracle_sample(W, U, b, nsites, seed=11):
    """One bounded sample of the workload for the FP64 oracle: its operator
    D = A - kappa H (clover built per site) at nsites sites of the workload's
    gauge field, applied to the workload's source.  Returns seconds."""
    from oracle import pyoracle as ora

    V = int(np.prod(W["L"]))
    sites = np.sort(np.random.Generator(np.random.Philox(seed)).choice(V, size=min(nsites, V), replace=False))
    x = b if b.ndim == 3 else b[0]
    t0 = time.perf_counter()
    ora.apply_D_sites(W["L"], U, W["csw"], W["kappa"], x, sites)
    return time.perf_counter() - t0


def oracle_sample_threads(W, U, b, nsites, nthreads, seed=11):
    """oracle_sample's sites split over nthreads host threads, each evaluating
    its share through the same C routine (which holds no shared state and runs
    outside the interpreter lock).  Returns seconds."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import pyoracle as ora

    V = int(np.prod(W["L"]))
    sites = np.sort(np.random.Generator(np.random.Philox(seed)).choice(V, size=min(nsites, V), replace=False))
    x = b if b.ndim == 3 else b[0]
    ora.apply_D_sites(W["L"], U, W["csw"], W["kappa"], x, sites[:1])  # its constant tables set up first
    chunks = np.array_split(sites, nthreads)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(nthreads) as ex:
        list(ex.map(lambda c: ora.apply_D_sites(W["L"], U, W["csw"], W["kappa"], x, c), chunks))
    return time.perf_counter() - t0


def oracle_baseline(W, U, b, nsites, units=None, iters=None, restarts=0):
    """cpu_baseline record: the measured sample time (ms) as the value, and
    time-to-solution estimates scaled from it in separately named keys."""
    V = int(np.prod(W["L"]))
    nsites = min(nsites, V)
    t = oracle_sample(W, U, b, nsites)
    full_op_ms = t / nsites * V * 1e3
    rec = {"value": t * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
           "sample": (f"FP64 oracle operator (clover built per site) at {nsites} sampled sites of the "
                      f"{'x'.join(map(str, W['L']))} workload's gauge field and source, single thread"),
           "host": host_info(), "scaled_full_operator_ms": full_op_ms}
    nthreads = os.cpu_count() or 1
    if nthreads > 1:
        ta = oracle_sample_threads(W, U, b, nsites, nthreads)
        rec["all_cores"] = {"value": ta * 1e3, "unit": "ms", "cores": nthreads,
                            "sample": "the same sites split over the host's cores, one thread each",
                            "speedup_over_one_core": t / ta}
    if units is not None:
        nr = W.get("nrhs", 1)
        rec["scaled_ms_per_fgmres_iteration"] = full_op_ms * units["per_iteration"] * nr
        rec["scaled_ms_fixed"] = full_op_ms * units["fixed"] * nr
        rec["cost_units_measured_on"] = units["lattice"]
        if iters is not None:
            rec["scaled_time_to_solution_ms"] = (rec["scaled_ms_fixed"] * (1 + restarts) +
                                                 rec["scaled_ms_per_fgmres_iteration"] * iters)
            rec["scaled_with"] = f"the GPU solve's {iters} iterations and {restarts} restarts"
    return rec


REF_SAMPLE_SITES = 1 << 18
CPU_SAMPLE_SITES = 1 << 20  # about 15-20 s of single-thread oracle work


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1502_04025_gb300 import inputs

    W = CONFIGS[args.config]
    U = inputs.gauge_field(W["L"], W["eps"], W["gauge_seed"])
    b = make_sources(W)
    units = oracle_cost_units(W)
    V = int(np.prod(W["L"]))
    nsites = min(REF_SAMPLE_SITES, V)
    ms = []
    for k in range(args.warmup + args.steps):
        t = oracle_sample(W, U, b, nsites, seed=11 + k)
        if k >= args.warmup:
            ms.append(t * 1e3)
    v = statistics.mean(ms)
    full_op_ms = v / nsites * V
    cpu = {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
           "sample": (f"per step: FP64 oracle operator (clover built per site) at {nsites} sampled sites "
                      f"of the {'x'.join(map(str, W['L']))} workload's gauge field and source, single thread"),
           "host": host_info()}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"], "config": args.config, "lattice": list(W["L"]),
                       "domain": list(W["dom"])},
            "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_sites": nsites,
            "scaled_full_operator_ms": full_op_ms,
            "scaled_ms_per_fgmres_iteration": full_op_ms * units["per_iteration"] * W.get("nrhs", 1),
            "scaled_ms_fixed": full_op_ms * units["fixed"] * W.get("nrhs", 1),
            "cost_units": units}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg

def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """The slowest rank's time (all ranks receive it); value itself with one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_sources(W):
    from paper_1502_04025_gb300 import inputs

    if W["source"] == "point12":
        return np.ascontiguousarray(inputs.point_sources(W["L"]))
    if W["source"] == "z2":
        return inputs.z2_source(W["L"], W["source_seed"])
    return inputs.gaussian_source(W["L"], W["source_seed"])


def sampled_residual(W, U, b, x, nsites=64, seed=7):
    """True residual of the returned solution at sampled sites, from the FP64
    oracle (max over right-hand sides of |b - D x|_S / |b|)."""
    from oracle import pyoracle as ora

    V = int(np.prod(W["L"]))
    sites = np.random.Generator(np.random.Philox(seed)).choice(V, size=min(nsites, V), replace=False)
    bs = b.reshape(-1, V, 4, 3)
    xs = x.reshape(-1, V, 4, 3)
    worst = 0.0
    for r in range(bs.shape[0]):
        dx = ora.apply_D_sites(W["L"], U, W["csw"], W["kappa"], xs[r], sites)
        res = np.linalg.norm(bs[r][sites] - dx) / np.linalg.norm(bs[r])
        worst = max(worst, float(res))
    return {"sites": int(len(sites)), "max_rel_residual_at_sites": worst}


def run_qdd(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    # one GPU per rank; with fewer GPUs than ranks (a check of the sharded path
    # with --dist-backend gloo) ranks share them
    local = int(os.environ.get("LOCAL_RANK", "0")) % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        if args.dist_backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1502_04025_gb300 import build, inputs

    build.build()
    from paper_1502_04025_gb300 import qdd

    W = CONFIGS[args.config]
    pk, pk_kind = peaks()
    ctx = qdd.qdd_create(local, 0)
    U = inputs.gauge_field(W["L"], W["eps"], W["gauge_seed"])
    b = make_sources(W)
    nrhs = W["nrhs"]
    # several ranks: the lattice is sharded in t (slabs of whole domains, strong
    # scaling) when it splits into equal slabs of an even number of domain
    # blocks; otherwise every rank solves its own copy (replicas)
    shard, shard_reason = None, ""
    if world > 1 and not args.replicas:
        from paper_1502_04025_gb300 import dist as qdist

        try:
            shard = qdist.slab_partition(W["L"][3], W["dom"][3], world)[rank]
        except ValueError as e:
            shard_reason = str(e)
    if shard is not None:
        t0, lt = shard
        comm = qdist.TorchComm(device=torch.device("cuda", local) if args.dist_backend == "nccl" else None)
        g = qdd.qdd_create_gauge_field_slab(ctx, qdist.local_lattice(W["L"], lt), W["dom"],
                                            qdist.extended_links(U, W["L"], W["dom"], t0, lt), comm)
        b = qdist.local_field(b, W["L"], t0, lt)
        parallelism = f"t-slabs over {world} GPUs: {lt} planes each, face slots and boundary planes exchanged"
    else:
        g = qdd.qdd_create_gauge_field(ctx, W["L"], W["dom"], U)
        parallelism = f"{world} replica(s)" + (f" ({shard_reason})" if world > 1 and not args.replicas else "")
    qdd.qdd_set_clover(g, W["csw"], W["kappa"])
    params = qdd.qdd_default_params(tol=W["tol"], restart_m=W["m"], nmr=W["nmr"], ncy=W["ncy"],
                                    sap_prec=W["sap_prec"], arnoldi_prec=W["arnoldi_prec"], max_restarts=200,
                                    nrhs=nrhs, relax_eta=W.get("relax_eta", 0.0), reorth=W.get("reorth", 1))
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # measured FMA-chain peaks (FP64 and FP32), before the timed region
    fma = {"fp64_tflops": qdd.qdd_measure_fma_peak(local, True, 200.0)[0],
           "fp32_tflops": qdd.qdd_measure_fma_peak(local, False, 200.0)[0],
           "how": "qdd_measure_fma_peak: 8 independent FMA chains per thread, 8 CTAs of 256 threads per SM, "
                  "about 200 ms, CUDA events"}

    rep = None
    # per-launch CUDA events on the Schwarz kernel (the dominant class); the
    # event pool is created here, before the timed region
    qdd.qdd_set_profiling(ctx, qdd.QDD_PROF_SAP)
    clocks = Clocks(local)
    clocks.start()  # the clock sampler starts during warm-up, before the timed region
    for _ in range(args.warmup):
        flush.fill_(1.0)
        _, rep = qdd.qdd_solve(g, bd, params, x=xd, allow_noconv=True)
    torch.cuda.synchronize()

    # ---- timed region: K solves, inputs resident, L2 flushed before each
    qdd.qdd_get_kernel_times(ctx, reset=True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        _, rep = qdd.qdd_solve(g, bd, params, x=xd, allow_noconv=True)
        reps.append(rep)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    kt = qdd.qdd_get_kernel_times(ctx, reset=True)
    qdd.qdd_set_profiling(ctx, 0)
    ms_step = max_over_ranks(ms_total / args.steps, dist, "cuda" if args.dist_backend == "nccl" else "cpu")
    launches = int(sum(r["kernel_launches"] for r in reps))

    # ---- kernel-class shares from one extra solve with every class event-timed
    qdd.qdd_set_profiling(ctx, qdd.QDD_PROF_ALL)
    qdd.qdd_get_kernel_times(ctx, reset=True)
    flush.fill_(1.0)
    qdd.qdd_solve(g, bd, params, x=xd, allow_noconv=True)
    work = qdd.qdd_get_kernel_work(ctx)
    shares = qdd.qdd_get_kernel_times(ctx, reset=True)
    qdd.qdd_set_profiling(ctx, 0)

    # ---- the FP64 vector algebra against its roofline: the time it needs at
    # the measured FP64 FMA rate or the measured HBM bandwidth, whichever binds
    blas_ms = shares["blas"][0]
    blas_flop, blas_bytes = work["blas"]
    t_alu = blas_flop / (fma["fp64_tflops"] * 1e12) * 1e3
    t_hbm = blas_bytes / (pk["hbm_gbs"] * 1e9) * 1e3
    blas_roof = {"kernel": "FP64 vector kernels of one solve (multi-dot, multi-axpy + norm, scaling, solution update)",
                 "bound": "fp64 alu" if t_alu >= t_hbm else "hbm", "ms": blas_ms, "launches": shares["blas"][1],
                 "flop": blas_flop, "bytes": blas_bytes,
                 "achieved_tflops": blas_flop / (blas_ms * 1e-3) / 1e12 if blas_ms > 0 else None,
                 "achieved_gbs": blas_bytes / (blas_ms * 1e-3) / 1e9 if blas_ms > 0 else None,
                 "peak_fp64_tflops": fma["fp64_tflops"], "peak_hbm_gbs": pk["hbm_gbs"],
                 "frac": max(t_alu, t_hbm) / blas_ms if blas_ms > 0 else None,
                 "frac_is": "roofline time (max of flop / measured FP64 FMA rate, bytes / measured HBM) over the "
                            "event-timed time"}

    # ---- roofline of the dominant kernel class (timed inside the timed region)
    classes = {k: v for k, v in shares.items() if v[1] > 0}
    dom_cls = max(classes, key=lambda k: classes[k][0])
    V = int(np.prod(W["L"]))
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = sm_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # TFLOP/s
    kt = kt if kt[dom_cls][0] > 0 else shares
    if dom_cls == "sap":
        ms_launch = kt["sap"][0] / kt["sap"][1]
        flop = nrhs * (V // 2) * sap_flop_per_site(W["dom"], W["nmr"])
        achieved = flop / (ms_launch * 1e-3) / 1e12
        roof = {"kernel": f"k_sap (Schwarz colour half-sweep, {W['sap_prec']} storage, FP32 arithmetic)"
                if W["sap_prec"] != "f64" else "k_sap (Schwarz colour half-sweep, FP64)",
                "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": ncu_traffic(f"k_sap_config{args.config}"),
                "ms_per_launch": ms_launch, "launches": kt["sap"][1],
                "flop_per_launch": flop,
                "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 flop x {pk.get('sm_max_mhz', 2070.0):.0f} MHz"}
    elif dom_cls == "dslash":
        ms_launch = kt["dslash"][0] / kt["dslash"][1]
        bytes_site = 576 + 576 + 96 + 192  # FP64-width links + clover, FP32 input, FP64 output
        achieved = nrhs * V * bytes_site / (ms_launch * 1e-3) / 1e9
        roof = {"kernel": "k_dslash (operator in the Arnoldi step)", "bound": "hbm", "achieved": achieved,
                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": None,
                "ms_per_launch": ms_launch, "launches": kt["dslash"][1]}
    else:
        ms_launch = kt["blas"][0] / kt["blas"][1]
        roof = {"kernel": "FP64 vector kernels", "bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": None, "traffic": None, "ms_per_launch": ms_launch,
                "launches": kt["blas"][1]}
    if roof["bound"] == "alu":
        # the FP32 peak is derived from the unit counts and the maximum SM clock
        # of the measured-peaks record; the FMA-chain probe's measured rate is in fma_peaks
        roof["peak_kind"] = ("derived from unit counts and the measured max SM clock" if pk_kind == "measured"
                             else "derived from unit counts and the fallback clock")
    else:
        roof["peak_kind"] = "of measured" if pk_kind == "measured" else "of fallback"
    roof["class_ms_one_solve"] = {k: round(v[0], 4) for k, v in shares.items()}

    # ---- end to end through the C ABI with host buffers (page-locked, so the
    # copies are direct DMA rather than staged through a driver buffer)
    e2e_ms = []
    b_pin = torch.from_numpy(b).pin_memory()
    x_pin = torch.empty(b.shape, dtype=torch.complex128, pin_memory=True)
    bh, xh = b_pin.numpy(), x_pin.numpy()  # numpy views of the page-locked tensors
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, r2 = qdd.qdd_solve(g, bh, params, x=xh, allow_noconv=True)
        t1 = time.perf_counter()
        if k > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e = {"value": statistics.mean(e2e_ms) if e2e_ms else None, "unit": "ms",
           "h2d_bytes_per_step": int(bh.nbytes), "d2h_bytes_per_step": int(xh.nbytes), "host_memory": "pinned"}
    parity = None
    if rank == 0 and e2e_ms and shard is None:
        parity = sampled_residual(W, U, b, xh)

    # ---- batching: the same sources one at a time (the first source's solve, times nrhs)
    unbatched = None
    if rank == 0 and world == 1 and nrhs > 1:
        p1 = qdd.qdd_default_params(tol=W["tol"], restart_m=W["m"], nmr=W["nmr"], ncy=W["ncy"],
                                    sap_prec=W["sap_prec"], arnoldi_prec=W["arnoldi_prec"], max_restarts=200,
                                    nrhs=1, relax_eta=W.get("relax_eta", 0.0), reorth=W.get("reorth", 1))
        b1 = bd[0].contiguous()
        x1 = torch.empty_like(b1)
        qdd.qdd_solve(g, b1, p1, x=x1, allow_noconv=True)
        ms1 = []
        for _ in range(2):
            flush.fill_(1.0)
            e0.record(stream)
            _, r1 = qdd.qdd_solve(g, b1, p1, x=x1, allow_noconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ms1.append(e0.elapsed_time(e1))
        t1 = statistics.median(ms1)
        unbatched = {"one_source_ms": t1, "iters": r1["iters"], "nrhs_times_one_ms": t1 * nrhs,
                     "gain_of_batching": t1 * nrhs / ms_step}

    # ---- the same system with FP64 throughout (Schwarz preconditioner and
    # Arnoldi operator): the plain FP64 GPU path the mixed-precision one is
    # measured against
    plain = None
    if rank == 0 and world == 1 and args.config in (2, 4) and not args.no_fp64_compare:
        p64 = qdd.qdd_default_params(tol=W["tol"], restart_m=W["m"], nmr=W["nmr"], ncy=W["ncy"], sap_prec="f64",
                                     arnoldi_prec="f64", max_restarts=200, nrhs=nrhs, reorth=1)
        qdd.qdd_solve(g, bd, p64, x=xd, allow_noconv=True)
        ms64 = []
        for _ in range(2):
            flush.fill_(1.0)
            e0.record(stream)
            _, r64 = qdd.qdd_solve(g, bd, p64, x=xd, allow_noconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ms64.append(e0.elapsed_time(e1))
        plain = {"ms": statistics.median(ms64), "iters": r64["iters"], "true_rel_res": r64["true_rel_res"],
                 "converged": bool(r64["converged"]), "speedup_of_mixed": statistics.median(ms64) / ms_step,
                 "params": "FP64 Schwarz (nmr 4, ncy 4), FP64 Arnoldi operator, re-orthogonalised Gram-Schmidt"}

    # ---- full-lattice operator throughput (FP32 and FP16 storage) on a lattice > L2
    dslash = None
    if not args.no_dslash and rank == 0 and world == 1 and args.config in (2, 4):
        Ud = inputs.gauge_field(DSL["L"], DSL["eps"], DSL["gauge_seed"])
        gd = qdd.qdd_create_gauge_field(ctx, DSL["L"], DSL["dom"], Ud)
        del Ud
        qdd.qdd_set_clover(gd, DSL["csw"], DSL["kappa"])
        xs = torch.from_numpy(inputs.gaussian_source(DSL["L"], DSL["source_seed"])).cuda()
        ys = torch.empty_like(xs)
        Vl = int(np.prod(DSL["L"]))
        two_rows, _ = qdd.qdd_link_compression(gd)
        dslash = {"lattice": list(DSL["L"]), "flop_per_site": 1848,
                  "link_rows": 2 if two_rows else 3}
        for name in ("f32", "f32_three_rows", "h16", "f16", "bf16", "df64", "f64"):
            prec = name.split("_")[0]
            rows3 = name.endswith("three_rows") or not two_rows
            qdd.qdd_set_link_compression(gd, not rows3)
            bps = op_bytes_per_site(prec, rows3)
            for _ in range(3):
                qdd.qdd_apply_D(gd, xs, prec, out=ys)
            qdd.qdd_set_profiling(ctx, qdd.QDD_PROF_DSLASH)
            qdd.qdd_get_kernel_times(ctx, reset=True)
            for _ in range(20):
                qdd.qdd_apply_D(gd, xs, prec, out=ys)
            kd = qdd.qdd_get_kernel_times(ctx, reset=True)
            qdd.qdd_set_profiling(ctx, 0)
            ms = kd["dslash"][0] / kd["dslash"][1]
            dslash[name] = {"ms": ms, "gflops": 1848 * Vl / (ms * 1e-3) / 1e9,
                            "gbs": bps * Vl / (ms * 1e-3) / 1e9,
                            "frac_hbm": bps * Vl / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                            "bytes_per_site": bps}
        qdd.qdd_set_link_compression(gd, two_rows)
        qdd.qdd_destroy_gauge(gd)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            if U is None:
                U = inputs.gauge_field(W["L"], W["eps"], W["gauge_seed"])
            cpu = oracle_baseline(W, U, b, CPU_SAMPLE_SITES, oracle_cost_units(W), reps[-1]["iters"],
                                  reps[-1]["restarts"])
        except Exception as e:  # the GPU number stands without it
            cpu = {"value": None, "unit": "ms", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    # a shorter serving mix (its own context; the workload's fields are freed first)
    serving = None
    if rank == 0 and world == 1 and args.serve_in_line > 0:
        qdd.qdd_destroy_gauge(g)
        qdd.qdd_destroy(ctx)
        g = ctx = None
        try:
            sv = serve_mix(args.serve_in_line)
            serving = {k: sv[k] for k in ("p50_ms", "p99_ms", "solves_per_s", "requests", "converged",
                                          "offered_rate_per_s", "gpu_busy_fraction", "wall_s")}
            serving["workload"] = sv["config"]["workload"]
        except Exception as e:  # the solve line stands without it
            serving = {"failed": repr(e)}

    if rank == 0:
        last = reps[-1]
        line = {"metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
                "scaling": "strong" if shard is not None else "weak",
                "vs_baseline": None,
                "dtype": ("f64" if W["sap_prec"] == "f64" else f"f64 outer / f32 arithmetic on {W['sap_prec']} "
                          "preconditioner storage"),
                "data": "synthetic",
                "config": {"workload": W["name"], "config": args.config, "lattice": list(W["L"]),
                           "domain": list(W["dom"]), "kappa": W["kappa"], "c_sw": W["csw"], "eps": W["eps"],
                           "nmr": W["nmr"], "ncy": W["ncy"], "restart_m": W["m"], "tol": W["tol"], "nrhs": nrhs,
                           "sap_prec": W["sap_prec"], "arnoldi_prec": W["arnoldi_prec"],
                           "relax_eta": W.get("relax_eta", 0.0), "reorth": W.get("reorth", 1),
                           "l2": "256 MB buffer written before every step; Krylov working set larger than L2",
                           "parallelism": parallelism},
                "iters": last["iters"], "restarts": last["restarts"], "true_rel_res": last["true_rel_res"],
                "converged": bool(last["converged"]),
                "roofline": roof, "roofline_fp64_vector_algebra": blas_roof, "fma_peaks": fma,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "dslash": dslash, "plain_fp64": plain, "unbatched": unbatched, "serving": serving}
        if parity is not None:
            line["parity"] = parity
        print(json.dumps(line), flush=True)
    if g is not None:
        qdd.qdd_destroy_gauge(g)
        qdd.qdd_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------ operator only

def run_op_bench(args):
    """Full-lattice Wilson-clover operator throughput (1848 flop/site) on a
    lattice larger than L2, per storage precision, event-timed per launch."""
    import torch

    from paper_1502_04025_gb300 import build, inputs

    build.build()
    from paper_1502_04025_gb300 import qdd

    pk, pk_kind = peaks()
    L = tuple(int(v) for v in args.op_lattice.split(","))
    ctx = qdd.qdd_create(0, 0)
    U = inputs.gauge_field(L, DSL["eps"], DSL["gauge_seed"])
    g = qdd.qdd_create_gauge_field(ctx, L, DSL["dom"], U)
    del U
    qdd.qdd_set_clover(g, DSL["csw"], DSL["kappa"])
    xs = torch.from_numpy(inputs.gaussian_source(L, DSL["source_seed"])).cuda()
    ys = torch.empty_like(xs)
    Vl = int(np.prod(L))
    out = {"metric": "Wilson-clover Dslash throughput", "unit": "GFLOP/s", "lattice": list(L),
           "domain": list(DSL["dom"]), "flop_per_site": 1848, "peak_hbm_gbs": pk["hbm_gbs"],
           "peak_kind": "of measured" if pk_kind == "measured" else "of fallback"}
    two_rows, _ = qdd.qdd_link_compression(g)
    out["link_rows"] = 2 if two_rows else 3
    for name in args.op_precs.split(","):
        # "<prec>_three_rows": the same operator reading whole links
        prec = name.split("_")[0]
        rows3 = name.endswith("_three_rows") or not two_rows
        qdd.qdd_set_link_compression(g, not rows3)
        for _ in range(3):
            qdd.qdd_apply_D(g, xs, prec, out=ys)
        qdd.qdd_set_profiling(ctx, qdd.QDD_PROF_DSLASH)
        qdd.qdd_get_kernel_times(ctx, reset=True)
        for _ in range(args.op_iters):
            qdd.qdd_apply_D(g, xs, prec, out=ys)
        kd = qdd.qdd_get_kernel_times(ctx, reset=True)
        qdd.qdd_set_profiling(ctx, 0)
        ms = kd["dslash"][0] / kd["dslash"][1]
        bps = op_bytes_per_site(prec, rows3)
        out[name] = {"ms": ms, "gflops": 1848 * Vl / (ms * 1e-3) / 1e9, "gbs": bps * Vl / (ms * 1e-3) / 1e9,
                     "frac_hbm": bps * Vl / (ms * 1e-3) / 1e9 / pk["hbm_gbs"], "bytes_per_site": bps}
    print(json.dumps(out), flush=True)
    qdd.qdd_destroy_gauge(g)
    qdd.qdd_destroy(ctx)


def run_sap_bench(args):
    """The Schwarz preconditioner alone (the headline workload's parameters:
    eps 0.7, c_sw 1.5, kappa 0.1355, 4^4 domains, nmr 4, 8 half-sweeps per
    application) on one lattice, per storage precision: 3 applications
    untimed, then --sap-iters event-timed.  A small lattice (the default,
    24^3x48, 1296 domains per colour) is the case the Schwarz kernel's ncu
    captures run on."""
    import torch

    from paper_1502_04025_gb300 import build, inputs

    build.build()
    from paper_1502_04025_gb300 import qdd

    pk, pk_kind = peaks()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = sm_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # TFLOP/s
    L = tuple(int(v) for v in args.sap_lattice.split(","))
    W = CONFIGS[4]
    ctx = qdd.qdd_create(0, 0)
    U = inputs.gauge_field(L, W["eps"], 1003)
    g = qdd.qdd_create_gauge_field(ctx, L, W["dom"], U)
    del U
    qdd.qdd_set_clover(g, W["csw"], W["kappa"])
    qdd.qdd_set_schwarz_variant(g, args.sap_form)
    eta = torch.from_numpy(inputs.gaussian_source(L, 2003)).cuda()
    V = int(np.prod(L))
    flop = sap_flop_per_site(W["dom"], W["nmr"]) * V / 2  # one half-sweep: half the sites' domains
    out = {"metric": "Schwarz half-sweep time", "unit": "ms", "lattice": list(L), "domain": list(W["dom"]),
           "nmr": W["nmr"], "form": args.sap_form, "peak_fp32_tflops": fp32_peak,
           "peak_kind": ("derived from unit counts and the measured max SM clock" if pk_kind == "measured"
                         else "derived from unit counts and the fallback clock")}
    for prec in args.sap_precs.split(","):
        for _ in range(3):
            qdd.qdd_sap_apply(g, eta, W["nmr"], 8, prec)
        torch.cuda.synchronize()
        qdd.qdd_set_profiling(ctx, qdd.QDD_PROF_SAP)
        qdd.qdd_get_kernel_times(ctx, reset=True)
        for _ in range(args.sap_iters):
            qdd.qdd_sap_apply(g, eta, W["nmr"], 8, prec)
        torch.cuda.synchronize()
        kt = qdd.qdd_get_kernel_times(ctx, reset=True)
        qdd.qdd_set_profiling(ctx, 0)
        ms = kt["sap"][0] / kt["sap"][1]
        out[prec] = {"ms_per_half_sweep": ms, "launches": kt["sap"][1],
                     "tflops": flop / (ms * 1e-3) / 1e12, "frac_fp32": flop / (ms * 1e-3) / 1e12 / fp32_peak}
    print(json.dumps(out), flush=True)
    qdd.qdd_destroy_gauge(g)
    qdd.qdd_destroy(ctx)


# ------------------------------------------------------------ multigrid

MGW = dict(L=(16, 16, 16, 32), dom=(8, 4, 4, 4), eps=0.5, csw=1.0, kappa=0.143, gauge_seed=1002, source_seed=2002,
           w0_seed=4001, nv=12, setup_iters=6, setup_ncy=4, nmr=4, post_ncy=4, coarse_iters=12, bootstrap=1, ncy=4,
           m=16, tol=1e-10)


def run_mg_bench(args):
    """The same near-critical system solved with Schwarz-preconditioned FGMRES
    and with FGMRES preconditioned by the two-level multigrid V-cycle (Schwarz
    smoother): time to a 1e-10 true residual, event-timed, L2 flushed before
    every solve; the multigrid setup is timed separately."""
    import torch

    from paper_1502_04025_gb300 import build, inputs

    build.build()
    from paper_1502_04025_gb300 import qdd

    W = MGW
    ctx = qdd.qdd_create(0, 0)
    U = inputs.gauge_field(W["L"], W["eps"], W["gauge_seed"])
    g = qdd.qdd_create_gauge_field(ctx, W["L"], W["dom"], U)
    del U
    qdd.qdd_set_clover(g, W["csw"], W["kappa"])
    b = torch.from_numpy(inputs.gaussian_source(W["L"], W["source_seed"])).cuda()
    w0 = torch.from_numpy(inputs.gaussian_source(W["L"], W["w0_seed"], nrhs=W["nv"])).cuda()
    x = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    common = dict(tol=W["tol"], restart_m=W["m"], max_restarts=200, arnoldi_prec="df64", relax_eta=1e-6, reorth=0)

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, rep = [], None
        for _ in range(steps):
            flush.fill_(1.0)
            e0.record(stream)
            rep = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms), rep

    p_sap = qdd.qdd_default_params(use_sap=1, nmr=W["nmr"], ncy=W["ncy"], sap_prec="f32", **common)
    p_mg = qdd.qdd_default_params(use_sap=2, **common)
    mg_kw = dict(nv=W["nv"], setup_iters=W["setup_iters"], setup_ncy=W["setup_ncy"], nmr=W["nmr"],
                 post_ncy=W["post_ncy"], coarse_iters=W["coarse_iters"], sap_prec="f32")
    timed(lambda: qdd.qdd_solve(g, b, p_sap, x=x)[1], args.warmup)
    ms_sap, r_sap = timed(lambda: qdd.qdd_solve(g, b, p_sap, x=x)[1], args.steps)
    mg = {}
    for boot in (0, W["bootstrap"]):  # the first build alone, then with the adaptive passes
        setup_ms, _ = timed(lambda: qdd.qdd_mg_setup(g, w0, bootstrap=boot, **mg_kw), 1 + max(args.warmup, 1))
        timed(lambda: qdd.qdd_solve(g, b, p_mg, x=x)[1], args.warmup)
        ms_mg, r_mg = timed(lambda: qdd.qdd_solve(g, b, p_mg, x=x)[1], args.steps)
        mg[boot] = {"ms": ms_mg, "iters": r_mg["iters"], "true_rel_res": r_mg["true_rel_res"],
                    "setup_ms": setup_ms, "bootstrap": boot}
    line = {"metric": "time to a 1e-10 residual near the critical kappa: Schwarz against two-level multigrid",
            "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
            "data": "synthetic",
            "config": {"workload": (f"16^3x32 Wilson-clover, c_sw {W['csw']}, kappa {W['kappa']}, eps {W['eps']} "
                                    f"links, 8x4x4x4 domains/aggregates, FGMRES({W['m']}), tol {W['tol']}"),
                       "multigrid": {k: W[k] for k in ("nv", "setup_iters", "setup_ncy", "nmr", "post_ncy",
                                                       "coarse_iters", "bootstrap")},
                       "schwarz": {"ncy": W["ncy"], "nmr": W["nmr"], "prec": "f32"},
                       "l2": "256 MB buffer written before every solve"},
            "schwarz": {"ms": ms_sap, "iters": r_sap["iters"], "true_rel_res": r_sap["true_rel_res"]},
            "multigrid": mg[W["bootstrap"]], "multigrid_no_bootstrap": mg[0],
            "speedup": ms_sap / mg[W["bootstrap"]]["ms"]}
    print(json.dumps(line), flush=True)
    qdd.qdd_destroy_gauge(g)
    qdd.qdd_destroy(ctx)


# ---------------------------------------------------------------- serving

SERVE_LATTICES = [((8, 8, 8, 8), (4, 4, 4, 4)), ((16, 16, 16, 32), (8, 4, 4, 4)),
                  ((24, 24, 24, 48), (4, 4, 4, 4)), ((32, 32, 32, 64), (4, 4, 4, 4))]
SERVE_KAPPAS = [0.120, 0.125, 0.130, 0.135]


def run_serve(args):
    """Poisson arrivals of solves on four lattice sizes with kappa in
    [0.120, 0.135] (four resident values) and 1-12 right-hand sides, FP32
    preconditioner, double-float Arnoldi operator, tol 1e-10, admission by an
    80% HBM budget; reports p50/p99 latency (submit to result) and solves/s."""
    from paper_1502_04025_gb300 import build

    build.build()
    print(json.dumps(serve_mix(args.serve_requests)), flush=True)


def serve_mix(n_requests):
    """The serving mix of run_serve with n_requests requests; returns its JSON record."""
    from paper_1502_04025_gb300 import inputs, qdd

    ctx = qdd.qdd_create(0, 0)
    qdd.qdd_serve_config(ctx, 4)
    gauges = {}
    for li, (L, dom) in enumerate(SERVE_LATTICES):
        U = inputs.gauge_field(L, 0.5, 1100 + li)
        for ki, k in enumerate(SERVE_KAPPAS):
            g = qdd.qdd_create_gauge_field(ctx, L, dom, U)
            qdd.qdd_set_clover(g, 1.0, k)
            gauges[(li, ki)] = g
        del U
    rng = np.random.Generator(np.random.Philox(3001))
    n = n_requests
    reqs = []
    for i in range(n):
        li = int(rng.integers(0, len(SERVE_LATTICES)))
        ki = int(rng.integers(0, len(SERVE_KAPPAS)))
        nrhs = int(rng.integers(1, 13))
        reqs.append((li, ki, nrhs))
    params = {r: qdd.qdd_default_params(tol=1e-10, sap_prec="f32", arnoldi_prec="df64", nrhs=r, max_restarts=200,
                                        relax_eta=1e-6, reorth=0)
              for r in range(1, 13)}
    srcs = {}
    for li, (L, dom) in enumerate(SERVE_LATTICES):
        srcs[li] = inputs.gaussian_source(L, 3100 + li, nrhs=12).reshape(12, -1, 4, 3)
    # calibrate: solve time of one request of each lattice with 1 and 12 rhs
    cal = {}
    for li in range(len(SERVE_LATTICES)):
        for r in (1, 12):
            bb = srcs[li][:r] if r > 1 else srcs[li][0]
            xx = np.zeros_like(bb)
            t0 = time.perf_counter()
            st, _ = qdd.qdd_poll(ctx, qdd.qdd_submit(ctx, gauges[(li, 0)], np.ascontiguousarray(bb), xx, params[r]),
                                 600.0)
            cal[(li, r)] = time.perf_counter() - t0
            del xx
    mean_service = np.mean([cal[(li, 1)] + (cal[(li, 12)] - cal[(li, 1)]) * (r - 1) / 11 for li, _, r in reqs])
    rate = 0.7 / mean_service  # requests per second for ~70% busy
    gaps = rng.exponential(1.0 / rate, size=n)
    import threading

    pending = []          # (ticket, x) in submission order; x freed once polled
    lock = threading.Lock()
    lat, ok, done, failures = [], [0], threading.Event(), []

    def poller():
        k = 0
        while k < n:
            with lock:
                item = pending[k] if k < len(pending) else None
            if item is None:
                time.sleep(0.0005)
                continue
            st, rep = qdd.qdd_poll(ctx, item[0], 600.0)
            if st == qdd.QDD_OK and rep["converged"]:
                ok[0] += 1
                lat.append(rep["seconds"])
            else:
                li, ki, r = reqs[k]
                failures.append({"lattice": list(SERVE_LATTICES[li][0]), "kappa": SERVE_KAPPAS[ki], "nrhs": r,
                                 "status": qdd.STATUS_NAMES[st] if 0 <= st < len(qdd.STATUS_NAMES) else st,
                                 "error": qdd.qdd_last_error(),
                                 "true_rel_res": rep["true_rel_res"] if rep else None})
            with lock:
                pending[k] = None  # release the output buffer
            k += 1
        done.set()

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    clocks = Clocks(0)
    clocks.start()
    t_start = time.perf_counter()
    t_next = t_start
    for i, (li, ki, r) in enumerate(reqs):
        t_next += gaps[i]
        while time.perf_counter() < t_next:
            time.sleep(max(0.0, min(0.001, t_next - time.perf_counter())))
        bb = srcs[li][:r] if r > 1 else srcs[li][0]
        x = np.zeros_like(bb)
        t = qdd.qdd_submit(ctx, gauges[(li, ki)], np.ascontiguousarray(bb), x, params[r])
        with lock:
            pending.append((t, x))
        del x
    done.wait()
    ok = ok[0]
    wall = time.perf_counter() - t_start
    clk = clocks.stop()
    used, budget = qdd.qdd_memory(ctx)
    line = {"metric": "SAP-FGMRES serving latency (submit to result)", "value": float(np.percentile(lat, 50)) * 1e3,
            "unit": "ms", "higher_is_better": False, "p50_ms": float(np.percentile(lat, 50)) * 1e3,
            "p99_ms": float(np.percentile(lat, 99)) * 1e3, "solves_per_s": ok / wall, "requests": n,
            "converged": ok, "failures": failures, "offered_rate_per_s": rate, "wall_s": wall,
            "gpu_busy_fraction": clk.get("gpu_busy_fraction"), "clocks": clk, "data": "synthetic",
            "config": {"workload": "serving mix: Poisson arrivals, lattices 8^4/16^3x32/24^3x48/32^3x64, "
                                   "kappa in {0.120,0.125,0.130,0.135}, 1-12 rhs, FP32 SAP, tol 1e-10",
                       "slots": 4, "hbm_budget_bytes": budget, "resident_gauge_bytes": used},
            "calibration_s": {f"{SERVE_LATTICES[li][0]}x{r}": v for (li, r), v in cal.items()}}
    for g in gauges.values():
        qdd.qdd_destroy_gauge(g)
    qdd.qdd_destroy(ctx)
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    elif args.op_bench:
        run_op_bench(args)
    elif args.sap_bench:
        run_sap_bench(args)
    elif args.mg:
        run_mg_bench(args)
    else:
        run_qdd(args)


if __name__ == "__main__":
    main()
