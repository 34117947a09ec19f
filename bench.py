"""Benchmark: unknowns x RHS solved to 1e-10 relative residual per second.

Workload: the 2048x2048 power-grid system (4,194,304 unknowns, log-uniform
branch conductances in [0.1, 10] S, 1% of nodes padded to ground by 10 S,
the rest sinking U[0, 1e-3] A) torn into 4096 tiles of 32x32 nodes, Zc = 1
ohm.  One step = one complete ``vtm_solve`` (x0 solves, VTM sweeps until
||b - A x|| <= 1e-10 ||b||, recovery, FP64 verification) with the inputs
already in HBM; plan and factorisation are set-up, timed separately.  L2 is
flushed (a 512 MB write) between timed steps.

``--impl reference`` times the CPU oracle instead (a bounded sample of the
same recipe, see ``reference_arm``).
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

METRIC = ("unknowns·RHS solved to 1e-10 rel. residual per sec (1 GB300), vs plain FP64 VTM; "
          "% HBM roofline")
UNIT = "unknowns*RHS/s"
TOL = 1e-10
SAMPLE_N = 512  # oracle sample: 512x512 instance of the same recipe


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vtm", choices=["vtm", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "fp32", "bf16", "fp16"])
    ap.add_argument("--workload", default="power_grid", choices=["power_grid", "thermal", "vccs", "grad"],
                    help="power_grid: the headline 2048^2 grid; thermal: 128x128x32 RC grid, 400 boxes, "
                         "64 RHS; vccs: 1024^2 grid with controlled sources, VTM and block Jacobi; "
                         "grad: 1024^2 grid, forward + adjoint solve + branch gradients")
    ap.add_argument("--grid", type=int, default=2048)
    ap.add_argument("--thermal-grid", type=int, default=128,
                    help="--workload thermal: the grid is N x N x 32 (a smaller case for profiling)")
    ap.add_argument("--thermal-boxes", type=int, default=400, help="--workload thermal: the number of boxes")
    ap.add_argument("--band-solve", type=int, default=0, choices=[0, 1],
                    help="FP32 single-column band solve: 0 bulk-copy ring, 1 register prefetch (same bits)")
    ap.add_argument("--zc", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-kernel", type=int, default=0, choices=list(range(6)),
                    help="batched sweep (thermal workload): 0 autotuned, 1/3 CUDA cores, 2/4 warp MMAs, "
                         "5 tcgen05")
    ap.add_argument("--l2-persist", type=int, default=0, choices=[0, 1],
                    help="1: reflection matrices persisting in L2 during low-precision sweeps, 0: off")
    ap.add_argument("--admittance", default="alpha", choices=["alpha", "diag", "wob", "sca"],
                    help="line admittance (Sec. VIII): alpha = 1/Zc on every line (default), diag = 2g, "
                         "wob = alpha 2g, sca = partial input admittance over --radius branches")
    ap.add_argument("--method", default="vtm", choices=["vtm", "async"],
                    help="vtm: synchronous sweeps; async: asynchronous VTM (tiles read the latest "
                         "waves of their neighbours, FP32/BF16/FP16 symmetric plans)")
    ap.add_argument("--alpha", type=float, default=0.5, help="the weight of --admittance wob")
    ap.add_argument("--radius", type=int, default=1, help="the neighbourhood of --admittance sca")
    ap.add_argument("--configs", default="all", choices=["all", "none"],
                    help="all: with the default power-grid line, also time the other configurations "
                         "(Zc = 0.25 / 4, thermal 64 RHS, VCCS grid VTM / block Jacobi / admittances, "
                         "gradient step) and report them under 'configs'")
    ap.add_argument("--config-steps", type=int, default=3, help="timed steps of each extra configuration")
    ap.add_argument("--sweep-kernel", type=int, default=0, choices=list(range(13)),
                    help="0: autotuned, 1: direct-load, 2: bulk-copy staged, 3/4: vector-load (256/128 "
                         "threads), 5/6: packed symmetric (128/64 threads), 7: packed symmetric, tile by "
                         "one bulk copy, 8: packed symmetric dataflow sweeps (one launch per inner solve), "
                         "9: packed symmetric, one warp per tile, 10: kernel 9's dataflow form, 11: kernel 9 "
                         "with the block products as warp MMAs (BF16/FP16), 12: kernel 9's organisation in "
                         "double-float arithmetic on packed hi/lo FP32 pairs (FP64 plans)")
    return ap.parse_args()


def admittance_config(args):
    extra = {"method": "asynchronous VTM (one cooperative launch, latest neighbour waves)"} \
        if args.method == "async" else {}
    if args.admittance == "alpha":
        return extra
    desc = {"diag": "W = diag(C) = 2g per line (Sec. VIII choice 2)",
            "wob": f"W = {args.alpha} C = {args.alpha} * 2g per line (Sec. VIII choice 4)",
            "sca": f"W = diagonal of the partial input admittance over {args.radius} branch(es), "
                   "lower-numbered end (Sec. VIII choice 5)"}[args.admittance]
    return dict(extra, admittance=desc)


def workload_config(args):
    l2 = "flushed (512 MB write) between timed steps"
    if args.workload == "thermal":
        tg, tb = args.thermal_grid, args.thermal_boxes
        return {"workload": f"RC thermal grid {tg}x{tg}x32 ({tg * tg * 32} unknowns), G + C/h, {tb} random boxes "
                            "(200-3000 nodes), Zc=1 ohm, 64 RHS", "n": tg * tg * 32, "nrhs": 64, "tol": TOL,
                "seed": 0, "l2": l2}
    if args.workload == "vccs":
        return {"workload": "1024x1024 resistor grid + VCCS at 5% of nodes (unsymmetric), 256 tiles of 64x64, "
                            "Zc=1 ohm, 1 RHS", "n": 1048576, "nrhs": 1, "tol": TOL, "seed": 0, "l2": l2}
    if args.workload == "grad":
        return {"workload": "1024x1024 SPD grid, 256 tiles of 64x64, Zc=1 ohm; step = forward solve + adjoint "
                            "solve + branch/injection gradients of sum(x^2)", "n": 1048576, "nrhs": 1,
                "tol": TOL, "seed": 0, "l2": l2}
    return {"workload": f"power grid {args.grid}x{args.grid} (5-point, {args.grid * args.grid} unknowns), "
                        f"32x32-node tiles ({(args.grid // 32) ** 2} sub-circuits), Zc={args.zc} ohm, 1 RHS",
            "n": args.grid * args.grid, "nrhs": 1, "tol": TOL, "seed": 0, "l2": l2}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return self
        # the timed region starts once the sampler has produced its first row
        t0 = time.perf_counter()
        while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
            time.sleep(0.01)
        self.lines.clear()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on the host (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(args, workers=None):
    """Run the oracle, as it stands, on the SAMPLE_N x SAMPLE_N instance of
    the same recipe (same tile size, distributions, Zc and tolerance), from
    scratch (tearing, factorisations, sweeps).  workers = None: the plain
    single-process oracle; else its iteration spread over that many host
    processes (the same sub-circuit solves, the same iterates).  Returns
    (unknowns/s, seconds, sweeps)."""
    from oracle import vtm_oracle as O
    from oracle.vtm_oracle_mp import vtm_midpoint_mp
    from paper_0910_0663_gb300 import workloads as wl
    w = wl.power_grid(SAMPLE_N, SAMPLE_N, 32, 32, Zc=args.zc, seed=0)
    A = w.csr()
    t0 = time.perf_counter()
    if workers is None:
        res = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1.0 / w.Zc, tol=TOL)
    else:
        res = vtm_midpoint_mp(A, w.partition, w.nparts, w.b, W=1.0 / w.Zc, tol=TOL, workers=workers)
    dt = time.perf_counter() - t0
    assert res.converged
    return w.n / dt, dt, res.sweeps


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def sample_text(sweeps=None, workers=None):
    how = ("the plain single-process oracle" if workers is None else
           f"the oracle's iteration over {workers} host processes (each owns a share of the "
           f"sub-circuits; same solves, same iterates)")
    s = (f"oracle VTM (numpy/scipy, FP64, literal Eq. 11 twin-row solves), {how}, on the "
         f"{SAMPLE_N}x{SAMPLE_N} instance of the same power-grid recipe (32x32 tiles, same Zc), solved to "
         f"1e-10 from scratch (tearing, local factorisations and sweeps)")
    if sweeps is not None:
        s += f"; {sweeps} sweeps"
    return s


def sample_config(args):
    return {"workload": f"power grid {SAMPLE_N}x{SAMPLE_N} (the oracle's bounded sample of the "
                        f"{args.grid}x{args.grid} power-grid recipe: {SAMPLE_N * SAMPLE_N} unknowns, "
                        f"{(SAMPLE_N // 32) ** 2} tiles of 32x32), Zc={args.zc} ohm, 1 RHS",
            "sample_of": workload_config(args)["workload"], "n": SAMPLE_N * SAMPLE_N, "nrhs": 1,
            "tol": TOL, "seed": 0}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.vtm_oracle_mp import cpu_model
    cores = host_cores()
    vals = []
    sweeps = None
    for i in range(args.warmup + args.steps):
        v, dt, sweeps = oracle_sample(args, workers=cores)
        if i >= args.warmup:
            vals.append(dt)
    t = float(np.mean(vals))
    value = SAMPLE_N * SAMPLE_N / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": sample_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(),
                             "kind": "oracle", "sample": sample_text(sweeps, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def job_value(units_local, t_local_ms, world, device=None):
    """Whole-job throughput of N replicas: the units all ranks processed
    divided by the slowest rank's time (max over ranks).  Returns (value,
    max_ms).  For world == 1 no collective is used."""
    if world <= 1:
        return units_local / (t_local_ms * 1e-3), t_local_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return u.item() / (t.item() * 1e-3), t.item()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "of measured"
    return 6800.0, "of fallback"


def sweep_bytes(stats, prec, nrhs=1):
    """(algorithmic, overhead) bytes of one sweep launch.

    Algorithmic: the stored reflection matrices once (the entries on and
    above the diagonal for the packed symmetric kernels, every entry
    otherwise) and, per port and right-hand side, five wave words: the
    incident wave gathered from the twin, c, the outgoing wave, and the two
    words of the residual term that comes from the twin.  Overhead (kept
    apart): per port the two further wave words the kernels read for their own
    residual term, the residual coefficients (g/W, d) (2 x 8 B in FP64 and in
    the batched sweep, 2 x 4 B otherwise), the twin index (4 B) and the
    node-run byte (1 B)."""
    s_t = {0: 8, 1: 4, 2: 2, 3: 2}[prec]
    s_w = 8 if prec == 0 else 4
    s_kd = 16 if (prec == 0 or nrhs > 1) else 8
    # the packed symmetric kernels need only the entries on and above the diagonal
    entries = stats["sum_tri"] if stats.get("sweep_kernel") in (5, 6, 7, 8, 9, 10, 11, 12) and nrhs == 1 else stats["sum_p2"]
    algorithmic = entries * s_t + stats["nports"] * 5 * s_w * nrhs
    overhead = stats["nports"] * (2 * s_w * nrhs + 5 + s_kd)
    return algorithmic, overhead


def plan_rowptr(w, dev):
    import torch
    return torch.from_numpy(w.indptr).to(dev)


def plan_colidx(w, dev):
    import torch
    return torch.from_numpy(w.indices).to(dev)


def sweep_kernel_name(kernel, nrhs, batch_kernel=0):
    if nrhs > 1:
        return {1: "batch_sweep_kernel (CUDA cores, persistent)", 2: "batch_sweep_mma_kernel (warp MMAs, persistent)",
                3: "batch_sweep_kernel (CUDA cores, item per CTA)", 4: "batch_sweep_mma_kernel (warp MMAs, item per CTA)",
                5: "batch_sweep_tc_kernel (tcgen05, TMEM accumulators, bulk-copy ring)"}.get(
                    batch_kernel, "batched sweep")
    return {1: "sweep_kernel (direct loads)", 2: "sweep_staged_kernel (bulk-copy ring)",
            3: "sweep_vec_kernel (256 threads)", 4: "sweep_vec_kernel (128 threads)",
            5: "sweep_sym_kernel (packed symmetric, 128 threads)",
            6: "sweep_sym_kernel (packed symmetric, 64 registers)",
            7: "sweep_symb_kernel (packed symmetric, one bulk copy per tile)",
            8: "sweep_flow_kernel (dataflow, one cooperative launch)",
            9: "sweep_wsym_kernel (packed symmetric, one warp per tile)",
            10: "sweep_wflow_kernel (dataflow, one warp per tile, one cooperative launch)",
            11: "sweep_wmma_kernel (packed symmetric, one warp per tile, block products as warp MMAs)",
            12: "sweep_wdf_kernel (packed symmetric FP64 bytes as hi/lo FP32 pairs, double-float arithmetic, "
                "one warp per tile)"}.get(
                kernel, str(kernel))


def sweep_kernel_source_hash():
    """sha256 of the device code of the launch-per-sweep packed kernels 5-11 in
    solve.cu and their shared block code (the text from their section header to
    the next section: the double-float kernel 12, or the dataflow kernels)."""
    src = open(os.path.join(ROOT, "paper_0910_0663_gb300", "csrc", "solve.cu")).read()
    i = src.find("// Packed symmetric sweep.")
    j = src.find("// FP64-accurate packed sweep", i)
    if j < 0:
        j = src.find("// Dataflow sweeps: one cooperative launch", i)
    return hashlib.sha256(src[i:j].encode()).hexdigest() if 0 <= i < j else None


def traffic_record(prec, stats, workload):
    """ncu DRAM bytes per sweep launch (profiles/sweep_traffic.json), if they
    were captured for this precision, this sweep kernel and the unchanged
    kernel source (the file records the hash of the packed kernels' source);
    else None."""
    path = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(path) or workload != "power_grid":
        return None
    with open(path) as fh:
        rec = json.load(fh)
    if rec.get("kernel_source_sha256") != sweep_kernel_source_hash():
        return None
    entry = rec.get("per_launch", {}).get({0: "fp64", 1: "fp32", 2: "bf16", 3: "fp16"}[prec])
    if not entry or stats.get("sweep_kernel") not in entry.get("sweep_kernels", []):
        return None
    return entry.get("bytes")


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_0910_0663_gb300 import build
    build.build()
    from paper_0910_0663_gb300 import workloads as wl

    if args.workload == "thermal" and (args.thermal_grid, args.thermal_boxes) != (128, 400):
        w = wl.thermal3d(32, args.thermal_grid, args.thermal_grid, args.thermal_boxes, nrhs=64, seed=0)
    elif args.workload == "thermal":
        w = wl.c3_thermal(nrhs=64)
    elif args.workload == "vccs":
        w = wl.c4_vccs()
    elif args.workload == "grad":
        w = wl.c5_grad_grid()
    else:
        w = wl.c2_power_grid(Zc=args.zc, ny=args.grid, nx=args.grid)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    if args.workload == "vccs":
        precs = ["fp64", "bj_fp64"]
    elif args.precision == "auto":
        precs = ["fp64", "fp32", "bf16", "fp16"] if args.workload != "grad" else ["fp64", "fp32"]
        if args.method == "async":
            precs = ["fp32", "bf16", "fp16"]  # asynchronous sweeps run in FP32/16-bit only
    else:
        precs = [args.precision]
    adm = None if args.admittance == "alpha" else (args.admittance, args.alpha, args.radius)
    results = {}
    errors = {}
    for prec in precs:
        try:
            results[prec] = run_mode(prec, w, dev, stream, flush, world, args.steps, args.warmup,
                                     method="bj" if prec.startswith("bj_") else args.method, adm=adm,
                                     grad=args.workload == "grad", sweep_kernel=args.sweep_kernel,
                                     l2_persist=args.l2_persist, e2e=True, batch_kernel=args.batch_kernel,
                                     band_solve=args.band_solve)
        except Exception as exc:  # a failing mode is reported, the others still run
            errors[prec] = repr(exc)
    if not results:
        raise RuntimeError(f"every mode failed: {errors}")
    best = max(results, key=lambda p: results[p]["value"])
    configs = None
    if (args.configs == "all" and args.workload == "power_grid" and args.grid == 2048 and args.method == "vtm"
            and adm is None and args.precision == "auto" and args.sweep_kernel == 0):
        configs = run_configs(args, w, dev, stream, flush, world)
    emit(args, results, errors, best, w, world, rank, configs)
    if world > 1:
        dist.destroy_process_group()


def run_mode(prec, w, dev, stream, flush, world, steps, warmup, method="vtm", adm=None, grad=False,
             sweep_kernel=0, l2_persist=0, e2e=True, Zc=None, batch_kernel=0, band_solve=0):
    """Plan, factor and time one mode on workload w: `steps` solves after
    `warmup` untimed ones, L2 flushed before each; with e2e also the same
    solves through the C ABI with pinned host buffers.  The plan is closed
    before returning."""
    import torch
    from paper_0910_0663_gb300 import vtm
    from paper_0910_0663_gb300 import _vtm as C
    prec_name = prec.split("_")[-1]
    bsrc = w.b if w.b.shape[0] > 1 else w.b[0]
    nrhs = 1 if bsrc.ndim == 1 else bsrc.shape[0]
    b_dev = torch.from_numpy(bsrc).to(dev)
    Zc = w.Zc if Zc is None else Zc
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=Zc,
                        precision=prec_name, device=dev, stream=stream, factor=False,
                        sweep_kernel=sweep_kernel, l2_persist=l2_persist, method=method,
                        batch_kernel=batch_kernel, band_solve=band_solve)
        if adm is not None and method != "bj":
            plan.set_admittance(adm[0], alpha=adm[1], radius=adm[2], factor=False)
        t1 = time.perf_counter()
        plan.factor()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    netmap = None
    if grad:
        netmap = C.vtm_netmap_create(w.n, plan_rowptr(w, dev), plan_colidx(w, dev),
                                     len(w.edges), torch.from_numpy(w.edges[:, 0]).to(dev),
                                     torch.from_numpy(w.edges[:, 1]).to(dev), stream.cuda_stream)
        gg = torch.empty(len(w.edges), dtype=torch.float64, device=dev)
        gr = torch.empty(w.n, dtype=torch.float64, device=dev)

    def step():
        x, info = plan.solve(b_dev, tol=TOL)
        if grad:
            lam, info2 = plan.adjoint(2.0 * x, tol=TOL)
            C.vtm_netmap_gradient(netmap, lam, x, 1, gg, gr)
            info = dict(info)
            for key in ("sweeps", "kernel_launches", "sweep_launches", "t_sweeps_ms"):
                info[key] = info[key] + info2[key]
            info["relres"] = max(info["relres"], info2["relres"])
        return x, info
    try:
        for _ in range(warmup):
            with torch.cuda.stream(stream):
                x, info = step()
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        times, infos = [], []
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        # clocks are sampled over both timed regions (device-resident and
        # host-buffer calls); the host-buffer warm-up sits between them
        sampler = ClockSampler(dev.index).__enter__()
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                ev0.record(stream)
                x, info = step()
                ev1.record(stream)
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
            infos.append(info)
        t_step = float(np.mean(times))
        value, t_step = job_value(w.n * nrhs, t_step, world, dev)
        e2e_value = None
        if e2e:
            # end to end through the C ABI with host buffers (copies inside);
            # warm-up through host buffers too (the plan's staging buffers are
            # allocated by the first such call), then the timed calls
            b_host = torch.from_numpy(bsrc).pin_memory()
            x_host = torch.empty_like(b_host).pin_memory()
            e2e_t = []
            for _ in range(max(1, warmup)):
                with torch.cuda.stream(stream):
                    C.vtm_solve(plan.handle, b_host, x_host, nrhs, TOL)
            torch.cuda.synchronize()
            for _ in range(max(1, steps)):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                h0 = time.perf_counter()
                with torch.cuda.stream(stream):
                    C.vtm_solve(plan.handle, b_host, x_host, nrhs, TOL)
                h1 = time.perf_counter()
                e2e_t.append(h1 - h0)
            e2e_value = w.n * nrhs * world / float(np.mean(e2e_t))
        sampler.__exit__(None, None, None)
        st = plan.stats()
    finally:
        if netmap is not None:
            C.vtm_netmap_destroy(netmap)
        plan.close()
    inf = infos[-1]
    alg, ovh = sweep_bytes(st, {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}[prec_name], nrhs)
    # the CUDA events bracket each batch of sweep launches on the plan's
    # stream; launches past convergence in the last batch return at once
    # and stay inside the time: per sweep = batch time / sweeps run
    sweeps_eff = max(1, inf["sweeps"])
    t_sweep_launch = inf["t_sweeps_ms"] / sweeps_eff
    achieved = alg * sweeps_eff / (inf["t_sweeps_ms"] * 1e-3) / 1e9
    return dict(t_step_ms=t_step, t_plan_s=t1 - t0, t_factor_s=t2 - t1, value=value, nrhs=nrhs,
                e2e_value=e2e_value, info=inf, stats=st, bytes_sweep=alg, overhead_bytes=ovh,
                achieved_gbs=achieved, t_sweep_ms=t_sweep_launch, clocks=sampler.summary(),
                relres=max(i["relres"] for i in infos))


def run_configs(args, w2, dev, stream, flush, world):
    """The other configurations of the method's benchmark set, each timed
    like the headline (fewer steps): the power grid at Zc = 0.25 and 4 ohm,
    the RC thermal grid with 64 right-hand sides, the unsymmetric grid with
    controlled sources (VTM, block Jacobi, VTM with Sec. VIII admittances) and
    the gradient step on the 1024x1024 grid."""
    from paper_0910_0663_gb300 import workloads as wl
    steps, warmup = args.config_steps, max(1, min(args.warmup, 2))
    peak, _ = measured_peaks()
    out = {}

    def entry(name, w, prec, **kw):
        try:
            r = run_mode(prec, w, dev, stream, flush, world, steps, warmup, e2e=False, **kw)
        except Exception as exc:
            out[name] = {"error": repr(exc)}
            return
        out[name] = {"mode": prec, "sweeps": r["info"]["sweeps"], "outer_steps": r["info"]["outer_steps"],
                     "ms_per_step": r["t_step_ms"], "value": r["value"], "unit": UNIT,
                     "relres": r["relres"], "n": w.n, "nrhs": r["nrhs"],
                     "sweep_kernel": r["stats"].get("sweep_kernel"),
                     "batch_kernel": r["stats"].get("batch_kernel"),
                     "sweep_ms_per_launch": r["t_sweep_ms"],
                     "sweep_hbm_frac": r["achieved_gbs"] / peak,
                     "t_plan_s": r["t_plan_s"], "t_factor_s": r["t_factor_s"], "clocks": r["clocks"]}

    for zc in (0.25, 4.0):
        for prec in ("fp16", "fp64"):
            entry(f"power_grid_2048_zc{zc:g}_{prec}", w2, prec, Zc=zc)
    w3 = wl.c3_thermal(nrhs=64)
    for prec in ("fp32", "bf16", "fp64"):
        entry(f"thermal_128x128x32_64rhs_{prec}", w3, prec)
    entry("thermal_128x128x32_64rhs_bf16_tcgen05", w3, "bf16", batch_kernel=5)
    entry("thermal_128x128x32_64rhs_bf16_mma_sync", w3, "bf16", batch_kernel=2)
    entry("thermal_128x128x32_64rhs_fp32_sca1", w3, "fp32", adm=("sca", 1.0, 1))
    del w3
    w4 = wl.c4_vccs()
    entry("vccs_1024_vtm_fp64", w4, "fp64")
    entry("vccs_1024_bj_fp64", w4, "bj_fp64", method="bj")
    entry("vccs_1024_vtm_sca1_fp64", w4, "fp64", adm=("sca", 1.0, 1))
    entry("vccs_1024_vtm_wob0.5_fp64", w4, "fp64", adm=("wob", 0.5, 1))
    del w4
    w5 = wl.c5_grad_grid()
    entry("grad_1024_forward_adjoint_gradient_fp32", w5, "fp32", grad=True)
    return out


def emit(args, results, errors, best, w, world, rank, configs=None):
    R = results[best]
    peak, peak_src = measured_peaks()
    prec_id = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}[best.split("_")[-1]]
    line = {
        "metric": METRIC, "value": R["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": R["t_step_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32+f64 refinement", "bf16": "bf16+f64 refinement",
                  "fp16": "f16+f64 refinement"}[best.split("_")[-1]],
        "data": "synthetic", "config": dict(workload_config(args), precision=best,
                                            **admittance_config(args)),
        "roofline": {"bound": "hbm", "kernel": sweep_kernel_name(R["stats"].get("sweep_kernel"), R["nrhs"],
                                                                 R["stats"].get("batch_kernel", 0)),
                     "achieved": R["achieved_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": R["achieved_gbs"] / peak, "peak_source": peak_src,
                     "traffic": traffic_record(prec_id, R["stats"], args.workload)
                     if args.grid == 2048 else None,
                     "algorithmic_bytes_per_launch": R["bytes_sweep"],
                     "overhead_bytes_per_launch": R["overhead_bytes"],
                     "avg_launch_ms": R["t_sweep_ms"]},
        "e2e": {"value": R["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": w.n * 8 * R["nrhs"],
                "d2h_bytes_per_step": w.n * 8 * R["nrhs"]},
        "gpu_launches": R["info"]["kernel_launches"],
        "clocks": R["clocks"],
        "sweeps": R["info"]["sweeps"], "outer_steps": R["info"]["outer_steps"],
        "relres": R["relres"],
        "setup": {"t_plan_s": R["t_plan_s"], "t_factor_s": R["t_factor_s"],
                  "t_plan_factor_solve_s": R["t_plan_s"] + R["t_factor_s"] + R["t_step_ms"] * 1e-3},
        "modes": {p: {"value": r["value"], "ms_per_step": r["t_step_ms"], "sweeps": r["info"]["sweeps"],
                      "outer_steps": r["info"]["outer_steps"], "relres": r["relres"],
                      "sweep_gbs": r["achieved_gbs"], "sweep_hbm_frac": r["achieved_gbs"] / peak,
                      "t_plan_s": r["t_plan_s"], "t_factor_s": r["t_factor_s"],
                      "sweep_ms_per_launch": r["t_sweep_ms"], "sweep_kernel": r["stats"].get("sweep_kernel"),
                      "gpu_launches": r["info"]["kernel_launches"]}
                  for p, r in results.items()},
    }
    if errors:
        line["mode_errors"] = errors
    if "fp64" in results:
        line["vs_plain_fp64"] = R["value"] / results["fp64"]["value"]
    if configs is not None:
        line["configs"] = configs
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "power_grid":
        from oracle.vtm_oracle_mp import cpu_model
        cores = host_cores()
        v, dt, sweeps = oracle_sample(args, workers=cores)
        v1, dt1, _ = oracle_sample(args)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(),
                                "kind": "oracle", "sample": sample_text(sweeps, cores), "seconds": dt,
                                "single_process": {"value": v1, "seconds": dt1, "cores": 1}}
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
