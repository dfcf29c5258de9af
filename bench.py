"""Benchmark: stationary DFM solves per second on one GB300 (or N replicas).

One step = the device-resident hot path on the 20^3 Kuhn-cube workload
(48,000 jittered tets, Np = 4, mu = 0.05, r = 0.95, one boundary-face source):
assemble the operator B (FP32 blocks, FP64 geometry set-up), project the
source, and solve (I - B) rho = rho0 by FP64-residual iterative refinement
around FP32 GMRES to a relative residual of 1e-8.  Inputs (mesh on device)
are resident when the timed region starts; the operator (518 MB) and Krylov
basis are larger than L2, so no flush is needed between steps.

The e2e figure runs the same metric through the C ABI from HOST buffers:
mesh arrays copied in (face matching and geometry run every step), the
solution copied back to pinned host memory, all inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
Under torchrun (N > 1) every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "stationary solves/s at 1e-6 rel err"
WORKLOAD = "kuhn20_np4"
WORKLOAD_DESC = ("20^3 Kuhn cube x 6 = 48,000 jittered tets (jitter 0.2h, seed 0); Np = 4 (15 Zernike functions); "
                 "mu = 0.05; boundary reflection 0.95; unit isotropic source on the x = 0 face at (0, 1/2, 1/2); "
                 "solve to FP64 relative residual 1e-8")
SOLVER_DESC = {
    "f32": "FP64-residual refinement around FP32 GMRES({restart}) right-preconditioned by sum_{{k<{d}}} B^k",
    "f16": ("FP64-residual refinement around flexible FP32 GMRES({restart}) right-preconditioned by sum_{{k<{d}}} B^k "
            "evaluated on an FP16 copy of the blocks"),
    "bf16": ("FP64-residual refinement around flexible FP32 GMRES({restart}) right-preconditioned by sum_{{k<{d}}} B^k "
             "evaluated on a BF16 copy of the blocks"),
    "fp8": ("FP64-residual refinement around flexible FP32 GMRES({restart}) right-preconditioned by sum_{{k<{d}}} B^k "
            "evaluated on an e4m3 copy of the blocks (one FP32 scale per row)"),
}
# Operator applications of the FP64 solve on the 20^3 workload: FP64 GMRES(128)
# right-preconditioned by sum_{k<16} B^k reaches the 1e-8 residual after 1,809
# applications (the count the FP64 comparator path records).  The oracle arm
# charges its measured per-application cost this many times.
REF_APPLICATIONS = {"kuhn20_np4": 1809}
FP32_LANES_PER_SM = 128
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# step's dominant kernel measured by ncu on this workload (mean of two
# launches; profiles/hop_e4m3_kuhn20_np4.md).  Keyed by the kernel instantiation and
# workload; an entry is dropped whenever its kernel changes.
PRECOND = {"f32": 0, "f16": 3, "bf16": 2, "fp8": 4}
MEASURED_TRAFFIC = {("hop_kernel<15, __nv_fp8_e4m3>", "kuhn20_np4"): 159.2e6}
HBM_PEAK_FALLBACK = 6800.0
# the timed region records CUDA events around every STATS_EVERY-th launch of
# each kernel (per-kernel durations); an event pair per launch would add ~9%
# to the step
STATS_EVERY = 16


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": HBM_PEAK_FALLBACK, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws, device):
    """The largest of every rank's `value` (a time): replicas run independently
    and the job takes as long as its slowest rank."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def flops_per_node(Np: int) -> int:
    """Counted FP32 operations per quadrature node of the assembly kernel: the
    rank-1 block update (2 nb^2), two Zernike vectors (complex powers 6 per
    order, radial recursion and angular products ~4 per function) and the node
    geometry (bilinear map, Jacobian, closed-form S, phi2: 130)."""
    nb = (Np + 1) * (Np + 2) // 2
    return 2 * nb * nb + 2 * (6 * Np + 4 * nb) + 130


def spmv_bytes(n_rows, nb, vec_bytes, with_x0=True, block_bytes=4):
    """Algorithmic bytes of one y = x0 + alpha B x: blocks and row map read
    once, x read once, x0 read once, y written once."""
    return n_rows * (3 * nb * nb * block_bytes + 4 + nb * vec_bytes * (3 if with_x0 else 2))


def summarize_kernels(kstats, n_rows, n_tets, Np, nodes, nsm, peaks, peak_src, workload, precond):
    """Per-kernel rooflines of a timed region and the dominant kernel's.
    kstats: name -> (launches, total ms) for assemble, spmv_f32, hop (the
    preconditioner's hops on the low-precision copy, precond "f16", "bf16" or
    "fp8"),
    spmv_f64vec, dot, axpy.  Returns (per-kernel dict, total ms per kernel,
    roofline of the kernel with the largest total among assemble/spmv)."""
    nb = (Np + 1) * (Np + 2) // 2
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tflops = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    kern = {}

    def hbm(name, n, ms, by):
        ach = by / (ms / n * 1e-3) / 1e9
        kern[name] = {"bound": "hbm", "launches": n, "ms_per_launch": ms / n, "achieved": ach, "peak": hbm_peak,
                      "unit": "GB/s", "frac": ach / hbm_peak, "bytes_per_launch": by}

    n_asm, ms_asm = kstats["assemble"]
    if n_asm:
        fl = nodes * flops_per_node(Np)  # per launch (every launch of the step is identical)
        ach = fl / (ms_asm / n_asm * 1e-3) / 1e12
        kern["assemble"] = {"bound": "alu", "launches": n_asm, "ms_per_launch": ms_asm / n_asm,
                            "achieved": ach, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                            "frac": ach / fp32_peak_tflops, "nodes_per_launch": nodes,
                            "flops_per_node": flops_per_node(Np),
                            "blocks_per_s": 12 * n_tets / (ms_asm / n_asm * 1e-3)}
    n, ms = kstats["spmv_f32"]
    if n:
        # with a 16-bit preconditioner copy the FP32 launches are the Krylov
        # operator w = z - B z (x0 = z); without it most are polynomial hops
        # without x0
        hbm("spmv_f32", n, ms, spmv_bytes(n_rows, nb, 4, with_x0=precond != "f32"))
    n, ms = kstats["hop"]
    if n:
        # unpadded copy values (+ the FP32 scale of an e4m3 row), row map, and
        # x, x0, y in the hop vectors' precision (FP16 with the FP16 and e4m3
        # copies, FP32 with the BF16 copy)
        eb = 1 if precond == "fp8" else 2
        vb = 4 if precond == "bf16" else 2
        hbm("hop", n, ms, spmv_bytes(n_rows, nb, vb, with_x0=True, block_bytes=eb) + (4 * n_rows if eb == 1 else 0))
    n, ms = kstats["spmv_f64vec"]
    if n:
        hbm("spmv_f64vec", n, ms, spmv_bytes(n_rows, nb, 8))
    for name in ("dot", "axpy"):
        n, ms = kstats[name]
        if n:
            kern[name] = {"launches": n, "ms_total": ms}
    total = {k: v[1] for k, v in kstats.items()}
    dominant = max((k for k in ("assemble", "spmv_f32", "hop") if k in kern), key=lambda k: total[k])
    d = kern[dominant]
    inst = {"spmv_f32": f"spmv_tma_kernel<{nb}, 1, float, float, float>",
            "hop": f"hop_kernel<{nb}, {dict(f16='__half', bf16='__nv_bfloat16', fp8='__nv_fp8_e4m3').get(precond)}>"
            }.get(dominant)
    traffic = MEASURED_TRAFFIC.get((inst, workload)) if inst else None
    roofline = {"bound": d["bound"], "achieved": round(d["achieved"], 3), "peak": round(d["peak"], 3),
                "unit": d["unit"], "frac": round(d["frac"], 4), "traffic": traffic, "kernel": dominant,
                "peak_source": peak_src if d["bound"] == "hbm" else
                f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz"}
    return kern, total, roofline


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    w = workload(args.workload)
    m = w["mesh"]
    Np = w["Np"]
    tol = args.tol if args.tol else w["tol"]
    mu = float(w["mu"][0])
    rows = np.asarray(w["sources"], dtype=np.int64)
    dfm.load()

    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])
    op = dfm.Operator(mesh, Np, mu=mu, precision=dfm.F32)
    method = dfm.GMRES_IR

    def step():
        op.reassemble(mu)
        rho0 = dfm.source(mesh, Np, rows)
        rho, info = op.solve(rho0, method=method, tol=tol, restart=args.restart, poly_degree=args.poly,
                             precond_precision=PRECOND[args.precond])
        return rho, info

    for _ in range(args.warmup):
        rho, info = step()
    torch.cuda.synchronize()

    # ---- timed region: device-resident steps --------------------------------
    sampler = ClockSampler(local)
    dfm.stats_reset()
    dfm.stats_enable(STATS_EVERY)
    l0 = dfm.launch_count()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    infos = []
    for _ in range(args.steps):
        rho, info = step()
        infos.append((info.iters, info.outer, info.resid))
    e1.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = dfm.launch_count() - l0
    dfm.stats_enable(False)
    elapsed_ms = e0.elapsed_time(e1)
    kstats = {k: dfm.kernel_stats(k) for k in (dfm.KERNEL_ASSEMBLE, dfm.KERNEL_SPMV, dfm.KERNEL_SPMV64,
                                                dfm.KERNEL_DOT, dfm.KERNEL_AXPY, dfm.KERNEL_SPMV16)}
    nodes = dfm.op_nodes(op)
    elapsed_ms = max_over_ranks(elapsed_ms, ws, "cuda")

    # ---- e2e: C ABI from host buffers, copies inside the timed region --------
    e2e = None
    if not args.no_e2e:
        host_rho = torch.empty((1, mesh.n_rows, op.nb), dtype=torch.float64, pin_memory=True)
        verts = np.ascontiguousarray(m.verts)
        tets = np.ascontiguousarray(m.tets)

        def e2e_step():
            mh = dfm.Mesh(verts, tets, refl=w["refl"])
            o = dfm.Operator(mh, Np, mu=mu, precision=dfm.F32)
            r0 = dfm.source(mh, Np, rows)
            x, inf = o.solve(r0, method=method, tol=tol, restart=args.restart, poly_degree=args.poly,
                             precond_precision=PRECOND[args.precond])
            host_rho.copy_(x, non_blocking=True)
            torch.cuda.synchronize()
            o.close()
            mh.close()
            return inf

        e2e_step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, ws, "cuda")
        h2d = verts.nbytes + tets.nbytes + 4 * m.n_tets * 8 + rows.nbytes
        d2h = host_rho.numel() * 8
        e2e = {"value": ws * max(1, args.steps) / dt, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    peaks, peak_src = _peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    nb = op.nb
    kern, total, roofline = summarize_kernels(
        {"assemble": kstats[dfm.KERNEL_ASSEMBLE], "spmv_f32": kstats[dfm.KERNEL_SPMV],
         "hop": kstats[dfm.KERNEL_SPMV16], "spmv_f64vec": kstats[dfm.KERNEL_SPMV64],
         "dot": kstats[dfm.KERNEL_DOT], "axpy": kstats[dfm.KERNEL_AXPY]},
        n_rows=mesh.n_rows, n_tets=int(m.n_tets), Np=Np, nodes=nodes, nsm=nsm, peaks=peaks, peak_src=peak_src,
        workload=args.workload, precond=args.precond)

    iters = [i[0] for i in infos]
    res = {
        "metric": METRIC,
        "value": ws * args.steps / (elapsed_ms * 1e-3),
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32 blocks/Krylov, f64 residual" if args.precond == "f32" else
                  f"f32 blocks, {args.precond} preconditioner copy, f32 Krylov, f64 residual"),
        "data": "synthetic",
        "config": {"workload": args.workload,
                   "desc": (WORKLOAD_DESC if args.workload == WORKLOAD else args.workload) + "; "
                   + SOLVER_DESC[args.precond].format(
                       restart=args.restart or 128, d=args.poly or (16 if args.precond == "f32" else 48)),
                   "n_tets": int(m.n_tets), "n_rows": int(mesh.n_rows), "nb": nb, "tol": tol,
                   "restart": args.restart or 128, "poly_degree": args.poly or (16 if args.precond == "f32" else 48), "precond": args.precond, "l2": "inputs larger than L2 (operator %.0f MB)" % (op.bytes / 1e6),
                   "parallelism": f"replicas x{ws}"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "assembly_blocks_per_s": kern.get("assemble", {}).get("blocks_per_s"),
        "solve": {"operator_applications": iters[-1], "refinements": infos[-1][1], "resid": infos[-1][2]},
        "kernels": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                    for k, v in kern.items()},
        "kernel_ms_per_step": {k: round(v / args.steps, 4) for k, v in total.items()},
    }
    if not args.no_comparator:
        res["fp64_gpu_path"] = fp64_comparator(dfm, mesh, Np, mu, rows, tol)
    if ws == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args.workload, op_apps=iters[-1], seconds=args.cpu_seconds)
    print(json.dumps(res))
    if ws > 1:
        dist.destroy_process_group()


def fp64_comparator(dfm, mesh, Np, mu, rows, tol):
    """The plain FP64 GPU path on the same workload: FP64 assembly and FP64
    GMRES (same polynomial preconditioner, restart) to the same residual.
    One warm-up and one timed solve."""
    import torch

    def once():
        op = dfm.Operator(mesh, Np, mu=mu, precision=dfm.F64)
        rho0 = dfm.source(mesh, Np, rows)
        rho, info = op.solve(rho0, method=dfm.GMRES, tol=tol, poly_degree=16)
        op.close()
        return info

    once()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    info = once()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": 1e3 / ms, "unit": "solves/s", "ms_per_solve": ms, "operator_applications": info.iters,
            "resid": info.resid, "desc": "FP64 blocks, FP64 GMRES(128) with sum_{k<16} B^k, same tolerance"}


# ---------------------------------------------------------------------------
# CPU oracle (reported baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_sample(wname, seconds, op_apps=None):
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload:
    (a) adaptive (1e-13) assembly of randomly drawn face pairs until about
    `seconds`/2 of wall time, giving seconds per block; (b) restarted GMRES
    iterations of the oracle at full size on an operator with the workload's
    sparsity, giving seconds per operator application (block values do not
    change the work).  Extrapolated solve time = (a) x 12 N + (b) x op_apps."""
    import oracle
    from paper_1608_04607_gb300.inputs import workload

    w = workload(wname)
    m = w["mesh"]
    Np = w["Np"]
    nb = (Np + 1) * (Np + 2) // 2
    threads = os.cpu_count() or 1
    topo = oracle.topology(m.tets)
    t, f, fp = oracle.pair_list(m.n_tets)
    rng = np.random.default_rng(0)
    mu = w["mu"] if "mu" in w else np.full(m.n_tets, 0.05)
    # (a) assembly sample, grown until the time budget is used
    n_pairs = 0
    t_asm = 0.0
    batch = max(threads, 8)
    while t_asm < 0.5 * seconds:
        sel = rng.integers(0, t.size, size=batch)
        t0 = time.perf_counter()
        oracle.blocks_for_pairs(m.verts, m.tets, topo, mu, w["refl"], Np, t[sel], f[sel], fp[sel], rtol=1e-13)
        t_asm += time.perf_counter() - t0
        n_pairs += batch
        batch *= 2
    per_block = t_asm / n_pairs
    # the same assembly on one thread (a fixed sample of 32 pairs)
    sel = rng.integers(0, t.size, size=32)
    t0 = time.perf_counter()
    oracle.blocks_for_pairs(m.verts, m.tets, topo, mu, w["refl"], Np, t[sel], f[sel], fp[sel], rtol=1e-13, nthreads=1)
    per_block_1t = (time.perf_counter() - t0) / 32
    # (b) oracle GMRES iterations at full size
    blocks = rng.standard_normal((4 * m.n_tets, 3, nb, nb)) * (0.3 / nb)
    dest = topo.recv[4 * np.repeat(np.arange(m.n_tets), 12) + fp].reshape(4 * m.n_tets, 3)
    op = oracle.Operator(Np=Np, blocks=blocks, dest=dest)
    rho0 = oracle.source_vector(m.verts, m.tets, w["sources"][:1], Np)
    k = 16
    t0 = time.perf_counter()
    oracle.solve_gmres(op, rho0, tol=1e-300, restart=64, maxit=k)
    per_app = (time.perf_counter() - t0) / k
    if op_apps is None:
        op_apps = 0
    est = per_block * 12 * m.n_tets + per_app * op_apps
    sample = (f"oracle assembly of {n_pairs} random face pairs (adaptive to 1e-13) and {k} oracle GMRES(64) "
              f"iterations at full size; extrapolated to 12 x {m.n_tets} blocks + {op_apps} operator applications")
    return est, sample, threads, per_block, per_app, per_block_1t


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def cpu_baseline(wname, op_apps, seconds=20.0):
    est, sample, threads, per_block, per_app, per_block_1t = _oracle_sample(wname, seconds, op_apps)
    return {"value": 1.0 / est, "unit": "solves/s", "cores": threads, "kind": "oracle", "sample": sample,
            "s_per_block": per_block, "s_per_block_1thread": per_block_1t, "s_per_application": per_app,
            "cpu_model": _cpu_model()}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    # a full oracle solve takes about half an hour of CPU time, so each step
    # times the oracle on a bounded sample (assembly of random face pairs and
    # full-size GMRES iterations) and extrapolates to the whole solve with the
    # FP64 path's application count
    from paper_1608_04607_gb300.inputs import workload

    wl = workload(args.workload)
    apps = args.ref_apps or REF_APPLICATIONS.get(args.workload, 2000)
    vals = []
    last = None
    for i in range(args.warmup + args.steps):
        est, sample, threads, _, _, _ = _oracle_sample(args.workload, args.cpu_seconds / 2, apps)
        if i >= args.warmup:
            vals.append(est)
        last = (sample, threads)
    v = 1.0 / statistics.mean(vals)
    res = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(vals) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload,
                      "desc": (WORKLOAD_DESC if args.workload == WORKLOAD else args.workload)
                      + "; FP64 CPU oracle (adaptive assembly to 1e-13, restarted GMRES), timed on a bounded sample",
                      "n_tets": int(wl["mesh"].n_tets), "n_rows": int(wl["mesh"].n_rows),
                      "nb": (wl["Np"] + 1) * (wl["Np"] + 2) // 2, "tol": args.tol or wl["tol"]},
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": last[1], "kind": "oracle", "sample": last[0]},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def run_apply(args):
    """Operator-application micro-benchmark: K timed y = x0 - B x launches
    (FP32 vectors) on the workload's assembled operator, for the SpMV roofline
    and for profiling the kernel in isolation."""
    import torch

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    torch.cuda.set_device(0)
    w = workload(args.workload)
    m = w["mesh"]
    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])
    op = dfm.Operator(mesh, w["Np"], mu=float(w["mu"][0]), precision=dfm.F32)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((1, mesh.n_rows, op.nb), device="cuda", dtype=torch.float32, generator=g)
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        op.apply(x, x0=x, alpha=-1.0, out=y)
    torch.cuda.synchronize()
    dfm.stats_reset()
    dfm.stats_enable(True)
    for _ in range(args.steps):
        op.apply(x, x0=x, alpha=-1.0, out=y)
    torch.cuda.synchronize()
    n, ms = dfm.kernel_stats(dfm.KERNEL_SPMV)
    dfm.stats_enable(False)
    peaks, src = _peaks()
    by = spmv_bytes(mesh.n_rows, op.nb, 4, with_x0=True)
    ach = by / (ms / n * 1e-3) / 1e9
    print(json.dumps({"mode": "apply", "workload": args.workload, "launches": n, "ms_per_launch": ms / n,
                      "bytes_per_launch": by, "achieved_gbs": ach, "peak_gbs": peaks.get("hbm_gbs"),
                      "frac": ach / float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)), "peak_source": src}))


def run_hop(args):
    """Preconditioner-hop micro-benchmark: z = sum_{k<9} B~^k x (8 hops per
    call) on the workload's low-precision copy (--precond) for --rhs
    right-hand sides (default 1), timed per hop launch with CUDA events."""
    import torch

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    torch.cuda.set_device(0)
    w = workload(args.workload)
    m = w["mesh"]
    R = args.rhs or 1
    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])
    prec = dfm.BF16 if w["Np"] >= 8 else dfm.F32
    op = dfm.Operator(mesh, w["Np"], mu=float(np.asarray(w["mu"]).reshape(-1)[0]), precision=prec)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((R, mesh.n_rows, op.nb), device="cuda", dtype=torch.float32, generator=g)
    x /= x.norm(dim=(1, 2), keepdim=True)
    pp = PRECOND[args.precond]
    for _ in range(args.warmup):
        op.precond(x, degree=9, precision=pp)
    torch.cuda.synchronize()
    dfm.stats_reset()
    dfm.stats_enable(True)
    for _ in range(args.steps):
        op.precond(x, degree=9, precision=pp)
    torch.cuda.synchronize()
    n, ms = dfm.kernel_stats(dfm.KERNEL_SPMV16)
    dfm.stats_enable(False)
    nb = op.nb
    eb = 1 if args.precond == "fp8" else 2
    vb = 4 if args.precond == "bf16" else 2
    by = mesh.n_rows * (3 * nb * nb * eb + 4 + (4 if eb == 1 else 0)) + 3 * nb * vb * mesh.n_rows * R
    peaks, src = _peaks()
    ach = by / (ms / n * 1e-3) / 1e9
    print(json.dumps({"mode": "hop", "workload": args.workload, "precond": args.precond, "rhs": R, "launches": n,
                      "ms_per_launch": ms / n, "bytes_per_launch": by, "achieved_gbs": ach,
                      "frac": ach / float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)), "peak_source": src}))


def fp64_sample(dfm, mesh, Np, mus, rows, tol, per_rhs_assembly):
    """The plain FP64 GPU path on a sample of a multi-source workload: FP64
    blocks and FP64 GMRES(128) with sum_{k<16} B^k (the settings of the
    single-source comparator), one solve per source, to the same residual.
    With per_rhs_assembly every source has its own damping, so its FP64
    operator is assembled inside the timed region, as the mixed-precision
    step assembles its moments; otherwise one operator serves all sources and
    only the solves are timed.  The first source is solved once untimed."""
    import torch

    shared = None if per_rhs_assembly else dfm.Operator(mesh, Np, mu=float(mus[0]), precision=dfm.F64)

    def one(mu, row):
        op = dfm.Operator(mesh, Np, mu=float(mu), precision=dfm.F64) if per_rhs_assembly else shared
        rho, info = op.solve(dfm.source(mesh, Np, [int(row)]), method=dfm.GMRES, tol=tol, poly_degree=16,
                             restart=128)
        if per_rhs_assembly:
            op.close()
        return info

    one(mus[0], rows[0])
    times, apps = [], []
    for mu, row in zip(mus, rows):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        info = one(mu, row)
        ev[1].record()
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
        apps.append(int(info.iters))
    if shared is not None:
        shared.close()
    ms = sum(times)
    return {"value": len(times) / (ms * 1e-3), "unit": "solves/s", "ms_per_solve": ms / len(times),
            "sample": f"the first {len(times)} sources", "operator_applications": apps,
            "assembly_in_timed_region": bool(per_rhs_assembly),
            "desc": "FP64 blocks, FP64 GMRES(128) with sum_{k<16} B^k, same tolerance"}


def run_batched(args):
    """Batched workload: 128 right-hand sides (random boundary-face sources) on
    the 30^3 Kuhn cube (162,000 tets, Np = 4), each with its own uniform damping
    mu_r ~ U[0.01, 0.2].  The operator depends on mu, so the step assembles
    K = 3 damping moments B^(k) = d^k B / d mu^k at mu_c = 0.105 once and
    solves all right-hand sides with B(mu_r) = sum_k (mu_r - mu_c)^k / k! B^(k)
    (truncation below 1e-7 for these tets), in lockstep groups that share
    every operator pass, to an FP64 relative residual of 1e-6.  With
    --precond f16/bf16/fp8 the polynomial preconditioner's hops run on a
    low-precision copy of B(mu_c) alone (flexible inner solve)."""
    import torch

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    torch.cuda.set_device(0)
    wname = args.workload if args.workload != WORKLOAD else "kuhn30_np4_rhs128"
    w = workload(wname)
    m = w["mesh"]
    Np = w["Np"]
    mu_rhs = w["mu_rhs"][: args.rhs] if args.rhs else w["mu_rhs"]
    rows = np.asarray(w["sources"], dtype=np.int64)[: len(mu_rhs)]
    R = len(mu_rhs)
    tol = args.tol if args.tol else w["tol"]
    mu_c, K = 0.105, 3
    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])
    ops = [dfm.Operator(mesh, Np, mu=mu_c, precision=dfm.F32, moment=k) for k in range(K)]

    def step():
        for o in ops:
            o.reassemble(mu_c)
        rho0 = dfm.source(mesh, Np, rows)
        # degree 64 with restart 32: 7.6 solves/s against 6.6 with degree 32, restart 128
        return dfm.solve_damped(ops, mu_rhs, rho0, tol=tol, batch=args.batch, poly_degree=args.poly or 64,
                                restart=args.restart or 32, precond_precision=PRECOND[args.precond])

    rho, info = step()
    torch.cuda.synchronize()
    dfm.stats_reset()
    dfm.stats_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    rho, info = step()
    e1.record()
    torch.cuda.synchronize()
    dfm.stats_enable(False)
    ms = e0.elapsed_time(e1)
    n_sp, ms_sp = dfm.kernel_stats(dfm.KERNEL_SPMV)
    n_as, ms_as = dfm.kernel_stats(dfm.KERNEL_ASSEMBLE)
    n_hop, ms_hop = dfm.kernel_stats(dfm.KERNEL_SPMV16)
    res = {"mode": "batched", "workload": wname, "n_tets": int(m.n_tets), "rhs": R, "K": K,
           "value": R / (ms * 1e-3), "unit": "solves/s", "ms_per_step": ms, "precond": args.precond,
           "operator_passes": info.iters, "resid_worst": info.resid,
           "assembly_ms": ms_as, "combo_launches": n_sp, "combo_ms": ms_sp,
           "hop_launches": n_hop, "hop_ms": ms_hop,
           "dot_ms": dfm.kernel_stats(dfm.KERNEL_DOT)[1], "axpy_ms": dfm.kernel_stats(dfm.KERNEL_AXPY)[1]}
    if args.fp64_sample:
        for o in ops:
            o.close()
        del rho
        n = min(args.fp64_sample, R)
        res["fp64_comparator"] = fp64_sample(dfm, mesh, Np, mu_rhs[:n], rows[:n], tol, per_rhs_assembly=True)
    print(json.dumps(res))


def run_cuboid(args):
    """Cuboid verification of Sec. 4.1 on the GPU: the Kuhn cuboid
    (0, 2) x (-1/2, 1/2)^2 with n cells per unit length (n = 4: 768 tets, the
    size of the paper's 972-tet mesh; n = 8: 6,144 tets), every wall
    reflecting (r = 1), mu = eta omega / (2c) = 0.4 pi (eta = 0.004,
    omega = 200 pi, c = 1) and a unit density entering the x = 0 side along
    its normal (Eq. RhoNeumann).  Each step of a case re-assembles B in FP32,
    solves to an FP64 relative residual of 1e-10 and reads rho_T at every
    centroid (Eq. IntDens); the line gives each case's median step time and
    the relative mean error (mean |rho_T - rho*| / mean rho*) against the
    exact ray solution rho* of Eq. ExactSol."""
    import torch

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import cuboid_rows_x0, kuhn_cuboid_mesh

    torch.cuda.set_device(0)
    mu, length = 0.4 * np.pi, 2.0
    cases = []
    for n in (4, 8):
        m = kuhn_cuboid_mesh(n, length=length)
        mesh = dfm.Mesh(m.verts, m.tets, refl=1.0)
        rows = cuboid_rows_x0(m)
        x = m.verts[m.tets].mean(axis=1)[:, 0]
        exact = (np.exp(-mu * x) + np.exp(-mu * (2 * length - x))) / (1 - np.exp(-2 * mu * length))
        tets = np.arange(m.n_tets)
        for Np in (4, 6, 8):
            op = dfm.Operator(mesh, Np, mu=mu, precision=dfm.F32)

            def step():
                op.reassemble(mu)
                rho0 = dfm.source_directed(mesh, Np, rows, combine=True)
                rho, info = op.solve(rho0, tol=1e-10)
                g, _ = dfm.interior_density(mesh, Np, tets, mu=mu)
                return dfm.tet_density(mesh, Np, g, rho), info

            for _ in range(max(args.warmup, 1)):
                step()
            times = []
            for _ in range(max(args.steps, 1)):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                torch.cuda.synchronize()
                ev[0].record()
                dens, info = step()
                ev[1].record()
                torch.cuda.synchronize()
                times.append(ev[0].elapsed_time(ev[1]))
            d = dens.cpu().numpy()
            err = float(np.mean(np.abs(d - exact)) / np.mean(exact))
            cases.append({"n_tets": m.n_tets, "Np": Np, "ms_per_step": statistics.median(times),
                          "rel_mean_err": err, "operator_applications": info.iters, "resid": info.resid})
            op.close()
        mesh.close()
    print(json.dumps({"metric": "cuboid relative mean error against the exact ray solution", "mode": "cuboid",
                      "value": cases[2]["rel_mean_err"], "unit": "fraction", "higher_is_better": False,
                      "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
                      "config": {"workload": "kuhn cuboid 2 x 1 x 1, n = 4 and 8 cells per unit length",
                                 "mu": mu, "refl": 1.0, "source": "normal incidence on x = 0", "tol": 1e-10},
                      "cases": cases}))


def run_many(args):
    """Many-source workload with a 45-function basis: the 32^3 Kuhn cube
    (196,608 tets, Np = 8, mu = 0.05, r = 0.95) with 64 random boundary-face
    sources.  One step assembles the operator in BF16 (9.6 GB), solves all 64
    right-hand sides to an FP64 relative residual of 1e-6 (FP64-residual
    refinement around flexible FP32 GMRES in lockstep groups, preconditioned by
    sum_{k<d} B~^k on an e4m3 copy of the blocks), and runs the adjoint of
    J = sum_r mean receiver density (cells [14,18)^3): one transposed solve and
    the dB/dmu contraction for all 64 solutions."""
    import torch

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    torch.cuda.set_device(0)
    wname = args.workload if args.workload != WORKLOAD else "kuhn32_np8_rhs64"
    w = workload(wname)
    m = w["mesh"]
    Np = w["Np"]
    rows = np.asarray(w["sources"], dtype=np.int64)[: (args.rhs or len(w["sources"]))]
    R = len(rows)
    tol = args.tol if args.tol else w["tol"]
    mu = float(w["mu"][0])
    receiver = w["receiver"]
    # degree 64 with restart 32 needs 36% fewer operator passes than degree 32
    # with restart 64 here (29,728 against 46,228 for the 64 sources)
    restart = args.restart or 32
    poly = args.poly or 64
    batch = args.batch or 8
    precond = PRECOND[args.precond]
    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])
    op = dfm.Operator(mesh, Np, mu=mu, precision=dfm.BF16)
    g, dg = dfm.interior_density(mesh, Np, receiver, weights=1.0 / len(receiver), mu=mu)

    def solve(rho0):
        return op.solve(rho0, tol=tol, restart=restart, poly_degree=poly, batch=batch, precond_precision=precond)

    rho, info = solve(dfm.source(mesh, Np, rows))  # warm-up (allocations)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    dfm.stats_reset()
    dfm.stats_enable(True)
    ev[0].record()
    op.reassemble(mu)
    ev[1].record()
    rho, info = solve(dfm.source(mesh, Np, rows))
    ev[2].record()
    lam, dj, ainfo = op.adjoint(rho, g, dg, tol=tol, restart=restart, poly_degree=poly, precond_precision=precond)
    ev[3].record()
    torch.cuda.synchronize()
    dfm.stats_enable(False)
    asm_ms, solve_ms, adj_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])
    peaks, peak_src = _peaks()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    ks = {name: dfm.kernel_stats(k) for name, k in (("assemble", dfm.KERNEL_ASSEMBLE), ("spmv", dfm.KERNEL_SPMV),
                                                    ("hop", dfm.KERNEL_SPMV16), ("spmv_t", dfm.KERNEL_SPMV_T),
                                                    ("spmv_f64vec", dfm.KERNEL_SPMV64), ("contract", dfm.KERNEL_CONTRACT),
                                                    ("dot", dfm.KERNEL_DOT), ("axpy", dfm.KERNEL_AXPY))}
    nb = op.nb
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    Rl = min(batch, R)
    kern = {}
    n, ms = ks["assemble"]
    if n:
        fl = dfm.op_nodes(op) * flops_per_node(Np)
        fp32_peak = nsm * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        ach = fl / (ms / n * 1e-3) / 1e12
        kern["assemble"] = {"bound": "alu", "ms_per_launch": ms / n, "achieved": ach, "peak": fp32_peak,
                            "unit": "TFLOP/s", "frac": ach / fp32_peak, "blocks_per_s": 12 * m.n_tets / (ms / n * 1e-3)}

    def hbm(name, by):
        n, ms = ks[name]
        if n:
            ach = by / (ms / n * 1e-3) / 1e9
            kern[name] = {"bound": "hbm", "launches": n, "ms_per_launch": ms / n, "bytes_per_launch": by,
                          "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak}

    # BF16 blocks read once per launch; up to `batch` right-hand sides of FP32 x, x0, y
    hbm("spmv", mesh.n_rows * (3 * nb * nb * 2 + 4) + 3 * nb * 4 * mesh.n_rows * Rl)
    # e4m3 copy (+ row scale) once per launch; FP16 x, x0, y per right-hand side
    hbm("hop", mesh.n_rows * (3 * nb * nb + 8) + 3 * nb * 2 * mesh.n_rows * Rl)
    # transposed BF16 application, one right-hand side (the adjoint)
    hbm("spmv_t", mesh.n_rows * (3 * nb * nb * 2 + 4) + 3 * nb * 4 * mesh.n_rows)
    for k2 in ("spmv_f64vec", "contract", "dot", "axpy"):
        n, ms = ks[k2]
        if n:
            kern[k2] = {"launches": n, "ms_total": ms}
    res = {"mode": "many", "workload": wname, "n_tets": int(m.n_tets), "nb": nb, "rhs": R,
           "metric": METRIC, "value": R / (solve_ms * 1e-3), "unit": "solves/s",
           "assembly_ms": asm_ms, "solve_ms": solve_ms, "adjoint_ms": adj_ms,
           "operator_passes": info.iters, "resid_worst": info.resid, "adjoint_passes": ainfo.iters,
           "adjoint_resid": ainfo.resid, "restart": restart, "batch": batch, "precond": args.precond,
           "poly_degree": poly, "operator_bytes": op.bytes, "J": float((g * rho).sum()),
           "grad_abs_max": float(dj.abs().max()), "kernels": kern,
           "kernel_ms": {k: round(v[1], 2) for k, v in ks.items()}, "peak_source": peak_src}
    if args.fp64_sample:
        # the BF16 operator and the solutions make room for the 38 GB FP64 operator
        op.close()
        del rho, lam
        n = min(args.fp64_sample, R)
        res["fp64_comparator"] = fp64_sample(dfm, mesh, Np, [mu] * n, rows[:n], tol, per_rhs_assembly=False)
    print(json.dumps(res))


def run_adjoint(args):
    """Adjoint workload: gradient of the mean receiver-region interior density
    with respect to per-tet damping (log-normal field) on the 40^3 Kuhn cube
    (384,000 tets, Np = 3).  Times forward assembly + solve, the receiver
    functional and the adjoint (transposed solve + fused dB/dmu contraction);
    optionally checks the gradient against central differences of the GPU
    forward solve on the sampled elements (step 1e-4).  The forward solve's
    preconditioner hops use the --precond copy, the transposed (adjoint) solve's
    the transposed copy."""
    import torch

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    torch.cuda.set_device(0)
    wname = args.workload if args.workload != WORKLOAD else "kuhn40_np3_adjoint"
    w = workload(wname)
    m = w["mesh"]
    Np = w["Np"]
    mu = torch.tensor(w["mu"], device="cuda")
    rows = np.asarray(w["sources"], dtype=np.int64)
    receiver = w["receiver"]
    tol = args.tol if args.tol else w["tol"]
    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])

    def forward(mu_vec, op=None, fp64=False):
        if op is None:
            op = dfm.Operator(mesh, Np, mu=mu_vec, precision=dfm.F64 if fp64 else dfm.F32)
        else:
            op.reassemble(mu_vec)
        rho0 = dfm.source(mesh, Np, rows)
        if fp64:
            rho, info = op.solve(rho0, method=dfm.GMRES, tol=1e-12, poly_degree=args.poly or 32,
                                 restart=args.restart or 256)
        else:
            rho, info = op.solve(rho0, method=dfm.GMRES_IR, tol=tol, poly_degree=args.poly or 32,
                                 restart=args.restart or 256, precond_precision=PRECOND[args.precond])
        g, dg = dfm.interior_density(mesh, Np, receiver, weights=1.0 / len(receiver), mu=mu_vec)
        return op, rho, g, dg, info

    akw = dict(tol=tol, poly_degree=args.poly or 32, restart=args.restart or 256,
               precond_precision=PRECOND[args.precond])
    op, rho, g, dg, info = forward(mu)
    lam, dj, ainfo = op.adjoint(rho, g, dg, **akw)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    op, rho, g, dg, info = forward(mu, op)
    ev[1].record()
    lam, dj, ainfo = op.adjoint(rho, g, dg, **akw)
    ev[2].record()
    torch.cuda.synchronize()
    J = float((g * rho[0]).sum())
    res = {"mode": "adjoint", "workload": wname, "n_tets": int(m.n_tets), "nb": op.nb, "J": J,
           "forward_ms": ev[0].elapsed_time(ev[1]), "adjoint_ms": ev[1].elapsed_time(ev[2]),
           "forward_applications": info.iters, "adjoint_applications": ainfo.iters,
           "grad_abs_max": float(dj.abs().max())}
    if args.fd:
        # central differences of the FP64 forward path (FP64 blocks, FP64 GMRES to 1e-12)
        grad = dj[0].cpu().numpy()
        els = w["fd"][:args.fd]
        rel = []
        ok = []
        h = 1e-4
        op64 = None
        for e in els:
            vals = []
            for sgn in (1, -1):
                mp = mu.clone()
                mp[int(e)] += sgn * h
                op64, r2, g2, _, _ = forward(mp, op64, fp64=True)
                vals.append(float((g2 * r2[0]).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            rel.append(abs(grad[int(e)] - fd) / max(abs(fd), 1e-300))
            ok.append(abs(grad[int(e)] - fd) <= 1e-3 * abs(fd) + 1e-6 * res["grad_abs_max"])
        res["fd_pass"] = int(sum(ok))
        res["fd_elements"] = len(els)
        res["fd_max_rel_err"] = float(max(rel))
        res["fd_median_rel_err"] = float(np.median(rel))
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--tol", type=float, default=0.0)
    ap.add_argument("--restart", type=int, default=0)
    ap.add_argument("--poly", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--precond", choices=["f32", "f16", "bf16", "fp8"], default="fp8",
                    help="precision of the blocks used by the polynomial preconditioner's hops")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-apps", type=int, default=0,
                    help="reference arm: operator applications charged per solve (0 = the FP64 path's count)")
    ap.add_argument("--mode", choices=["solve", "apply", "hop", "adjoint", "batched", "many", "cuboid"], default="solve")
    ap.add_argument("--rhs", type=int, default=0, help="batched mode: number of right-hand sides (0 = all)")
    ap.add_argument("--batch", type=int, default=0, help="batched mode: right-hand sides per lockstep group")
    ap.add_argument("--fp64-sample", type=int, default=0,
                    help="batched and many modes: time the plain FP64 GPU path on this many sources")
    ap.add_argument("--fd", type=int, default=0, help="adjoint mode: elements checked by central differences")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "apply":
        run_apply(args)
    elif args.mode == "hop":
        run_hop(args)
    elif args.mode == "adjoint":
        run_adjoint(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "many":
        run_many(args)
    elif args.mode == "cuboid":
        run_cuboid(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
