"""Benchmark: stationary DFM solves per second with adjoint gradients on one
GB300 (or N replicas).

Default workload (the largest single-GPU configuration, 45-function basis):
the 32^3 Kuhn cube (196,608 jittered tets, N_p = 8, mu = 0.05, r = 0.95),
operator blocks in BF16 (9.6 GB), 64 random boundary-face sources and the
mean interior density of the receiver cells [14, 18)^3 as the functional.
A job assembles B for the 64 sources, solves them and the adjoint equation
and forms every source's gradient; its 4 steps take the sources 16 at a time.
One step: project the group's sources, solve (I - B) rho = rho0 for all 16 in
one block Krylov space to an FP64 relative residual of 1e-6 (FP64-residual
refinement around block flexible FP32 GMRES(24) right-preconditioned by
sum_{k<64} B~^k on an e4m3 copy, hops on tensor cores, the Horner chains
replayed as CUDA graphs), then the adjoint: the transposed solve
(I - B)^T lambda = g to 1e-6 (at the job's first step, which also assembles
B; the later steps start from that lambda, whose residual the refinement
checks) and the fused lambda^T (dB/dmu) rho_r contraction, giving
dJ_r/dmu_e for the 16 sources.  Assembly is also timed on its own (assembly
blocks/s).  The timed steps start a job (4 steps by default: one whole job
with its assembly and adjoint solve).  Inputs are resident when the timed
region starts; the operator
and Krylov vectors are far larger than L2, so no flush is needed between
steps.  The value is sources per second, each with its solve and gradient.

The e2e figure runs the same steps through the C ABI with the step's source
rows copied from host memory and its gradients dJ/dmu copied back to pinned
host memory inside the timed region.

--workload kuhn20_np4 runs the 48,000-tet single-source solve instead (one
step = assembly + source + GMRES-IR solve to 1e-8), which is also reported in
the default line under "kuhn20_np4".

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
WORKLOAD = "kuhn20_np4"          # the single-source solve of the 48,000-tet cube
HEADLINE = "kuhn32_np8_rhs64"    # the default: 45 functions, BF16 blocks, sources in groups with adjoint
HEADLINE_GROUP = 16              # sources per step (one block Krylov space)
HEADLINE_RESTART = 24            # block steps per restart cycle
# workloads the source-group benchmark runs: the default and its 16^3 case for profiling
GROUP_WORKLOADS = {"kuhn32_np8_rhs64": None,
                   "kuhn16_np8": ("16^3 Kuhn cube x 6 = 24,576 jittered tets, Np = 8, 16 sources, one job per step; "
                                  "{krylov} GMRES({restart}), sum_{{k<{d}}} B~^k, {group} sources per step "
                                  "(the default workload's steps at 1/8 of its size, for profiling)")}
HEADLINE_DESC = ("32^3 Kuhn cube x 6 = 196,608 jittered tets (jitter 0.2h, seed 0); Np = 8 (45 Zernike functions); "
                 "mu = 0.05; boundary reflection 0.95; jobs of 64 random boundary-face unit sources (seed 2), {group} per "
                 "step, each job assembling B once at its first step; "
                 "BF16 operator blocks; FP64-residual refinement around flexible FP32 {krylov} GMRES({restart}) "
                 "right-preconditioned by sum_{{k<{d}}} B~^k on an e4m3 copy (tensor-core hops, CUDA graphs of the "
                 "Horner chains); relative residual "
                 "1e-6; adjoint of the mean receiver density (cells [14,18)^3): transposed solve to 1e-6 on the "
                 "transposed e4m3 copy at each job's first step (later steps start from it and check its residual) "
                 "and the fused dB/dmu contraction for every step's sources")
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
REF_APPLICATIONS = {"kuhn20_np4": 1809, "kuhn32_np8_rhs64": 2600}
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


def run_gpu(args, extra=False):
    """The single-source solve of a workload (by default the 48,000-tet cube).
    extra: a short run of it inside the default benchmark (5 steps, 2 warm-up,
    a 10 s CPU sample), returned instead of printed."""
    import copy

    import torch
    import torch.distributed as dist

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    ws, rank, local = _dist()
    if extra:
        args = copy.copy(args)
        args.workload, args.steps, args.warmup = WORKLOAD, min(args.steps, 5), min(args.warmup, 2)
        args.cpu_seconds = min(args.cpu_seconds, 10.0)
        args.restart, args.poly, args.tol, args.batch = 0, 0, 0.0, 0
        ws, rank = 1, 0
    torch.cuda.set_device(local)
    if ws > 1 and not extra:
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
                             precond_precision=PRECOND[args.precond], coarse=args.coarse)
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
                             precond_precision=PRECOND[args.precond], coarse=args.coarse)
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
                   "coarse_aggregates": args.coarse ** 3,
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
    if extra:
        op.close()
        mesh.close()
        return res
    print(json.dumps(res))
    if ws > 1:
        dist.destroy_process_group()


def _hop_bytes(n_rows, nb, R):
    """Algorithmic bytes of one hop on the e4m3 copy: the values (one byte
    each) and the row scale, the row map, and x, x0, y in FP16 per
    right-hand side."""
    return n_rows * (3 * nb * nb + 8) + 3 * nb * 2 * n_rows * R


def _apply_bytes(n_rows, nb, block_bytes, vec_bytes, R):
    """Algorithmic bytes of one application y = x0 + alpha B x on R
    right-hand sides: blocks and row map once, x, x0 and y per right-hand side."""
    return n_rows * (3 * nb * nb * block_bytes + 4) + 3 * nb * vec_bytes * n_rows * R


def headline_kernels(ks, n_rows, n_tets, Np, nodes, nsm, peaks, peak_src, B):
    """Per-kernel rooflines of the default workload's timed steps (ks: name ->
    (launches, total ms)) and the roofline of the kernel with the largest
    total time among the hops and applications."""
    nb = (Np + 1) * (Np + 2) // 2
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    kern = {}
    by = {"hop": _hop_bytes(n_rows, nb, B), "hop_t": _hop_bytes(n_rows, nb, 1),
          "spmv": _apply_bytes(n_rows, nb, 2, 4, B), "spmv_t": _apply_bytes(n_rows, nb, 2, 4, 1),
          "spmv_f64vec": _apply_bytes(n_rows, nb, 2, 8, B), "spmv_f64vec_t": _apply_bytes(n_rows, nb, 2, 8, 1)}
    for name, b in by.items():
        n, ms = ks.get(name, (0, 0.0))
        if n:
            ach = b / (ms / n * 1e-3) / 1e9
            kern[name] = {"bound": "hbm", "launches": n, "ms_per_launch": ms / n, "bytes_per_launch": b,
                          "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak}
    for name in ("contract", "dot", "axpy"):
        n, ms = ks.get(name, (0, 0.0))
        if n:
            kern[name] = {"launches": n, "ms_total": ms}
    total = {k: v[1] for k, v in ks.items()}
    dominant = max((k for k in by if k in kern), key=lambda k: total[k])
    d = kern[dominant]
    inst = {"hop": f"hop_frag_kernel<{nb}, __nv_fp8_e4m3, 8>", "hop_t": f"hop_frag_kernel<{nb}, __nv_fp8_e4m3, 1>"}
    traffic = MEASURED_TRAFFIC.get((inst.get(dominant), HEADLINE))
    roofline = {"bound": "hbm", "achieved": round(d["achieved"], 3), "peak": round(d["peak"], 3), "unit": "GB/s",
                "frac": round(d["frac"], 4), "traffic": traffic, "kernel": dominant, "peak_source": peak_src}
    return kern, total, roofline


def run_headline(args):
    """The default workload: source groups solved with adjoint gradients (see
    the module docstring).  Prints the JSON line."""
    import torch
    import torch.distributed as dist

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    wname = args.workload if args.workload in GROUP_WORKLOADS else HEADLINE
    w = workload(wname)
    m = w["mesh"]
    Np = w["Np"]
    tol = args.tol if args.tol else w["tol"]
    mu = float(w["mu"][0])
    sources = np.asarray(w["sources"], dtype=np.int64)
    receiver = w["receiver"]
    B = args.batch or HEADLINE_GROUP
    restart = args.restart or (HEADLINE_RESTART if B == HEADLINE_GROUP else 32)
    poly = args.poly or 64
    precond = PRECOND[args.precond]
    dfm.load()
    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])
    op = dfm.Operator(mesh, Np, mu=mu, precision=dfm.BF16)
    g, dg = dfm.interior_density(mesh, Np, receiver, weights=1.0 / len(receiver), mu=mu)
    skw = dict(tol=tol, restart=restart, poly_degree=poly, precond_precision=precond)

    # a job: assemble B, solve all sources and the adjoint equation, and form
    # every source's gradient; its steps take the sources B at a time, the
    # first step assembles and solves the adjoint equation (lambda depends on
    # the operator and the functional, not on the sources), the later steps
    # start the adjoint refinement from that lambda (its FP64 residual is
    # checked, then the contraction runs)
    per_job = max(1, sources.size // B)
    state = {"lam": None}

    def group(i):
        idx = (np.arange(B) + (i % per_job) * B) % sources.size
        return sources[idx]

    def step(i, rows=None):
        first = i % per_job == 0
        if first:
            op.reassemble(mu)
        rho0 = dfm.source(mesh, Np, group(i) if rows is None else rows)
        rho, info = op.solve(rho0, batch=B, block=0 if args.lockstep else 1, **skw)
        lam, dj, ainfo = op.adjoint(rho, g, dg, lam0=None if first else state["lam"], **skw)
        state["lam"] = lam
        return rho, dj, info, ainfo

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    # ---- timed region: device-resident steps --------------------------------
    sampler = ClockSampler(local)
    dfm.stats_reset()
    dfm.stats_enable(STATS_EVERY)
    l0 = dfm.launch_count()
    g0 = dfm.hop_graph_replays()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    infos = []
    for i in range(args.steps):
        rho, dj, info, ainfo = step(i)  # the timed steps start a job: its assembly and adjoint solve included
        infos.append((info.iters, info.outer, info.resid, ainfo.iters, ainfo.resid))
    e1.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = dfm.launch_count() - l0
    graph_replays = dfm.hop_graph_replays() - g0
    dfm.stats_enable(False)
    elapsed_ms = e0.elapsed_time(e1)
    names = {"assemble": dfm.KERNEL_ASSEMBLE, "hop": dfm.KERNEL_SPMV16, "hop_t": dfm.KERNEL_SPMV16_T,
             "spmv": dfm.KERNEL_SPMV,
             "spmv_t": dfm.KERNEL_SPMV_T, "spmv_f64vec": dfm.KERNEL_SPMV64, "spmv_f64vec_t": dfm.KERNEL_SPMV64_T,
             "contract": dfm.KERNEL_CONTRACT, "dot": dfm.KERNEL_DOT, "axpy": dfm.KERNEL_AXPY}
    ks = {k: dfm.kernel_stats(v) for k, v in names.items()}
    elapsed_ms = max_over_ranks(elapsed_ms, ws, "cuda")
    J = float((g * rho).sum())

    # ---- assembly (timed on its own: re-assembly into the same operator) -----
    dfm.stats_reset()
    dfm.stats_enable(True)
    for _ in range(2):
        op.reassemble(mu)
    torch.cuda.synchronize()
    n_as, ms_as = dfm.kernel_stats(dfm.KERNEL_ASSEMBLE)
    dfm.stats_enable(False)
    nodes = dfm.op_nodes(op)

    # ---- e2e: C ABI with host source rows in and host gradients out ----------
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(1, min(args.steps, args.e2e_steps or per_job))
        host_dj = torch.empty((B, m.n_tets), dtype=torch.float64, pin_memory=True)
        host_rows = [np.ascontiguousarray(group(i)) for i in range(e2e_steps)]
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            _, dj_i, _, _ = step(i, rows=host_rows[i])
            host_dj.copy_(dj_i, non_blocking=True)
            torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, ws, "cuda")
        e2e = {"value": ws * B * e2e_steps / dt, "unit": "solves/s", "steps": e2e_steps,
               "h2d_bytes_per_step": int(host_rows[0].nbytes), "d2h_bytes_per_step": int(host_dj.numel() * 8)}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    peaks, peak_src = _peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    kern, total, roofline = headline_kernels(ks, mesh.n_rows, int(m.n_tets), Np, nodes, nsm, peaks, peak_src, B)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    asm_ach = nodes * flops_per_node(Np) / (ms_as / n_as * 1e-3) / 1e12
    it = np.array(infos)
    res = {
        "metric": METRIC,
        "value": ws * B * args.steps / (elapsed_ms * 1e-3),
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16 blocks, e4m3 preconditioner copy, f16 hop vectors, f32 Krylov, f64 residual",
        "data": "synthetic",
        "config": {"workload": wname,
                   "desc": (HEADLINE_DESC if wname == HEADLINE else GROUP_WORKLOADS[wname]).format(
                       restart=restart, d=poly, group=B, krylov="lockstep" if args.lockstep else "block"),
                   "krylov": "lockstep" if args.lockstep else f"block (one Krylov space per group of {B} sources)",
                   "hop_graph_replays": int(graph_replays),
                   "n_tets": int(m.n_tets), "n_rows": int(mesh.n_rows), "nb": op.nb, "sources_per_step": B,
                   "tol": tol, "restart": restart, "poly_degree": poly, "precond": args.precond,
                   "unit_of_work": "one source solved to 1e-6 with its gradient dJ/dmu; a job of 64 sources "
                                   f"({per_job} steps) assembles B and solves the adjoint equation once, at its first step",
                   "l2": "inputs larger than L2 (operator %.0f MB)" % (op.bytes / 1e6),
                   "parallelism": f"replicas x{ws}"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "assembly": {"ms": ms_as / n_as, "blocks_per_s": 12 * m.n_tets / (ms_as / n_as * 1e-3),
                     "roofline": {"bound": "alu", "achieved": asm_ach, "peak": fp32_peak, "unit": "TFLOP/s",
                                  "frac": asm_ach / fp32_peak, "nodes": nodes, "flops_per_node": flops_per_node(Np),
                                  "peak_source": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz"}},
        "assembly_blocks_per_s": 12 * m.n_tets / (ms_as / n_as * 1e-3),
        "solve": {"operator_passes_per_step": int(np.median(it[:, 0])), "adjoint_passes_per_step": int(np.median(it[:, 3])),
                  "resid_worst": float(it[:, 2].max()), "adjoint_resid_worst": float(it[:, 4].max()), "J": J},
        "kernels": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                    for k, v in kern.items()},
        "kernel_ms_per_step": {k: round(v / args.steps, 3) for k, v in total.items()},
        "autotune": [{k: e[k] for k in ("nb", "rhs_per_group", "groups", "transpose", "rows", "chosen")}
                     | {"candidates": len(e["tried"])} for e in dfm.autotune_report()
                     if e["rows"] == mesh.n_rows],
    }
    op.close()
    del rho, dj
    torch.cuda.synchronize()
    if not args.no_comparator:
        res["fp64_gpu_path"] = fp64_sample(dfm, mesh, Np, [mu], sources[:1], tol, per_rhs_assembly=False,
                                           warm=False)
    if ws == 1 and not args.no_cpu_baseline:
        apps = int(np.median(it[:, 0])) if "fp64_gpu_path" not in res else res["fp64_gpu_path"]["operator_applications"][0]
        res["cpu_baseline"] = cpu_baseline(wname, op_apps=apps, seconds=args.cpu_seconds, group=B)
    mesh.close()
    if not args.no_extra:
        res["kuhn20_np4"] = run_gpu(args, extra=True)
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

def _oracle_sample(wname, seconds, op_apps=None, group=1):
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload:
    (a) adaptive (1e-13) assembly of randomly drawn face pairs until about
    `seconds`/2 of wall time, giving seconds per block; (b) restarted GMRES
    iterations of the oracle on an operator with the workload's sparsity,
    giving seconds per operator application (block values do not change the
    work): at full size, or, when the FP64 blocks would pass 2 GB, on the
    8^3 cube with the same basis, scaled by the ratio of operator rows.
    Extrapolated time of one benchmark step = (a) x 12 N x (the step's share
    of the assembly) + (b) x op_apps x (solves per step).  The default
    workload's step solves `group` sources and one adjoint equation and is
    charged group / (number of sources) of the assembly; a single-source step
    one solve and the whole assembly."""
    import oracle
    from paper_1608_04607_gb300.inputs import kuhn_cube_mesh, workload

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
    # the same assembly on one thread (a fixed sample of 32 pairs; 4 for large bases)
    n1 = 32 if nb <= 15 else 4
    sel = rng.integers(0, t.size, size=n1)
    t0 = time.perf_counter()
    oracle.blocks_for_pairs(m.verts, m.tets, topo, mu, w["refl"], Np, t[sel], f[sel], fp[sel], rtol=1e-13, nthreads=1)
    per_block_1t = (time.perf_counter() - t0) / n1
    # (b) oracle GMRES iterations, at full size or on the 8^3 cube scaled by rows
    ms = m
    if 4 * m.n_tets * 3 * nb * nb * 8 > 2e9:
        ms = kuhn_cube_mesh(8, jitter=0.2, seed=0)
    tops = topo if ms is m else oracle.topology(ms.tets)
    _, _, fps = oracle.pair_list(ms.n_tets)
    blocks = rng.standard_normal((4 * ms.n_tets, 3, nb, nb)) * (0.3 / nb)
    dest = tops.recv[4 * np.repeat(np.arange(ms.n_tets), 12) + fps].reshape(4 * ms.n_tets, 3)
    op = oracle.Operator(Np=Np, blocks=blocks, dest=dest)
    rho0 = oracle.source_vector(ms.verts, ms.tets, [int(np.nonzero(tops.recv == np.arange(4 * ms.n_tets))[0][0])], Np)
    k = 16 if ms is m else 8
    t0 = time.perf_counter()
    oracle.solve_gmres(op, rho0, tol=1e-300, restart=64, maxit=k)
    per_app = (time.perf_counter() - t0) / k * (m.n_tets / ms.n_tets)
    if op_apps is None:
        op_apps = 0
    headline = wname == HEADLINE
    share = group / len(w["sources"]) if headline else 1.0
    solves = group + 1 if headline else 1
    est = per_block * 12 * m.n_tets * share + per_app * op_apps * solves
    where = "at full size" if ms is m else f"on the 8^3 cube ({4 * ms.n_tets} rows) scaled to {4 * m.n_tets} rows"
    sample = (f"extrapolated: oracle assembly of {n_pairs} random face pairs (adaptive to 1e-13) and {k} oracle "
              f"GMRES(64) iterations {where}; per step {share:g} x 12 x {m.n_tets} blocks + {solves} x {op_apps} "
              f"operator applications")
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


def cpu_baseline(wname, op_apps, seconds=20.0, group=1):
    est, sample, threads, per_block, per_app, per_block_1t = _oracle_sample(wname, seconds, op_apps, group)
    return {"value": group / est, "unit": "solves/s", "cores": threads, "kind": "oracle", "sample": sample,
            "operator_applications_charged": op_apps,
            "s_per_block": per_block, "s_per_block_1thread": per_block_1t, "s_per_application": per_app,
            "cpu_model": _cpu_model()}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    # a full oracle solve takes hours of CPU time, so each step times the
    # oracle on a bounded sample (assembly of random face pairs and GMRES
    # iterations) and extrapolates to the whole step with the FP64 GPU path's
    # application count
    from paper_1608_04607_gb300.inputs import workload

    wname = args.workload or HEADLINE
    wl = workload(wname)
    apps = args.ref_apps or REF_APPLICATIONS.get(wname, 2000)
    group = (args.batch or HEADLINE_GROUP) if wname == HEADLINE else 1
    vals = []
    last = None
    for i in range(args.warmup + args.steps):
        est, sample, threads, _, _, _ = _oracle_sample(wname, args.cpu_seconds / 2, apps, group)
        if i >= args.warmup:
            vals.append(est)
        last = (sample, threads)
    v = group / statistics.mean(vals)
    desc = (HEADLINE_DESC.format(restart=HEADLINE_RESTART, d=64, krylov="block", group=HEADLINE_GROUP)
            if wname == HEADLINE else
            WORKLOAD_DESC if wname == WORKLOAD else wname)
    res = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(vals) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wname,
                      "desc": desc + "; FP64 CPU oracle (adaptive assembly to 1e-13, restarted GMRES), timed on a "
                      "bounded sample and extrapolated",
                      "sources_per_step": group, "operator_applications_charged": apps,
                      "n_tets": int(wl["mesh"].n_tets), "n_rows": int(wl["mesh"].n_rows),
                      "nb": (wl["Np"] + 1) * (wl["Np"] + 2) // 2, "tol": args.tol or wl["tol"]},
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": last[1], "kind": "oracle", "sample": last[0]},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def run_apply(args):
    """Operator-application micro-benchmark: K timed y = x0 - B x launches
    (FP32 vectors, --rhs right-hand sides, default 1) on the workload's
    assembled operator (BF16 blocks for N_p = 8, else FP32), for the
    application's roofline and for profiling the kernel in isolation."""
    import torch

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import workload

    torch.cuda.set_device(0)
    w = workload(args.workload)
    m = w["mesh"]
    mesh = dfm.Mesh(m.verts, m.tets, refl=w["refl"])
    bf16 = w["Np"] >= 8
    op = dfm.Operator(mesh, w["Np"], mu=float(w["mu"][0]), precision=dfm.BF16 if bf16 else dfm.F32)
    R = args.rhs or 1
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((R, mesh.n_rows, op.nb), device="cuda", dtype=torch.float32, generator=g)
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
    by = _apply_bytes(mesh.n_rows, op.nb, 2 if bf16 else 4, 4, R)
    ach = by / (ms / n * 1e-3) / 1e9
    print(json.dumps({"mode": "apply", "workload": args.workload, "rhs": R, "launches": n, "ms_per_launch": ms / n,
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
                      "frac": ach / float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)), "peak_source": src,
                      "autotune": [e for e in dfm.autotune_report() if e["rows"] == mesh.n_rows]}))


def fp64_sample(dfm, mesh, Np, mus, rows, tol, per_rhs_assembly, warm=True):
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

    if warm:
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
            "sample": f"the first {len(times)} sources" + ("" if warm else " (no warm-up solve)"),
            "operator_applications": apps,
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
    wname = args.workload
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
    exact ray solution rho* of Eq. ExactSol.  Each order runs with the
    piecewise-constant spatial function per face and, up to N_p = 8, with the
    linear spatial basis (three functions per face)."""
    import torch

    from paper_1608_04607_gb300 import dfm
    from paper_1608_04607_gb300.inputs import cuboid_rows_x0, kuhn_cuboid_mesh

    torch.cuda.set_device(0)
    mu, length = 0.4 * np.pi, 2.0
    cases = []
    plan = []
    spatials = [int(v) for v in args.cuboid_spatial.split(",")]
    for part in args.cuboid_cases.split(";"):
        n_s, nps = part.split(":")
        plan.append((int(n_s), [int(v) for v in nps.split(",")]))
    for n, nps in plan:
        m = kuhn_cuboid_mesh(n, length=length)
        mesh = dfm.Mesh(m.verts, m.tets, refl=1.0)
        rows = cuboid_rows_x0(m)
        x = m.verts[m.tets].mean(axis=1)[:, 0]
        exact = (np.exp(-mu * x) + np.exp(-mu * (2 * length - x))) / (1 - np.exp(-2 * mu * length))
        tets = np.arange(m.n_tets)
        for Np, spatial in [(a, b) for b in spatials for a in nps if b == 0 or a <= 8]:
            code = dfm.basis(Np, spatial)
            op = dfm.Operator(mesh, code, mu=mu, precision=dfm.F32)

            def step():
                op.reassemble(mu)
                rho0 = dfm.source_directed(mesh, code, rows, combine=True)
                rho, info = op.solve(rho0, tol=1e-10)
                g, _ = dfm.interior_density(mesh, code, tets, mu=mu)
                return dfm.tet_density(mesh, code, g, rho), info

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
            cases.append({"n_tets": m.n_tets, "Np": Np, "spatial": "linear" if spatial else "constant",
                          "unknowns_per_face": op.nb, "ms_per_step": statistics.median(times),
                          "rel_mean_err": err, "operator_applications": info.iters, "resid": info.resid})
            op.close()
        mesh.close()
    best = min(cases, key=lambda c: c["rel_mean_err"])
    print(json.dumps({"metric": "cuboid relative mean error against the exact ray solution", "mode": "cuboid",
                      "value": best["rel_mean_err"], "unit": "fraction", "higher_is_better": False,
                      "best_case": {"n_tets": best["n_tets"], "Np": best["Np"], "spatial": best["spatial"]},
                      "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
                      "config": {"workload": "kuhn cuboid 2 x 1 x 1, " + args.cuboid_cases + " (cells per unit length: "
                                             "basis orders)",
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
    wname = args.workload
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
    wname = args.workload
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
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 8 = one whole job of the default workload, else 5)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default=None,
                    help="default: the 196,608-tet 45-function workload (solve mode); see each mode for its own")
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
    ap.add_argument("--cuboid-cases", default="4:4,6,8,10,12,16,20;8:4,6,8,12,16",
                    help="cuboid mode: 'n:Np,Np,...;n:...' (n cells per unit length, basis orders)")
    ap.add_argument("--coarse", type=int, default=2,
                    help="single-source solves: two-level preconditioner on coarse^3 aggregates (0 = off; "
                         "2 measured fastest on the 48,000-tet workload: 1,932 applications against 2,164)")
    ap.add_argument("--cuboid-spatial", default="0,1",
                    help="cuboid mode: spatial bases per face, 0 = constant, 1 = linear (orders <= 8 only)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="default workload: steps of the e2e measurement (0 = one job)")
    ap.add_argument("--no-extra", action="store_true", help="default workload: skip the 48,000-tet solve's key")
    ap.add_argument("--lockstep", action="store_true",
                    help="default workload: each source in its own Krylov space (lockstep) instead of block GMRES")
    ap.add_argument("--autotune", type=int, choices=[0, 1], default=1,
                    help="1: tune the hop launch geometry on first use (default); 0: fixed default geometry")
    args = ap.parse_args()
    if args.steps is None:
        # the default workload: one whole job (its assembly and adjoint solve included)
        args.steps = 64 // (args.batch or HEADLINE_GROUP) if args.mode == "solve" and args.workload in (None, HEADLINE) \
            else 5
    if args.workload is None and args.impl != "reference":
        args.workload = {"solve": HEADLINE, "batched": "kuhn30_np4_rhs128", "many": HEADLINE,
                         "adjoint": "kuhn40_np3_adjoint"}.get(args.mode, WORKLOAD)
    if args.impl != "reference" and args.autotune == 0:
        from paper_1608_04607_gb300 import dfm

        dfm.autotune(0)
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
    elif args.workload in GROUP_WORKLOADS:
        run_headline(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
