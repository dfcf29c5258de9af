"""Host-side logic of bench.py: roofline bookkeeping and the multi-rank
(replica) timing reduction, on CPU with the gloo backend."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}
N_ROWS, NB, NP = 192_000, 15, 4


def _stats(**kw):
    base = {"assemble": (0, 0.0), "spmv_f32": (0, 0.0), "hop": (0, 0.0), "spmv_f64vec": (0, 0.0),
            "dot": (0, 0.0), "axpy": (0, 0.0)}
    base.update(kw)
    return base


def _summ(stats, precond):
    return bench.summarize_kernels(stats, n_rows=N_ROWS, n_tets=N_ROWS // 4, Np=NP, nodes=10_000_000, nsm=152,
                                   peaks=PEAKS, peak_src="measured", workload="kuhn20_np4", precond=precond)


def test_spmv_bytes_counts_each_operand_once():
    # FP32 blocks, row map, x, x0 read once, y written once
    assert bench.spmv_bytes(10, 15, 4) == 10 * (3 * 225 * 4 + 4 + 15 * 4 * 3)
    assert bench.spmv_bytes(10, 15, 4, with_x0=False) == 10 * (3 * 225 * 4 + 4 + 15 * 4 * 2)
    assert bench.spmv_bytes(10, 15, 4, block_bytes=2) == 10 * (3 * 225 * 2 + 4 + 15 * 4 * 3)
    assert bench.spmv_bytes(10, 15, 8) == 10 * (3 * 225 * 4 + 4 + 15 * 8 * 3)


def test_sixteen_bit_hops_dominate_with_their_own_bytes():
    st = _stats(assemble=(1, 22.0), spmv_f32=(120, 12.0), hop=(1880, 110.0), dot=(250, 17.0))
    kern, total, roof = _summ(st, "f16")
    assert roof["kernel"] == "hop" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    by = N_ROWS * (3 * NB * NB * 2 + 4 + NB * 2 * 3)  # FP16 copy, FP16 hop vectors
    assert kern["hop"]["bytes_per_launch"] == by
    ach = by / (110.0 / 1880 * 1e-3) / 1e9
    assert roof["achieved"] == pytest.approx(ach, rel=1e-6)
    assert roof["peak"] == 6000.0 and roof["frac"] == pytest.approx(ach / 6000.0, abs=1e-4)
    # the FP32 launches are the Krylov operator w = z - B z, which reads x0
    assert kern["spmv_f32"]["bytes_per_launch"] == bench.spmv_bytes(N_ROWS, NB, 4, with_x0=True)
    assert total["dot"] == 17.0
    key = ("hop_kernel<15, __half>", "kuhn20_np4")
    assert roof["traffic"] == bench.MEASURED_TRAFFIC.get(key)


def test_fp8_hops_count_one_byte_per_value_and_the_row_scale():
    st = _stats(assemble=(1, 22.0), spmv_f32=(60, 6.0), hop=(1900, 60.0))
    kern, _, roof = _summ(st, "fp8")
    assert roof["kernel"] == "hop"
    assert kern["hop"]["bytes_per_launch"] == N_ROWS * (3 * NB * NB * 1 + 4 + NB * 2 * 3 + 4)
    kern, _, _ = _summ(st, "bf16")  # BF16 copy: FP32 hop vectors
    assert kern["hop"]["bytes_per_launch"] == N_ROWS * (3 * NB * NB * 2 + 4 + NB * 4 * 3)


def test_fp32_preconditioner_hops_read_no_x0():
    st = _stats(assemble=(1, 22.0), spmv_f32=(2000, 175.0))
    kern, _, roof = _summ(st, "f32")
    assert roof["kernel"] == "spmv_f32"
    assert kern["spmv_f32"]["bytes_per_launch"] == bench.spmv_bytes(N_ROWS, NB, 4, with_x0=False)


def test_assembly_dominated_step_reports_alu_roofline():
    st = _stats(assemble=(2, 300.0), spmv_f32=(10, 1.0))
    kern, _, roof = _summ(st, "f32")
    assert roof["kernel"] == "assemble" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    peak = 152 * bench.FP32_LANES_PER_SM * 2 * 2000.0 * 1e6 / 1e12
    assert roof["peak"] == pytest.approx(peak, rel=1e-6)
    fl = 10_000_000 * bench.flops_per_node(NP)
    assert kern["assemble"]["achieved"] == pytest.approx(fl / 0.150 / 1e12, rel=1e-9)
    assert roof["traffic"] is None


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
ws, rank, local = bench._dist()
t = bench.max_over_ranks(1.5 + rank, ws, "cpu")
print(json.dumps({"rank": rank, "ws": ws, "max": t}))
dist.destroy_process_group()
"""


def test_max_over_ranks_gloo_world_size_2():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    assert sorted(r["rank"] for r in res) == [0, 1]
    assert all(r["ws"] == 2 and r["max"] == 2.5 for r in res)


def test_max_over_ranks_single_process_is_identity():
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25


def test_reference_arm_non_zero_rank_prints_nothing():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_headline_kernels_count_each_kernel_with_its_own_operands():
    """The default workload's kernels: hops with 8 right-hand sides (e4m3
    copy, FP16 vectors), transposed hops with one, BF16 applications with FP32
    and FP64 vectors; the roofline goes to the kernel with the largest time."""
    rows, Np, B = 786_432, 8, 8
    nb = 45
    ks = {"hop": (3600, 3600 * 0.9), "hop_t": (3500, 3500 * 0.74), "spmv": (60, 60 * 13.0),
          "spmv_t": (60, 60 * 2.3), "spmv_f64vec": (2, 120.0), "spmv_f64vec_t": (2, 10.0),
          "contract": (1, 120.0), "dot": (100, 300.0), "axpy": (100, 200.0)}
    kern, total, roof = bench.headline_kernels(ks, rows, rows // 4, Np, 10_000_000, 152, PEAKS, "measured", B)
    assert kern["hop"]["bytes_per_launch"] == rows * (3 * nb * nb + 8) + 3 * nb * 2 * rows * B
    assert kern["hop_t"]["bytes_per_launch"] == rows * (3 * nb * nb + 8) + 3 * nb * 2 * rows
    assert kern["spmv"]["bytes_per_launch"] == rows * (3 * nb * nb * 2 + 4) + 3 * nb * 4 * rows * B
    assert kern["spmv_f64vec_t"]["bytes_per_launch"] == rows * (3 * nb * nb * 2 + 4) + 3 * nb * 8 * rows
    assert roof["kernel"] == "hop" and roof["unit"] == "GB/s"
    ach = kern["hop"]["bytes_per_launch"] / 0.9e-3 / 1e9
    assert roof["achieved"] == pytest.approx(ach, rel=1e-6) and roof["frac"] == pytest.approx(ach / 6000.0, abs=1e-4)
    assert total["dot"] == 300.0
