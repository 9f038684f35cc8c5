#!/usr/bin/env python
"""Benchmark of the VoxCap GB300 hot path.

One step = one full capacitance extraction of the workload: voxcap_setup
from device-resident voxel labels (panels, Toeplitz tensors -- FP64 near
field, FP32 far-field sums under FP32+refinement --, circulant embedding and
kernel spectra, preconditioner) followed by the batched FP32 +
FP64-refinement GMRES solve of all conductors and the capacitance
reduction.  ``value`` is seconds per capacitance matrix over the whole job
(lower is better).  The same JSON line also carries the plain-FP64 time,
the FP32 fused-product throughput (matvecs/s), the HBM roofline of the
product on the step's workload (``roofline``) and on the 128x128x64 bus
crossing with its 8 columns (``roofline_large``), the end-to-end number
through the C ABI with host buffers, the oracle's CPU time on a bounded
sample, clocks and the kernel-launch count.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload plates|cube|bus|pillars]

Under torchrun (N > 1) every rank runs its own replica of the workload
(independent extractions, no data-path collective): weak scaling.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matvecs/s, s per C-matrix at 1e-4 rel err: FP32+refine vs FP64; % HBM roofline"
TOL = 1e-5          # GMRES relative residual; gives C to well below 1e-4 (checked in the line)


def workload(name):
    from paper_2004_02609_gb300 import workloads as W
    if name == "plates":
        return W.plates(), "two parallel plates 24x24x2 voxels, 4 apart, eps_r=3.9 slab, 32x32x16 grid"
    if name == "cube":
        return W.cube(4), "conductor cube 4x4x4 voxels in vacuum"
    if name == "bus":
        return W.bus_crossing(), "4x4 bus crossing in 3 dielectric layers, 128x128x64 grid"
    if name == "pillars":
        return W.pillars_field()[0], "two pillars in a smooth random dielectric, 64^3 grid"
    if name == "meanders":
        return W.meanders(), ("two interleaved meanders (width 4, spacing 4, thickness 8, 32 legs) "
                              "in eps_r=3.9, 512x512x64 grid")
    raise SystemExit(f"unknown workload {name}")


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        fd, self.path = tempfile.mkstemp(prefix="voxcap_clocks_", suffix=".csv")
        os.close(fd)
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
            os.remove(self.path)
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1.0)        # writes 256 MB > 129 MB L2


def mvm_model_bytes(vc, nrhs):
    """Algorithmic bytes of one FP32 product per right-hand side: panel I/O
    (x, y, face index: 12 N), the kernel spectra in reduced real octant form
    (15 * 4 * (Mx/2+1)(My/2+1)(Mz/2+1), shared by the nrhs columns), and one
    HBM round trip of the 3 forward and 6 inverse z-unpadded half spectra
    (2 * 9 * 8 * (Mx/2+1) * My * (Nz+1))."""
    Mx, My, Mz = vc.fft_lengths()
    nx, ny, nz = vc.shape
    Hx = Mx // 2 + 1
    spectra = 15 * 4 * Hx * (My // 2 + 1) * (Mz // 2 + 1)
    inter = 2 * 9 * 8 * Hx * My * (nz + 1)
    return 12 * vc.N + spectra / nrhs + inter


# DRAM bytes (read + write) of one batched FP32 product, summed over its five
# kernels, from `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum`
# (profiles/product_traffic.md); None where no capture matches the current
# kernels.
TRAFFIC = {"plates": 11909376, "bus": 4548623360}


def product_roofline(vc, dev, reps, workload_name):
    """Time `reps` batched FP32 products (all conductor columns) with CUDA
    events on the launching stream and relate the model bytes to the
    measured HBM peak."""
    import torch
    m = vc.n_conductors
    x = torch.randn(m, vc.N, device=dev, dtype=torch.float32)
    for _ in range(3):
        vc.matvec(x)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        vc.matvec(x)
    ev[1].record(stream)
    ev[1].synchronize()
    t = ev[0].elapsed_time(ev[1]) / 1e3 / reps
    hbm, peak_src = read_peaks()
    b = mvm_model_bytes(vc, m) * m
    return m / t, {"kernel": "fused FP32 product (5 passes: xfwd, yfwd, zmac, yinv, xinv), "
                             f"{m} columns, {workload_name}",
                   "bound": "hbm", "achieved": b / t / 1e9, "peak": hbm, "unit": "GB/s",
                   "frac": b / t / 1e9 / hbm, "traffic": TRAFFIC.get(workload_name),
                   "peak_source": peak_src, "bytes_per_launch": b, "launch_s": t,
                   "fft_lengths": list(vc.fft_lengths())}


def max_over_ranks(x, world, device):
    """The largest x over the ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def run_ours(args, rank, world):
    import torch
    import __graft_entry__ as ge
    from paper_2004_02609_gb300 import voxcap as V
    if rank == 0:
        ge.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    V.lib()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w, desc = workload(args.workload)
    lab_dev = torch.tensor(w.labels, device=dev)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def extraction(precision, labels):
        vc = V.VoxCap(labels, w.conductor_id, w.eps_r, w.voxel_size, precision=precision)
        C, st = vc.capacitance(tol=TOL)
        n = vc.N
        vc.close()
        return C, st, n

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- warm-up ----
    for _ in range(args.warmup):
        extraction("fp32_refine", lab_dev)
    # ---- timed: FP32 + refinement ----
    times = []
    barrier()
    torch.cuda.synchronize()
    launches0 = V.launch_count()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            C32, st32, N = extraction("fp32_refine", lab_dev)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    barrier()
    launches = V.launch_count() - launches0
    t_step = sum(times) / len(times)
    t_max = max_over_ranks(sum(times), world, dev) / len(times)
    # ---- plain FP64 for comparison ----
    extraction("fp64", lab_dev)
    t64 = []
    for _ in range(max(1, args.steps // 2)):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        C64, st64, _ = extraction("fp64", lab_dev)
        e1.record(stream)
        e1.synchronize()
        t64.append(e0.elapsed_time(e1) / 1e3)
    # accuracy of the FP32+refine matrix against a tight FP64 solve
    vc = V.VoxCap(lab_dev, w.conductor_id, w.eps_r, w.voxel_size, precision="fp64")
    Ct, _ = vc.capacitance(tol=1e-10)
    cerr = float(np.max(np.abs(C32 - Ct)) / np.max(np.abs(Ct)))
    # ---- fused FP32 product throughput and roofline ----
    m = vc.n_conductors
    matvecs_per_s, roof = product_roofline(vc, dev, 20, args.workload)
    vc.close()
    # ---- the product on the bus crossing (8 columns, 110,848 panels) ----
    roof_large = None
    if args.workload != "bus":
        wb, _ = workload("bus")
        vb = V.VoxCap(torch.tensor(wb.labels, device=dev), wb.conductor_id, wb.eps_r, wb.voxel_size)
        _, roof_large = product_roofline(vb, dev, 10, "bus")
        vb.close()
    # ---- end to end through the C ABI with host buffers ----
    e2e = []
    lab_host = np.ascontiguousarray(w.labels, dtype=np.int32)
    for _ in range(max(1, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C, st, _ = extraction("fp32_refine", lab_host)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    h2d = lab_host.nbytes + w.conductor_id.astype(np.int32).nbytes + w.eps_r.astype(np.float64).nbytes
    d2h = int(np.asarray(C).size) * 8
    res = {
        "metric": METRIC,
        "value": t_max / world,
        "unit": "s/C-matrix",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 products in f64 refinement",
        "data": "synthetic",
        "config": {"workload": desc, "panels": N, "conductors": m, "gmres_tol": TOL,
                   "restart": 35, "precond": "bdd nv=10",
                   "step": "setup from device labels + batched capacitance solve",
                   "l2": "flushed between timed steps (256 MB write)"},
        "fp32_refine": {"s_per_C": t_step, "iterations": st32["iterations"], "sweeps": st32["sweeps"],
                        "products": st32["matvecs"], "c_rel_err_vs_fp64_1e-10": cerr},
        "fp64": {"s_per_C": sum(t64) / len(t64), "iterations": st64["iterations"],
                 "products": st64["matvecs"]},
        "matvecs_per_s": matvecs_per_s,
        "roofline": roof,
        "roofline_large": roof_large,
        "e2e": {"value": statistics.median(e2e), "unit": "s/C-matrix", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(w, budget_s=args.cpu_budget)
    return res


def run_products(args):
    """Product-only timing (--products): setup once, then K batched FP32
    products with all conductor columns; used for kernel profiling."""
    import torch
    import __graft_entry__ as ge
    from paper_2004_02609_gb300 import voxcap as V
    ge.build()
    w, desc = workload(args.workload)
    vc = V.VoxCap(torch.tensor(w.labels, device="cuda"), w.conductor_id, w.eps_r, w.voxel_size)
    if args.path >= 0:
        vc.set_product_path(args.path)
    m = vc.n_conductors
    x = torch.randn(m, vc.N, device="cuda", dtype=torch.float32)
    for _ in range(args.warmup):
        vc.matvec(x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        vc.matvec(x)
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    hbm, src = read_peaks()
    b = mvm_model_bytes(vc, m) * m
    return {"mode": "products", "workload": desc, "panels": vc.N, "columns": m, "path": vc.set_product_path(args.path) if args.path >= 0 else None,
            "fft_lengths": vc.fft_lengths(), "s_per_batched_product": t, "matvecs_per_s": m / t,
            "model_bytes": b, "achieved_GBps": b / t / 1e9, "frac_of_" + src + "_hbm": b / t / 1e9 / hbm}


def cpu_baseline(w, budget_s=20.0):
    """The oracle as it stands on the host cores, on a bounded sample: the
    dense assembly integrates every distinct panel-pair integral; a random
    sample of those is timed and scaled by their total count; the LU solve
    and capacitance reduction run in full."""
    import oracle as O
    t0 = time.perf_counter()
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    n = ps.n
    c2 = np.rint(2.0 * ps.centers).astype(np.int64)
    span = int(2 * (max(ps.nx, ps.ny, ps.nz) + 2))
    Wd = 2 * span + 1
    kr = ps.kind.astype(np.int64)
    orr = ps.orient.astype(np.int64)
    keys = []
    for k0 in range(0, n, 1024):
        k1 = min(n, k0 + 1024)
        d = c2[k0:k1, None, :] - c2[None, :, :] + span
        kk = ((kr[k0:k1, None] * 3 + orr[k0:k1, None]) * 3 + orr[None, :])
        keys.append(np.unique(((kk * Wd + d[..., 0]) * Wd + d[..., 1]) * Wd + d[..., 2]))
    uniq = np.unique(np.concatenate(keys))
    t_keys = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    sample = 64
    spent, done = 0.0, 0
    while spent < budget_s and done < len(uniq):
        pick = uniq[rng.integers(0, len(uniq), sample)]
        dz = pick % Wd - span
        r = pick // Wd
        dy = r % Wd - span
        r //= Wd
        dx = r % Wd - span
        r //= Wd
        ol = r % 3
        r //= 3
        ot = r % 3
        kd = r // 3
        t1 = time.perf_counter()
        O.entries(kd, ot, ol, np.stack([dx, dy, dz], 1) / 2.0, rtol=1e-13)
        spent += time.perf_counter() - t1
        done += sample
    per_entry = spent / done
    A = np.random.default_rng(1).standard_normal((n, n)) + n * np.eye(n)
    t2 = time.perf_counter()
    np.linalg.solve(A, np.ones((n, ps.n_conductors)))
    t_lu = time.perf_counter() - t2
    total = t_keys + per_entry * len(uniq) + t_lu
    return {"value": total, "unit": "s/C-matrix", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} of {len(uniq)} distinct panel-pair integrals timed "
                      f"({spent:.1f} s) and scaled; panel keys and an N={n} LU timed in full"}


def run_reference(args, rank, world):
    """The oracle (plain FP64 CPU) on the same workload and metric."""
    if rank != 0:
        return None
    w, desc = workload(args.workload)
    t = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(w, budget_s=max(2.0, args.cpu_budget / max(1, args.steps)))
        if i >= args.warmup:
            t.append(cb["value"])
    v = statistics.median(t)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/C-matrix",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": v, "unit": "s/C-matrix", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "s/C-matrix", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plates")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--products", action="store_true",
                    help="time only the batched FP32 products of the workload (profiling aid)")
    ap.add_argument("--path", type=int, default=-1,
                    help="with --products: FP32 product kernels 0 generic, 1 compiled plans, -1 tuned")
    args = ap.parse_args()
    if args.products:
        print(json.dumps(run_products(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
