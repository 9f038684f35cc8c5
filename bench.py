#!/usr/bin/env python
"""Benchmark of the VoxCap GB300 hot path.

Headline workload: two interleaved meanders (line width 4, spacing 4,
thickness 8, 32 legs) in eps_r = 3.9 on a 512 x 512 x 64 grid, 1,410,624
panels, 2 conductors, with the block-Toeplitz tensors restored from Tucker
factors compressed at tolerance 1e-6 (installed once before timing, as the
paper's installation stage), GMRES tolerance 1e-6.

One step = one full capacitance extraction: voxcap_setup from device-resident
voxel labels (panels, Tucker restoration of the Toeplitz tensors on the
tensor cores, circulant embedding and kernel spectra, preconditioner)
followed by the batched FP32 + FP64-refinement GMRES solve of both
conductors and the capacitance reduction.  ``value`` is seconds per
capacitance matrix over the whole job (lower is better).  The line also
carries the plain-FP64 time of the same extraction, the set-up phases
(Tucker restoration against FP64 generation), the HBM roofline of the FP32
product, a cuFFT-based product of the same sizes timed beside it, the
end-to-end number through the C ABI with host buffers, the smaller
configurations (plates, bus crossing with 16 small structures, pillars with
the adjoint gradient), the oracle's CPU time, clocks and the kernel-launch
count.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --products --workload bus [--path P]     (product timing only;
                                                            meanders256: a profiling size)
  python bench.py --setup --workload pillars                (set-up timing only)

Under torchrun (N > 1) every rank runs its own replica of the workload
(independent extractions, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matvecs/s, s per C-matrix at 1e-4 rel err: FP32+refine vs FP64; % HBM roofline"
TUCKER_TOL = 1e-6
# plain-FP64 products of the headline extraction (GMRES at 1e-6 with the
# paper's preconditioner), the count the CPU product time is scaled by when
# the reference arm runs without a GPU solve beside it
FP64_PRODUCTS_MEANDERS = 90


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
    if name == "meanders256":
        return W.meanders(256, 256, 64, 16), ("two interleaved meanders (width 4, spacing 4, thickness 8, "
                                              "16 legs) in eps_r=3.9, 256x256x64 grid (profiling size)")
    raise SystemExit(f"unknown workload {name}")


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


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


def product_sources_hash():
    """Digest of the sources of the product kernels: a DRAM-traffic capture
    applies to the current build only while this matches."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2004_02609_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                    glob.glob(os.path.join(csrc, "*.h"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def captured_traffic(workload_name):
    """DRAM bytes (read + write) of one batched FP32 product, summed over its
    kernels, from the ncu capture summarised in the profiles folder for this
    workload -- or None when no capture exists or the kernels have changed
    since it was taken (its recorded source digest differs)."""
    p = os.path.join(ROOT, "profiles", f"product_traffic_{workload_name}.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"traffic_bytes_per_product:\s*(\d+)\s+sources:\s*([0-9a-f]+)", txt)
    if not m or m.group(2) != product_sources_hash():
        return None
    return int(m.group(1))


def time_products(vc, x, reps):
    """Mean seconds of one batched product, CUDA events on the launching stream."""
    import torch
    for _ in range(3):
        vc.matvec(x)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        vc.matvec(x)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def product_roofline(vc, dev, reps, workload_name):
    """Time `reps` batched FP32 products (all conductor columns) with CUDA
    events on the launching stream and relate the model bytes to the
    measured HBM peak."""
    import torch
    x = torch.randn(vc.n_conductors, vc.N, device=dev, dtype=torch.float32)
    t = time_products(vc, x, reps)
    hbm, peak_src = read_peaks()
    b = mvm_model_bytes(vc, vc.n_conductors) * vc.n_conductors
    return vc.n_conductors / t, {
        "kernel": "FP32 product, 5 passes (x scatter+R2C, y, z+spectral MAC+inverse z, inverse y, "
                  f"C2R+gather), {vc.n_conductors} columns, {workload_name}",
        "bound": "hbm", "achieved": b / t / 1e9, "peak": hbm, "unit": "GB/s",
        "frac": b / t / 1e9 / hbm, "target_frac": 0.6, "target_met": b / t / 1e9 / hbm >= 0.6,
        "traffic": captured_traffic(workload_name),
        "peak_source": peak_src, "bytes_per_launch": b, "launch_s": t,
        "fft_lengths": list(vc.fft_lengths()), "path": vc.set_product_path(-2)}


def max_over_ranks(x, world, device):
    """The largest x over the ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


# ---------------------------------------------------------------- pieces of the GPU arm
def install_tucker(D, tol, rank, world):
    """The installation stage (Sec. II.C): the four canonical Toeplitz tensors
    on a D^3 cube, compressed at `tol`.  Rank 0 installs; under torchrun the
    other ranks load its file.  Returns (model, seconds)."""
    from paper_2004_02609_gb300 import tucker as T
    t0 = time.perf_counter()
    path = os.path.join(tempfile.gettempdir(), f"voxcap_tucker_D{D}_tol{tol:g}.npz")
    if rank == 0:
        model = T.install(D, tol)
        if world > 1:
            model.save(path)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        if rank != 0:
            model = T.TuckerModel.load(path)
    return model, time.perf_counter() - t0


def extraction(V, w, labels, precision, tol, tucker=None, **kw):
    """One capacitance extraction: set-up + batched solve; returns
    (C, stats, panels, set-up phase times)."""
    vc = V.VoxCap(labels, w.conductor_id, w.eps_r, w.voxel_size, precision=precision, tucker=tucker, **kw)
    C, st = vc.capacitance(tol=tol)
    n, ph = vc.N, vc.setup_times()
    vc.close()
    return C, st, n, ph


def timed(fn, stream, flush=None):
    """fn() bracketed by CUDA events on `stream` (L2 flushed first)."""
    import torch
    if flush is not None:
        flush_l2(flush)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def rel_c_err(A, B):
    A, B = np.asarray(A), np.asarray(B)
    return float(np.max(np.abs(A - B)) / np.max(np.abs(B)))


def config_line(V, name, dev, stream, flush, tol, reps=2, roof_reps=10, grad=False, small=False):
    """A smaller configuration as an extra key: FP32+refine and plain FP64
    seconds per capacitance matrix, iterations, product roofline; the bus
    crossing adds its 16 small box structures batched in one handle, the
    pillars the adjoint gradient of all C entries."""
    import torch
    w, desc = workload(name)
    lab = torch.tensor(w.labels, device=dev)
    extraction(V, w, lab, "fp32_refine", tol)
    t32 = [timed(lambda: extraction(V, w, lab, "fp32_refine", tol), stream, flush) for _ in range(reps)]
    (C32, st32, N, _) = t32[-1][1]
    t64, (C64, st64, _, _) = timed(lambda: extraction(V, w, lab, "fp64", tol), stream, flush)
    out = {"workload": desc, "panels": N, "conductors": int(np.asarray(C32).shape[0]), "gmres_tol": tol,
           "fp32_refine": {"s_per_C": statistics.median(t for t, _ in t32), "iterations": st32["iterations"],
                           "products": st32["matvecs"]},
           "fp64": {"s_per_C": t64, "iterations": st64["iterations"], "products": st64["matvecs"]},
           "c_rel_err_fp32_refine_vs_fp64": rel_c_err(C32, C64)}
    vc = V.VoxCap(lab, w.conductor_id, w.eps_r, w.voxel_size)
    out["matvecs_per_s"], out["roofline"] = product_roofline(vc, dev, roof_reps, name)
    if grad:
        m = vc.n_conductors
        vc.capacitance(tol=tol)
        tg, _ = timed(lambda: vc.capacitance_grad(np.ones((m, m)), tol=tol), stream, flush)
        out["adjoint_gradient_s"] = tg
    vc.close()
    if small:
        from paper_2004_02609_gb300 import workloads as W
        boxes = W.small_boxes(16, 16)
        labs = torch.tensor(np.stack([b.labels for b in boxes]), device=dev)
        b0 = boxes[0]

        def batch():
            v = V.VoxCap(labs, b0.conductor_id, b0.eps_r, 1e-6)
            C, st = v.capacitance(tol=tol)
            v.close()
            return st
        batch()
        ts, st = timed(batch, stream, flush)
        out["small_structures"] = {"count": 16, "grid": "16^3", "s_for_all_16_C": ts,
                                   "iterations": st["iterations"]}
    return out


def cufft_product(vc, dev, reps):
    """The same product with cuFFT (torch.fft, which calls cuFFT) in place
    of the library's passes, for timing only: panel scatter onto the three
    face grids, R2C along x and C2C along y and z at the handle's padded
    lengths (zero padding implicit, as in the library), the multiply-
    accumulate with 15 real kernel spectra on the full half spectrum
    (random values: the cost does not depend on them; the half-voxel phases
    are left out), the inverse transforms truncated to the face box, and the
    gather.  Never reachable from the library."""
    import torch
    Mx, My, Mz = vc.fft_lengths()
    nx, ny, nz = vc.shape
    Lx, Ly, Lz = nx + 1, ny + 1, nz + 1
    Hx = Mx // 2 + 1
    m = vc.n_conductors
    pm = vc.panel_map()
    o = pm["orient"].astype(np.int64)
    f = pm["face"].astype(np.int64)
    Fx = np.where(o == 0, nx + 1, nx)
    Fy = np.where(o == 1, ny + 1, ny)
    i, jj, k = f % Fx, (f // Fx) % Fy, f // (Fx * Fy)
    flat = torch.tensor(((o * Lz + k) * Ly + jj) * Lx + i, device=dev)
    kind = torch.tensor(pm["kind"].astype(np.int64), device=dev)
    x = torch.randn(m, vc.N, device=dev)
    spec = torch.randn(15, Mz, My, Hx, device=dev)
    pairs = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
    epairs = [[6, 9, 10], [12, 7, 11], [13, 14, 8]]

    def product():
        g = torch.zeros(m, 3 * Lz * Ly * Lx, device=dev)
        g[:, flat] = x
        g = g.view(m, 3, Lz, Ly, Lx)
        q = torch.fft.rfft(g, n=Mx, dim=-1)
        q = torch.fft.fft(q, n=My, dim=-2)
        q = torch.fft.fft(q, n=Mz, dim=-3)
        outs = []
        for tab in (pairs, epairs):
            for a in range(3):
                acc = q[:, 0] * spec[tab[a][0]] + q[:, 1] * spec[tab[a][1]] + q[:, 2] * spec[tab[a][2]]
                c = torch.fft.ifft(acc, dim=-3)[:, :Lz]
                c = torch.fft.ifft(c, dim=-2)[:, :, :Ly]
                outs.append(torch.fft.irfft(c, n=Mx, dim=-1)[..., :Lx])
        pot = torch.stack(outs[:3], 1).reshape(m, -1)
        fld = torch.stack(outs[3:], 1).reshape(m, -1)
        return torch.where(kind == 0, pot[:, flat], fld[:, flat])

    product()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        product()
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    del spec
    torch.cuda.empty_cache()
    return t


def cpu_fft_product_seconds(w, workers):
    """Seconds of one product of the oracle's CPU FFT method (scipy FFTs on
    `workers` threads) on workload w, with stand-in spectra (see
    oracle.fft_gmres.FFTProduct.timing_stand_in)."""
    import oracle as O
    from oracle import fft_gmres as F
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    prod = F.FFTProduct.timing_stand_in(ps, workers=workers)
    x = np.random.default_rng(0).standard_normal(ps.n)
    t0 = time.perf_counter()
    prod(x)
    return time.perf_counter() - t0, ps.n


def cpu_baseline(fp64_products):
    """The oracle on the host cores: the CPU FFT product of the headline grid
    timed once (stand-in spectra) and scaled by the plain-FP64 product count
    of the GPU extraction; the dense oracle (Galerkin integrals, LU, Eq. 8)
    timed in full on the 4^3 cube."""
    import oracle as O
    from paper_2004_02609_gb300 import workloads as W
    cores = os.cpu_count()
    w, _ = workload("meanders")
    t_mvm, n = cpu_fft_product_seconds(w, cores)
    c = W.cube(4)
    t0 = time.perf_counter()
    O.capacitance(O.panels(c.labels, c.conductor_id, c.eps_r), voxel_size=c.voxel_size)
    t_dense = time.perf_counter() - t0
    return {"value": t_mvm * fp64_products, "unit": "s/C-matrix", "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": (f"one CPU FFT product of the oracle (scipy.fft, {cores} workers) on the meanders grid "
                       f"({n} panels, stand-in spectra) timed at {t_mvm:.2f} s and scaled by the "
                       f"{fp64_products} products of the plain-FP64 GPU extraction (extrapolated); "
                       f"dense oracle extraction of the 4^3 cube timed in full: {t_dense:.2f} s"),
            "cpu_product_s": t_mvm, "dense_cube4_s": t_dense}


# ---------------------------------------------------------------- the GPU arm
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
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    w, desc = workload("meanders")
    tol = args.tol
    lab_dev = torch.tensor(w.labels, device=dev)
    D = max(w.labels.shape) + 2
    model, t_install = install_tucker(D, TUCKER_TOL, rank, world)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step(precision="fp32_refine", labels=lab_dev):
        return extraction(V, w, labels, precision, tol, tucker=model)

    # ---- warm-up, then exactly K timed steps: FP32 products + FP64 refinement
    for _ in range(args.warmup):
        step()
    times = []
    barrier()
    torch.cuda.synchronize()
    launches0 = V.launch_count()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            t, (C32, st32, N, ph32) = timed(step, stream, flush)
            times.append(t)
    torch.cuda.synchronize()
    barrier()
    launches = V.launch_count() - launches0
    t_step = sum(times) / len(times)
    t_max = max_over_ranks(sum(times), world, dev) / len(times)
    # ---- plain FP64, same extraction (Tucker-restored tensors)
    t64, (C64, st64, _, ph64) = timed(lambda: step("fp64"), stream, flush)
    # ---- the fast refinement option (FP32 Gram-Schmidt arithmetic, FP32
    # residuals for early sweeps; the headline keeps FP64 there)
    fast_step = lambda: extraction(V, w, lab_dev, "fp32_refine", tol, tucker=model, fast_refine=1)
    fast_step()
    tf = []
    for _ in range(3):
        t, (Cf, stf, _, _) = timed(fast_step, stream, flush)
        tf.append(t)
    # ---- set-up: Tucker restoration against generating the tensors in FP64
    _, _, _, ph_gen = extraction(V, w, lab_dev, "fp64", tol)
    # ---- the FP32 product: roofline, cuFFT beside it
    vc = V.VoxCap(lab_dev, w.conductor_id, w.eps_r, w.voxel_size, tucker=model)
    matvecs_per_s, roof = product_roofline(vc, dev, 10, "meanders")
    t_cufft = cufft_product(vc, dev, 3)
    m = vc.n_conductors
    vc.close()
    # ---- end to end through the C ABI: host labels in, host C out
    lab_host = np.ascontiguousarray(w.labels, dtype=np.int32)
    e2e = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        extraction(V, w, lab_host, "fp32_refine", tol, tucker=model)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    h2d = lab_host.nbytes + w.conductor_id.astype(np.int32).nbytes + w.eps_r.astype(np.float64).nbytes
    d2h = int(np.asarray(C32).size) * 8
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
        "config": {"workload": desc, "panels": N, "conductors": m, "gmres_tol": tol, "restart": 35,
                   "precond": "bdd nv=10", "toeplitz": f"Tucker-restored, tolerance {TUCKER_TOL:g}",
                   "step": "setup from device labels (Tucker restoration) + batched capacitance solve",
                   "l2": "flushed between timed steps (256 MB write)"},
        "fp32_refine": {"s_per_C": t_step, "iterations": st32["iterations"], "sweeps": st32["sweeps"],
                        "products": st32["matvecs"], "setup_phases_s": ph32,
                        "c_rel_err_vs_fp64": rel_c_err(C32, C64)},
        "fp64": {"s_per_C": t64, "iterations": st64["iterations"], "products": st64["matvecs"],
                 "setup_phases_s": ph64},
        "fp32_refine_fast": {"s_per_C": sum(tf) / len(tf), "steps": len(tf), "iterations": stf["iterations"],
                             "sweeps": stf["sweeps"], "products": stf["matvecs"],
                             "c_rel_err_vs_fp64": rel_c_err(Cf, C64),
                             "option": "fast_refine=1: FP32 Gram-Schmidt arithmetic for the FP32 basis, FP32 "
                                       "residual after sweeps that only had to reach >= 1e-5"},
        "toeplitz_tensors": {"tucker_restore_s": ph32["toeplitz"], "fp64_generation_s": ph_gen["toeplitz"],
                             "install_s_untimed": t_install, "ranks": model.ranks,
                             "compressed_bytes": int(model.nbytes())},
        "matvecs_per_s": matvecs_per_s,
        "roofline": roof,
        "cufft_product_s": t_cufft,
        "e2e": {"value": statistics.median(e2e), "unit": "s/C-matrix", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": d2h, "steps": len(e2e)},
        "gpu_launches": int(launches),
        "gpu_launches_per_step": int(launches / max(1, args.steps)),
        "clocks": clk.summary(),
    }
    if not args.no_configs:
        res["configs"] = {
            "plates": config_line(V, "plates", dev, stream, flush, tol, reps=3),
            "bus": config_line(V, "bus", dev, stream, flush, tol, small=True),
            "pillars": config_line(V, "pillars", dev, stream, flush, tol, grad=True),
        }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(st64["matvecs"])
    return res


def run_products(args):
    """Product-only timing (--products): set-up once, then K batched FP32
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
    return {"mode": "products", "workload": desc, "panels": vc.N, "columns": m,
            "path": vc.set_product_path(-2), "fft_lengths": vc.fft_lengths(), "s_per_batched_product": t,
            "matvecs_per_s": m / t, "model_bytes": b, "achieved_GBps": b / t / 1e9,
            "frac_of_" + src + "_hbm": b / t / 1e9 / hbm, "sources": product_sources_hash()}


def run_setup(args):
    """Set-up only (--setup): the workload's set-up with its Toeplitz tensors
    restored from Tucker factors (tolerance 1e-6, installed first) and with
    them generated in FP64, K times each; prints the phase times (profiling
    aid for the tensor-core restoration)."""
    import torch
    import __graft_entry__ as ge
    from paper_2004_02609_gb300 import voxcap as V
    ge.build()
    w, desc = workload(args.workload)
    lab = torch.tensor(w.labels, device="cuda")
    model, t_install = install_tucker(max(w.labels.shape) + 2, TUCKER_TOL, 0, 1)
    out = {"mode": "setup", "workload": desc, "install_s": t_install, "ranks": model.ranks}
    for name, kw in (("tucker", {"tucker": model}), ("fp64_generated", {"entries": "fp64"})):
        ph = []
        for _ in range(args.warmup + args.steps):
            vc = V.VoxCap(lab, w.conductor_id, w.eps_r, w.voxel_size, **kw)
            ph.append(vc.setup_times())
            vc.close()
        out[name] = {k: statistics.median(p[k] for p in ph[args.warmup:]) for k in ph[0]}
    return out


# ---------------------------------------------------------------- the reference arm
def run_reference(args, rank, world):
    """The oracle (plain FP64 CPU; the paper publishes no code) on the same
    workload and metric: every step times one product of the oracle's CPU
    FFT method on the meanders grid (stand-in spectra: the same FFT, multiply
    and scatter work as the real product), and seconds per C-matrix are that
    time scaled by the plain-FP64 product count of the extraction.  The
    warm-up steps run the same product on the plates grid."""
    if rank != 0:
        return None
    w, desc = workload("meanders")
    wp, _ = workload("plates")
    cores = os.cpu_count()
    for _ in range(args.warmup):
        cpu_fft_product_seconds(wp, cores)
    per = []
    n = 0
    for _ in range(args.steps):
        t, n = cpu_fft_product_seconds(w, cores)
        per.append(t)
    t_mvm = statistics.median(per)
    v = t_mvm * FP64_PRODUCTS_MEANDERS
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/C-matrix",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(per) * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "panels": n, "conductors": 2, "gmres_tol": args.tol, "restart": 35,
                       "toeplitz": "oracle FFT product, stand-in spectra (timing)"},
            "cpu_baseline": {"value": v, "unit": "s/C-matrix", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": (f"each step one CPU FFT product (scipy.fft, {cores} workers, {n} panels) "
                                        f"timed; value = median product time {t_mvm:.2f} s x "
                                        f"{FP64_PRODUCTS_MEANDERS} products of the plain-FP64 extraction "
                                        "(extrapolated); ms_per_step is the measured time of one step")},
            "e2e": {"value": v, "unit": "s/C-matrix", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--workload", default="meanders", help="with --products: the workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the smaller configurations")
    ap.add_argument("--products", action="store_true",
                    help="time only the batched FP32 products of the workload (profiling aid)")
    ap.add_argument("--path", type=int, default=-1,
                    help="with --products: FP32 product kernels 0 generic, 1 compiled plans (+ variant bits), -1 tuned")
    ap.add_argument("--setup", action="store_true",
                    help="time only the set-up of the workload, Tucker-restored and generated (profiling aid)")
    args = ap.parse_args()
    if args.products:
        print(json.dumps(run_products(args)), flush=True)
        return
    if args.setup:
        print(json.dumps(run_setup(args)), flush=True)
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
