"""Benchmark of the AxLocal hot path on GB300 (one JSON line on rank 0).

Workload (the order sweep at its headline order): perturbed trilinear box of
64 x 64 x 32 = 131072 elements at N = 7 (67.1M local DOFs), X ~ U(-1, 1)
float64.  One step = one AxLocal over the whole mesh (all steps of the hot
path: geometry, forward contractions, geometric product, transposed
contractions) in the FP64-accurate trilinear-recompute kernel.  Inputs
(1.07 GB per step) are larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-sweep]

Multi-GPU (torchrun): every rank runs its own replica of the workload
(weak scaling, no collective on the data path); value = all ranks' DOFs /
max-over-ranks time.  The reference arm (--impl reference) times the FP64
CPU oracle on the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "AxLocal GDOF/s & % roofline vs N (recompute vs stored G); PCG time-to-1e-8"
UNIT = "GDOF/s"
HEADLINE_N = 7
HEADLINE_KIND = "trilinear"
HEADLINE_PREC = "f64dw"
SM_COUNT = 152  # GB300; run() reads the live count from the device
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (4 SMSPs x 32): the unit-count peak
FP32_FFMA_MEASURED_PER_SM_CLK = 116  # FFMA per SM per clock reached by a dependent-chain probe (91% of 128)
FP64_OPS_PER_SM_CLK = 2  # FP64 FMA instructions per SM per clock on GB300 (measured 1.19 TFLOP/s)

# dram bytes per launch from committed ncu captures, valid while the kernel
# sources hash to the recorded value (else reported as null).
# DRAM traffic per launch of the headline kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) on the 32^3-element case of
# the same kernel (profiles/ax_dw_trilinear_n7_e32768_traffic.md), scaled by
# elements to the 64x64x32 workload (traffic grows with the element count);
# valid while the kernel's sources hash to "src".
TRAFFIC = {"ax_fiber_kernel<DW, 8, 1, 1>": {"bytes": 4.0 * (140.625664e6 + 90.101504e6), "src": "396301e52c1c9ebc"}}


# the sources that define the headline kernel (double-word AxLocal, N = 7)
KERNEL_SOURCES = ("ax_fiber.cuh", "dw.cuh", "dw2.cuh", "inst_fiber.inc", "ax_dw_g1.cu", "tables.cuh", "ax_internal.h",
                  "gll.cpp", "gll.h")


def _src_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2504_07042_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        load = sorted(sm)[len(sm) // 4:] or sm  # drop the idle head of the record
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


def _host_link(torch, Xh, Yh, X, Y, reps=5):
    """Copy-engine bandwidth between pinned host memory and the device, GB/s:
    host to device, device to host, and both at once on two streams."""
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    nbytes = X.numel() * X.element_size()

    def timed(fn, nb):
        fn()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream()
        t0.record(cur)
        for _ in range(reps):
            fn()
        t1.record(cur)
        torch.cuda.synchronize()
        return nb * reps / (t0.elapsed_time(t1) * 1e-3) / 1e9

    def both():
        cur = torch.cuda.current_stream()
        sa.wait_stream(cur)
        sb.wait_stream(cur)
        with torch.cuda.stream(sa):
            X.copy_(Xh, non_blocking=True)
        with torch.cuda.stream(sb):
            Yh.copy_(Y, non_blocking=True)
        cur.wait_stream(sa)
        cur.wait_stream(sb)

    return {"h2d_gbs": timed(lambda: X.copy_(Xh, non_blocking=True), nbytes),
            "d2h_gbs": timed(lambda: Yh.copy_(Y, non_blocking=True), nbytes),
            "both_gbs": timed(both, 2 * nbytes)}


def _build_case(ax, torch, dev, N, kind, prec, mesh="trilinear", box=None):
    from paper_2504_07042_gb300 import inputs
    ex, ey, ez = box or inputs.sweep_box(N)
    if mesh == "parallelepiped":
        V = inputs.parallelepiped_vertices(ex, ey, ez)
    else:
        V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0)
    op = ax.Ax(torch.from_numpy(V).to(dev), N, kind, prec)
    X = torch.from_numpy(inputs.element_vectors(V.shape[0], N, seed=1)).to(dev, op.dtype)
    Y = torch.empty_like(X)
    return op, X, Y, V


def _time_launches(torch, fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        fn()
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps  # ms


def _median_launch_ms(torch, fn, launches, warmup, stream):
    """Median over `launches` launches, each timed alone by CUDA events on the
    launching stream, after `warmup` untimed launches."""
    for _ in range(warmup):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(launches)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def reduce_max_ms(torch, ms, device):
    """Max over ranks of a per-rank time (ms); identity on one process."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, dofs_per_rank, ms_max):
    """Replicas: every rank processes dofs_per_rank local DOFs per step; the
    job's throughput is all ranks' DOFs over the slowest rank's time (GDOF/s)."""
    return world * dofs_per_rank / (ms_max * 1e-3) / 1e9


def _pipe_peak(info, sm_mhz, sms=SM_COUNT):
    clk = (sm_mhz or 1980.0) * 1e6
    if info["pipe"] == 0:
        return FP64_OPS_PER_SM_CLK * sms * clk, "FP64 pipe"
    return FP32_LANES_PER_SM * sms * clk, "FP32 pipe"


def _roofline(info, ms, sm_mhz, hbm_gbs, sms=SM_COUNT):
    """Time-based roofline of Sec. 3.4: T_mem = bytes / measured HBM bandwidth,
    T_cmp = pipe instructions / pipe peak; frac = max(T_cmp, T_mem) / T_meas."""
    E = info["E"]
    t = ms * 1e-3
    bytes_ = info["bytes_per_element"] * E
    ops = info["pipe_ops_per_element"] * E
    pipe_peak, pipe_name = _pipe_peak(info, sm_mhz, sms)
    t_mem = bytes_ / (hbm_gbs * 1e9)
    t_cmp = ops / pipe_peak
    F = info["flops_ax_per_element"] * E
    r = {
        "t_mem_ms": t_mem * 1e3, "t_cmp_ms": t_cmp * 1e3, "t_meas_ms": ms,
        "P_eff_gflops": F / t / 1e9, "R_eff_gflops": F / max(t_mem, t_cmp) / 1e9,
        "frac_time_roofline": max(t_mem, t_cmp) / t,
        "hbm_gbs_achieved": bytes_ / t / 1e9, "pipe": pipe_name,
    }
    if t_cmp >= t_mem:
        r.update({"bound": "alu", "achieved": ops / t / 1e12, "peak": pipe_peak / 1e12,
                  "unit": "Tinst/s (%s lane-instructions)" % pipe_name})
    else:
        r.update({"bound": "hbm", "achieved": bytes_ / t / 1e9, "peak": hbm_gbs, "unit": "GB/s"})
    r["frac"] = r["achieved"] / r["peak"]
    if r["bound"] == "alu" and info["pipe"] != 0:
        # the same work against the FFMA rate a probe kernel actually reaches
        r["frac_vs_measured_ffma"] = r["frac"] * FP32_LANES_PER_SM / FP32_FFMA_MEASURED_PER_SM_CLK
    return r


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_oracle_rate_single_thread(seconds=3.0, N=HEADLINE_N):
    """cpu_oracle_rate on one host thread (the oracle's OpenMP team set to 1,
    then restored); returns (GDOF/s, sample)."""
    from oracle import oracle
    n = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        rate, _, sample = cpu_oracle_rate(seconds, N)
    finally:
        oracle.set_num_threads(n)
    return rate, sample


def cpu_oracle_rate(seconds=10.0, N=HEADLINE_N):
    """FP64 oracle AxLocal (Eq. 9 + Eq. 7 + Algorithm 1, OpenMP over elements)
    on a bounded sample of the workload mesh; returns (GDOF/s, cores, sample)."""
    from oracle import oracle
    from paper_2504_07042_gb300 import inputs
    ex, ey, ez = inputs.sweep_box(N)
    V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0)
    n3 = (N + 1) ** 3
    pilot = 512
    X = inputs.element_vectors(pilot, N, seed=1)
    t = time.perf_counter()
    oracle.axlocal_vertices(V[:pilot], X, N)
    dt = time.perf_counter() - t
    m = int(min(V.shape[0], max(pilot, pilot * seconds / max(dt, 1e-6))))
    X = inputs.element_vectors(m, N, seed=1)
    reps, t = 0, time.perf_counter()
    while True:  # whole passes over the sample until about `seconds` of CPU work
        oracle.axlocal_vertices(V[:m], X, N)
        reps += 1
        dt = time.perf_counter() - t
        if dt >= seconds:
            break
    return (reps * m * n3 / dt / 1e9, oracle.num_threads(),
            "%d pass(es) over the first %d of %d elements (%.1f s)" % (reps, m, V.shape[0], dt))


def host_cpu():
    """The host's CPU model and logical CPU count (lscpu where present)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": model, "logical_cpus": os.cpu_count()}


def cpu_oracle_sweep(seconds=1.5):
    """The FP64 oracle AxLocal on every order-sweep mesh (N in {3,5,7,9,11,15},
    perturbed trilinear box and parallelepiped box), all host threads, each on
    a bounded sample of about `seconds` of CPU work; GDOF/s per case."""
    from oracle import oracle
    from paper_2504_07042_gb300 import inputs
    out = []
    for N in (3, 5, 7, 9, 11, 15):
        ex, ey, ez = inputs.sweep_box(N)
        n3 = (N + 1) ** 3
        for mesh in ("trilinear", "parallelepiped"):
            if mesh == "parallelepiped":
                V = inputs.parallelepiped_vertices(ex, ey, ez)
            else:
                V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0)
            m = max(64, min(V.shape[0], int(2 ** 21 // n3)))
            X = inputs.element_vectors(m, N, seed=1)
            reps, t = 0, time.perf_counter()
            while True:
                oracle.axlocal_vertices(V[:m], X, N)
                reps += 1
                dt = time.perf_counter() - t
                if dt >= seconds:
                    break
            out.append({"N": N, "mesh": mesh, "gdofs": reps * m * n3 / dt / 1e9, "elements_in_sample": m,
                        "passes": reps, "seconds": dt, "threads": oracle.num_threads()})
    return out


def headline_config(world):
    """The workload the bench line measures (both arms report it)."""
    return {"workload": "order sweep at N=7: perturbed trilinear box 64x64x32 = 131072 elements, "
                        "67.1M local DOFs, X~U(-1,1) float64",
            "kind": HEADLINE_KIND, "precision": "float64 in/out, double-word FP32-pair arithmetic",
            "l2": "inputs larger than L2 (1.07 GB per step); no flush",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle
    from paper_2504_07042_gb300 import inputs
    N = HEADLINE_N
    ex, ey, ez = inputs.sweep_box(N)
    V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=0)
    n3 = (N + 1) ** 3
    m = 2048  # elements per step: a bounded sample of the workload
    X = inputs.element_vectors(m, N, seed=1)
    for _ in range(args.warmup):
        oracle.axlocal_vertices(V[:m], X, N)
    t = time.perf_counter()
    for s in range(args.steps):
        lo = (s * m) % (V.shape[0] - m)
        oracle.axlocal_vertices(V[lo:lo + m], X, N)
    dt = (time.perf_counter() - t) / args.steps
    val = m * n3 / dt / 1e9
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": headline_config(world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "FP64 CPU oracle on %d elements per step (a bounded sample of the "
                                       "131072-element workload), float64 arithmetic" % m},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _detail_path(args):
    if args.detail:
        return args.detail
    return os.path.join(ROOT, "bench_out", "bench_detail.json")


def _write_detail(path, detail):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(detail, f, indent=1)
        return path
    except OSError as e:
        sys.stderr.write("bench: could not write %s: %s\n" % (path, e))
        return None


def run(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    from paper_2504_07042_gb300 import ax
    peaks, peak_src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    op, X, Y, V = _build_case(ax, torch, dev, HEADLINE_N, HEADLINE_KIND, HEADLINE_PREC)
    info = op.ax_query()
    stream = torch.cuda.current_stream()
    E, n3 = op.E, op.n3
    fn = lambda: op.ax_local(X, Y, stream)  # noqa: E731
    for _ in range(max(args.warmup, 3)):
        fn()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    with Clocks(local) as ck:
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
    ms = reduce_max_ms(torch, t0.elapsed_time(t1) / args.steps, dev)
    clocks = ck.summary()
    value = whole_job_value(world, E * n3, ms)
    roof = _roofline(info, ms, clocks.get("sm_mhz"), hbm, sms)
    src = _src_hash()
    kname = "ax_fiber_kernel<DW, 8, %d, 1>" % info["kind"]
    traffic = TRAFFIC.get(kname)
    alu = roof["bound"] == "alu"
    roof_line = {"bound": roof["bound"], "achieved": roof["achieved"], "peak": roof["peak"], "unit": roof["unit"],
                 "frac": roof["frac"], "traffic": traffic["bytes"] if traffic and traffic["src"] == src else None,
                 "kernel": kname,
                 "peak_source": ("%s: %d lanes/SM x %d SMs x median SM clock (unit counts)"
                                 % (roof["pipe"], FP32_LANES_PER_SM, sms) if alu
                                 else "hbm_gbs of MEASURED_PEAKS.json (%s)" % peak_src)}
    if "frac_vs_measured_ffma" in roof:
        roof_line["frac_vs_measured_ffma"] = roof["frac_vs_measured_ffma"]
    roof_line["hbm_frac_of_measured"] = roof["hbm_gbs_achieved"] / hbm

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    Xh = torch.from_numpy(X.cpu().numpy()).pin_memory()
    Yh = torch.empty_like(Xh).pin_memory()
    for _ in range(2):
        op.ax_local_host(Xh, Yh, stream)
    t = time.perf_counter()
    e2e_steps = max(2, min(args.steps, 10))
    for _ in range(e2e_steps):
        op.ax_local_host(Xh, Yh, stream)
    e2e_s = (time.perf_counter() - t) / e2e_steps
    nbytes = X.numel() * X.element_size()
    e2e = {"value": world * E * n3 / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}
    # the host link's own bound on this leg: the same bytes moved by the copy
    # engines alone, both directions at once, no kernel
    link = _host_link(torch, Xh, Yh, X, Y)
    e2e["link_gbs"] = round(link["both_gbs"], 1)
    e2e["frac_of_link"] = round((2 * nbytes / e2e_s / 1e9) / link["both_gbs"], 3)
    del Xh, Yh
    op.ax_destroy()
    del X, Y
    torch.cuda.empty_cache()

    detail = {"headline": {"roofline_time_based": {k: roof[k] for k in (
        "t_mem_ms", "t_cmp_ms", "t_meas_ms", "P_eff_gflops", "R_eff_gflops", "frac_time_roofline",
        "hbm_gbs_achieved")}, "sms": sms, "src_hash": src}, "host_link": link}
    if not args.no_sweep and rank == 0:
        for name, f in (("sweep", lambda: run_sweep(ax, torch, dev, hbm, clocks.get("sm_mhz"), sms)),
                        ("pcg", lambda: run_pcg(ax, torch, dev)),
                        ("batch", lambda: run_batch(ax, torch, dev)),
                        ("learned", lambda: run_learned(ax, torch, dev))):
            t = time.perf_counter()
            detail[name] = f()
            sys.stderr.write("bench: %s section done in %.1f s\n" % (name, time.perf_counter() - t))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64dw", "data": "synthetic",
            "config": headline_config(world),
            "roofline": roof_line, "e2e": e2e,
            # per step: the AxLocal kernel and its scaled fix-up pass (an empty list: no work)
            "gpu_launches": 2 * args.steps, "clocks": clocks}
    if rank == 0:
        rate, cores, sample = cpu_oracle_rate()
        rate1, sample1 = cpu_oracle_rate_single_thread()
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                                "single_thread_value": rate1}
        detail["cpu_baseline_single_thread"] = {"value": rate1, "unit": UNIT, "sample": sample1}
        detail["host_cpu"] = host_cpu()
        if not args.no_sweep:
            detail["cpu_oracle_sweep"] = cpu_oracle_sweep()
        line["detail"] = os.path.relpath(_write_detail(_detail_path(args), detail) or "", ROOT)
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def cpu_oracle_pcg(N=7, n=16):
    """CPU-baseline leg for the solver: the FP64 oracle's Jacobi-PCG on the
    16^3 N = 7 Poisson problem to 1e-10 on the host cores, with its own
    factors (Eq. 7), nodal coordinates, mass and gather.  Returns its solution
    (the reference for the GPU solvers' errors) and its timing."""
    from oracle import oracle
    from paper_2504_07042_gb300 import inputs
    V = inputs.box_vertices(n, n, n, perturb=0.1, seed=0)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    G, _ = oracle.factors(V, N)
    P = oracle.nodal_coords(V, N)
    f = 3 * np.pi ** 2 * np.sin(np.pi * P[:, 0]) * np.sin(np.pi * P[:, 1]) * np.sin(np.pi * P[:, 2])
    b = oracle.gather(G[:, 6, :] * f, gid, ng)
    t = time.perf_counter()
    x, it, rr, ok = oracle.pcg(G, gid, ng, mask, b, N, rtol=1e-10, maxit=20000)
    dt = time.perf_counter() - t
    return x, {"seconds": dt, "iterations": it, "relres": rr, "converged": bool(ok), "rtol": 1e-10,
               "threads": oracle.num_threads(), "what": "FP64 CPU oracle Jacobi-PCG (Eq. 1; Algorithm 1 with "
                                                        "Eq. 7 factors), right-hand side built by the oracle"}


def run_pcg(ax, torch, dev):
    """Poisson -lap u = 3 pi^2 u, u = sin(pi x) sin(pi y) sin(pi z), homogeneous
    Dirichlet, 16^3 perturbed trilinear elements at N = 7: wall time to 1e-8
    relative residual for FP64-accurate Jacobi-PCG (double-word AxLocal) and
    for the mixed-precision solver (FP64 refinement around a float32 inner PCG
    whose AxLocal contracts in FP32, TF32, BF16 or FP16), and each solution's
    error against the FP64 oracle's own PCG solve of the same problem (its
    right-hand side built by the oracle), which is timed on the host cores."""
    from paper_2504_07042_gb300 import inputs
    N, n = 7, 16
    V = inputs.box_vertices(n, n, n, perturb=0.1, seed=0)
    gid, ng = inputs.box_global_ids(n, n, n, N)
    mask = inputs.box_boundary_mask(n, n, n, N)
    Vd = torch.from_numpy(V).to(dev)
    hi = ax.Ax(Vd, N, "trilinear", "f64dw")
    hi.gs_setup(torch.from_numpy(gid).to(dev), ng, torch.from_numpy(mask).to(dev))
    XYZ = torch.empty((V.shape[0], 3, (N + 1) ** 3), dtype=torch.float64, device=dev)
    hi.ax_node_coords(XYZ)
    u = torch.sin(torch.pi * XYZ[:, 0]) * torch.sin(torch.pi * XYZ[:, 1]) * torch.sin(torch.pi * XYZ[:, 2])
    b = hi.gs_gather(hi.ax_mass(3 * torch.pi ** 2 * u, torch.empty_like(u)), torch.empty(ng, dtype=torch.float64, device=dev))
    ug = torch.zeros(ng, dtype=torch.float64, device=dev)
    ug[torch.from_numpy(gid.reshape(-1)).to(dev)] = u.reshape(-1)

    x_orc, orc_pcg = cpu_oracle_pcg()
    x_orc_d = torch.from_numpy(x_orc).to(dev)
    nrm = float(x_orc_d.abs().max())
    out = {"workload": "16^3 perturbed trilinear elements, N=7, %d global nodes, rtol 1e-8" % ng,
           "oracle_pcg": orc_pcg}
    los = {p: ax.Ax(Vd, N, "trilinear", p) for p in ("fp32", "tf32", "bf16", "fp16")}
    runs = [("fp64_jacobi_pcg", lambda x: hi.pcg_solve(b, x, rtol=1e-8, maxit=20000, precond=1))]
    for p, inner_rtol in (("fp32", 1e-3), ("tf32", 1e-2), ("bf16", 1e-2), ("fp16", 1e-2)):
        runs.append(("mixed_fp64_refinement_%s_inner" % p,
                     lambda x, lo=los[p], r=inner_rtol: hi.pcg_solve_mixed(lo, b, x, rtol=1e-8, inner_rtol=r,
                                                                           max_outer=100)))
    for name, fn in runs:
        x = torch.zeros(ng, dtype=torch.float64, device=dev)
        fn(x)  # warm-up (allocations, module loading)
        x.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = fn(x)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        out[name] = {"seconds": dt, "result": list(res), "max_error_vs_exact": float((x - ug).abs().max()),
                     "rel_error_vs_oracle_solve": float((x - x_orc_d).abs().max()) / nrm}
        # the same solver to 1e-10 (the refinement's stated tolerance): error against the oracle solve
        x.zero_()
        if name == "fp64_jacobi_pcg":
            hi.pcg_solve(b, x, rtol=1e-10, maxit=20000, precond=1)
        else:
            lo = los[name.split("_")[3]]
            hi.pcg_solve_mixed(lo, b, x, rtol=1e-10, inner_rtol=1e-3 if lo is los["fp32"] else 1e-2, max_outer=100)
        out[name]["rel_error_vs_oracle_solve_at_1e-10"] = float((x - x_orc_d).abs().max()) / nrm
    out["speedup_mixed_over_fp64"] = out["fp64_jacobi_pcg"]["seconds"] / out["mixed_fp64_refinement_fp32_inner"]["seconds"]
    hi.ax_destroy()
    for lo in los.values():
        lo.ax_destroy()
    return out


def run_batch(ax, torch, dev):
    """64 perturbed-box meshes, E log-uniform on [64, 4096] (near-cubic boxes),
    N uniform on {3,5,7,9}, FP32, trilinear recompute.  AxLocal of the whole
    batch as ONE persistent launch over a (mesh, element tile) queue
    (untuned and autotuned), against one launch per order group and one
    launch per mesh; Jacobi-PCG to 1e-5 with one CUDA-graph launch per CG
    iteration holding one persistent kernel, against the grouped graph (one
    launch per phase and order) and the meshes solved in turn; then the
    grouped path with TF32 tensor-core contractions."""
    from paper_2504_07042_gb300 import inputs
    spec = inputs.batch_meshes()
    meshes = []
    for s, (ex, ey, ez, N) in enumerate(spec):
        V = inputs.box_vertices(ex, ey, ez, perturb=0.1, seed=s)
        gid, ng = inputs.box_global_ids(ex, ey, ez, N)
        mask = inputs.box_boundary_mask(ex, ey, ez, N)
        meshes.append((torch.from_numpy(V).to(dev), N, torch.from_numpy(gid).to(dev), ng,
                       torch.from_numpy(mask).to(dev)))
    bt = ax.AxBatch(meshes, "trilinear", "fp32")
    per = [ax.Ax(m[0], m[1], "trilinear", "fp32") for m in meshes]
    stream = torch.cuda.current_stream()
    X = torch.rand(bt.n_local, device=dev, dtype=torch.float32) * 2 - 1
    Y = torch.empty_like(X)
    slices = []
    for m, op in enumerate(per):
        n = op.E * op.n3
        lo = bt.local_offsets[m]
        slices.append((op, X[lo:lo + n], Y[lo:lo + n]))

    def per_mesh():
        for op, xs, ys in slices:
            op.ax_local(xs, ys, stream)

    local = lambda: bt.ax_batch_local(X, Y, stream)  # noqa: E731
    info = bt.ax_batch_info()
    untuned = _time_launches(torch, local, 10, 3, stream)
    tune = bt.ax_batch_tune()
    tuned = _time_launches(torch, local, 10, 3, stream)
    bt.ax_batch_set_persistent(False)
    grouped_untuned = _time_launches(torch, local, 10, 3, stream)
    gtune = bt.ax_batch_tune()
    grouped = _time_launches(torch, local, 10, 3, stream)
    ginfo = bt.ax_batch_info()
    bt.ax_batch_set_persistent(True)
    single = _time_launches(torch, per_mesh, 10, 3, stream)
    gd = lambda ms: bt.n_local / (ms * 1e-3) / 1e9  # noqa: E731
    out = {"meshes": len(spec), "elements": int(sum(m[0].shape[0] for m in meshes)), "local_dofs": bt.n_local,
           "global_dofs": bt.n_global, "orders": sorted(set(int(m[1]) for m in meshes)),
           "persistent": {"launches_per_axlocal": info["local_launches"],
                          "launches_per_cg_iteration": info["iteration_launches"],
                          "tuned_blocks_per_item_and_grid_per_order": {str(k): list(v) for k, v in tune.items()},
                          "axlocal_untuned_ms": untuned, "axlocal_tuned_ms": tuned,
                          "autotune_saves_pct": 100.0 * (untuned - tuned) / untuned,
                          "axlocal_tuned_gdofs": gd(tuned)},
           "grouped": {"launches_per_axlocal": ginfo["local_launches"],
                       "launches_per_cg_iteration": ginfo["iteration_launches"],
                       "tuned_tile_grid_per_order": {str(k): list(v) for k, v in gtune.items()},
                       "axlocal_untuned_ms": grouped_untuned, "axlocal_tuned_ms": grouped,
                       "axlocal_tuned_gdofs": gd(grouped)},
           "per_mesh": {"launches_per_axlocal": len(spec), "axlocal_ms": single, "axlocal_gdofs": gd(single)},
           "speedup_persistent_over_per_mesh": single / tuned, "speedup_persistent_over_grouped": grouped / tuned}
    bvec = torch.ones(bt.n_global, device=dev, dtype=torch.float32)

    def solve(graph, name):
        x = torch.zeros_like(bvec)
        bt.ax_batch_pcg(bvec, x, rtol=1e-5, maxit=20000, graph=graph)  # warm-up
        x.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        it, rr, st = bt.ax_batch_pcg(bvec, x, rtol=1e-5, maxit=20000, graph=graph)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t, "status": st, "max_iterations": max(it),
                     "total_iterations": sum(it), "max_relres": max(rr)}

    solve(1, "pcg_graph_persistent")
    bt.ax_batch_set_persistent(False)
    solve(1, "pcg_graph_grouped")
    bt.ax_batch_set_persistent(True)
    solve(0, "pcg_per_mesh")
    out["pcg_speedup_persistent_over_per_mesh"] = out["pcg_per_mesh"]["seconds"] / out["pcg_graph_persistent"]["seconds"]
    out["pcg_speedup_persistent_over_grouped"] = (out["pcg_graph_grouped"]["seconds"]
                                                  / out["pcg_graph_persistent"]["seconds"])
    for op in per:
        op.ax_destroy()
    bt.ax_batch_destroy()
    # the same batch with TF32 tensor-core contractions (FP32 accumulation): grouped launches
    bt = ax.AxBatch(meshes, "trilinear", "tf32")
    bt.ax_batch_tune()
    t_tc = _time_launches(torch, lambda: bt.ax_batch_local(X, Y, stream), 10, 3, stream)
    x = torch.zeros_like(bvec)
    bt.ax_batch_pcg(bvec, x, rtol=1e-5, maxit=20000, graph=1)  # warm-up
    x.zero_()
    torch.cuda.synchronize()
    t = time.perf_counter()
    it, rr, st = bt.ax_batch_pcg(bvec, x, rtol=1e-5, maxit=20000, graph=1)
    torch.cuda.synchronize()
    out["tf32_grouped"] = {"axlocal_batched_ms": t_tc, "axlocal_batched_gdofs": gd(t_tc),
                           "pcg_graph": {"seconds": time.perf_counter() - t, "status": st, "max_iterations": max(it),
                                         "total_iterations": sum(it), "max_relres": max(rr)}}
    bt.ax_batch_destroy()
    return out


def run_learned(ax, torch, dev):
    """Learned preconditioner on 32^3 = 32768 perturbed trilinear elements at
    N=7 (16.8M local DOFs): the MLP is trained (tcgen05 BF16 kernels) on
    residual/error pairs of 200 seeded solves with random smooth sources, the
    checkpoint and damping are picked on a held-out source, and flexible CG
    with it is timed against FP64-accurate Jacobi-PCG to 1e-8 relative
    residual on a third source (both with the double-word AxLocal)."""
    from paper_2504_07042_gb300 import inputs, learned
    N = 7

    def problem(n):
        V = inputs.box_vertices(n, n, n, perturb=0.1, seed=0)
        gid, ng = inputs.box_global_ids(n, n, n, N)
        mask = inputs.box_boundary_mask(n, n, n, N)
        Vd = torch.from_numpy(V).to(dev)
        op = ax.Ax(Vd, N, "trilinear", "f64dw")
        op.gs_setup(torch.from_numpy(gid).to(dev), ng, torch.from_numpy(mask).to(dev))
        return op, ng

    op, ng = problem(32)
    t = time.perf_counter()
    F, T = learned.collect_pairs(op, ng, seeds=range(100, 300), per_snapshot=1024)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t
    XYZ = learned.node_coords(op).cpu().numpy()
    b = learned.rhs_from_f(op, torch.from_numpy(inputs.smooth_rhs(XYZ, 300)).to(dev), ng)
    # validation: a held-out source (seed 301) on the same mesh picks the checkpoint and omega
    b_val = learned.rhs_from_f(op, torch.from_numpy(inputs.smooth_rhs(XYZ, 301)).to(dev), ng)
    mlp = ax.AxMLP(seed=2)
    t = time.perf_counter()
    omega, it_val, hist, trace = learned.train_select(mlp, F, T, op, b_val, chunks=(3, 3, 3, 3), omegas=(0.5, 0.75),
                                                      lr=3e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t
    samples = int(F.shape[0])
    del F, T
    out = {"workload": "32^3 perturbed trilinear elements N=7, %d global nodes; training pairs from 200 seeded "
                       "solves (smooth exact solutions, seeds 100-299), validation source seed 301, test source "
                       "seed 300, rtol 1e-8" % ng,
           "training": {"pairs": samples, "pair_collection_s": t_pairs, "train_and_select_s": t_train,
                        "epochs": len(hist), "loss_first_epoch": float(hist[0]), "loss_last_epoch": float(hist[-1]),
                        "selected_omega": omega, "validation_iterations": it_val,
                        "selection_trace": [list(x) for x in trace]}}
    if omega is None:
        omega = 0.5
    runs = (("fp64_jacobi_pcg", lambda x: op.pcg_solve(b, x, rtol=1e-8, maxit=20000, precond=1)),
            ("learned_flexible_pcg", lambda x: ax.pcg_solve_learned(op, mlp, b, x, rtol=1e-8, maxit=20000, omega=omega,
                                                                     check=False)))
    sol = {}
    for name, fn in runs:
        x = torch.zeros(ng, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = fn(x)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t, "result": list(res)}
        sol[name] = x
    out["max_diff_learned_vs_jacobi"] = float((sol["learned_flexible_pcg"] - sol["fp64_jacobi_pcg"]).abs().max()
                                              / sol["fp64_jacobi_pcg"].abs().max())
    out["iteration_ratio"] = out["learned_flexible_pcg"]["result"][0] / max(1, out["fp64_jacobi_pcg"]["result"][0])
    out["speedup_learned_over_jacobi"] = out["fp64_jacobi_pcg"]["seconds"] / out["learned_flexible_pcg"]["seconds"]
    mlp.ax_mlp_destroy()
    op.ax_destroy()
    return out


def run_sweep(ax, torch, dev, hbm, sm_mhz, sms=SM_COUNT):
    """Per-N GDOF/s and roofline fraction, recompute vs stored, per precision:
    the median of 20 launches, each timed alone, after 3 warm-up launches."""
    out = []
    stream = torch.cuda.current_stream()
    for N in (3, 5, 7, 9, 11, 15):
        for mesh, kinds in (("trilinear", ("stored", "trilinear", "partial")), ("parallelepiped", ("parallelepiped",))):
            for prec in ("fp64", "f64dw", "fp32", "tf32", "bf16", "fp16"):
                for kind in kinds:
                    if prec in ("tf32", "bf16", "fp16") and kind in ("stored", "partial"):
                        continue  # tensor-core contractions: the recompute kinds only
                    op, X, Y, _ = _build_case(ax, torch, dev, N, kind, prec, mesh)
                    info = op.ax_query()
                    ms = _median_launch_ms(torch, lambda: op.ax_local(X, Y, stream), 20, 3, stream)
                    roof = _roofline(info, ms, sm_mhz, hbm, sms)
                    out.append({"N": N, "mesh": mesh, "kind": kind, "prec": prec, "E": op.E,
                                "gdofs": op.E * op.n3 / (ms * 1e-3) / 1e9, "ms": ms, "bound": roof["bound"],
                                "frac": roof["frac"], "frac_vs_measured_ffma": roof.get("frac_vs_measured_ffma"),
                                "P_eff_gflops": roof["P_eff_gflops"],
                                "hbm_gbs": roof["hbm_gbs_achieved"]})
                    op.ax_destroy()
                    del X, Y
                    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--detail", default=None, help="side file for the sweep and solver sections "
                    "(default bench_out/bench_detail.json)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
