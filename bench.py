#!/usr/bin/env python3
"""Benchmark of the p-norm (x,max) semiring product on GB300.

Metric: effective semiring Gop/s, counted as M*N*K (n^3) per product, of the
p-norm tensor-core estimate, next to the exact CUDA-core product and the FP64
CPU oracle, with the estimate's error stated against the exact product.

Workload (default): one square product, n = 16384, entries exp(-Exponential(4))
(= U^(1/4)), BF16 powered operands, P = {1, 2, ..., 64}.  A step is one full
call: maxima and scales, powered operand images, the tensor-core level
launches with the fused stable-p epilogue, writing C and p_sel.  Inputs (1 GiB
each) are larger than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch under torch.distributed.run; every rank computes its own
product (independent replicas, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--k", type=int, default=0,
                    help="contraction length of the default product (0: n); M = N = n")
    ap.add_argument("--compute", default="bf16")
    ap.add_argument("--tile-n", type=int, default=0)
    ap.add_argument("--tile-m", type=int, default=0,
                    help="0 automatic, 128 one CTA per tile, 256 a CTA pair per 256 x 256 tile")
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--err-samples", type=int, default=4096)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-exact", action="store_true")
    ap.add_argument("--no-e4m3", action="store_true",
                    help="skip the E4M3 run of the default product")
    ap.add_argument("--count", type=int, default=4096,
                    help="grouped workload: number of problems")
    ap.add_argument("--estimator", type=int, default=0, choices=[0, 1, 2],
                    help="0: plain largest-stable-p norm; 1 / 2: r = 1 / r = 2 multiset "
                         "projection")
    ap.add_argument("--correction", type=int, default=0, choices=[0, 1, 2],
                    help="1: divide by K^(1/p*); 2: affine model fitted on --n-fit exact samples")
    ap.add_argument("--n-fit", type=int, default=1024)
    ap.add_argument("--workload", default="pnorm",
                    choices=["pnorm", "apsp", "backward", "grouped", "maxconv", "maxconv-long",
                             "topk", "peaks"],
                    help="pnorm: the default product; the others measure the other paths")
    return ap.parse_args()


P_LOG2 = list(range(7))


def launches_per_step(args):
    """maxima + (A images, B images, GEMM) per level; the r = 2 projection adds
    a level at 3p/4 below every p whose p/2 and p/4 are in P; the affine
    correction its two fit kernels."""
    levels = len(P_LOG2) + (len(P_LOG2) - 2 if args.estimator == 2 else 0)
    return 1 + 3 * levels + (2 if args.correction == 2 else 0)


def workload_name(n, compute, estimator=0, correction=0, n_fit=0):
    est = "" if estimator == 0 else f" r={estimator} projection estimator;"
    if correction == 1:
        est += " estimate / K^(1/p*);"
    elif correction == 2:
        est += f" affine correction from {n_fit} exact samples;"
    return (f"maxprod_pnorm n={n} {compute} P={{1..64}} entries exp(-Exp(4));{est} "
            f"exact CUDA-core (x,max) product as the comparison")


# ---------------------------------------------------------------- clocks ---
class ClockSampler:
    """Samples nvidia-smi (SM clock, throttle reasons) every 100 ms; only the
    samples whose timestamps fall inside the timed region are reported (the
    nearest one if the region is shorter than the sampling period)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark_begin(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        from datetime import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        samples = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    samples.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inside = [x for x in samples if self.t0 <= x[0] <= self.t1]
        how = "inside timed region"
        if not inside:
            mid = 0.5 * (self.t0 + self.t1)
            inside = [min(samples, key=lambda x: abs(x[0] - mid))]
            how = "nearest sample (timed region shorter than the 100 ms period)"
        reasons = set()
        for x in inside:
            for nm, val in zip(self.NAMES, x[3]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(x[1] for x in inside),
                "sm_max_mhz": max(x[2] for x in inside), "reasons": sorted(reasons),
                "samples": len(inside), "sampling": how}


# --------------------------------------------------------------- helpers ---
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


TENSOR_PEAKS_PROFILE = "tensor_peaks_tf32_e4m3.md"


def tensor_peaks():
    """TF32 and E4M3 dense peaks measured on the GB300s with the library
    GEMMs (``bench.py --workload peaks``), recorded in profiles/; {} if absent."""
    out = {}
    try:
        text = open(os.path.join(ROOT, "profiles", TENSOR_PEAKS_PROFILE)).read()
    except OSError:
        return out
    for key in ("tf32_tflops", "tf32_tflops_sustained", "e4m3_tflops", "e4m3_tflops_sustained"):
        m = re.search(rf"^{key}:\s*([0-9.eE+]+)\s*$", text, re.M)
        if m:
            out[key] = float(m.group(1))
    return out


def gemm_peak_tflops(compute, peaks, burst=True, measured=None):
    """Dense tensor peak of the operand format and where it comes from.  burst:
    the figure for a kernel timed alone in a short region (else the sustained,
    seconds-long one).  BF16 / FP16 take the measured BF16 figure; TF32 and
    E4M3 their own measured figures when `measured` holds them, else the BF16
    figure times the nominal format ratio; 3xTF32 issues three TF32 products."""
    sfx = "" if burst else "_sustained"
    measured = measured or {}
    bf16 = peaks["bf16_tflops" + sfx]
    if compute in ("bf16", "f16"):
        return bf16, "measured bf16_tflops" + sfx
    base = {"tf32": "tf32", "f32": "tf32", "e4m3": "e4m3"}[compute]
    div = 3.0 if compute == "f32" else 1.0
    key = f"{base}_tflops{sfx}"
    if key in measured:
        return measured[key] / div, f"measured {key}" + (" / 3 (3xTF32)" if div > 1 else "")
    ratio = {"tf32": 0.5, "e4m3": 2.0}[base]
    return bf16 * ratio / div, (f"bf16_tflops{sfx} x nominal {base} ratio {ratio}"
                                + (" / 3 (3xTF32)" if div > 1 else ""))


def gemm_source_sha():
    """Hash of every source the tensor-core level kernel is compiled from."""
    h = hashlib.sha256()
    for f in ("pn_gemm_kernel.cuh", "pn_device.cuh", "pn_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1511_05690_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(compute):
    """DRAM bytes per top-level GEMM launch recorded by ncu in profiles/, if the
    kernel source is unchanged since the capture (else None)."""
    prof = os.path.join(ROOT, "profiles", f"gemm_level_{compute}_n16384.md")
    try:
        sha = gemm_source_sha()
        text = open(prof).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1))


def cpu_baseline(A_h, B_h, n, seconds, oracle):
    """The FP64 oracle (exact max + every p-sum) on sampled output entries,
    sized to about `seconds` of CPU time; Gop/s counted as K per entry."""
    g = workloads.rng(None, 99)
    rows = np.unique(g.integers(0, n, 64))
    A64 = A_h[rows].astype(np.float64)  # only sampled rows are read
    B64 = B_h.astype(np.float64)
    r = oracle.row_scales(A64)
    c = oracle.col_scales(B64)

    Kc = A_h.shape[1]  # semiring ops per output entry

    def run(E):
        loc = g.integers(0, len(rows), E)
        jj = g.integers(0, n, E)
        t0 = time.perf_counter()
        oracle.entries(A64, B64, loc, jj, P_LOG2, r, c)
        return time.perf_counter() - t0

    E0 = 64
    t0 = run(E0)
    E = max(E0, int(E0 * seconds / max(t0, 1e-3)))
    t = run(E)
    cores = oracle.num_threads()
    out = {"value": E * Kc / t / 1e9, "unit": "Gop/s", "cores": cores, "kind": "oracle",
           "sample": f"{E} random output entries of the n={n} product (exact max and "
                     f"the {len(P_LOG2)} p-sums each, FP64); {t:.1f} s"}
    # the same oracle on one thread, on a quarter of the time budget
    oracle.set_num_threads(1)
    try:
        t1 = run(16)
        E1 = max(16, int(16 * 0.25 * seconds / max(t1, 1e-3)))
        t1 = run(E1)
    finally:
        oracle.set_num_threads(cores)
    out["single_thread"] = {"value": E1 * Kc / t1 / 1e9, "unit": "Gop/s", "cores": 1,
                            "sample": f"{E1} random output entries, same work per entry; "
                                      f"{t1:.1f} s"}
    return out


def gpu_local_cpus(torch):
    """CPUs on the current GPU's NUMA node (from sysfs), or None."""
    try:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        bus = f"{props.pci_domain_id:04x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
        text = open(f"/sys/bus/pci/devices/{bus}/local_cpulist").read().strip()
    except (OSError, AttributeError):
        return None
    cpus = set()
    for part in text.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus or None


def pinned_on_gpu_node(torch, arrays):
    """Pinned host copies of `arrays`, allocated and first touched while this
    process runs only on the GPU's NUMA-local CPUs (so their pages live on the
    GPU's node); the previous CPU affinity is restored afterwards.  Returns
    (tensors, note for the JSON line)."""
    local = gpu_local_cpus(torch)
    prev = None
    note = "GPU NUMA node unknown; affinity unchanged"
    try:
        if local:
            prev = os.sched_getaffinity(0)
            both = prev & local
            if both and both != prev:
                os.sched_setaffinity(0, both)
                note = f"allocated on the GPU-local CPUs ({len(both)} of {len(prev)})"
            else:
                note = "already on the GPU-local CPUs" if both else "no GPU-local CPU allowed"
                prev = None
    except (OSError, AttributeError):
        note, prev = "affinity unavailable", None
    try:
        out = [torch.from_numpy(a).pin_memory() if a is not None else None for a in arrays]
    finally:
        if prev is not None:
            os.sched_setaffinity(0, prev)
    return out, note


def link_probe(torch, host_in, host_out, dev_in, dev_out):
    """Host link rates of the pinned buffers: one host->device copy alone, one
    device->host copy alone, and both at once on two streams (GB/s, best of 3),
    with the GPU's NUMA node and local CPUs and this process's CPU affinity."""
    def timed(pairs):
        best = None
        streams = [torch.cuda.Stream() for _ in pairs]
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for st, (dst, src) in zip(streams, pairs):
                with torch.cuda.stream(st):
                    dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        return best
    nb_in = host_in.numel() * host_in.element_size()
    nb_out = dev_out.numel() * dev_out.element_size()
    t_in = timed([(dev_in, host_in)])
    t_out = timed([(host_out, dev_out)])
    t_both = timed([(dev_in, host_in), (host_out, dev_out)])
    out = {"h2d_alone_gbs": nb_in / t_in / 1e9, "d2h_alone_gbs": nb_out / t_out / 1e9,
           "h2d_d2h_concurrent_gbs": (nb_in + nb_out) / t_both / 1e9}
    try:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        bus = f"{props.pci_domain_id:04x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
        base = f"/sys/bus/pci/devices/{bus}"
        out["gpu_numa_node"] = open(base + "/numa_node").read().strip()
        out["gpu_local_cpus"] = open(base + "/local_cpulist").read().strip()
    except (OSError, AttributeError):
        pass
    try:
        cpus = sorted(os.sched_getaffinity(0))
        out["process_cpus"] = f"{cpus[0]}-{cpus[-1]} ({len(cpus)})" if cpus else ""
    except (OSError, AttributeError):
        pass
    return out


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Max of a per-rank number over all ranks (the slowest rank sets the time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, ops_per_step: float, steps: int, ms_max: float) -> float:
    """Whole-job throughput in G ops/s: every rank computes its own product
    (weak scaling), over the slowest rank's time."""
    return world * ops_per_step * steps / (ms_max / 1e3) / 1e9


# ----------------------------------------------------------------- ours ---
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1511_05690_gb300 as pn

    n = args.n
    Kc = args.k if args.k > 0 else n  # contraction length
    A_h, B_h = workloads.wide_range_pair(n, n, Kc)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    corr = dict(estimator=args.estimator, correction=args.correction)
    if args.correction == 2:
        # sample entries of the affine model, drawn apart from the error samples
        gfit = workloads.rng(None, 150)
        fit_ii, fit_jj = gfit.integers(0, n, args.n_fit), gfit.integers(0, n, args.n_fit)
        corr.update(fit_i=torch.from_numpy(fit_ii.astype(np.int32)).cuda(),
                    fit_j=torch.from_numpy(fit_jj.astype(np.int32)).cuda())

    def step(ev0=None, ev1=None):
        return pn.maxprod_pnorm(A, B, p_log2=P_LOG2, compute=args.compute, tile_n=args.tile_n,
                                tile_m=args.tile_m, out=C, want_ssel=False, check=False,
                                ev_begin=ev0, ev_end=ev1, **corr)

    for _ in range(max(args.warmup, 0)):
        step()
    pn.check_device_status(A.device, "warmup")
    K = args.steps
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)  # let the sampler come up before the timed region
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_begin()
    t_begin.record(stream)
    for s in range(K):
        _, psel, _ = step(*gev[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    pn.check_device_status(A.device, "timed steps")
    ms = t_begin.elapsed_time(t_end)
    gemm_ms = [a.elapsed_time(b) for a, b in gev]
    ms_max = max_over_ranks(ms, world, device="cuda")
    ops = float(n) * n * Kc
    value = job_value(world, ops, K, ms_max)

    # error of the estimate at sampled entries: vs exact and vs the FP64 p-norm
    err = None
    if rank == 0 and args.err_samples > 0:
        import oracle
        ii, jj = workloads.wide_range_entries(n, args.err_samples)
        rows = np.unique(ii)
        A64 = A_h[rows].astype(np.float64)
        B64 = B_h.astype(np.float64)
        r = np.ones(n)
        r[rows] = oracle.row_scales(A64)
        c = oracle.col_scales(B64)
        loc = np.searchsorted(rows, ii)
        exact, S = oracle.entries(A64, B64, loc, jj, P_LOG2, r[rows], c)
        del B64
        ti, tj = torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()
        Cs = C[ti, tj].double().cpu().numpy()
        ps = (psel[ti, tj].cpu().numpy() & 0x7F).astype(np.int64)
        if args.estimator == 0 and args.correction == 0:
            S_at = S[np.arange(len(ii)), ps]
            pn_ref = r[ii] * c[jj] * np.power(S_at, 1.0 / 2.0 ** ps)
        else:
            # the oracle's estimator (and correction) on its own p-sums of the
            # sampled entries
            tau = oracle.default_tau(Kc, {"f32": 0, "tf32": 1, "bf16": 2, "f16": 3,
                                         "e4m3": 4}[args.compute])
            rc = r[ii] * c[jj]
            S34 = None
            if args.estimator == 2:
                S34 = oracle.entries_real(A64, B_h.astype(np.float64), loc, jj,
                                          [0.75 * 2.0 ** lp for lp in P_LOG2], r[rows], c)
                S34 = S34.T[:, None, :]
            pn_ref, ps_o, _ = oracle.estimate(S.T[:, None, :], P_LOG2, np.ones(1), rc, tau,
                                              estimator=args.estimator, S34=S34)
            coef = None
            if args.correction == 2:
                frows = np.unique(fit_ii)
                rf = np.ones(n)
                rf[frows] = oracle.row_scales(A_h[frows].astype(np.float64))
                coef = oracle.fit_coefficients(A_h[frows].astype(np.float64),
                                               B_h.astype(np.float64),
                                               np.searchsorted(frows, fit_ii), fit_jj, P_LOG2,
                                               rf[frows], c, tau, args.estimator)
            if args.correction:
                oracle.apply_correction(pn_ref, ps_o, P_LOG2, Kc, np.ones(1), rc,
                                        args.correction, coef)
            pn_ref = pn_ref[0]
        samples = dict(ii=ii, jj=jj, ti=ti, tj=tj, exact=exact, S=S, rc=r[ii] * c[jj])
        e_exact = np.abs(Cs - exact) / exact
        e_orc = np.abs(Cs - pn_ref) / pn_ref
        err = {"samples": int(len(ii)), "max_rel_vs_exact": float(e_exact.max()),
               "median_rel_vs_exact": float(np.median(e_exact)),
               "max_rel_vs_fp64_pnorm": float(e_orc.max()),
               "median_rel_vs_fp64_pnorm": float(np.median(e_orc)),
               "p_sel_histogram": {str(2 ** int(k)): int(v) for k, v in
                                   zip(*np.unique(ps, return_counts=True))}}

    # the same product with E4M3 operands (the n = 16384 configuration names
    # both formats): its own short timed region, the top GEMM's events, and
    # the error at the same sampled entries
    e4m3_info = None
    if (rank == 0 and args.compute == "bf16" and args.estimator == 0 and args.correction == 0
            and not args.no_e4m3):
        C8 = torch.empty_like(C)

        def step8(ev0=None, ev1=None):
            return pn.maxprod_pnorm(A, B, p_log2=P_LOG2, compute="e4m3", tile_n=args.tile_n,
                                    tile_m=args.tile_m, out=C8, want_ssel=False, check=False,
                                    ev_begin=ev0, ev_end=ev1)
        for _ in range(max(args.warmup, 3)):
            step8()
        K8 = max(1, min(K, 20))
        ev8 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K8)]
        a8, b8 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a8.record(stream)
        for s8 in range(K8):
            _, ps8, _ = step8(*ev8[s8])
        b8.record(stream)
        torch.cuda.synchronize()
        pn.check_device_status(A.device, "e4m3 steps")
        ms8 = a8.elapsed_time(b8) / K8
        g8 = statistics.mean(x.elapsed_time(y) for x, y in ev8)
        tp8 = tensor_peaks()
        pk8, pk8_how = gemm_peak_tflops("e4m3", measured_peaks()[0], True, tp8)
        ach8 = 2.0 * ops / (g8 / 1e3) / 1e12
        e4m3_info = {"ms_per_step": ms8, "value": ops / (ms8 / 1e3) / 1e9, "unit": "Gop/s",
                     "steps": K8,
                     "roofline": {"bound": "tensor", "achieved": ach8, "peak": pk8,
                                  "unit": "TFLOP/s", "frac": ach8 / pk8, "launch_ms": g8,
                                  "peak_source": pk8_how}}
        if err is not None:
            sm = samples
            C8s = C8[sm["ti"], sm["tj"]].double().cpu().numpy()
            q8 = (ps8[sm["ti"], sm["tj"]].cpu().numpy() & 0x7F).astype(np.int64)
            ref8 = sm["rc"] * np.power(sm["S"][np.arange(len(q8)), q8], 1.0 / 2.0 ** q8)
            x8 = np.abs(C8s - sm["exact"]) / sm["exact"]
            o8 = np.abs(C8s - ref8) / ref8
            e4m3_info["err"] = {
                "samples": int(len(q8)), "max_rel_vs_exact": float(x8.max()),
                "median_rel_vs_exact": float(np.median(x8)),
                "max_rel_vs_fp64_pnorm": float(o8.max()),
                "median_rel_vs_fp64_pnorm": float(np.median(o8)),
                "p_sel_histogram": {str(2 ** int(k)): int(v) for k, v in
                                    zip(*np.unique(q8, return_counts=True))}}
        del C8

    # exact CUDA-core product of the same inputs, for the comparison in the metric
    exact_info = None
    if rank == 0 and not args.no_exact:
        E = torch.empty_like(C)
        pn.maxprod_exact(A, B, out=E)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pn.maxprod_exact(A, B, out=E)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        exact_info = {"ms": ems, "gops": ops / (ems / 1e3) / 1e9,
                      "speedup_of_pnorm": (ops / (ms_max / K / 1e3) / 1e9) / (ops / (ems / 1e3) / 1e9)}
        del E

    # end to end through the public API from pinned host buffers: every step
    # copies its inputs in, runs the product and copies C out; consecutive
    # independent steps overlap on three streams (paper_1511_05690_gb300.pipeline)
    from paper_1511_05690_gb300.pipeline import HostPipeline
    (Ah, Bh, Ch), numa_note = pinned_on_gpu_node(
        torch, [A_h, B_h, np.zeros((n, n), dtype=np.float32)])
    del C
    torch.cuda.empty_cache()
    pipe = HostPipeline(n, n, Kc, compute=args.compute, tile_n=args.tile_n, tile_m=args.tile_m,
                        p_log2=P_LOG2,
                        **corr)
    KE = max(1, args.e2e_steps)
    pipe.run([(Ah, Bh, Ch)] * 2)  # warm-up
    # three timed runs of KE steps each, the median reported: the host link is
    # shared with the other GPU of the same CPU, whose transfers can halve it
    # for a while (every run's time is in the line)
    runs = []
    for _ in range(3):
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        stages = []
        pipe.run([(Ah, Bh, Ch)] * KE, ev_start=x0, ev_end=x1, stages=stages)
        runs.append((max_over_ranks(x0.elapsed_time(x1) / KE, world, device="cuda"), stages))
    e2e_runs_ms = [r[0] for r in runs]
    e2e_ms, stages = sorted(runs, key=lambda r: r[0])[1]
    e2e_value = job_value(world, ops, 1, e2e_ms)
    pn.check_device_status(A.device, "e2e")
    from paper_1511_05690_gb300.pipeline import stage_summary
    e2e_stages = stage_summary(stages, pipe.h2d_bytes, pipe.d2h_bytes)
    e2e_link = link_probe(torch, Ah, Ch, pipe.A[0], pipe.C[0])
    e2e_link["host_buffers"] = numa_note
    del pipe

    peaks, peak_src = measured_peaks()
    gemm_avg = statistics.mean(gemm_ms)
    achieved = 2.0 * ops / (gemm_avg / 1e3) / 1e12
    # the GEMM is timed inside a short region (K steps, about 0.1 s): the burst
    # figure; the sustained one is reported beside it
    tp = tensor_peaks()
    peak, peak_how = gemm_peak_tflops(args.compute, peaks, burst=True, measured=tp)
    peak_s, _ = gemm_peak_tflops(args.compute, peaks, burst=False, measured=tp)
    line = {
        "metric": "Effective semiring Gop/s (n^3/s): p-norm TC vs exact GPU kernel at stated err",
        "value": value, "unit": "Gop/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.compute, "data": "synthetic",
        "config": {"workload": workload_name(n, args.compute, args.estimator, args.correction,
                                             args.n_fit), "n": n, "k": Kc,
                   "p_log2": P_LOG2,
                   "outputs": "C and p_sel", "l2": "inputs larger than L2 (1 GiB each), no flush",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "Gop/s", "h2d_bytes_per_step": 2 * 4 * n * Kc,
                "d2h_bytes_per_step": 4 * n * n, "steps": KE, "ms_per_step": e2e_ms,
                "runs_ms_per_step": e2e_runs_ms,
                "how": "pinned host A, B in / C out every step; steps overlap copy-in, "
                       "compute and copy-out on three streams (one per copy direction); "
                       "median of three timed runs of `steps` steps",
                "stages": e2e_stages, "link": e2e_link},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic_from_profile(args.compute),
                     "kernel": "k_gemm_level (largest p), 2*n^3 FLOP per launch",
                     "launch_ms": gemm_avg,
                     "peak_source": f"{peak_how} ({peak_src}; burst: the launch is timed "
                                    f"inside a short region)",
                     "peak_sustained": peak_s, "frac_of_sustained": achieved / peak_s},
        "clocks": clk,
        "gpu_launches": launches_per_step(args) * K,
        "err": err,
        "exact_kernel": exact_info,
    }
    if e4m3_info is not None:
        if exact_info is not None:
            e4m3_info["speedup_over_exact_kernel"] = exact_info["ms"] / e4m3_info["ms_per_step"]
        line["e4m3"] = e4m3_info
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        line["cpu_baseline"] = cpu_baseline(A_h, B_h, n, args.cpu_seconds, oracle)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------ reference ---
def run_reference(args):
    """The FP64 oracle as the reference arm, on a bounded sample per step."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    n = args.n
    g = workloads.rng(None, 98)
    rows = np.unique(g.integers(0, n, 16))
    # only the sampled rows of A and all of B are needed: draw the full pair once
    A_h, B_h = workloads.wide_range_pair(n, n, n)
    A64 = A_h[rows].astype(np.float64)
    B64 = B_h.astype(np.float64)
    r = oracle.row_scales(A64)
    c = oracle.col_scales(B64)
    per_step_s = 4.0

    def run(E):
        ii = g.integers(0, len(rows), E)
        jj = g.integers(0, n, E)
        t0 = time.perf_counter()
        oracle.entries(A64, B64, ii, jj, P_LOG2, r, c)
        return time.perf_counter() - t0

    t0 = run(32)
    E = max(32, int(32 * per_step_s / max(t0, 1e-3)))
    for _ in range(max(args.warmup, 0)):
        run(max(8, E // 8))
    t_total = 0.0
    for _ in range(args.steps):
        t_total += run(E)
    value = args.steps * E * n / t_total / 1e9
    sample = (f"{E} random output entries per step of the n={n} product (exact max and "
              f"{len(P_LOG2)} p-sums each, FP64)")
    line = {
        "metric": "Effective semiring Gop/s (n^3/s): p-norm TC vs exact GPU kernel at stated err",
        "impl": "reference", "value": value, "unit": "Gop/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(n, args.compute), "n": n, "p_log2": P_LOG2},
        "cpu_baseline": {"value": value, "unit": "Gop/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Gop/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ other workloads ---
def _timed(torch, fn, K, warmup, stream):
    for _ in range(max(warmup, 1)):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(K):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / K


def measure_tensor_peaks(torch, stream, n=8192, sustain_s=4.0):
    """Dense tensor peaks of the library GEMMs, measured like the BF16 figure
    of the measured-peaks file: 2 n^3 FLOP per product, n = 8192, best of 10
    (burst) and back to back for a few seconds (sustained), CUDA events,
    clocks sampled.  BF16: torch.matmul; TF32: torch.matmul on FP32 with TF32
    allowed; E4M3: torch._scaled_mm (FP8 E4M3 operands, FP32 scales, BF16
    out)."""
    torch.manual_seed(0)
    out = {"workload": "peaks", "n": n}

    def run(name, fn):
        try:
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            best = None
            for _ in range(10):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                best = ms if best is None else min(best, ms)
            clocks = ClockSampler(torch.cuda.current_device())
            clocks.start()
            time.sleep(0.3)
            reps = max(1, int(sustain_s * 1e3 / best))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            clocks.mark_begin()
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            clocks.mark_end()
            sus = a.elapsed_time(b) / reps
            flop = 2.0 * n ** 3
            out[f"{name}_tflops"] = flop / (best / 1e3) / 1e12
            out[f"{name}_tflops_sustained"] = flop / (sus / 1e3) / 1e12
            out[f"{name}_clocks"] = clocks.stop()
        except Exception as e:  # a format the library GEMM does not offer here
            out[f"{name}_error"] = f"{type(e).__name__}: {e}"[:300]

    a16 = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    b16 = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    run("bf16", lambda: torch.matmul(a16, b16))
    del a16, b16
    a32 = torch.randn(n, n, device="cuda")
    b32 = torch.randn(n, n, device="cuda")
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    run("tf32", lambda: torch.matmul(a32, b32))
    torch.backends.cuda.matmul.allow_tf32 = prev
    del a32, b32
    a8 = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
    b8 = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()  # column-major
    one = torch.ones((), device="cuda", dtype=torch.float32)
    run("e4m3", lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one,
                                         out_dtype=torch.bfloat16))
    return out


def run_other(args):
    """APSP n=4096 (12 squarings, 3xTF32), forward+backward n=2048 (3xTF32),
    or 4096 grouped products (BF16, CUDA-graph replay).  One JSON line."""
    import torch
    import paper_1511_05690_gb300 as pn
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    K = args.steps
    line = {"metric": "Effective semiring Gop/s (n^3/s): p-norm TC vs exact GPU kernel at stated err",
            "unit": "Gop/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic"}
    if args.workload == "peaks":
        line = measure_tensor_peaks(torch, stream)
        print(json.dumps(line), flush=True)
        return
    if args.workload == "topk":
        # approximate top-k of x_i y_j (Alg. 9 with the NormQueue) for a batch
        # of pairs, with the index recovery (two calls: y and y reversed)
        batch, n, k = 256, 4096, 1024
        g = workloads.rng(None, 7)
        xh = g.random((batch, n)).astype(np.float32)
        yh = g.random((batch, n)).astype(np.float32)
        x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        P13 = list(range(13))
        res = {}

        def fwd():
            res["out"] = pn.topk_xy(x, y, k, p_log2=P13, check=False)
        ms = _timed(torch, fwd, K, args.warmup, stream)
        pn.check_device_status(x.device, "topk_xy")
        vals, ii, jj = (t.cpu().numpy() for t in res["out"])
        errs, recov = [], []
        for b in range(4):  # exact top-k of 4 problems on the host
            ex = np.sort(np.outer(xh[b].astype(np.float64), yh[b]).ravel())[::-1][:k]
            errs.append(np.abs(np.sort(vals[b])[::-1] - ex) / ex)
            recov.append(float(np.mean(ii[b] >= 0)))
        errs = np.concatenate(errs)
        line.update(value=batch * float(n) * n / (ms / 1e3) / 1e9, ms_per_step=ms,
                    dtype="f64 (FFT) + FP64 NormQueue",
                    config={"workload": f"topk_xy batch={batch} n={n} k={k}, x, y U[0,1), "
                            "P={1..4096}, tau=1e-12, both calls and the index recovery",
                            "batch": batch, "n": n, "k": k,
                            "value_counts": "n^2 products x_i y_j per problem"},
                    err={"problems": 4, "max_rel_vs_exact_topk": float(errs.max()),
                         "median_rel_vs_exact_topk": float(np.median(errs)),
                         "indices_recovered": float(np.mean(recov))})
    elif args.workload == "maxconv-long":
        # one long max-convolution (Sec. 1): n = 2^21 per vector, 2^22 - 1
        # outputs, four-step FP64 FFT through a workspace
        n = 1 << 21
        g = workloads.rng(None, 6)
        xh = ((1.0 - g.random(n)) ** 0.25).astype(np.float32)
        yh = ((1.0 - g.random(n)) ** 0.25).astype(np.float32)
        x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        nz = 2 * n - 1
        z = torch.empty((1, nz), dtype=torch.float32, device="cuda")
        ze = torch.empty_like(z)
        res = {}

        def fwd():
            res["psel"] = pn.maxconv_pnorm(x, y, out=z, check=False)[1]
        ms = _timed(torch, fwd, K, args.warmup, stream)
        pn.check_device_status(x.device, "maxconv_pnorm_long")
        ems = _timed(torch, lambda: pn.maxconv_exact(x, y, out=ze), 1, 1, stream)
        ops = float(n) * n
        psel = res["psel"].cpu().numpy()[0]
        zz, zex = z.cpu().numpy()[0], ze.cpu().numpy()[0]
        rel = np.abs(zz - zex) / zex
        # FP64 work: per FFT level two transforms of N = 2^22 (5 N log2 N
        # flops each) plus the inter-step twiddles and the spectrum (~40 N)
        N, logN = 1 << 22, 22
        mm = np.arange(nz)
        L = np.minimum(mm, n - 1) - np.maximum(0, mm - n + 1) + 1
        lp = (psel & 0x7F).astype(np.int64)
        P = list(range(7))
        levels = 0
        for q in range(len(P) - 1, -1, -1):
            levels += 1
            W = int(L[lp < P[q]].sum())
            if W == 0 or q == 0 or W * (8 + 2 * q) <= 10 * N * logN:
                break
        flops = levels * (10.0 * N * logN + 40.0 * N)
        line.update(value=ops / (ms / 1e3) / 1e9, ms_per_step=ms, dtype="f64 (FFT)",
                    config={"workload": f"maxconv_pnorm (long) n={n} per vector ({nz} outputs), "
                            "entries exp(-Exp(4)), P={1..64}, tau=1e-12, four-step FP64 FFT",
                            "n": n},
                    exact_kernel={"ms": ems, "gops": ops / (ems / 1e3) / 1e9,
                                  "speedup_of_pnorm": ems / ms},
                    err={"outputs": int(rel.size), "max_rel_vs_exact": float(rel.max()),
                         "median_rel_vs_exact": float(np.median(rel)),
                         "p_sel_histogram": {str(2 ** int(k)): int(v) for k, v in
                                             zip(*np.unique(lp, return_counts=True))}},
                    roofline={"bound": "fp64", "achieved": flops / (ms / 1e3) / 1e12,
                              "peak": 1.25, "unit": "TFLOP/s",
                              "frac": flops / (ms / 1e3) / 1e12 / 1.25, "traffic": None,
                              "fft_levels": levels,
                              "peak_source": "nominal FP64 rate of the profiling recipe"})
    elif args.workload == "maxconv":
        # batch of max-convolutions (Sec. 1), H = FP64 FFT, one CTA per problem
        batch, n = args.count if args.count != 4096 else 1024, 4096
        g = workloads.rng(None, 5)
        xh = ((1.0 - g.random((batch, n))) ** 0.25).astype(np.float32)
        yh = ((1.0 - g.random((batch, n))) ** 0.25).astype(np.float32)
        x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        nz = 2 * n - 1
        z = torch.empty((batch, nz), dtype=torch.float32, device="cuda")
        ze = torch.empty_like(z)
        res = {}

        def fwd():
            res["psel"] = pn.maxconv_pnorm(x, y, out=z, check=False)[1]
        ms = _timed(torch, fwd, K, args.warmup, stream)
        pn.check_device_status(x.device, "maxconv_pnorm")
        ems = _timed(torch, lambda: pn.maxconv_exact(x, y, out=ze), max(1, K // 5), 1, stream)
        ops = float(batch) * n * n  # (x,max) terms of the exact max-convolution
        psel = res["psel"].cpu().numpy()
        zz, zex = z.cpu().numpy(), ze.cpu().numpy()
        rel = np.abs(zz - zex) / zex
        # FP64 work actually done: the FFT levels each problem ran, replaying
        # the kernel's rule from
        # p_sel -- after level q the open indices (p* below that level) either
        # end the loop (none), go to the direct sums (few terms) or need the
        # next FFT level
        P = list(range(7))
        N, logN = 8192, 13
        mm = np.arange(nz)
        L = np.minimum(mm, n - 1) - np.maximum(0, mm - n + 1) + 1
        levels = np.zeros(batch, dtype=np.int64)
        for b in range(batch):
            lp = (psel[b] & 0x7F).astype(np.int64)
            for q in range(len(P) - 1, -1, -1):
                levels[b] += 1
                W = int(L[lp < P[q]].sum())
                if W == 0 or q == 0 or W * (8 + 2 * q) <= 10 * N * logN:
                    break
        # per level: forward FFT of length N (a multiply-free radix-4 first
        # pass, 4N flops, then N/2 butterflies of 10 flops per stage), the
        # spectrum (about 28 flops per output pair), inverse of length M = N/2
        M = N // 2
        per_level = 4 * N + 5 * N * (logN - 2) + 28 * M + 4 * M + 5 * M * (logN - 3)
        flops = float(levels.sum()) * per_level
        line.update(value=ops / (ms / 1e3) / 1e9, ms_per_step=ms, dtype="f64 (FFT)",
                    config={"workload": f"maxconv_pnorm batch={batch} n={n} (2n-1 outputs), "
                            "entries exp(-Exp(4)), P={1..64}, tau=1e-12, FP64 FFT per problem "
                            "in shared memory", "batch": batch, "n": n},
                    exact_kernel={"ms": ems, "gops": ops / (ems / 1e3) / 1e9,
                                  "speedup_of_pnorm": ems / ms},
                    err={"outputs": int(rel.size), "max_rel_vs_exact": float(rel.max()),
                         "median_rel_vs_exact": float(np.median(rel)),
                         "p_sel_histogram": {str(2 ** int(k)): int(v) for k, v in
                                             zip(*np.unique(psel & 0x7F, return_counts=True))}},
                    roofline={"bound": "fp64", "achieved": flops / (ms / 1e3) / 1e12,
                              "peak": 1.25, "unit": "TFLOP/s",
                              "frac": flops / (ms / 1e3) / 1e12 / 1.25,
                              "traffic": None, "levels_run_mean": float(levels.mean()),
                              "peak_source": "nominal FP64 rate of the profiling recipe"})
    elif args.workload == "apsp":
        n, T = 4096, 12
        W = torch.from_numpy(workloads.apsp_weights(n, density=0.1, index=1)).cuda()
        D = torch.empty_like(W)
        shape = dict(tile_n=args.tile_n, tile_m=args.tile_m)
        pn.apsp_pnorm(W, out=D, **shape)
        graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s):
                pn.apsp_pnorm(W, out=D, check=False, stream=s, **shape)
        stream.wait_stream(s)
        ms = _timed(torch, graph.replay, K, args.warmup, stream)
        E = torch.empty_like(W)
        ems = _timed(torch, lambda: [pn.maxprod_exact(W, W, semiring=1, out=E) for _ in range(1)],
                     1, 1, stream)
        # the exact closure by as many exact (+,min) squarings: the estimate's
        # error at this configuration (it never exceeds the exact distance)
        X = W.clone()
        for _ in range(T):
            X = pn.maxprod_exact(X, X, semiring=1)
        fin = torch.isfinite(X)
        dd, xx = D[fin].double(), X[fin].double()
        apsp_err = {"max_abs_vs_exact": float((dd - xx).abs().max()),
                    "median_abs_vs_exact": float((dd - xx).abs().median()),
                    "exact_median_distance": float(xx.median()),
                    "exact_max_distance": float(xx.max()),
                    "zero_estimate_fraction": float((dd == 0).double().mean()),
                    "never_above_exact": bool((dd <= xx + 1e-5 + 1e-5 * xx).all())}
        del X, E
        line.update(value=T * n ** 3 / (ms / 1e3) / 1e9, ms_per_step=ms, dtype="f32 (3xTF32)",
                    config={"workload": "apsp_pnorm n=4096 density 0.1 U[0,1] weights, 12 "
                            "squarings, P={1..64}, diag reset + clamp, CUDA graph", "n": n},
                    exact_kernel={"one_minplus_squaring_ms": ems,
                                  "gops": n ** 3 / (ems / 1e3) / 1e9},
                    err=apsp_err,
                    gpu_launches=K * (1 + T * 22 + 1))
    elif args.workload == "backward":
        n = 2048
        A_h, B_h = workloads.uniform_pair(n, n, n, index=2)
        A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
        out = {}
        for name, pl in (("p16", [4]), ("p1_64", list(range(7)))):
            C, psel, ssel = pn.maxprod_pnorm(A, B, p_log2=pl, compute="f32")
            G = 1.0 / C
            fwd = _timed(torch, lambda: pn.maxprod_pnorm(A, B, p_log2=pl, compute="f32",
                                                         check=False), K, args.warmup, stream)
            bwd = _timed(torch, lambda: pn.maxprod_pnorm_backward(A, B, C, ssel, psel, G,
                                                                  p_log2=pl, compute="f32",
                                                                  check=False),
                         K, args.warmup, stream)
            import ctypes
            o = pn.make_opts(pl, "f32")
            ws_b = pn.lib().pn_backward_workspace_size(n, n, n, ctypes.byref(o))
            out[name] = {"fwd_ms": fwd, "bwd_ms": bwd,
                         "fwd_bwd_gops": n ** 3 / ((fwd + bwd) / 1e3) / 1e9,
                         "recompute_workspace_bytes": int(ws_b),
                         "saved_powered_tiles_bytes": 2 * n * n * 4 * len(pl)}
        line.update(value=out["p1_64"]["fwd_bwd_gops"],
                    ms_per_step=out["p1_64"]["fwd_ms"] + out["p1_64"]["bwd_ms"],
                    dtype="f32 (3xTF32)",
                    config={"workload": "maxprod_pnorm forward + backward n=2048 U(0,1], "
                            "loss sum log C, P={16} and P={1..64}", "n": n, "detail": out})
    else:
        sizes = workloads.grouped_sizes(args.count)
        g = torch.Generator(device="cuda")
        g.manual_seed(workloads.SEED_BASE + 3)
        As = [1 - torch.rand((int(m), int(m)), generator=g, device="cuda") for m in sizes]
        Bs = [1 - torch.rand((int(m), int(m)), generator=g, device="cuda") for m in sizes]
        plan = pn.GroupedProduct(As, Bs, compute="bf16", tile_n=args.tile_n)
        plan.run(check=True)
        chosen = plan.autotune() if args.tile_n == 0 else args.tile_n
        graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s):
                plan.run(stream=s)
        stream.wait_stream(s)
        ms = _timed(torch, graph.replay, K, args.warmup, stream)
        ops = float(np.sum(sizes.astype(np.float64) ** 3))
        line.update(value=ops / (ms / 1e3) / 1e9, ms_per_step=ms, dtype="bf16",
                    config={"workload": f"{args.count} square products, n = round(16 * 64^U), "
                            "BF16, P={1..64}, an image-strip launch then one persistent launch "
                            "over every p level, CUDA graph replay",
                            "sum_n3": ops, "tile_n": chosen})
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "pnorm":
        run_other(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
