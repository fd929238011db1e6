"""Benchmark: field-sample RK4IP steps per second on one GB300 (or N replicas).

A step is one RK4IP step (Eq. 4a-4f: four linear-operator applications and four
Kerr evaluations) over all fields of the workload.  The default workload is the
45-mode x 2-polarisation link (90 fields, N_t = 2^17 complex64, 9 WDM 16-QAM
channels per mode, h = 25 m); --workload c3 selects the 120-mode link.

Prints one JSON line (rank 0).  `value` is the device-timed throughput with the
fields resident in HBM; `e2e` is the same metric through mmf_propagate_host with
pinned host buffers, the host<->device copies inside the timed region.
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import make_workload  # noqa: E402

METRIC = "field-sample RK4IP steps/s"
UNIT = "field-sample steps/s"
L2_BYTES = 126.5e6
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
KERR_NAMES = {"fp32": 0, "bf16x3": 1, "bf16": 2, "tf32x3": 3}
CSRC = os.path.join(ROOT, "paper_1901_01895_gb300", "csrc")
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# (summaries in profiles/), valid only while the kernel source hashes to the same value.
TRAFFIC = {
    ("kerr_tcr", "c2", "bf16x3"): {"bytes": 147.79776e6, "src": "kerr_tcr.cu", "sha": "36b4f2bb709720a6"},
    ("kerr_tcr", "c2", "tf32x3"): {"bytes": 150.077696e6, "src": "kerr_tcr.cu", "sha": "36b4f2bb709720a6"},
    ("kerr_tcr", "c3", "bf16x3"): {"bytes": 1613.955584e6, "src": "kerr_tcr.cu", "sha": "36b4f2bb709720a6"},
    ("lin", "c2"): {"bytes": 645.184832e6, "src": "lin.cu", "sha": "487b20fb67a6cbc4"},
    ("lin", "c3k"): {"bytes": 1978.45472e6, "src": "lin.cu", "sha": "487b20fb67a6cbc4"},
    ("kerr_kappa_tc", "c3k", "bf16x3"): {"bytes": 931.402816e6, "src": "kerr_kappa_tc.cu", "sha": "a01c44371d52ed6a"},
    ("kerr_kappa", "c3k", "fp32"): {"bytes": 461.734144e6, "src": "kerr_kappa.cu", "sha": "7963614e83ad800b"},
    ("kerr_simt", "c2", "fp32"): {"bytes": 253.03936e6, "src": "kerr_pairs.cu", "sha": "1e2fbe75c8615854"},
}


def measured_traffic(key):
    """Profiled DRAM bytes per launch, or None when the kernel changed since the capture."""
    import hashlib
    t = TRAFFIC.get(key)
    if not t:
        return None
    sha = hashlib.sha256(open(os.path.join(CSRC, t["src"]), "rb").read()).hexdigest()[:16]
    return t["bytes"] if sha == t["sha"] else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []          # (host time of arrival, csv line)
        self.window = None       # (start, end) of the timed region, host clock

    def mark(self, start: float, end: float):
        """Keep only the samples that arrive inside [start, end] (plus one polling interval)."""
        self.window = (start, end + 0.06)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if self.window and not (self.window[0] <= ts <= self.window[1]):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, device) -> float:
    """The job's time of a timed region: the slowest rank's, by an all-reduce (MAX) followed
    by a barrier. NCCL with a CUDA device on the GPU machine; gloo with the CPU in the tests."""
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.barrier()
    return float(t.item())


def sum_over_ranks(v: float, device) -> float:
    """Sum of a per-rank rate over the ranks (independent replicas of the serving mix)."""
    import torch
    t = torch.tensor([v], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the job's time (weak scaling,
    replicas: each rank runs the same workload)."""
    return units_per_rank * ws / (ms / 1e3)


def kerr_flops_per_sample(M: int, n_pol: int, parity) -> float:
    """Algorithmic flops of one Kerr evaluation per time sample, counted on the factored
    pair contraction over nonzero parity blocks: 2 * rows * sum_c n_c^2 (rows = 3 for two
    polarisations, 2 for one) plus the epilogue contraction."""
    cls = {}
    for i in range(M):
        for j in range(i, M):
            c = int(parity[i]) ^ int(parity[j])
            cls[c] = cls.get(c, 0) + 1
    rows = 3 if n_pol == 2 else 2
    gemm = 2.0 * rows * sum(n * n for n in cls.values())
    return gemm


def kernel_times(f, x, stream, hstep, reps):
    """Mean duration (ms, CUDA events on the launching stream, back-to-back launches after two
    untimed ones) of each kernel variant one RK4IP step launches (Eq. 4a-4f):
      Kerr    one input twice (T = h N(A); k4 = h N(v)), two inputs twice (k2, k3: the stage
              input A_I + k/2 formed on the load);
      linear  one input twice (A_I, k1), two inputs once (A_I + k3), four inputs plus the added
              k4/6 once (Eq. 4f).
    The per-launch figures are the means over the step's eight launches."""
    import torch
    bufs = [torch.empty_like(x) for _ in range(5)]
    for i, b in enumerate(bufs):
        b.copy_(x)
        b.mul_(0.05 * (i + 1))
    out = torch.empty_like(x)
    p = [b.data_ptr() for b in bufs]

    def timed(fn):
        for _ in range(2):
            fn()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / reps

    xp, op = x.data_ptr(), out.data_ptr()
    k1 = timed(lambda: f.kerr_stage(xp, 0, 0.0, op, hstep))
    k2 = timed(lambda: f.kerr_stage(xp, p[0], 0.5, op, hstep))
    l1 = timed(lambda: f.linear_stage([xp], [1.0], 0, 0.0, op, hstep / 2))
    l2 = timed(lambda: f.linear_stage([xp, p[0]], [1.0, 1.0], 0, 0.0, op, hstep / 2))
    l4 = timed(lambda: f.linear_stage([xp, p[0], p[1], p[2]], [1.0, 1 / 6, 1 / 3, 1 / 3], p[3], 1 / 6, op, hstep / 2))
    del bufs, out
    return {"kerr_ms": (2 * k1 + 2 * k2) / 4, "lin_ms": (2 * l1 + l2 + l4) / 4,
            "kerr_1in_ms": k1, "kerr_2in_ms": k2, "lin_1in_ms": l1, "lin_2in_ms": l2, "lin_4in_add_ms": l4}


def roofline(wl, kerr_path, kerr, kt, peaks, workload):
    """Roofline of the step's dominant kernel, per launch averaged over the step's variants.

    Kerr: algorithmic flops = the factored pair contraction over nonzero parity blocks
    (kerr_flops_per_sample) x N_t; the kernels are timed in isolation (back-to-back
    launches of one kernel), so the peak is the BURST BF16 tensor rate, a third of it for
    BF16x3 (three BF16 products per term).  FP32 CUDA-core paths: the FP32 FMA rate.
    Linear step: algorithmic bytes = 8 B per field-sample for each input row, each added
    row and the output row (16 B for a single input); the propagator table is this design's
    constant, not the method's data, and shows up only in the measured DRAM traffic."""
    P, N = wl.P, wl.N_t
    kappa = kerr_path.startswith("kappa")
    kflops = (2.0 * P * P if kappa else kerr_flops_per_sample(wl.n_modes, wl.n_pol, wl.parity)) * N
    # Kerr bytes per field-sample: one input row and the output twice, two inputs and the output twice
    kerr_bytes = P * N * (16.0 + 16.0 + 24.0 + 24.0) / 4
    kerr_unit, kerr_scale = "TFLOP/s", 1e12
    if kerr_path == "kappa-tcgen05":
        # the kappa GEMM on the tensor cores takes a few % of the BF16x3 peak: the launch is bound by
        # its field traffic (the rows in, the Kerr term out)
        kerr_peak, kerr_bound, peak_kind = peaks["hbm_gbs"], "hbm", "hbm copy"
        kerr_unit, kerr_scale = "GB/s", 1e9
        kerr_key = ("kerr_kappa_tc", workload, kerr)
    elif kerr_path.startswith("pairs-tcgen05"):
        if kerr == "tf32x3":
            # TF32 peak = the measured BF16 burst peak x the nominal dense ratio 1.1 / 2.25 (PFLOP/s)
            kerr_peak = peaks["bf16_tflops"] * (1.1 / 2.25) / 3.0
            peak_kind = "tf32 (bf16 burst x 1.1/2.25) / 3 (tf32x3)"
        else:
            kerr_peak = peaks["bf16_tflops"] * (1.0 / 3.0 if kerr == "bf16x3" else 1.0)
            peak_kind = "bf16 burst" + (" / 3 (bf16x3)" if kerr == "bf16x3" else "")
        kerr_bound = "tensor"
        kerr_key = ("kerr_tcr", workload, kerr)
    else:
        # FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x max SM clock
        kerr_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        kerr_bound, peak_kind = "alu", "fp32 fma (152 x 128 x 2 x max SM clock)"
        kerr_key = ("kerr_kappa" if kappa else "kerr_simt", workload, kerr)
    kerr_ms, lin_ms = kt["kerr_ms"], kt["lin_ms"]
    # bytes per field-sample of the step's four linear launches: (in + out) x2, 2 in + out, 4 in + add + out
    lin_bpfs = (16.0 + 16.0 + 24.0 + 48.0) / 4
    lin_bytes = P * N * lin_bpfs
    lin_gbs = lin_bytes / (lin_ms / 1e3) / 1e9
    kerr_tf = kflops / (kerr_ms / 1e3) / 1e12
    kerr_ach = (kerr_bytes if kerr_unit == "GB/s" else kflops) / (kerr_ms / 1e3) / kerr_scale
    if 4 * kerr_ms >= 4 * lin_ms:
        roof = {"kernel": "kerr", "bound": kerr_bound, "achieved": kerr_ach, "peak": kerr_peak, "unit": kerr_unit,
                "frac": kerr_ach / kerr_peak, "traffic": measured_traffic(kerr_key), "peak_kind": peak_kind,
                "per_launch": {"flop": kflops, "ms": kerr_ms, "algorithmic_bytes": kerr_bytes}}
    else:
        roof = {"kernel": "lin", "bound": "hbm", "achieved": lin_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": lin_gbs / peaks["hbm_gbs"], "traffic": measured_traffic(("lin", workload)),
                "peak_kind": "hbm copy", "per_launch": {"bytes": lin_bytes, "ms": lin_ms}}
    roof["peak_source"] = peaks["_source"]
    roof["other"] = dict(kt)
    roof["other"].update({"lin_GBps": lin_gbs, "lin_frac_hbm": lin_gbs / peaks["hbm_gbs"],
                          "lin_bytes_per_field_sample": lin_bpfs, "kerr_TFLOPs": kerr_tf,
                          "kerr_frac": kerr_ach / kerr_peak, "kerr_bound": kerr_bound})
    return roof


def run_ours(args, ws, rank, local):
    import torch
    import paper_1901_01895_gb300 as mmf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kappa_form = args.workload == "c3k"
    wl = make_workload("c3" if kappa_form else args.workload, with_S=not kappa_form)
    P, N = wl.P, wl.N_t
    hstep = wl.L / wl.n_steps
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    if kappa_form:
        # the paper's own Kerr operator (Eq. 1: self- and cross-phase matrix) at its largest size
        from workloads import kappa_hg
        if args.kerr not in ("fp32", "bf16x3"):
            raise SystemExit("the kappa form runs in FP32 (CUDA cores) or BF16x3 (tensor cores)")
        kappa = kappa_hg(wl.modes, 10e-6, wl.n_pol)
        f = mmf.Fiber.from_kappa(kappa, wl.betas, wl.alpha, wl.gamma, N, wl.dt, KERR_NAMES[args.kerr], sp)
    else:
        flags = KERR_NAMES[args.kerr]
        f = mmf.Fiber.from_workload(wl, flags=flags, stream=sp)
    info = f.info()
    x0 = torch.from_numpy(wl.fields.astype(np.complex64)).to(dev)
    x = x0.clone()
    torch.cuda.synchronize()

    # warm-up (also captures the step graph)
    for _ in range(args.warmup):
        f.propagate(x.data_ptr(), hstep, 1)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    # timed region: K RK4IP steps; every step streams ~1.5 GB through HBM (> L2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.5)          # nvidia-smi is polling before the timed region starts
        torch.cuda.synchronize()
        w0 = time.time()
        e0.record(stream)
        f.propagate(x.data_ptr(), hstep * args.steps, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark(w0, time.time())
    ms = e0.elapsed_time(e1)
    if ws > 1:
        ms = max_over_ranks(ms, dev)
    value = job_rate(float(P) * N * args.steps, ws, ms)

    # per-kernel timing of the step's two kernels, on the stream they run on, in the variants
    # the step launches (Eq. 4a-4f)
    kt = kernel_times(f, x, stream, hstep, reps=max(3, min(50, args.steps * 4)))

    # end to end through the host-buffer entry point (pinned host memory)
    hin = torch.from_numpy(wl.fields.astype(np.complex64)).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    hin_np, hout_np = hin.numpy(), hout.numpy()
    f.propagate_host(hin_np, hout_np, hstep, 1)      # warm the staging buffer
    # every step: copy the fields in, one RK4IP step, copy the result out (chained on the host)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f.propagate_host(hin_np, hout_np, hstep, 1)
        hin_np, hout_np = hout_np, hin_np
    e2e_ms = (time.perf_counter() - t0) * 1e3
    if ws > 1:
        e2e_ms = max_over_ranks(e2e_ms, dev)
    bi = P * N * 8
    e2e_value = job_rate(float(P) * N * args.steps, ws, e2e_ms)

    peaks = load_peaks()
    kerr_path = info["kerr_path"]
    roof = roofline(wl, kerr_path, args.kerr, kt, peaks, args.workload)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, budget_s=args.cpu_budget)
    f.close()
    del x, x0
    torch.cuda.empty_cache()
    parity = parity_check(args.workload, wl_full=wl if args.workload == "c2" else None) \
        if rank == 0 and args.parity and not kappa_form else None
    if rank == 0 and args.parity and kappa_form:
        parity = parity_check_kappa()
    kbp = kerr_by_precision(wl) if rank == 0 and args.workload == "c2" and args.c3_block else None
    c3 = c3_block() if rank == 0 and args.workload == "c2" and args.c3_block else None
    serving = None
    if rank == 0 and args.serving_requests > 0:
        serving = serving_bench(args.serving_requests, args.serving_length_scale, args.serving_kerr)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.kerr == "fp32" else f"f32+{args.kerr}-kerr", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl.n_modes} HG modes x {wl.n_pol} pol = {P} fields, "
                               f"N_t={N}, h={hstep:g} m" + (", Kerr in the kappa form of Eq. 1" if kappa_form else ""),
                   "P": P, "N_t": N, "kerr": args.kerr,
                   "kerr_path": kerr_path, "l2": "inputs larger than L2 (working set %.2f GB)" %
                   (7 * P * N * 8 / 1e9), "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bi},
        # per step: four Kerr evaluations (one launch each, the stage input formed on the load)
        # and four linear steps, each three launches above N_t = 2^14 (scratch-row path), one below
        "gpu_launches": (4 + 4 * (3 if N > 1 << 14 else 1)) * args.steps,
        "clocks": clk.summary(),
        "parity": parity,
        "kerr_by_precision": kbp,
        "c3": c3,
        "serving": serving,
    }
    return out


def parity_check(workload: str, n_steps: int = 2, N_t: int = 256, wl_full=None):
    """rel-L2 of the GPU path (each Kerr precision) against the FP64 oracle:
      window       all fields and the full Kerr tensor on a reduced window (N_t samples,
                   n_steps steps);
      full_length  (when the workload's own rows are given) whole rows at the workload's
                   N_t, one step, every field, with the overlap tensor thinned to 0.2 % of its
                   symmetry orbits (SPM kept) so that the oracle's term-by-term sum finishes in
                   seconds: the same launch shapes, passes and stage combines as the timed step."""
    import dataclasses
    import torch
    import oracle
    import paper_1901_01895_gb300 as mmf
    from workloads import thinned_tensor

    def run(w, n, Lp, ref):
        res = {}
        for name, fl in KERR_NAMES.items():
            f = mmf.Fiber.from_workload(w, flags=fl, stream=torch.cuda.current_stream().cuda_stream)
            x = torch.from_numpy(w.fields.astype(np.complex64)).cuda()
            f.propagate(x.data_ptr(), Lp, n)
            y = x.cpu().numpy().astype(np.complex128)
            f.close()
            del x
            res[f"rel_l2_{name}"] = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
        return res

    wl = make_workload(workload, N_t=N_t)
    Lp = n_steps * wl.L / wl.n_steps
    ref = oracle.propagate_workload(wl, n_steps=n_steps, L=Lp)
    out = {"window": f"{workload} fields and Kerr tensor, N_t={N_t}, {n_steps} steps of h={wl.L / wl.n_steps:g} m"}
    out.update(run(wl, n_steps, Lp, ref))
    if wl_full is not None:
        w = dataclasses.replace(wl_full, S=thinned_tensor(wl_full.S, 0.002, 5))
        Lp = w.L / w.n_steps
        ref = oracle.propagate_workload(w, n_steps=1, L=Lp)
        full = {"case": f"{workload} fields at N_t={w.N_t} (all {w.P} rows), overlap tensor thinned to 0.2 % of "
                        f"its orbits, 1 step of h={Lp:g} m"}
        full.update(run(w, 1, Lp, ref))
        out["full_length"] = full
    return out


def kerr_by_precision(wl, reps: int = 10):
    """One Kerr evaluation of the workload in every precision (CUDA-event timing of back-to-back
    launches on the launching stream, single-input variant), with its algorithmic rate and the
    fraction of that precision's peak (see roofline())."""
    import torch
    import paper_1901_01895_gb300 as mmf
    peaks = load_peaks()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    x = torch.from_numpy(wl.fields.astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    hstep = wl.L / wl.n_steps
    out = {}
    for name, fl in KERR_NAMES.items():
        f = mmf.Fiber.from_workload(wl, flags=fl, stream=stream.cuda_stream)
        path = f.info()["kerr_path"]
        n = reps if name != "fp32" else max(3, reps // 4)
        for _ in range(2):
            f.kerr_stage(x.data_ptr(), 0, 0.0, y.data_ptr(), hstep)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            f.kerr_stage(x.data_ptr(), 0, 0.0, y.data_ptr(), hstep)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n
        f.close()
        r = roofline(wl, path, name, {"kerr_ms": ms, "lin_ms": 1e-9}, peaks, "")
        out[name] = {"kerr_path": path, "ms": ms, "TFLOPs": r["achieved"], "peak": r["peak"], "frac": r["frac"],
                     "peak_kind": r["peak_kind"]}
    del x, y
    return out


def c3_block(steps: int = 3, warmup: int = 1, kerr: str = "bf16x3"):
    """The 120-mode link (240 fields x 2^17, h = 50 m) next to the default line: device-timed
    RK4IP steps, the Kerr kernel against its roofline, and rel-L2 against the FP64 oracle on a
    64-sample window of the same fields and tensor (one step, BF16x3 and FP32)."""
    import torch
    import oracle
    import paper_1901_01895_gb300 as mmf
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = make_workload("c3")
    hstep = wl.L / wl.n_steps
    stream = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    f = mmf.Fiber.from_workload(wl, flags=KERR_NAMES[kerr], stream=stream.cuda_stream)
    create_s = time.perf_counter() - t0
    x = torch.from_numpy(wl.fields.astype(np.complex64)).to(dev)
    torch.cuda.synchronize()
    for _ in range(warmup):
        f.propagate(x.data_ptr(), hstep, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    f.propagate(x.data_ptr(), hstep * steps, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    status = f.device_status()
    kt = kernel_times(f, x, stream, hstep, reps=3)
    info = f.info()
    f.close()
    del x
    torch.cuda.empty_cache()
    roof = roofline(wl, info["kerr_path"], kerr, kt, load_peaks(), "c3")
    win = make_workload("c3", N_t=64)
    Lp = win.L / win.n_steps
    ref = oracle.propagate_workload(win, n_steps=1, L=Lp)
    par = {"window": "c3 fields and Kerr tensor, N_t=64, 1 step of h=50 m"}
    for name in (kerr, "fp32"):
        g = mmf.Fiber.from_workload(win, flags=KERR_NAMES[name], stream=torch.cuda.current_stream().cuda_stream)
        y = torch.from_numpy(win.fields.astype(np.complex64)).cuda()
        g.propagate(y.data_ptr(), Lp, 1)
        yh = y.cpu().numpy().astype(np.complex128)
        g.close()
        par[f"rel_l2_{name}"] = float(np.linalg.norm(yh - ref) / np.linalg.norm(ref))
    return {"workload": f"c3: {wl.n_modes} HG modes x {wl.n_pol} pol = {wl.P} fields, N_t={wl.N_t}, h={hstep:g} m",
            "kerr": kerr, "kerr_path": info["kerr_path"], "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "value": wl.P * wl.N_t * steps / (ms / 1e3), "unit": UNIT,
            "device_status": status, "create_s": create_s, "roofline": roof, "parity": par}


def parity_check_kappa(n_steps: int = 2, N_t: int = 256):
    """rel-L2 of the kappa-form GPU path (FP32 CUDA cores and BF16x3 tensor cores) against the
    FP64 oracle on a reduced window of the 120-mode link (all 240 rows, N_t samples, n_steps
    steps)."""
    import torch
    import oracle
    import paper_1901_01895_gb300 as mmf
    from workloads import kappa_hg
    wl = make_workload("c3", N_t=N_t, with_S=False)
    kappa = kappa_hg(wl.modes, 10e-6, wl.n_pol)
    Lp = n_steps * wl.L / wl.n_steps
    ref = oracle.propagate_kappa(kappa, wl.betas, wl.alpha, wl.gamma, wl.dt, wl.fields, Lp, n_steps)
    out = {"window": f"c3k rows and kappa, N_t={N_t}, {n_steps} steps of h={wl.L / wl.n_steps:g} m"}
    for name in ("fp32", "bf16x3"):
        f = mmf.Fiber.from_kappa(kappa, wl.betas, wl.alpha, wl.gamma, N_t, wl.dt, KERR_NAMES[name],
                                 torch.cuda.current_stream().cuda_stream)
        x = torch.from_numpy(wl.fields.astype(np.complex64)).cuda()
        f.propagate(x.data_ptr(), Lp, n_steps)
        y = x.cpu().numpy().astype(np.complex128)
        f.close()
        out["rel_l2_" + name] = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    return out


def run_serving(args, ws, rank, local):
    """--workload c4: the serving mix as its own JSON line."""
    import torch
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        sv = serving_bench(args.serving_requests_c4, args.serving_length_scale, args.serving_kerr)
    peaks = load_peaks()
    # replicas: every rank serves its own copy of the mix; the job's rate is their sum
    value = sum_over_ranks(sv["value"], torch.device("cuda", local)) if ws > 1 else sv["value"]
    return {
        "metric": "served field-sample RK4IP steps/s (serving mix, Poisson arrivals)", "value": value,
        "unit": UNIT, "n_gpus": ws, "steps": sv["requests"], "warmup": 1,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if sv["kerr"] == "fp32" else f"f32+{sv['kerr']}-kerr", "data": "synthetic",
        "config": {"workload": "c4: " + sv["sample"], "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 for every N_t >= 2^14 at 12+ fields x slots"},
        "serving": sv,
        "roofline": None,
        "e2e": {"value": value, "unit": UNIT, "note": "served requests are end to end: pinned host in and out"},
        "gpu_launches": sv["gpu_launches"],
        "clocks": clk.summary(),
        "peak_source": peaks["_source"],
    }


def serving_bench(n_req: int, length_scale: float, kerr: str, load: float = 0.8, seed: int | None = None):
    """Serving mix (continuous batching through mmf_server_*) against one-at-a-time solves.

    The request stream is the seeded mix of workloads.serving with every length scaled by
    length_scale (dz = 10 m).  Three measurements, all on the same requests and inputs:
      capacity   all requests submitted at once (closed loop): field-sample steps/s;
      served     Poisson arrivals at `load` x capacity (open loop): p50/p99 latency from
                 submission to the result in host memory, and throughput;
      one-at-a-time  each request alone through the public single-link calls
                 (mmf_create, mmf_propagate_host, mmf_destroy): its solve time; the
                 latency it would see under the same arrivals is that of a FIFO queue
                 in front of it (computed from the measured solve times).
    Host buffers are pinned; inputs and outputs are separate buffers.
    """
    import torch
    import paper_1901_01895_gb300 as mmf
    from workloads.serving import serving_requests, fiber_type, SignalBank

    reqs = serving_requests(n_req, seed=seed, length_scale=length_scale)
    bank = SignalBank()
    xin = [torch.from_numpy(bank.fields(r)).pin_memory() for r in reqs]
    xout = [torch.empty_like(x).pin_memory() for x in xin]
    ins = [x.numpy() for x in xin]
    outs = [x.numpy() for x in xout]
    work = np.array([r.work for r in reqs])
    flags = KERR_NAMES[kerr]
    ftypes = {M: fiber_type(M) for M in sorted({r.n_modes for r in reqs})}

    srv = mmf.Server()
    fid = {M: srv.add_fiber(M, 2, ft["S"], ft["parity"], ft["gamma"], flags) for M, ft in ftypes.items()}

    def run(arrivals):
        t0 = time.perf_counter()
        ids = []
        for r, a, xi, xo in zip(reqs, arrivals, ins, outs):
            while True:
                now = time.perf_counter() - t0
                if now >= a:
                    break
                time.sleep(min(0.002, a - now))
            ids.append(srv.submit(fid[r.n_modes], r.betas, 0.0, r.N_t, r.dt, r.L, r.n_steps, xi, xo))
        lat = np.array([srv.wait(i, 3600.0) for i in ids])
        makespan = time.perf_counter() - t0
        for i in ids:
            srv.release(i)
        return lat, makespan

    # warm-up: one short request per shape builds every pool and its graph
    shapes = {}
    for r, xi in zip(reqs, ins):
        shapes.setdefault((r.n_modes, r.N_t), (r, xi))
    wids = [srv.submit(fid[r.n_modes], r.betas, 0.0, r.N_t, r.dt, 10.0, 1, xi, np.empty_like(xi))
            for r, xi in shapes.values()]
    for i in wids:
        srv.wait(i, 600.0)
        srv.release(i)
    st0 = srv.stats()
    lat_c, span_c = run(np.zeros(len(reqs)))
    capacity = work.sum() / span_c
    rate = load * capacity / work.mean()                 # requests per second
    arr = np.array([r.arrival for r in reqs]) / rate
    st1 = srv.stats()
    lat_s, span_s = run(arr)
    st2 = srv.stats()
    srv.close()
    served = work.sum() / span_s

    # one request at a time through the single-link calls, in the plain FP32 path and in the
    # served precision
    pct = lambda v, q: float(np.percentile(v, q))

    def one_at_a_time(fl):
        solve = []
        for r, xi, xo in zip(reqs, ins, outs):
            ft = ftypes[r.n_modes]
            t0 = time.perf_counter()
            f = mmf.Fiber(r.n_modes, 2, ft["S"], ft["parity"], r.betas, 0.0, ft["gamma"], r.N_t, r.dt, fl, 0)
            f.propagate_host(xi, xo, r.L, r.n_steps)
            f.close()
            solve.append(time.perf_counter() - t0)
        solve = np.array(solve)
        done, q_lat = 0.0, []
        for a, sv in zip(arr, solve):
            done = max(done, a) + sv
            q_lat.append(done - a)
        q_lat = np.array(q_lat) * 1e3
        return {"value": work.sum() / solve.sum(), "unit": UNIT,
                "solve_p50_ms": pct(solve * 1e3, 50), "solve_p99_ms": pct(solve * 1e3, 99),
                "queued_p50_ms": pct(q_lat, 50), "queued_p99_ms": pct(q_lat, 99)}
    oat_fp32 = one_at_a_time(KERR_NAMES["fp32"])
    oat_same = oat_fp32 if kerr == "fp32" else one_at_a_time(flags)
    return {
        "requests": len(reqs), "kerr": kerr,
        "sample": f"first {len(reqs)} requests of the seeded serving mix (6/15/36/45 HG modes x 2 pol, "
                  f"N_t 2^14..2^17, -4..+4 dBm), lengths x{length_scale:g} ({int(min(r.n_steps for r in reqs))}-"
                  f"{int(max(r.n_steps for r in reqs))} steps at dz = 10 m)",
        "capacity": capacity, "load": load, "arrival_rate_per_s": rate,
        "value": served, "unit": UNIT,
        "p50_ms": pct(lat_s, 50), "p99_ms": pct(lat_s, 99),
        "closed_loop_p50_ms": pct(lat_c, 50), "closed_loop_p99_ms": pct(lat_c, 99),
        "pools": st2["pools"], "peak_running": st2["peak_running"],
        "gpu_launches": int(st2["kernel_launches"] - st1["kernel_launches"]),
        "one_at_a_time_fp32": oat_fp32,
        "one_at_a_time_same_precision": oat_same,
        "capacity_vs_one_at_a_time_fp32": capacity / oat_fp32["value"],
        "capacity_vs_one_at_a_time_same_precision": capacity / oat_same["value"],
        "warmup_kernel_launches": int(st0["kernel_launches"]),
    }


def cpu_baseline(workload: str, budget_s: float = 20.0):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload: all
    fields and the full Kerr tensor, N_t reduced so one step takes a few seconds."""
    import oracle
    if workload == "c3k":
        from workloads import kappa_hg
        wl = make_workload("c3", with_S=False)
        kappa = kappa_hg(wl.modes, 10e-6, wl.n_pol)
        n = 64
        while True:
            s_ = make_workload("c3", N_t=n, with_S=False)
            t0 = time.perf_counter()
            oracle.propagate_kappa(kappa, s_.betas, s_.alpha, s_.gamma, s_.dt, s_.fields, s_.L / s_.n_steps, 1)
            dt_s = time.perf_counter() - t0
            if dt_s > budget_s / 4 or n * 2 > wl.N_t:
                break
            n *= 2
        return {"value": s_.P * n / dt_s, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                "sample": f"c3k rows and kappa, N_t={n} (of {wl.N_t}), 1 RK4IP step, {dt_s:.1f} s"}
    wl = make_workload(workload, N_t=None, with_S=True)
    # pick N_t so that one step costs ~budget_s/3 on this host (measure a tiny run first)
    n_small = 64 if wl.N_t >= 64 else wl.N_t
    sps = {"c0": 16, "c1": 32, "c2": 64, "c3": 32}.get(workload, 32)
    n_small = max(sps, n_small)
    small = make_workload(workload, N_t=n_small)
    t0 = time.perf_counter()
    oracle.propagate(small.S, small.n_pol, small.betas, small.alpha, small.gamma, small.dt, small.fields,
                     small.L / small.n_steps, 1)
    t_small = time.perf_counter() - t0
    scale = max(1, int((budget_s / 3) / max(t_small, 1e-6)))
    n = n_small
    while n * 2 <= min(wl.N_t, n_small * scale):
        n *= 2
    sample = make_workload(workload, N_t=n)
    steps = 1
    t0 = time.perf_counter()
    oracle.propagate(sample.S, sample.n_pol, sample.betas, sample.alpha, sample.gamma, sample.dt, sample.fields,
                     sample.L / sample.n_steps * steps, steps)
    dt_s = time.perf_counter() - t0
    return {"value": sample.P * n * steps / dt_s, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{workload} fields and Kerr tensor, N_t={n} (of {wl.N_t}), {steps} RK4IP step, "
                      f"{dt_s:.1f} s"}


def run_reference(args, ws, rank):
    """The FP64 oracle, as it stands, on the host cores: each timed step is one oracle RK4IP
    step on a bounded window of the workload (all fields and the full Kerr operator, fewer
    samples); for the serving mix (c4), one step of each request in turn, one at a time."""
    if rank != 0:
        return None
    import oracle
    w = args.workload
    if w == "c4":
        from workloads.serving import serving_requests, fiber_type
        reqs = serving_requests(8)
        ft = {M: fiber_type(M) for M in {r.n_modes for r in reqs}}
        sample_nt = 64
        rng = np.random.default_rng(0)

        def one(i):
            r = reqs[i % len(reqs)]
            x = (rng.standard_normal((r.P, sample_nt)) + 1j * rng.standard_normal((r.P, sample_nt))) * 1e-2
            oracle.propagate(ft[r.n_modes]["S"], 2, r.betas, 0.0, ft[r.n_modes]["gamma"], r.dt, x, 10.0, 1)
            return r.P * sample_nt
        for i in range(args.warmup):
            one(i)
        t0 = time.perf_counter()
        units = sum(one(i) for i in range(args.steps))
        el = time.perf_counter() - t0
        P_desc, Nt_desc = "6/15/36/45 HG modes x 2 pol", "2^14..2^17"
        sample = f"serving-mix requests one at a time, one RK4IP step each at N_t={sample_nt}"
    else:
        base = "c3" if w == "c3k" else w
        wl = make_workload(base, with_S=False)
        sample_nt = {"c0": 4096, "c1": 1024, "c2": 256, "c3": 64, "c3k": 1024}[w]
        s = make_workload(base, N_t=sample_nt, with_S=(w != "c3k"))
        hstep = s.L / s.n_steps
        if w == "c3k":
            from workloads import kappa_hg
            kappa = kappa_hg(s.modes, 10e-6, s.n_pol)
            step = lambda A: oracle.propagate_kappa(kappa, s.betas, s.alpha, s.gamma, s.dt, A, hstep, 1)
        else:
            step = lambda A: oracle.propagate(s.S, s.n_pol, s.betas, s.alpha, s.gamma, s.dt, A, hstep, 1)
        A = s.fields.copy()
        for _ in range(args.warmup):
            A = step(A)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            A = step(A)
        el = time.perf_counter() - t0
        units = s.P * sample_nt * args.steps
        P_desc, Nt_desc = f"{wl.n_modes} HG modes x {wl.n_pol} pol = {wl.P} fields", wl.N_t
        sample = f"{w} fields and Kerr operator at N_t={sample_nt} (of {wl.N_t}), one step per timed step"
    value = units / el
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{w}: {P_desc}", "N_t": Nt_desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c0", "c1", "c2", "c3", "c3k", "c4"])
    ap.add_argument("--kerr", default="bf16x3", choices=list(KERR_NAMES))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-parity", dest="parity", action="store_false",
                    help="skip the rel-L2 check against the FP64 oracle on a reduced window")
    ap.add_argument("--no-c3", dest="c3_block", action="store_false",
                    help="skip the 120-mode block of the default line")
    ap.add_argument("--serving-requests", type=int, default=48,
                    help="serving-mix sample added to the default line (0 = none)")
    ap.add_argument("--serving-requests-c4", type=int, default=200, help="requests of --workload c4")
    ap.add_argument("--serving-length-scale", type=float, default=0.01)
    ap.add_argument("--serving-kerr", default="bf16x3", choices=list(KERR_NAMES),
                    help="Kerr precision of the served requests (one-at-a-time solves are timed in FP32 and in this)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out))
        return
    if ws > 1:
        import torch
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    out = run_serving(args, ws, rank, local) if args.workload == "c4" else run_ours(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
