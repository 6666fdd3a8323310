"""Benchmark of the stochastic MDD hot path: SGD steps (forward MDC on a source batch, residual, adjoint,
update) on synthetic data shaped like the paper's workloads.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload NAME]

Default workload: 48 independent MDD problems of uneven sizes (nr, nv in [64, 600], ns in [64, 800], nt in
{256, 512, 1024, 1500}, the largest member nt = 1500 with nr = nv = ns = 1200), batch 32, split-BF16
tensor-core products; a step of this line is one epoch of every member, replayed from one captured CUDA
graph.  Single problems: --workload smdd_nt512_n201_nb16_recip etc.

Prints one JSON line (rank 0).  `value` is the algorithmic FLOP rate of the whole job: per SGD step
    F_gemm = 16 nb nr nv nf                      (forward + adjoint complex products, 8 real flops / MAC)
    F_fft  = 5 N log2(N) (nr nv + nb nv)         (two real FFTs per model trace and per residual trace,
                                                  2.5 N log2 N flops each; with reciprocity the model is
                                                  symmetric and nr nv becomes its nv (nv + 1) / 2 distinct
                                                  traces, the step the library runs)
with N the smallest 2^a 3^b 5^c >= 2 nt - 1 and nf = N/2 + 1 (the shortest transform that keeps the
linear convolution exact, whatever length the library pads to), summed over the steps of all ranks and
divided by the max over ranks of the device time.  The roofline figures divide the same algorithmic work
by the measured peaks: compulsory bytes (the model read and written, the gathered kernel spectra, the
observed rows of the batch) over the measured HBM copy bandwidth, FFT flops over the measured FP32 FMA
rate, product flops over the FP32 rate (FP32 products) or the sustained BF16 tensor rate (split-BF16
products).  Bytes a staged pipeline moves in addition (the model and gradient spectra written by one
kernel and read by the next) are reported per kernel as `staged_bytes`, not counted as algorithmic.

--impl reference times the FP64 oracle (direct time-domain sums, OpenMP on the host cores) on a bounded
sample of each step (a subset of virtual-source columns; forward and adjoint cost are linear in the
number of columns) and reports the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2202_04486_gb300 import synth  # noqa: E402

BATCH_WORKLOAD = "smdd_batch48_nb32"
DEFAULT_WORKLOAD = BATCH_WORKLOAD
DEFAULT_PRECISION = "bf16x3"
FIXED_ERROR_WORKLOADS = ("smdd_nt1024_n301_ns401_nb32", "smdd_nt1024_n301_ns401_nb64")
METRIC = "MDC fwd+adj GFLOP/s (SMDD step)"
UNIT = "GFLOP/s"


# ------------------------------------------------------------------------------------------------
# work model (algorithmic)
# ------------------------------------------------------------------------------------------------
def nfft_for(nt: int) -> int:
    """Smallest 2^a 3^b 5^c >= 2 nt - 1: the shortest FFT whose circular convolution equals the linear
    one on [0, nt) (the algorithmic length; the library may pad further)."""
    n = max(2 * nt - 1, 1)
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return n
        n += 1


def nf_of(nt: int) -> int:
    return nfft_for(nt) // 2 + 1


def fft_flops(nt: int) -> float:
    """2.5 N log2 N for one real FFT of the algorithmic length N."""
    n = nfft_for(nt)
    return 2.5 * n * math.log2(n)


def model_traces(nr, nv, sym=False) -> int:
    """Distinct model traces: nr nv, or nv (nv + 1) / 2 for a symmetric model (reciprocity, Eq. 4: the
    model X = C_r z is symmetric, so the traces on and above the diagonal determine it)."""
    return nv * (nv + 1) // 2 if sym else nr * nv


def step_work(nt, nr, nv, nb, sym=False) -> tuple[float, float]:
    """(F_gemm, F_fft) of one SGD step (sym: the model transforms of the distinct traces only)."""
    return 16.0 * nb * nr * nv * nf_of(nt), 2.0 * fft_flops(nt) * (model_traces(nr, nv, sym) + nb * nv)


def step_flops(nt, nr, nv, nb, sym=False) -> float:
    return sum(step_work(nt, nr, nv, nb, sym))


def step_bytes_compulsory(nt, nr, nv, nb, recip, sym=False) -> float:
    """Model read + write, the gathered kernel spectra, the batch rows of U_obs (and, with reciprocity,
    the round trip of the gradient that couples trace (r, v) with (v, r)).  sym: a symmetric model is read
    on its distinct traces and written whole; the symmetric gradient is formed in the adjoint product, so
    there is no gradient round trip."""
    if sym:
        return float((model_traces(nr, nv, True) + nr * nv) * nt * 4 + nf_of(nt) * nb * nr * 8 + nb * nv * nt * 4)
    b = 2 * nr * nv * nt * 4 + nf_of(nt) * nb * nr * 8 + nb * nv * nt * 4
    if recip:
        b += 2 * nr * nv * nt * 4
    return float(b)


def kernel_work(stage, nt, nr, nv, nb, sym=False):
    """Algorithmic bytes and flops of one launch of a stage, and the bytes the staged pipeline moves in
    addition (spectra written by one kernel and read by the next), at the algorithmic FFT length.  sym: the
    update of a symmetric model (its distinct traces transformed, the model written whole, the spectra below
    the block diagonal copied from above it)."""
    nf = nf_of(nt)
    ff = fft_flops(nt)
    if stage == "update" and sym:
        # gradient spectra read and model spectra written on the distinct traces (the forward product reads the
        # rest transposed)
        up = model_traces(nr, nv, True)
        return dict(bytes=(up + nr * nv) * nt * 4, flops=2 * ff * up, staged=2 * up * nf * 8, tensor=False)
    if stage == "update":      # inverse FFT of the gradient, update, FFT of the new model, per model trace
        return dict(bytes=2 * nv * nr * nt * 4, flops=2 * ff * nv * nr, staged=2 * nv * nr * nf * 8, tensor=False)
    if stage == "cgemm_fwd":   # products with the gathered kernel rows; model spectra in, batch spectra out
        return dict(bytes=nf * nb * nr * 8, flops=8.0 * nv * nr * nb * nf, staged=nf * (nv * nr + nv * nb) * 8,
                    tensor=True)
    if stage == "cgemm_adj":   # residual spectra and gathered kernel rows in, gradient spectra out
        return dict(bytes=nf * nb * nr * 8, flops=8.0 * nv * nr * nb * nf, staged=nf * (nv * nb + nv * nr) * 8,
                    tensor=True)
    if stage == "residual":    # inverse FFT, window, subtraction of the observed rows, loss, FFT
        return dict(bytes=nb * nv * nt * 4, flops=2 * ff * nb * nv, staged=2 * nb * nv * nf * 8, tensor=False)
    if stage == "rfft":        # model spectra of the first step
        return dict(bytes=nv * nr * nt * 4, flops=ff * nv * nr, staged=nv * nr * nf * 8, tensor=False)
    return dict(bytes=0, flops=0, staged=0, tensor=False)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 SIMT peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


class Peaks:
    """The roofline denominators: HBM copy bandwidth and sustained BF16 tensor rate from
    MEASURED_PEAKS.json, FP32 FMA rate measured in this run by the library's probe."""

    def __init__(self, fp32_tflops: float, fp32_derived: float):
        pk, src = load_peaks()
        self.hbm = float(pk["hbm_gbs"]) * 1e9
        self.bf16 = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))) * 1e12
        self.fp32 = fp32_tflops * 1e12
        self.fp32_derived = fp32_derived
        self.source = src

    def kernel_roof(self, stage, work, ms, tensor_products: bool):
        """Roofline of one launch: T_roof = max(bytes / HBM, flops / arithmetic peak); the binding resource
        names the bound; frac = T_roof / measured duration (= achieved / peak in the binding unit)."""
        t = ms * 1e-3
        on_tc = work["tensor"] and tensor_products
        p_ar = self.bf16 if on_tc else self.fp32
        t_mem, t_ar = work["bytes"] / self.hbm, work["flops"] / p_ar
        if t_mem >= t_ar:
            roof = {"bound": "hbm", "achieved": round(work["bytes"] / t / 1e9, 1), "peak": round(self.hbm / 1e9, 1),
                    "unit": "GB/s", "peak_source": f"{self.source} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
        else:
            roof = {"bound": "tensor" if on_tc else "alu", "achieved": round(work["flops"] / t / 1e12, 3),
                    "peak": round(p_ar / 1e12, 2), "unit": "TFLOP/s",
                    "peak_source": ("sustained BF16 dense tensor rate (MEASURED_PEAKS.json bf16_tflops_sustained); "
                                    "algorithmic complex-product flops, not the split products" if on_tc else
                                    "FP32 FMA rate measured in this run (mdc_alu_probe)")}
        roof["frac"] = round(max(t_mem, t_ar) / t, 4)
        roof["kernel"] = stage
        roof["launch_ms"] = round(ms, 5)
        roof["algorithmic_bytes"] = int(work["bytes"])
        roof["algorithmic_flops"] = float(work["flops"])
        roof["staged_bytes"] = int(work["staged"])
        roof["staged_gbs"] = round((work["bytes"] + work["staged"]) / t / 1e9, 1)
        return roof

    def step_roof_s(self, nt, nr, nv, nb, recip, tensor_products: bool, sym=False) -> float:
        """T_roof of one step: max(B / HBM, F_gemm / P_gemm + F_fft / P_FP32)."""
        fg, ff = step_work(nt, nr, nv, nb, sym)
        p_gemm = self.bf16 if tensor_products else self.fp32
        return max(step_bytes_compulsory(nt, nr, nv, nb, recip, sym) / self.hbm, fg / p_gemm + ff / self.fp32)


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2202_04486_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(stage: str, workload: str):
    """DRAM bytes per launch of `stage` from the committed ncu summary, or None when the summary is
    missing or was taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    src_hash, table = None, {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("source_hash:"):
                src_hash = line.split(":", 1)[1].strip()
            elif line and not line.startswith("#") and ":" not in line:
                parts = line.split()
                if len(parts) >= 2:
                    try:
                        table[parts[0]] = float(parts[1])
                    except ValueError:
                        pass
    if src_hash != kernel_source_hash():
        return None
    return table.get(stage)


# ------------------------------------------------------------------------------------------------
# combining the ranks (one independent replica per GPU)
# ------------------------------------------------------------------------------------------------
def combine_ranks(times, flops: float, device=None):
    """Max over ranks of each time and sum over ranks of the flops (all ranks call it; a no-op without
    an initialised process group of more than one rank).  Returns (times, flops)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(times), float(flops)
    tt = torch.tensor(list(times), dtype=torch.float64, device=device)
    ff = torch.tensor([float(flops)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(ff, op=dist.ReduceOp.SUM)
    return tt.tolist(), ff.item()


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.out is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.out.seek(0)
        sm, smmax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smmax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smmax) if smmax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# problem set-up (both arms)
# ------------------------------------------------------------------------------------------------
def make_inputs(w, seed):
    n = w.get("n") or 0
    nt, nb = w["nt"], w["nb"]
    nr, nv, ns = w.get("nr", n), w.get("nv", n), w.get("ns", n)
    p = synth.make_problem(nt, nr, nv, ns, dx=w["dx"], n_reflectors=w["n_reflectors"],
                           n_multiples=w["n_multiples"], seed=seed)
    return p


def workload_dims(name):
    w = dict(synth.WORKLOADS[name])
    for k in ("nr", "nv", "ns"):
        w.setdefault(k, w.get("n"))
    return w


# ------------------------------------------------------------------------------------------------
# oracle (CPU) timing: used for cpu_baseline and for --impl reference
# ------------------------------------------------------------------------------------------------
def oracle_step_sample(D, X, U_obs, idx, vsel):
    import oracle
    U = oracle.mdc_forward(D, X, idx, vsel=vsel)
    R = U - U_obs[idx][:, vsel]
    G = oracle.mdc_adjoint(D, R, idx, vsel=np.arange(len(vsel)))
    return G


def time_oracle(w, D, X, U_obs, batches, target_s=12.0, max_cols=None):
    """Time the oracle's forward+adjoint on a sample of virtual-source columns and extrapolate to a
    full step.  Returns (GFLOP/s equivalent, seconds per full step, sample description, threads)."""
    import oracle
    nv = w["nv"]
    idx = batches[0][0]
    cols = min(2, nv)
    t0 = time.perf_counter()
    oracle_step_sample(D, X, U_obs, idx, np.arange(cols))
    t1 = time.perf_counter()
    per_col = max((t1 - t0) / cols, 1e-6)
    k = int(min(nv if max_cols is None else max_cols, max(1, target_s / per_col)))
    vsel = np.linspace(0, nv - 1, k).round().astype(np.int64)
    t0 = time.perf_counter()
    oracle_step_sample(D, X, U_obs, idx, vsel)
    t1 = time.perf_counter()
    t_step = (t1 - t0) * nv / k
    f = step_flops(w["nt"], w["nr"], w["nv"], len(idx), bool(w["reciprocity"]))
    sample = (f"forward+adjoint direct sums (FP64) for {k} of {nv} virtual-source columns of one batch of "
              f"{len(idx)} sources, extrapolated linearly in the column count ({t1 - t0:.1f} s measured)")
    return f / t_step / 1e9, t_step, sample, oracle.num_threads()


def oracle_extra(w, D, X, U_obs, idx, target_s=3.0):
    """The oracle's other timings for one step: the direct sums on one thread, and the FP64 FFT tier
    (numpy) -- each on a column sample of about target_s, extrapolated in the column count."""
    import oracle
    nv = w["nv"]
    cores = oracle.num_threads()
    res = {}
    try:
        oracle.set_num_threads(1)
        t0 = time.perf_counter()
        oracle_step_sample(D, X, U_obs, idx, np.arange(1))
        per_col = max(time.perf_counter() - t0, 1e-6)
        k = int(min(nv, max(1, target_s / per_col)))
        vsel = np.linspace(0, nv - 1, k).round().astype(np.int64)
        t0 = time.perf_counter()
        oracle_step_sample(D, X, U_obs, idx, vsel)
        t1 = (time.perf_counter() - t0) * nv / k
    finally:
        oracle.set_num_threads(cores)
    macs = 2.0 * len(idx) * w["nv"] * w["nr"] * w["nt"] * (w["nt"] + 1) / 2   # forward + adjoint direct sums
    res["tier_a_1thread_s_per_step"] = round(t1, 3)
    res["tier_a_1thread_gflops"] = round(step_flops(w["nt"], w["nr"], w["nv"], len(idx), bool(w["reciprocity"])) / t1 / 1e9, 5)
    res["tier_a_1thread_direct_mac_per_s"] = round(macs / t1, 1)
    t0 = time.perf_counter()
    k = max(1, min(nv, 4))
    vsel = np.arange(k)
    Uf = oracle.mdc_forward_fft(D, X[vsel], idx)
    oracle.mdc_adjoint_fft(D, Uf - U_obs[idx][:, vsel], idx)
    res["tier_b_fft_s_per_step"] = round((time.perf_counter() - t0) * nv / k, 3)
    res["tier_b_sample"] = f"{k} of {nv} virtual-source columns, extrapolated"
    return res


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def measured_peaks(dev):
    """FP32 FMA rate measured now by the library's probe (and the lane-count figure beside it)."""
    import torch

    from paper_2202_04486_gb300 import binding

    props = torch.cuda.get_device_properties(dev)
    pk, _ = load_peaks()
    fp32_derived = fp32_alu_peak_tflops(props.multi_processor_count, pk.get("sm_max_mhz", 2070.0))
    return Peaks(binding.alu_peak_tflops(0), fp32_derived), binding.alu_peak_tflops(1)


def stage_roofs(peaks, stage, member, tensor_products, sym=False):
    """Per-stage roofline of the timed steps: stage -> (ms, launches) from the library's stage timers."""
    nt, nr, nv, nb = member
    out = {}
    for k, (ms, n) in stage.items():
        if n <= 0 or k not in ("rfft", "cgemm_fwd", "residual", "cgemm_adj", "update"):
            continue
        out[k] = peaks.kernel_roof(k, kernel_work(k, nt, nr, nv, nb, sym), ms / n, tensor_products)
        out[k]["launches"] = int(n)
    tot = sum(v["launch_ms"] * v["launches"] for v in out.values())
    for v in out.values():
        v["share"] = round(v["launch_ms"] * v["launches"] / tot, 4)
    return out


def run_gpu(args, rank, world, w):
    import torch

    from paper_2202_04486_gb300 import binding, build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or not os.path.exists(binding.LIB_PATH):
        build.build()
    if world > 1:
        torch.distributed.barrier()
    binding.load_library()
    nt, nr, nv, ns, nb = w["nt"], w["nr"], w["nv"], w["ns"], w["nb"]
    recip = bool(w["reciprocity"])

    p = make_inputs(w, seed=rank)
    D = torch.from_numpy(p.D.astype(np.float32)).to(dev)
    X_true = torch.from_numpy(p.X_true.astype(np.float32)).to(dev)
    # observed data: forward of the true model over all sources (GPU path) plus seeded noise
    gen = binding.MDCPlan(D, nv, nb_max=ns)
    U_obs = gen.forward(X_true, torch.arange(ns, dtype=torch.int32, device=dev))
    if w["noise"] > 0:
        rms = U_obs.pow(2).mean().sqrt()
        U_obs += w["noise"] * rms * torch.from_numpy(p.noise.astype(np.float32)).to(dev)
    gen.close()

    tc = args.precision == "bf16x3"
    prec = binding.MDC_PREC_BF16X3 if tc else binding.MDC_PREC_FP32
    plan = binding.MDCPlan(D, nv, nb_max=nb, precision=prec)
    chosen = plan.autotune(nb, binding.SMDD_RECIPROCITY if recip else 0, reps=5) if args.autotune else plan.get_config()
    sigma2 = plan.sigma2_max(60)
    alpha = 0.5 * 2.0 / sigma2
    # the model starts at zero, so with reciprocity it stays symmetric: the update runs on its distinct traces
    flags = ((binding.SMDD_RECIPROCITY | binding.SMDD_SYMMETRIC) if recip else 0) | binding.SMDD_KEEP_XHAT
    X = torch.zeros((nv, nr, nt), device=dev)
    n_ep = 2 * (args.warmup + args.steps) // math.ceil(ns / nb) + 3
    batches = [b for ep in synth.epoch_batches(ns, nb, n_ep, seed=rank) for b in ep]
    idx_dev = [torch.from_numpy(b).to(dev) for b in batches]
    loss = torch.zeros(len(batches), device=dev, dtype=torch.float64)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)
    # L2 policy (the same for the device-timed and the end-to-end loop): flush before every timed step
    # unless the step's own traffic is far larger than L2 (then back-to-back steps, as an SGD run issues
    # them, and the inputs themselves evict L2)
    l2_bytes = 126 * 1024 * 1024
    step_traffic = step_bytes_compulsory(nt, nr, nv, nb, recip, recip) + 4.0 * nf_of(nt) * nv * nr * 8
    do_flush = args.l2 == "flush" or (args.l2 == "auto" and step_traffic < 4 * l2_bytes)
    stream = torch.cuda.current_stream()

    def one_step(k):
        fl = flags | (binding.SMDD_REUSE_XHAT if k > 0 else 0)
        binding.smdd_step(plan.handle, X, U_obs, idx_dev[k], alpha, fl, loss[k])

    for k in range(args.warmup):
        if do_flush:
            flush.fill_(float(k))
        one_step(k)
    torch.cuda.synchronize()

    # timed region: K steps, per-step CUDA events on the launching stream, stage timers off
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = binding.mdc_plan_launch_count(plan.handle)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    try:
        smi_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        smi_id = str(local)
    with ClockSampler(smi_id) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            k = args.warmup + i
            if do_flush:
                flush.fill_(float(k))
            ev[i][0].record(stream)
            one_step(k)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    launches = binding.mdc_plan_launch_count(plan.handle) - l0
    status = plan.sync_status()
    if status != binding.MDC_OK:
        raise RuntimeError(f"device status {binding.status_string(status)}")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(step_ms) / 1e3
    flops = sum(step_flops(nt, nr, nv, len(batches[args.warmup + i]), recip) for i in range(args.steps))
    losses = loss[: args.warmup + args.steps].cpu().numpy()

    # stage shares: the same steps once more with the library's per-kernel CUDA events (outside the timed
    # region, same L2 policy)
    binding.mdc_plan_set_profiling(plan.handle, True)
    binding.mdc_plan_stage_times(plan.handle, reset=True)
    for i in range(args.steps):
        k = args.warmup + args.steps + i
        if do_flush:
            flush.fill_(float(k))
        one_step(k)
    stage = binding.mdc_plan_stage_times(plan.handle, reset=True)
    binding.mdc_plan_set_profiling(plan.handle, False)

    # e2e: the same steps through smdd_step_host with host inputs: every step the plan copies the batch
    # index list and the batch rows of U_obs (pinned) host -> device on its copy stream, overlapping the
    # previous step, and the step's loss comes back device -> host (pinned); the host reads the loss of
    # step k - 1 once step k is queued, and the last one after the loop.  Same L2 policy as above.
    U_host = U_obs.cpu().pin_memory()
    Xe = torch.zeros_like(X)
    idx_host = [torch.from_numpy(np.ascontiguousarray(b, dtype=np.int32)) for b in batches]
    loss_host = torch.zeros(len(batches), dtype=torch.float64).pin_memory()
    h2d = d2h = 0

    def e2e_run(ks, count):
        nonlocal h2d, d2h
        done = []
        for j, k in enumerate(ks):
            if do_flush:
                flush.fill_(float(k))
            fl = flags | (binding.SMDD_REUSE_XHAT if k > 0 else 0)
            binding.smdd_step_host(plan.handle, Xe, U_host, idx_host[k], alpha, fl, loss_host[k:k + 1], stream)
            e = torch.cuda.Event()
            e.record(stream)
            done.append(e)
            if j > 0:
                done[j - 1].synchronize()
                _ = float(loss_host[ks[j - 1]])
            if count:
                h2d += idx_host[k].numel() * 4 + idx_host[k].numel() * nv * nt * 4
                d2h += 8
        done[-1].synchronize()
        _ = float(loss_host[ks[-1]])

    e2e_run(list(range(args.warmup)), False)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    e2e_run([args.warmup + i for i in range(args.steps)], True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - e0

    # max over ranks
    (t_dev, t_e2e, wall), flops_all = combine_ranks([t_dev, t_e2e, wall], flops, dev)
    if rank != 0:
        return None

    peaks, fp64_peak = measured_peaks(dev)
    kern = stage_roofs(peaks, stage, (nt, nr, nv, nb), tc, recip)
    dom = max(kern, key=lambda k: kern[k]["share"])
    roof = dict(kern[dom])
    roof["traffic"] = ncu_traffic(dom, args.workload)
    t_roof = peaks.step_roof_s(nt, nr, nv, nb, recip, tc, recip)
    ms_per_step = t_dev / args.steps * 1e3
    nfft_impl, _ = binding.mdc_plan_info(plan.handle)

    out = {
        "metric": METRIC, "value": round(flops_all / t_dev / 1e9, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if not tc else "f32 FFTs, bf16x3 (split hi+lo) tensor-core products",
        "data": "synthetic (seeded Ricker/hyperbola generator; U_obs = GPU forward of the true model + 5% noise)",
        "config": {"workload": args.workload, "nt": nt, "nr": nr, "nv": nv, "ns": ns, "nb": nb,
                   "nfft_algorithmic": nfft_for(nt), "nfft_library": nfft_impl, "reciprocity": recip,
                   "precision": args.precision, "solver": "SGD, alpha = 0.5 * 2/sigma^2_max",
                   "l2": ("flushed before every step (256 MiB write, outside the step events; also in the e2e loop)"
                          if do_flush else
                          f"inputs larger than L2: no flush, back-to-back steps (per-step traffic "
                          f"{step_traffic / 2**20:.0f} MiB against {l2_bytes / 2**20:.0f} MiB of L2)"),
                   "per_rank": "independent problem replica, seed = rank (no data-path collective)",
                   "autotuned": bool(args.autotune), "kernel_config": chosen},
        "e2e": {"value": round(flops_all / t_e2e / 1e9, 2), "unit": UNIT,
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": int(launches) * world,
        "roofline": roof,
        "kernels": kern,
        "step_roofline": {"t_roof_us": round(t_roof * 1e6, 2), "t_step_us": round(ms_per_step * 1e3, 2),
                          "frac": round(t_roof / (ms_per_step * 1e-3), 4),
                          "definition": ("max(compulsory bytes / HBM, F_gemm / P_gemm + F_fft / P_FP32); P_gemm = "
                                         + ("sustained BF16 tensor rate" if tc else "measured FP32 FMA rate")),
                          "fp32_tflops_measured": round(peaks.fp32 / 1e12, 2),
                          "fp32_tflops_derived": round(peaks.fp32_derived, 2),
                          "bf16_tflops_sustained": round(peaks.bf16 / 1e12, 1),
                          "fp64_tflops_measured": round(fp64_peak, 3)},
        "clocks": clk.summary(),
        "steps_per_s": round(args.steps / t_dev, 2),
        "wall_s_timed_region": round(wall, 4),
        "loss_first_last": [float(losses[0]), float(losses[-1])],
    }
    if args.fixed_error_epochs > 0:
        out["fixed_error"] = precision_comparison(args, dev, D, U_obs, X_true, w, rank)
    if args.solver_epochs > 0:
        out["solvers"] = solver_comparison(args, dev, D, U_obs, X_true, w, rank)
    if world == 1 or rank == 0:
        D64 = p.D.astype(np.float32).astype(np.float64)
        Xs = np.zeros((nv, nr, nt))
        Uo = U_obs.double().cpu().numpy()
        val, t_step, sample, cores = time_oracle(w, D64, Xs, Uo, [batches[args.warmup:]])
        macs = 2.0 * nb * nv * nr * nt * (nt + 1) / 2
        out["cpu_baseline"] = {"value": round(val, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample, "s_per_step_extrapolated": round(t_step, 3),
                               "steps_per_s": round(1.0 / t_step, 5), "direct_mac_per_s": round(macs / t_step, 1)}
        out["cpu_baseline"].update(oracle_extra(w, D64, Xs, Uo, batches[args.warmup]))
    return out


def precision_comparison(args, dev, D, U_obs, X_true, w, rank):
    """FP32 products against split-BF16 products at the same final-model error: both run the same
    epochs from the same batches (autotuned configurations when --autotune); the model error is the
    relative L2 distance to the true model, and the BF16x3 path runs until its error is at most the FP32
    path's (or twice the epochs).  Device time of the steps only."""
    import torch

    from paper_2202_04486_gb300 import binding

    nt, nr, nv, ns, nb = w["nt"], w["nr"], w["nv"], w["ns"], w["nb"]
    recip = bool(w["reciprocity"])
    n_ep = args.fixed_error_epochs
    batches = synth.epoch_batches(ns, nb, 2 * n_ep, seed=100 + rank)
    idx_dev = [[torch.from_numpy(b).to(dev) for b in ep] for ep in batches]
    xt_norm = X_true.double().norm().item()
    res, x_at = {}, {}
    for name, prec in (("fp32", binding.MDC_PREC_FP32), ("bf16x3", binding.MDC_PREC_BF16X3)):
        plan = binding.MDCPlan(D, nv, nb_max=nb, precision=prec)
        flags = binding.SMDD_RECIPROCITY if recip else 0
        cfg = plan.autotune(nb, flags, reps=3) if args.autotune else plan.get_config()
        alpha = 0.5 * 2.0 / plan.sigma2_max(60)
        X = torch.zeros((nv, nr, nt), device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t, steps, errs, k = 0.0, 0, [], 0
        target = res.get("fp32", {}).get("model_error")
        for ep in range(2 * n_ep if target is not None else n_ep):
            e0.record()
            for ii in idx_dev[ep]:
                fl = flags | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
                binding.smdd_step(plan.handle, X, U_obs, ii, alpha, fl)
                k += 1
            e1.record()
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) / 1e3
            steps += len(idx_dev[ep])
            errs.append((X.double() - X_true.double()).norm().item() / xt_norm)
            if ep + 1 == n_ep:
                x_at[name] = X.clone()
            if target is not None and ep + 1 >= n_ep and errs[-1] <= target * (1 + 1e-3):
                break
        if plan.sync_status() != binding.MDC_OK:
            raise RuntimeError("device status after the precision comparison")
        res[name] = {"epochs": len(errs), "steps": steps, "model_error": errs[-1], "device_s": round(t, 4),
                     "steps_per_s": round(steps / t, 2), "kernel_config": cfg}
        plan.close()
    res["bf16x3_vs_fp32_steps_per_s"] = round(res["bf16x3"]["steps_per_s"] / res["fp32"]["steps_per_s"], 3)
    res["bf16x3_vs_fp32_time_to_error"] = round(res["fp32"]["device_s"] / res["bf16x3"]["device_s"], 3)
    a, b = x_at["bf16x3"].double(), x_at["fp32"].double()
    res["x_rel_l2_bf16x3_vs_fp32_after_n_epochs"] = float((a - b).norm() / b.norm())
    res["nb"] = nb
    res["tolerance"] = ("FP64-oracle parity of these paths (the -m gpu tests, nt 1024 301 x 301 x 401 batch 32, "
                        "sampled columns): FP32 <= 1e-5 and BF16x3 <= 1e-4 relative L2 on U and the gradient; "
                        "X after 50 epochs <= 1e-4 (FP32) and 1e-3 (BF16x3)")
    res["definition"] = ("same batches from X = 0; model error = ||X - X_true|| / ||X_true||; BF16x3 runs until "
                         "its error is within 0.1% of the FP32 error after the FP32 epochs (the two differ by "
                         "rounding only); device time of the steps")
    return res


def fixed_error_run(args, dev, name, rank):
    """precision_comparison on a single-problem workload built here (the batched line carries it for the
    mixed-precision workloads: nt 1024, 301 x 301 x 401, batch 32 and 64)."""
    import torch

    from paper_2202_04486_gb300 import binding

    w = workload_dims(name)
    p = make_inputs(w, seed=rank)
    D = torch.from_numpy(p.D.astype(np.float32)).to(dev)
    X_true = torch.from_numpy(p.X_true.astype(np.float32)).to(dev)
    gen = binding.MDCPlan(D, w["nv"], nb_max=w["nb"])
    U_obs = torch.empty((w["ns"], w["nv"], w["nt"]), device=dev)
    for s0 in range(0, w["ns"], w["nb"]):
        ii = torch.arange(s0, min(w["ns"], s0 + w["nb"]), device=dev, dtype=torch.int32)
        gen.forward(X_true, ii, out=U_obs[s0:s0 + ii.numel()])
    gen.close()
    res = precision_comparison(args, dev, D, U_obs, X_true, w, rank)
    res["workload"] = name
    del D, X_true, U_obs
    torch.cuda.empty_cache()
    return res


def solver_comparison(args, dev, D, U_obs, X_true, w, rank):
    """The paper's comparison of solvers on the same problem, in epochs (one epoch = every source once:
    ceil(ns/nb) stochastic steps, or one full-gradient LSQR iteration): SGD (alpha = 0.5 * 2/sigma^2),
    N-SGD (mu = 0.9, alpha = 0.25 * 2/sigma^2) and LSQR, all with the workload's reciprocity flag, from
    X = 0.  Reports the model error ||X - X_true|| / ||X_true|| after every epoch, the device time, and the
    epochs each solver needs to reach SGD's final error."""
    import torch

    from paper_2202_04486_gb300 import binding

    nt, nr, nv, ns, nb = w["nt"], w["nr"], w["nv"], w["ns"], w["nb"]
    recip = bool(w["reciprocity"])
    n_ep = args.solver_epochs
    batches = synth.epoch_batches(ns, nb, n_ep, seed=200 + rank)
    idx_dev = [[torch.from_numpy(b).to(dev) for b in ep] for ep in batches]
    xt = X_true.double()
    xt_norm = xt.norm().item()
    rflag = binding.SMDD_RECIPROCITY if recip else 0
    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for solver in ("sgd", "nsgd", "lsqr"):
        plan = binding.MDCPlan(D, nv, nb_max=ns if solver == "lsqr" else nb)
        sigma2 = plan.sigma2_max(60)
        X = torch.zeros((nv, nr, nt), device=dev)
        V = torch.zeros_like(X)
        errs, t = [], 0.0
        if solver == "lsqr":
            # LSQR cannot be resumed from its iterate alone: each checkpoint count runs from zero
            checks = sorted({k for k in (1, 2, 3, 5, 10, 20, 30, 50, 100, 200) if k < n_ep} | {n_ep})
            for k in checks:
                X.zero_()
                e0.record()
                binding.smdd_lsqr(plan.handle, X, U_obs, k, rflag)
                e1.record()
                torch.cuda.synchronize()
                if k == n_ep:
                    t = e0.elapsed_time(e1) / 1e3
                errs.append((k, (X.double() - xt).norm().item() / xt_norm))
        else:
            alpha = (0.5 if solver == "sgd" else 0.25) * 2.0 / sigma2
            k = 0
            for ep in idx_dev:
                e0.record()
                for ii in ep:
                    fl = rflag | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
                    if solver == "sgd":
                        binding.smdd_step(plan.handle, X, U_obs, ii, alpha, fl)
                    else:
                        binding.smdd_step_ex(plan.handle, X, U_obs, ii, alpha, fl | binding.SMDD_NESTEROV, V=V, mu=0.9)
                    k += 1
                e1.record()
                torch.cuda.synchronize()
                t += e0.elapsed_time(e1) / 1e3
                errs.append((len(errs) + 1, (X.double() - xt).norm().item() / xt_norm))
        if plan.sync_status() != binding.MDC_OK:
            raise RuntimeError(f"device status after {solver}")
        res[solver] = {"model_error_at_epoch": {k: round(e, 5) for k, e in errs}, "device_s": round(t, 4)}
        plan.close()
    # batch-size sweep of SGD (same epochs, alpha = 0.5 * 2/sigma^2 for every batch size)
    sweep = {}
    for nbs in sorted({4, 8, nb, 2 * nb, 4 * nb} & set(range(1, ns + 1))):
        plan = binding.MDCPlan(D, nv, nb_max=nbs)
        alpha = 0.5 * 2.0 / plan.sigma2_max(60)
        X = torch.zeros((nv, nr, nt), device=dev)
        bl = synth.epoch_batches(ns, nbs, n_ep, seed=300 + rank)
        k, t = 0, 0.0
        e0.record()
        for ep in bl:
            for b in ep:
                fl = rflag | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if k else 0)
                binding.smdd_step(plan.handle, X, U_obs, torch.from_numpy(b).to(dev), alpha, fl)
                k += 1
        e1.record()
        torch.cuda.synchronize()
        if plan.sync_status() != binding.MDC_OK:
            raise RuntimeError("device status after the batch-size sweep")
        sweep[str(nbs)] = {"model_error": round((X.double() - xt).norm().item() / xt_norm, 5),
                           "steps": k, "device_s": round(e0.elapsed_time(e1) / 1e3, 4)}
        plan.close()
    res["sgd_batch_size_sweep"] = sweep
    target = res["sgd"]["model_error_at_epoch"][n_ep]
    for solver in ("sgd", "nsgd", "lsqr"):
        errs = res[solver]["model_error_at_epoch"]
        res[solver]["epochs_to_sgd_final_error"] = next((k for k in sorted(errs) if errs[k] <= target), None)
    res["definition"] = ("model error = ||X - X_true|| / ||X_true|| after each epoch (the batch-size sweep: after "
                         f"all {n_ep} epochs); an epoch is ceil(ns/nb) "
                         "stochastic steps or one LSQR iteration (every source once); LSQR is evaluated at "
                         f"checkpoint iteration counts, each run from zero; LSQR device_s is for {n_ep} iterations")
    return res


# ------------------------------------------------------------------------------------------------
# GPU arm, many independent problems: whole epochs of every member replayed from one CUDA graph
# ------------------------------------------------------------------------------------------------
def oracle_member_sample(m, target_s, seed=0):
    """Time the oracle's forward + adjoint of one SGD step of batch member m (nt, nr, nv, nb) on a sample of
    virtual-source columns sized to about target_s, extrapolated linearly in the column count.  The
    direct sums cost the same for any values, so the batch rows of D and the model columns are seeded
    random traces (no full-size FP64 generation on the host).  Returns (GFLOP/s, s per step, columns)."""
    import oracle

    nt, nr, nv, nb = m["nt"], m["nr"], m["nv"], m["nb"]
    rng_seed = 7000 + seed
    Dr = synth.random_traces((nb, nr, nt), rng_seed)
    idx = np.arange(nb, dtype=np.int32)

    def run(k):
        Xs = synth.random_traces((k, nr, nt), rng_seed + 1)
        t0 = time.perf_counter()
        U = oracle.mdc_forward(Dr, Xs, idx)
        oracle.mdc_adjoint(Dr, U, idx)
        return time.perf_counter() - t0

    per_col = max(run(1), 1e-6)
    k = int(min(nv, max(1, target_s / per_col)))
    t = run(k) if k > 1 else per_col
    t_step = t * nv / k
    return step_flops(nt, nr, nv, nb, m["reciprocity"]) / t_step / 1e9, t_step, k


def largest_shape(args):
    """(nt, nr, nv, ns) of the batch's fixed largest member, or None."""
    if not args.batch_largest:
        return None
    return tuple(int(v) for v in args.batch_largest_shape.split(","))


def run_gpu_batch(args, rank, world):
    import torch

    from paper_2202_04486_gb300 import binding, build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or not os.path.exists(binding.LIB_PATH):
        build.build()
    if world > 1:
        torch.distributed.barrier()
    binding.load_library()
    specs = synth.batch_members(args.batch_n, seed=1000 + 100000 * rank,
                                largest=largest_shape(args))
    tc = args.precision == "bf16x3"
    prec = binding.MDC_PREC_BF16X3 if tc else binding.MDC_PREC_FP32
    n_perm = args.warmup + args.steps
    members, setup = [], []
    t_setup = time.perf_counter()
    for m in specs:
        nt, nr, nv, ns, nb = m["nt"], m["nr"], m["nv"], m["ns"], m["nb"]
        D, Xt = synth.make_problem_device(nt, nr, nv, ns, dx=m["dx"], n_reflectors=m["n_reflectors"],
                                          n_multiples=m["n_multiples"], seed=m["seed"], device=dev)
        plan = binding.MDCPlan(D, nv, nb_max=nb, precision=prec)
        U_obs = torch.empty((ns, nv, nt), device=dev)
        for s0 in range(0, ns, nb):
            ii = torch.arange(s0, min(ns, s0 + nb), device=dev, dtype=torch.int32)
            plan.forward(Xt, ii, out=U_obs[s0:s0 + ii.numel()])
        del D, Xt
        alpha = 0.5 * 2.0 / plan.sigma2_max(30)
        # every member starts at X = 0: a reciprocity member stays symmetric (update on its distinct traces)
        flags = (binding.SMDD_RECIPROCITY | binding.SMDD_SYMMETRIC) if m["reciprocity"] else 0
        cfg = plan.autotune(nb, flags, reps=3) if args.autotune else plan.get_config()
        perm = np.stack([np.concatenate(ep) for ep in synth.epoch_batches(ns, nb, n_perm, seed=m["seed"])])
        steps = -(-ns // nb)
        members.append(dict(plan=plan, X=torch.zeros((nv, nr, nt), device=dev), U_obs=U_obs,
                            perm=torch.from_numpy(perm).to(dev), nb=nb, alpha=alpha, flags=flags,
                            loss=torch.zeros((n_perm, steps), device=dev, dtype=torch.float64)))
        setup.append(dict(m, steps=steps, cfg=cfg, perm_host=torch.from_numpy(perm).pin_memory(),
                          nfft_library=binding.mdc_plan_info(plan.handle)[0]))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    mode = binding.MDC_BATCH_QUEUE if args.batch_mode == "queue" else binding.MDC_BATCH_BRANCHES
    batch = binding.MDCBatch(members, n_branches=args.branches, mode=mode)
    step_sizes = [(m["nt"], m["nr"], m["nv"], min(m["nb"], m["ns"] - s * m["nb"]), m["reciprocity"])
                  for m in setup for s in range(m["steps"])]
    epoch_flops = sum(step_flops(nt, nr, nv, nb, rc) for nt, nr, nv, nb, rc in step_sizes)
    stream = torch.cuda.current_stream()

    batch.run(0, args.warmup)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    try:
        smi_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        smi_id = str(local)
    with ClockSampler(smi_id) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            ev[i][0].record(stream)
            batch.run(args.warmup + i, 1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    for m in members:
        st = m["plan"].sync_status()
        if st != binding.MDC_OK:
            raise RuntimeError(f"device status {binding.status_string(st)}")
    t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    launches = (batch.kernels_per_epoch + 1) * args.steps
    loss_first = [float(m["loss"][0, 0]) for m in members]
    loss_last = [float(m["loss"][args.warmup + args.steps - 1, -1]) for m in members]

    # e2e: every epoch's permutations go host -> device (pinned) before the replay and every member's
    # step losses come back device -> host after it (inputs larger than L2 in both loops: no flush)
    loss_host = [torch.empty_like(m["loss"][0], device="cpu").pin_memory() for m in members]
    h2d = d2h = 0
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(args.steps):
        e = args.warmup + i
        for m, sp in zip(members, setup):
            m["perm"][e % n_perm].copy_(sp["perm_host"][e % n_perm], non_blocking=True)
            h2d += sp["perm_host"][0].numel() * 4
        batch.run(e, 1)
        for m, lh in zip(members, loss_host):
            lh.copy_(m["loss"][e % n_perm], non_blocking=True)
            d2h += lh.numel() * 8
        stream.synchronize()
    t_e2e = time.perf_counter() - e0

    # per-kernel figures of the largest member, from a few profiled steps outside the graph
    big = max(range(len(setup)), key=lambda k: step_flops(setup[k]["nt"], setup[k]["nr"], setup[k]["nv"], setup[k]["nb"],
                                                          setup[k]["reciprocity"]))
    mb, sb = members[big], setup[big]
    plan = mb["plan"]
    binding.mdc_plan_set_profiling(plan.handle, True)
    binding.mdc_plan_stage_times(plan.handle, reset=True)
    for s in range(3):
        ii = mb["perm"][0, s * sb["nb"]:(s + 1) * sb["nb"]]
        binding.smdd_step(plan.handle, mb["X"], mb["U_obs"], ii, mb["alpha"],
                          mb["flags"] | binding.SMDD_KEEP_XHAT | (binding.SMDD_REUSE_XHAT if s else 0))
    stage = binding.mdc_plan_stage_times(plan.handle, reset=True)
    binding.mdc_plan_set_profiling(plan.handle, False)
    if plan.sync_status() != binding.MDC_OK:
        raise RuntimeError("device status after the profiled steps")

    (t_dev, t_e2e, wall), flops_all = combine_ranks([t_dev, t_e2e, wall], epoch_flops * args.steps, dev)
    if rank != 0:
        return None
    peaks, fp64_peak = measured_peaks(dev)
    kern = stage_roofs(peaks, stage, (sb["nt"], sb["nr"], sb["nv"], sb["nb"]), tc, sb["reciprocity"])
    dom = max(kern, key=lambda k: kern[k]["share"])
    roof = dict(kern[dom])
    roof["traffic"] = ncu_traffic(dom, BATCH_WORKLOAD)
    roof["member"] = {k: sb[k] for k in ("nt", "nr", "nv", "ns", "nb")}
    t_roof_epoch = sum(peaks.step_roof_s(nt, nr, nv, nb, rc, tc, rc) for nt, nr, nv, nb, rc in step_sizes)
    ms_epoch = t_dev / args.steps * 1e3
    cfgs, nffts = {}, {}
    for sp in setup:
        key = f"fft{sp['cfg']['fft_variant']}_fwd{sp['cfg']['gemm_fwd']}_adj{sp['cfg']['gemm_adj']}"
        cfgs[key] = cfgs.get(key, 0) + 1
        nk = f"{sp['nt']}:{nfft_for(sp['nt'])}/{sp['nfft_library']}"
        nffts[nk] = nffts.get(nk, 0) + 1
    out = {
        "metric": METRIC, "value": round(flops_all / t_dev / 1e9, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_epoch, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if not tc else "f32 FFTs, bf16x3 (split hi+lo) tensor-core products",
        "data": "synthetic (seeded Ricker/hyperbola generator per member, evaluated on the device; U_obs = GPU forward)",
        "config": {"workload": BATCH_WORKLOAD, "members": len(specs),
                   "largest_member": list(largest_shape(args)) if args.batch_largest else False,
                   "steps_per_epoch_all_members": sum(sp["steps"] for sp in setup), "nb": 32,
                   "precision": args.precision, "a_step_of_this_line": "one epoch of every member (one graph replay)",
                   "branches": batch.n_branches, "kernels_per_epoch": batch.kernels_per_epoch,
                   "epoch_layout": args.batch_mode,
                   "autotuned": bool(args.autotune), "chosen_configs": cfgs,
                   "members_by_nt_nfft_algorithmic_library": nffts,
                   "l2": "inputs larger than L2 (no flush)", "setup_s": round(t_setup, 1),
                   "per_rank": "independent member set, seeds offset by rank (no data-path collective)"},
        "e2e": {"value": round(flops_all / t_e2e / 1e9, 2), "unit": UNIT,
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": int(launches) * world,
        "roofline": roof,
        "kernels_largest_member": kern,
        "step_roofline": {"t_roof_ms_per_epoch": round(t_roof_epoch * 1e3, 3), "t_epoch_ms": round(ms_epoch, 3),
                          "frac": round(t_roof_epoch / (ms_epoch * 1e-3), 4),
                          "definition": ("sum over every step of every member of max(compulsory bytes / HBM, "
                                         "F_gemm / P_gemm + F_fft / P_FP32); P_gemm = "
                                         + ("sustained BF16 tensor rate" if tc else "measured FP32 FMA rate")),
                          "fp32_tflops_measured": round(peaks.fp32 / 1e12, 2),
                          "fp32_tflops_derived": round(peaks.fp32_derived, 2),
                          "bf16_tflops_sustained": round(peaks.bf16 / 1e12, 1),
                          "fp64_tflops_measured": round(fp64_peak, 3)},
        "clocks": clk.summary(),
        "epochs_per_s": round(args.steps / t_dev, 3),
        "wall_s_timed_region": round(wall, 3),
        "loss_first_last_sum": [sum(loss_first), sum(loss_last)],
    }
    # the other epoch layout on the same members, timed the same way (a few epochs): the branch graph
    # against the waves of persistent work-queue kernels
    batch.close()
    other = binding.MDC_BATCH_BRANCHES if mode == binding.MDC_BATCH_QUEUE else binding.MDC_BATCH_QUEUE
    try:
        if other == binding.MDC_BATCH_QUEUE:   # the queue layout runs every product on the tile kernel
            for m in members:
                c = m["plan"].get_config()
                if c["gemm_fwd"] == binding.MDC_GEMM_TC_STREAM:
                    m["plan"].set_config(gemm_fwd=binding.MDC_GEMM_TC)
        b2 = binding.MDCBatch(members, n_branches=args.branches, mode=other)
        b2.run(0, 1)
        k2 = min(args.steps, 5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b2.run(1, k2)
        e1.record(stream)
        torch.cuda.synchronize()
        for m in members:
            if m["plan"].sync_status() != binding.MDC_OK:
                raise RuntimeError("device status after the other epoch layout")
        t_other = e0.elapsed_time(e1) / k2
        out["batch_layouts"] = {
            "timed_layout": args.batch_mode, "timed_ms_per_epoch": round(ms_epoch, 3),
            "other_layout": "queue" if other == binding.MDC_BATCH_QUEUE else "branches",
            "other_ms_per_epoch": round(t_other, 3), "other_epochs_timed": k2,
            "other_kernels_per_epoch": b2.kernels_per_epoch,
            "definition": ("branches: every member's steps as its plan's own launches on parallel graph branches; "
                           "queue: the epoch in waves (step w of every member), each stage one launch per kernel "
                           "family of persistent CTAs taking (problem, tile) items from a device work queue")}
        b2.close()
    except binding.MDCError as e:
        out["batch_layouts"] = {"timed_layout": args.batch_mode, "other_layout_error": str(e)}
    # release the members before the mixed-precision comparison
    for m in members:
        m["plan"].close()
    members.clear()
    torch.cuda.empty_cache()
    if args.fixed_error_epochs > 0:
        out["fixed_error"] = {name.rsplit("_", 1)[-1]: fixed_error_run(args, dev, name, rank)
                              for name in FIXED_ERROR_WORKLOADS}
    # oracle on the host cores: one step of the largest member on a column sample
    val, t_step, k = oracle_member_sample(sb, args.oracle_seconds)
    import oracle
    out["cpu_baseline"] = {"value": round(val, 4), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                           "sample": (f"largest member (nt {sb['nt']}, {sb['nr']} x {sb['nv']}, batch {sb['nb']}): FP64 "
                                      f"direct-sum forward + adjoint of one step on {k} of {sb['nv']} virtual-source "
                                      f"columns, extrapolated linearly in the column count"),
                           "s_per_step_extrapolated": round(t_step, 2)}
    return out


# ------------------------------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ------------------------------------------------------------------------------------------------
def run_reference_batch(args, rank, world):
    """The oracle on the batched workload: each of the W + K steps of this arm times one SGD step of one
    member (members in turn, largest first) on a column sample of about 150 / (W + K) seconds,
    extrapolated to the member's full step; the K timed samples give the epoch-weighted rate
    sum(steps_m F_m) / sum(steps_m t_m) over the members they cover."""
    if rank != 0:
        return None
    import oracle
    specs = synth.batch_members(args.batch_n, seed=1000, largest=largest_shape(args))
    for m in specs:
        m["steps"] = -(-m["ns"] // m["nb"])
    order = sorted(specs, key=lambda m: -step_flops(m["nt"], m["nr"], m["nv"], m["nb"], m["reciprocity"]))
    budget = 150.0 / max(1, args.steps + args.warmup)
    f_tot = t_tot = 0.0
    used = []
    for k in range(args.warmup + args.steps):
        # warm-up samples on the smallest members, timed samples from the largest member on
        m = order[(k - args.warmup) % len(order)] if k >= args.warmup else order[-1 - k % len(order)]
        val, t_step, cols = oracle_member_sample(m, budget, seed=k)
        if k >= args.warmup:
            f_tot += m["steps"] * step_flops(m["nt"], m["nr"], m["nv"], m["nb"], m["reciprocity"])
            t_tot += m["steps"] * t_step
            used.append(f"{m['nt']}/{m['nr']}x{m['nv']}:{cols}")
    val = f_tot / t_tot / 1e9
    epoch_flops = sum(m["steps"] * step_flops(m["nt"], m["nr"], m["nv"], m["nb"], m["reciprocity"]) for m in specs)
    sample = ("each step: FP64 direct-sum forward + adjoint of one SGD step of one member (largest first, in "
              "turn) on a column sample, extrapolated in the column count; epoch-weighted over the members "
              "timed (nt/nr x nv:columns): " + ", ".join(used) + "; ms_per_step = the epoch of all members at "
              "that rate")
    return {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(epoch_flops / (val * 1e9) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "seeded random traces of each member's shape (the direct sums cost the same for any values)",
            "config": {"workload": BATCH_WORKLOAD, "members": len(specs), "nb": 32},
            "cpu_baseline": {"value": round(val, 4), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args, rank, world, w):
    if rank != 0:
        return None
    import oracle
    nt, nr, nv, ns, nb = w["nt"], w["nr"], w["nv"], w["ns"], w["nb"]
    p = make_inputs(w, seed=0)
    D = p.D.astype(np.float32).astype(np.float64)
    X = np.zeros((nv, nr, nt))
    U_obs = oracle.mdc_forward_fft(D, p.X_true.astype(np.float32), np.arange(ns))
    batches = [b for ep in synth.epoch_batches(ns, nb, 2 + (args.steps + args.warmup) // math.ceil(ns / nb),
                                               seed=0) for b in ep]
    # per step: a column sample sized so the whole run stays within a few minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    _, _, _, cores = time_oracle(w, D, X, U_obs, [batches], target_s=0.2, max_cols=2)
    t_tot, f_tot = 0.0, 0.0
    cols_used = []
    per_col = None
    for k in range(args.warmup + args.steps):
        idx = batches[k]
        if per_col is None:
            t0 = time.perf_counter()
            oracle_step_sample(D, X, U_obs, idx, np.arange(1))
            per_col = max(time.perf_counter() - t0, 1e-6)
        ncols = int(max(1, min(nv, budget / per_col)))
        vsel = np.linspace(0, nv - 1, ncols).round().astype(np.int64)
        t0 = time.perf_counter()
        oracle_step_sample(D, X, U_obs, idx, vsel)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            t_tot += dt * nv / ncols
            f_tot += step_flops(nt, nr, nv, len(idx), bool(w["reciprocity"]))
            cols_used.append(ncols)
    val = f_tot / t_tot / 1e9
    sample = (f"each step: FP64 direct-sum forward+adjoint on {min(cols_used)}-{max(cols_used)} of {nv} "
              f"virtual-source columns, extrapolated linearly in the column count")
    return {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_tot / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Ricker/hyperbola generator)",
            "config": {"workload": args.workload, "nt": nt, "nr": nr, "nv": nv, "ns": ns, "nb": nb,
                       "reciprocity": bool(w["reciprocity"])},
            "cpu_baseline": {"value": round(val, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(synth.WORKLOADS) + [BATCH_WORKLOAD])
    ap.add_argument("--autotune", dest="autotune", action="store_true", default=True,
                    help="let the plan autotuner choose the FFT variant and the product kernels (default)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use the plans' default kernel configuration")
    ap.add_argument("--batch-n", type=int, default=48, help=f"{BATCH_WORKLOAD}: number of members")
    ap.add_argument("--batch-largest", type=int, default=1,
                    help=f"{BATCH_WORKLOAD}: 1 = the last member is the fixed largest one (nt 1500, 1200^3)")
    ap.add_argument("--batch-largest-shape", default="1500,1200,1200,1200",
                    help=f"{BATCH_WORKLOAD}: nt,nr,nv,ns of the fixed largest member (a smaller one, with --batch-n 1, "
                         "makes a single-member run small enough for a multi-pass ncu capture)")
    ap.add_argument("--branches", type=int, default=8, help=f"{BATCH_WORKLOAD}: parallel graph branches")
    ap.add_argument("--batch-mode", default="branches", choices=["branches", "queue"],
                    help=f"{BATCH_WORKLOAD}: epoch layout of the timed run (the other one is timed beside it)")
    ap.add_argument("--solver-epochs", type=int, default=0,
                    help="also compare SGD, N-SGD and full-gradient LSQR over this many epochs (model error per epoch)")
    ap.add_argument("--l2", default="auto", choices=["auto", "flush", "none"],
                    help="L2 between timed steps (single problems): auto (default: flush unless a step moves > 4x L2), "
                         "flush, or none; the end-to-end loop follows the same policy")
    ap.add_argument("--fixed-error-epochs", type=int, default=None,
                    help="compare FP32 and BF16x3 products at the same final-model error after this many epochs "
                         f"(default: 50 on {BATCH_WORKLOAD}, where it runs the nt 1024 301 x 301 x 401 workload at "
                         "batch 32 and 64; 0 elsewhere)")
    ap.add_argument("--oracle-seconds", type=float, default=12.0, help="CPU time of the oracle sample for cpu_baseline")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16x3"],
                    help=f"arithmetic of the per-frequency products (the FFTs are FP32 in both); default "
                         f"{DEFAULT_PRECISION} on {BATCH_WORKLOAD}, fp32 elsewhere")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    batch_mode = args.workload == BATCH_WORKLOAD
    if args.precision is None:
        args.precision = DEFAULT_PRECISION if batch_mode else "fp32"
    if args.fixed_error_epochs is None:
        args.fixed_error_epochs = 50 if batch_mode else 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference_batch(args, rank, world) if batch_mode else run_reference(args, rank, world,
                                                                                     workload_dims(args.workload))
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_gpu_batch(args, rank, world) if batch_mode else run_gpu(args, rank, world, workload_dims(args.workload))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
