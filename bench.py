"""Benchmark of the stochastic MDD hot path: one SGD step (forward MDC on a source batch, residual,
adjoint, reciprocity-preconditioned update) per timed iteration, on synthetic data shaped like the
paper's workloads.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload NAME]

Prints one JSON line (rank 0).  `value` is the algorithmic FLOP rate of the whole job:
F_step = 16 nb nr nv nf (forward + adjoint complex products, 8 real flops per complex MAC)
       + 5 nfft log2(nfft) (nr nv + nb nv) (two real FFTs per model trace and per residual trace,
         2.5 N log2 N flops each), summed over the steps of all ranks, divided by the max over ranks of
the device time of the K timed steps.  L2 is flushed (256 MiB write, outside the per-step CUDA events)
before every timed step; --l2 none / auto run the steps back to back (auto: when a step's own HBM traffic
exceeds four times the L2 size), which measured within 0.5 % of the flushed steps on the default workload.

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

DEFAULT_WORKLOAD = "smdd_nt512_n201_nb16_recip"
METRIC = "MDC fwd+adj GFLOP/s (SMDD step)"
UNIT = "GFLOP/s"


# ------------------------------------------------------------------------------------------------
# work model
# ------------------------------------------------------------------------------------------------
def nfft_for(nt: int) -> int:
    n = 64
    while n < 2 * nt - 1:
        n *= 2
    return n


def step_flops(nt, nr, nv, nb) -> float:
    nfft = nfft_for(nt)
    nf = nfft // 2 + 1
    return 16.0 * nb * nr * nv * nf + 5.0 * nfft * math.log2(nfft) * (nr * nv + nb * nv)


def nf_of(nt: int) -> int:
    return nfft_for(nt) // 2 + 1


def step_bytes_compulsory(nt, nr, nv, nb, recip) -> float:
    nfft = nfft_for(nt)
    nf = nfft // 2 + 1
    b = 2 * nr * nv * nt * 4 + nf * nb * nr * 8 + nb * nv * nt * 4
    if recip:
        b += 2 * nr * nv * nt * 4
    return float(b)


def kernel_work(stage, nt, nr, nv, nb):
    """Algorithmic bytes and flops of one launch of a stage (see the design notes for the derivation)."""
    nfft = nfft_for(nt)
    nf = nfft // 2 + 1
    fft_flops = 2.5 * nfft * math.log2(nfft)
    if stage == "update":      # read Gh, read X, write X, write Xh (fused re-transform)
        return dict(bytes=nv * nr * (2 * nf * 8 + 2 * nt * 4), flops=2 * fft_flops * nv * nr)
    if stage == "cgemm_fwd":   # read Xh, gathered kernel rows, write Uh
        return dict(bytes=nf * (nv * nr + nb * nr + nv * nb) * 8, flops=8.0 * nv * nr * nb * nf)
    if stage == "cgemm_adj":   # read Rh, gathered kernel rows, write Gh
        return dict(bytes=nf * (nv * nb + nb * nr + nv * nr) * 8, flops=8.0 * nv * nr * nb * nf)
    if stage == "residual":    # read Uh, read U_obs rows, write Rh
        return dict(bytes=nb * nv * (2 * nf * 8 + nt * 4), flops=2 * fft_flops * nb * nv)
    if stage == "rfft":        # read X, write Xh
        return dict(bytes=nv * nr * (nt * 4 + nf * 8), flops=fft_flops * nv * nr)
    return dict(bytes=0, flops=0)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 SIMT peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


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
    f = step_flops(w["nt"], w["nr"], w["nv"], len(idx))
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
    res["tier_a_1thread_gflops"] = round(step_flops(w["nt"], w["nr"], w["nv"], len(idx)) / t1 / 1e9, 5)
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
    if args.fixed_error_epochs <= 0 and args.solver_epochs <= 0:
        del X_true

    prec = binding.MDC_PREC_BF16X3 if args.precision == "bf16x3" else binding.MDC_PREC_FP32
    plan = binding.MDCPlan(D, nv, nb_max=nb, precision=prec)
    chosen = plan.autotune(nb, binding.SMDD_RECIPROCITY if recip else 0, reps=5) if args.autotune else plan.get_config()
    sigma2 = plan.sigma2_max(60)
    alpha = 0.5 * 2.0 / sigma2
    flags = (binding.SMDD_RECIPROCITY if recip else 0) | binding.SMDD_KEEP_XHAT
    X = torch.zeros((nv, nr, nt), device=dev)
    n_ep = (args.warmup + args.steps) // math.ceil(ns / nb) + 2
    batches = [b for ep in synth.epoch_batches(ns, nb, n_ep, seed=rank) for b in ep]
    idx_dev = [torch.from_numpy(b).to(dev) for b in batches]
    loss = torch.zeros(len(batches), device=dev, dtype=torch.float64)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)
    # L2 policy: flush before every timed step unless the step's own traffic is far larger than L2
    # (then back-to-back steps, as an SGD run issues them, and the inputs themselves evict L2)
    l2_bytes = 126 * 1024 * 1024
    step_traffic = step_bytes_compulsory(nt, nr, nv, nb, recip) + 4.0 * nf_of(nt) * nv * nr * 8
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

    # timed region: K steps, L2 flushed before each, per-step CUDA events on the launching stream
    binding.mdc_plan_set_profiling(plan.handle, True)
    binding.mdc_plan_stage_times(plan.handle, reset=True)
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
    stage = binding.mdc_plan_stage_times(plan.handle, reset=True)
    binding.mdc_plan_set_profiling(plan.handle, False)
    status = plan.sync_status()
    if status != binding.MDC_OK:
        raise RuntimeError(f"device status {binding.status_string(status)}")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(step_ms) / 1e3
    flops = sum(step_flops(nt, nr, nv, len(batches[args.warmup + i])) for i in range(args.steps))
    losses = loss[: args.warmup + args.steps].cpu().numpy()

    # e2e: the same steps through smdd_step_host with host inputs: every step the plan copies the batch
    # index list and the batch rows of U_obs (pinned) host -> device on its copy stream, overlapping the
    # previous step, and the step's loss comes back device -> host (pinned); the host reads the loss of
    # step k - 1 once step k is queued, and the last one after the loop
    U_host = U_obs.cpu().pin_memory()
    Xe = torch.zeros_like(X)
    idx_host = [torch.from_numpy(np.ascontiguousarray(b, dtype=np.int32)) for b in batches]
    loss_host = torch.zeros(len(batches), dtype=torch.float64).pin_memory()
    h2d = d2h = 0

    def e2e_run(ks, count):
        nonlocal h2d, d2h
        done = []
        for j, k in enumerate(ks):
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

    peaks, peak_src = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    # dominant kernel: largest share of the device time of the timed steps
    st = {k: v for k, v in stage.items() if v[1] > 0 and k in ("rfft", "cgemm_fwd", "residual", "cgemm_adj", "update")}
    dom = max(st, key=lambda k: st[k][0])
    dom_ms = st[dom][0] / st[dom][1]
    kw = kernel_work(dom, nt, nr, nv, nb)
    if dom in ("cgemm_fwd", "cgemm_adj") and args.precision == "fp32":
        peak = fp32_alu_peak_tflops(props.multi_processor_count, peaks.get("sm_max_mhz", 2070.0))
        ach = kw["flops"] / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": ncu_traffic(dom, args.workload),
                "kernel": dom, "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                                             f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz"}
    else:
        peak = float(peaks["hbm_gbs"])
        ach = kw["bytes"] / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": ncu_traffic(dom, args.workload),
                "kernel": dom, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"}
    roof["algorithmic_per_launch"] = kw["bytes"] if roof["bound"] == "hbm" else kw["flops"]
    roof["launch_ms"] = round(dom_ms, 5)
    stage_share = {k: {"ms_per_launch": round(v[0] / v[1], 5), "launches": v[1],
                       "share": round(v[0] / sum(x[0] for x in st.values()), 4)} for k, v in st.items()}

    # step-level roofline: max(compulsory bytes / HBM, flops / FP32 ALU peak)
    # FP32 peak: measured FMA throughput (probe launched after the timed region), lane count x clock beside it
    fp32_derived = fp32_alu_peak_tflops(props.multi_processor_count, peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = binding.alu_peak_tflops(0)
    fp64_peak = binding.alu_peak_tflops(1)
    t_roof = max(step_bytes_compulsory(nt, nr, nv, nb, recip) / (peaks["hbm_gbs"] * 1e9),
                 step_flops(nt, nr, nv, nb) / (fp32_peak * 1e12))
    ms_per_step = t_dev / args.steps * 1e3

    out = {
        "metric": METRIC, "value": round(flops_all / t_dev / 1e9, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f32 FFTs, bf16x3 (split hi+lo) tensor-core products",
        "data": "synthetic (seeded Ricker/hyperbola generator; U_obs = GPU forward of the true model + 5% noise)",
        "config": {"workload": args.workload, "nt": nt, "nr": nr, "nv": nv, "ns": ns, "nb": nb,
                   "nfft": nfft_for(nt), "reciprocity": recip, "precision": args.precision, "solver": "SGD, alpha = 0.5 * 2/sigma^2_max",
                   "l2": ("flushed before every timed step (256 MiB write, outside the step events)" if do_flush else
                          f"inputs larger than L2: no flush, back-to-back steps (per-step traffic "
                          f"{step_traffic / 2**20:.0f} MiB against {l2_bytes / 2**20:.0f} MiB of L2)"),
                   "per_rank": "independent problem replica, seed = rank (no data-path collective)",
                   "autotuned": bool(args.autotune), "kernel_config": chosen},
        "e2e": {"value": round(flops_all / t_e2e / 1e9, 2), "unit": UNIT,
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": int(launches) * world,
        "roofline": roof,
        "stage_share": stage_share,
        "step_roofline": {"t_roof_us": round(t_roof * 1e6, 2), "t_step_us": round(ms_per_step * 1e3, 2),
                          "frac": round(t_roof / (ms_per_step * 1e-3), 4),
                          "definition": "max(compulsory bytes / measured HBM GB/s, algorithmic flops / measured FP32 FMA peak)",
                          "fp32_tflops_measured": round(fp32_peak, 2), "fp32_tflops_derived": round(fp32_derived, 2),
                          "fp64_tflops_measured": round(fp64_peak, 3)},
        "clocks": clocks,
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
    res = {}
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
            if target is not None and ep + 1 >= n_ep and errs[-1] <= target * (1 + 1e-3):
                break
        if plan.sync_status() != binding.MDC_OK:
            raise RuntimeError("device status after the precision comparison")
        res[name] = {"epochs": len(errs), "steps": steps, "model_error": errs[-1], "device_s": round(t, 4),
                     "steps_per_s": round(steps / t, 2), "kernel_config": cfg}
        plan.close()
    res["bf16x3_vs_fp32_steps_per_s"] = round(res["bf16x3"]["steps_per_s"] / res["fp32"]["steps_per_s"], 3)
    res["bf16x3_vs_fp32_time_to_error"] = round(res["fp32"]["device_s"] / res["bf16x3"]["device_s"], 3)
    res["definition"] = ("same batches from X = 0; model error = ||X - X_true|| / ||X_true||; BF16x3 runs until "
                         "its error is within 0.1% of the FP32 error after the FP32 epochs (the two differ by "
                         "rounding only); device time of the steps")
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
BATCH_WORKLOAD = "smdd_batch48_nb32"


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
                                largest=(1500, 1200, 1200, 1200) if args.batch_largest else None)
    prec = binding.MDC_PREC_BF16X3 if args.precision == "bf16x3" else binding.MDC_PREC_FP32
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
        flags = binding.SMDD_RECIPROCITY if m["reciprocity"] else 0
        cfg = plan.autotune(nb, flags, reps=3) if args.autotune else plan.get_config()
        perm = np.stack([np.concatenate(ep) for ep in synth.epoch_batches(ns, nb, n_perm, seed=m["seed"])])
        steps = -(-ns // nb)
        members.append(dict(plan=plan, X=torch.zeros((nv, nr, nt), device=dev), U_obs=U_obs,
                            perm=torch.from_numpy(perm).to(dev), nb=nb, alpha=alpha, flags=flags,
                            loss=torch.zeros((n_perm, steps), device=dev, dtype=torch.float64)))
        setup.append(dict(m, steps=steps, cfg=cfg, perm_host=torch.from_numpy(perm).pin_memory()))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    batch = binding.MDCBatch(members, n_branches=args.branches)
    epoch_flops = sum(step_flops(m["nt"], m["nr"], m["nv"], min(m["nb"], m["ns"] - s * m["nb"]))
                      for m in setup for s in range(m["steps"]))
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
    # step losses come back device -> host after it
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

    # dominant kernel of the largest member, from a few profiled steps outside the graph
    big = max(range(len(setup)), key=lambda k: step_flops(setup[k]["nt"], setup[k]["nr"], setup[k]["nv"], setup[k]["nb"]))
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
    peaks, peak_src = load_peaks()
    st = {k: v for k, v in stage.items() if v[1] > 0 and k in ("cgemm_fwd", "residual", "cgemm_adj", "update")}
    dom = max(st, key=lambda k: st[k][0] / st[k][1])
    dom_ms = st[dom][0] / st[dom][1]
    kw = kernel_work(dom, sb["nt"], sb["nr"], sb["nv"], sb["nb"])
    if dom in ("cgemm_fwd", "cgemm_adj") and args.precision == "bf16x3":
        ach = kw["flops"] / (dom_ms * 1e-3) / 1e12
        pk = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
        roof = {"bound": "tensor", "achieved": round(ach, 2), "peak": pk, "unit": "TFLOP/s", "frac": round(ach / pk, 4),
                "traffic": None, "kernel": dom,
                "peak_source": f"{peak_src} bf16 sustained (algorithmic complex flops, not the 9 split products)"}
    elif dom in ("cgemm_fwd", "cgemm_adj"):
        props = torch.cuda.get_device_properties(dev)
        pk = fp32_alu_peak_tflops(props.multi_processor_count, peaks.get("sm_max_mhz", 2070.0))
        ach = kw["flops"] / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 2), "peak": round(pk, 2), "unit": "TFLOP/s",
                "frac": round(ach / pk, 4), "traffic": None, "kernel": dom, "peak_source": "derived FP32 SIMT peak"}
    else:
        pk = float(peaks["hbm_gbs"])
        ach = kw["bytes"] / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk, "unit": "GB/s", "frac": round(ach / pk, 4),
                "traffic": None, "kernel": dom, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"}
    roof["launch_ms"] = round(dom_ms, 4)
    roof["member"] = {k: sb[k] for k in ("nt", "nr", "nv", "ns", "nb")}
    roof["stage_ms_per_launch"] = {k: round(v[0] / v[1], 4) for k, v in st.items()}

    (t_dev, t_e2e, wall), flops_all = combine_ranks([t_dev, t_e2e, wall], epoch_flops * args.steps, dev)
    if rank != 0:
        return None
    cfgs = {}
    for sp in setup:
        key = f"fft{sp['cfg']['fft_variant']}_fwd{sp['cfg']['gemm_fwd']}_adj{sp['cfg']['gemm_adj']}"
        cfgs[key] = cfgs.get(key, 0) + 1
    out = {
        "metric": METRIC, "value": round(flops_all / t_dev / 1e9, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_dev / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f32 FFTs, bf16x3 (split hi+lo) tensor-core products",
        "data": "synthetic (seeded Ricker/hyperbola generator per member, evaluated on the device; U_obs = GPU forward)",
        "config": {"workload": BATCH_WORKLOAD, "members": len(specs), "largest_member": bool(args.batch_largest),
                   "steps_per_epoch_all_members": sum(sp["steps"] for sp in setup), "nb": 32,
                   "precision": args.precision, "a_step_of_this_line": "one epoch of every member (one graph replay)",
                   "branches": batch.n_branches, "kernels_per_epoch": batch.kernels_per_epoch,
                   "autotuned": bool(args.autotune), "chosen_configs": cfgs,
                   "l2": "inputs larger than L2 (no flush)", "setup_s": round(t_setup, 1),
                   "per_rank": "independent member set, seeds offset by rank (no data-path collective)"},
        "e2e": {"value": round(flops_all / t_e2e / 1e9, 2), "unit": UNIT,
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": int(launches) * world,
        "roofline": roof,
        "clocks": clk.summary(),
        "epochs_per_s": round(args.steps / t_dev, 3),
        "wall_s_timed_region": round(wall, 3),
        "loss_first_last_sum": [sum(loss_first), sum(loss_last)],
    }
    # oracle on the host cores: the smallest member, a column sample of one step
    small = min(specs, key=lambda m: m["nt"] * m["nr"] * m["nv"])
    w = dict(small)
    p = synth.make_problem(w["nt"], w["nr"], w["nv"], w["ns"], dx=w["dx"], n_reflectors=w["n_reflectors"],
                           n_multiples=w["n_multiples"], seed=w["seed"])
    D64 = p.D.astype(np.float32).astype(np.float64)
    Uo = np.zeros((w["ns"], w["nv"], w["nt"]))
    bt = synth.epoch_batches(w["ns"], w["nb"], 1, seed=w["seed"])
    val, t_step, sample, cores = time_oracle(w, D64, np.zeros((w["nv"], w["nr"], w["nt"])), Uo, bt, target_s=10.0)
    out["cpu_baseline"] = {"value": round(val, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"member nt={w['nt']} nr={w['nr']} nv={w['nv']} ns={w['ns']}: " + sample}
    return out


# ------------------------------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ------------------------------------------------------------------------------------------------
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
            f_tot += step_flops(nt, nr, nv, len(idx))
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
    ap.add_argument("--steps", type=int, default=50)
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
    ap.add_argument("--branches", type=int, default=8, help=f"{BATCH_WORKLOAD}: parallel graph branches")
    ap.add_argument("--solver-epochs", type=int, default=0,
                    help="also compare SGD, N-SGD and full-gradient LSQR over this many epochs (model error per epoch)")
    ap.add_argument("--l2", default="flush", choices=["auto", "flush", "none"],
                    help="L2 between timed steps: flush (default), none, or auto (flush unless a step moves > 4x L2; "
                         "measured within 0.5%% of flush on the default workload)")
    ap.add_argument("--fixed-error-epochs", type=int, default=0,
                    help="also compare FP32 and BF16x3 products at the same final-model error after this many epochs")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3"],
                    help="arithmetic of the per-frequency products (the FFTs are FP32 in both)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.workload == BATCH_WORKLOAD:
        if args.impl == "reference":
            ap.error(f"--impl reference times single problems; {BATCH_WORKLOAD} has no reference arm")
        if world > 1:
            import torch
            torch.distributed.init_process_group("nccl")
        out = run_gpu_batch(args, rank, world)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    w = workload_dims(args.workload)
    if args.impl == "reference":
        out = run_reference(args, rank, world, w)
    else:
        if world > 1:
            import torch
            torch.distributed.init_process_group("nccl")
        out = run_gpu(args, rank, world, w)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
