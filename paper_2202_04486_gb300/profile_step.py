"""SGD steps of one plan with given sizes and kernel configuration, for kernel timing and profiler captures.

    python -m paper_2202_04486_gb300.profile_step --nt 1500 --nr 1200 --nv 100 --ns 64 --nb 32 \
        [--precision bf16x3|fp32] [--recip] [--symmetric] [--config '{"fft_variant": 0, ...}'] \
        [--steps 3] [--warmup 2] [--stages]

Builds a plan on seeded random kernel traces (the kernels' work does not depend on the values), a model
(symmetrised with --recip) and observed data, runs one step that transforms the model, `warmup` steps that
reuse the kept spectra, and `steps` timed steps (CUDA events); prints one JSON line with the mean device
time per step and, with --stages, the mean time per launch of every stage from the library's own events.
The timed steps make one launch of each stage kernel in order (forward product, residual, adjoint product,
update), so a profiler can select them by launch count.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding, build


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--nt", type=int, default=1500)
    ap.add_argument("--nr", type=int, default=1200)
    ap.add_argument("--nv", type=int, default=100)
    ap.add_argument("--ns", type=int, default=64)
    ap.add_argument("--nb", type=int, default=32)
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp32"])
    ap.add_argument("--recip", action="store_true", help="reciprocity preconditioner (needs nr == nv)")
    ap.add_argument("--symmetric", action="store_true", help="with --recip: the symmetric-model step")
    ap.add_argument("--config", default=None, help="JSON kernel configuration (mdc_plan_set_config fields)")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--stages", action="store_true", help="per-stage times from the library's events")
    a = ap.parse_args(argv)
    if not torch.cuda.is_available():
        raise RuntimeError("profile_step needs a CUDA device")
    build.build()
    binding.load_library()
    dev = torch.device("cuda:0")
    g = torch.Generator(device=dev).manual_seed(0)
    D = torch.randn(a.ns, a.nr, a.nt, device=dev, generator=g) * 0.01
    prec = binding.MDC_PREC_BF16X3 if a.precision == "bf16x3" else binding.MDC_PREC_FP32
    plan = binding.MDCPlan(D, a.nv, nb_max=a.nb, precision=prec)
    if a.config:
        plan.set_config(**json.loads(a.config))
    X = torch.randn(a.nv, a.nr, a.nt, device=dev, generator=g) * 1e-3
    if a.recip:
        X = (0.5 * (X + X.transpose(0, 1))).contiguous()
    U = torch.randn(a.ns, a.nv, a.nt, device=dev, generator=g)
    idx = torch.randperm(a.ns, device=dev, generator=g)[: a.nb].int()
    base = (binding.SMDD_RECIPROCITY if a.recip else 0) | (binding.SMDD_SYMMETRIC if a.symmetric else 0)
    flags = base | binding.SMDD_KEEP_XHAT | binding.SMDD_REUSE_XHAT
    plan.step(X, U, idx, 1e-6, base | binding.SMDD_KEEP_XHAT)
    for _ in range(a.warmup):
        plan.step(X, U, idx, 1e-6, flags)
    torch.cuda.synchronize()
    binding.mdc_plan_set_profiling(plan.handle, a.stages)
    if a.stages:
        binding.mdc_plan_stage_times(plan.handle, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        plan.step(X, U, idx, 1e-6, flags)
    e1.record()
    torch.cuda.synchronize()
    out = {"shape": {"nt": a.nt, "nr": a.nr, "nv": a.nv, "ns": a.ns, "nb": a.nb}, "precision": a.precision,
           "recip": a.recip, "symmetric": a.symmetric, "config": plan.get_config(), "nfft": plan.nfft,
           "ms_per_step": round(e0.elapsed_time(e1) / max(a.steps, 1), 4)}
    if a.stages:
        st = binding.mdc_plan_stage_times(plan.handle)
        out["stage_ms_per_launch"] = {k: round(ms / n, 4) for k, (ms, n) in st.items() if n}
    status = plan.sync_status()
    if status != binding.MDC_OK:
        raise RuntimeError(f"device status {binding.status_string(status)}")
    plan.close()
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
