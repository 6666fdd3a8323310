"""Thin ctypes binding of libsmdd_gb300.so (the C ABI declared in include/smdd.h).

Argument marshalling only: every function here checks the torch tensors it is given (device, dtype,
contiguity, shape), passes their device pointers and the current CUDA stream to the C function of the
same name, and raises MDCError on a non-zero status.  All arithmetic runs in the library's CUDA
kernels; there is no CPU fallback.  If the library is missing or no CUDA device is present, the first
call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmdd_gb300.so")

MDC_OK = 0
MDC_ERR_INVALID_ARG = 1
MDC_ERR_SHAPE = 2
MDC_ERR_INDEX_RANGE = 3
MDC_ERR_OOM = 4
MDC_ERR_CUDA = 5
MDC_ERR_TIMEOUT = 6
MDC_ERR_UNSUPPORTED = 7

SMDD_RECIPROCITY = 1
SMDD_KEEP_XHAT = 2
SMDD_REUSE_XHAT = 4
SMDD_UOBS_GATHERED = 8
SMDD_NESTEROV = 16
SMDD_ADAM = 32
SMDD_SYMMETRIC = 64

MDC_NUM_STAGES = 7

MDC_PREC_FP32 = 0
MDC_PREC_BF16X3 = 1

MDC_GEMM_SIMT = 0
MDC_GEMM_SIMT32 = 1
MDC_GEMM_SIMT64 = 2
MDC_GEMM_TC = 3
MDC_GEMM_GEMV = 4
MDC_GEMM_TC_STREAM = 5

MDC_BATCH_BRANCHES = 0
MDC_BATCH_QUEUE = 1

EXPORTED = (
    "mdc_plan_create", "mdc_plan_destroy", "mdc_plan_info", "mdc_plan_sigma2_max", "mdc_forward",
    "mdc_adjoint", "smdd_step", "mdc_plan_sync_status", "mdc_status_string", "mdc_plan_set_profiling",
    "mdc_plan_stage_times", "mdc_stage_name", "mdc_plan_launch_count", "mdc_forward_static",
    "mdc_plan_get_config", "mdc_plan_set_config", "mdc_plan_autotune", "smdd_step_ex", "smdd_lsqr", "mdc_plan_set_band",
    "mdc_batch_create", "mdc_batch_run", "mdc_batch_info", "mdc_batch_destroy", "mdc_alu_probe",
    "smdd_step_host", "mdc_plan_set_wait_probe", "mdc_batch_create_ex",
)


class MDCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class smdd_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("flags", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class smdd_step_ex_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("flags", ctypes.c_int), ("mu", ctypes.c_float), ("t", ctypes.c_int),
                ("V", ctypes.c_void_p), ("mute", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("reserved", ctypes.c_int)]


class mdc_config(ctypes.Structure):
    _fields_ = [("fft_variant", ctypes.c_int), ("gemm_fwd", ctypes.c_int), ("gemm_adj", ctypes.c_int),
                ("fft_prefetch", ctypes.c_int), ("reserved", ctypes.c_int * 4)]

    def as_dict(self) -> dict:
        return {"fft_variant": self.fft_variant, "gemm_fwd": self.gemm_fwd, "gemm_adj": self.gemm_adj,
                "fft_prefetch": self.fft_prefetch}


class smdd_member(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("X", ctypes.c_void_p), ("U_obs", ctypes.c_void_p),
                ("perm", ctypes.c_void_p), ("n_perm", ctypes.c_int), ("nb", ctypes.c_int), ("alpha", ctypes.c_float),
                ("flags", ctypes.c_int), ("loss", ctypes.c_void_p), ("loss_rows", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the in-tree library (no GPU needed to load it).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2202_04486_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i, f, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
    lib.mdc_plan_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i, f, vp, i, vp]
    lib.mdc_plan_destroy.argtypes = [vp]
    lib.mdc_plan_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.mdc_plan_sigma2_max.argtypes = [vp, i, ctypes.POINTER(d), vp]
    lib.mdc_forward.argtypes = [vp, vp, vp, i, vp, vp]
    lib.mdc_adjoint.argtypes = [vp, vp, vp, i, vp, vp]
    lib.smdd_step.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(smdd_params), vp, vp]
    lib.mdc_plan_sync_status.argtypes = [vp]
    lib.mdc_status_string.argtypes = [i]
    lib.mdc_status_string.restype = ctypes.c_char_p
    lib.mdc_plan_set_profiling.argtypes = [vp, i]
    lib.mdc_plan_stage_times.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong), i]
    lib.mdc_stage_name.argtypes = [i]
    lib.mdc_stage_name.restype = ctypes.c_char_p
    lib.mdc_forward_static.argtypes = [i, i, i, i, f, vp, vp, vp, i, vp, vp, vp]
    lib.smdd_step_ex.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(smdd_step_ex_params), vp, vp]
    lib.smdd_lsqr.argtypes = [vp, vp, vp, i, i, vp, vp, vp]
    lib.mdc_plan_set_band.argtypes = [vp, i]
    lib.mdc_plan_get_config.argtypes = [vp, ctypes.POINTER(mdc_config)]
    lib.mdc_plan_set_config.argtypes = [vp, ctypes.POINTER(mdc_config)]
    lib.mdc_plan_autotune.argtypes = [vp, i, i, i, ctypes.POINTER(mdc_config), vp]
    lib.mdc_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(smdd_member), i, i, vp]
    lib.mdc_batch_create_ex.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(smdd_member), i, i, i, vp]
    lib.mdc_batch_run.argtypes = [vp, ctypes.c_longlong, i, vp]
    lib.mdc_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i)]
    lib.mdc_batch_destroy.argtypes = [vp]
    lib.mdc_plan_launch_count.argtypes = [vp]
    lib.mdc_alu_probe.argtypes = [i, i, i, vp, ctypes.POINTER(d), vp]
    lib.smdd_step_host.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(smdd_params), vp, vp]
    lib.mdc_plan_set_wait_probe.argtypes = [vp, ctypes.c_longlong]
    lib.mdc_plan_launch_count.restype = ctypes.c_longlong
    for name in EXPORTED:
        if name not in ("mdc_status_string", "mdc_stage_name", "mdc_plan_launch_count"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load_library().mdc_status_string(int(status)).decode()
    except ImportError:
        return f"status {status}"


def _check(rc: int, where: str) -> None:
    if rc != MDC_OK:
        raise MDCError(rc, where)


def _stream_ptr(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype, shape=None) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _shape(t: torch.Tensor, name: str, shape) -> None:
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the stochastic MDD kernels run only on the GPU")


# ------------------------------------------------------------------------------------------------
# functions with the C names (plan handles are plain integers)
# ------------------------------------------------------------------------------------------------
def mdc_plan_create(D: torch.Tensor, nv: int, nb_max: int = 0, nfft: int = 0, scale: float = 1.0,
                    precision: int = 0, stream=None) -> int:
    _require_cuda()
    lib = load_library()
    ns, nr, nt = D.shape
    h = ctypes.c_void_p()
    _check(lib.mdc_plan_create(ctypes.byref(h), nt, nr, nv, ns, nb_max, nfft, float(scale),
                               _dev(D, "D", torch.float32), precision, _stream_ptr(stream)), "mdc_plan_create")
    return h.value


def mdc_plan_destroy(plan: int) -> None:
    _check(load_library().mdc_plan_destroy(ctypes.c_void_p(plan)), "mdc_plan_destroy")


def mdc_plan_info(plan: int) -> tuple[int, int]:
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load_library().mdc_plan_info(ctypes.c_void_p(plan), ctypes.byref(a), ctypes.byref(b)), "mdc_plan_info")
    return a.value, b.value


def mdc_plan_sigma2_max(plan: int, n_iter: int = 60, stream=None) -> float:
    out = ctypes.c_double()
    _check(load_library().mdc_plan_sigma2_max(ctypes.c_void_p(plan), n_iter, ctypes.byref(out), _stream_ptr(stream)),
           "mdc_plan_sigma2_max")
    return out.value


def mdc_forward(plan: int, X: torch.Tensor, idx: torch.Tensor, U: torch.Tensor, stream=None) -> torch.Tensor:
    nb = idx.numel()
    _check(load_library().mdc_forward(ctypes.c_void_p(plan), _dev(X, "X", torch.float32), _dev(idx, "idx", torch.int32),
                                      nb, _dev(U, "U", torch.float32), _stream_ptr(stream)), "mdc_forward")
    return U


def mdc_adjoint(plan: int, R: torch.Tensor, idx: torch.Tensor, G: torch.Tensor, stream=None) -> torch.Tensor:
    nb = idx.numel()
    _check(load_library().mdc_adjoint(ctypes.c_void_p(plan), _dev(R, "R", torch.float32), _dev(idx, "idx", torch.int32),
                                      nb, _dev(G, "G", torch.float32), _stream_ptr(stream)), "mdc_adjoint")
    return G


def smdd_step(plan: int, X: torch.Tensor, U_obs: torch.Tensor, idx: torch.Tensor, alpha: float, flags: int = 0,
              loss: torch.Tensor | None = None, stream=None) -> None:
    p = smdd_params(float(alpha), int(flags))
    lp = ctypes.c_void_p(0) if loss is None else _dev(loss, "loss", torch.float64)
    _check(load_library().smdd_step(ctypes.c_void_p(plan), _dev(X, "X", torch.float32),
                                    _dev(U_obs, "U_obs", torch.float32), _dev(idx, "idx", torch.int32), idx.numel(),
                                    ctypes.byref(p), lp, _stream_ptr(stream)), "smdd_step")


def _host(t: torch.Tensor, name: str, dtype) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def smdd_step_host(plan: int, X: torch.Tensor, U_obs_host: torch.Tensor, idx_host: torch.Tensor, alpha: float,
                   flags: int = 0, loss_host: torch.Tensor | None = None, stream=None) -> None:
    """SGD step with the batch taken from host memory: U_obs_host [ns][nv][nt] float32 (pinned for
    asynchronous copies), idx_host int32 [nb] (CPU), loss_host a CPU float64 tensor whose first element
    receives 1/2 ||R||^2 once the stream has run the step (pinned for an asynchronous copy), or None."""
    p = smdd_params(float(alpha), int(flags))
    lp = ctypes.c_void_p(0) if loss_host is None else _host(loss_host, "loss_host", torch.float64)
    _check(load_library().smdd_step_host(ctypes.c_void_p(plan), _dev(X, "X", torch.float32),
                                         _host(U_obs_host, "U_obs_host", torch.float32),
                                         _host(idx_host, "idx_host", torch.int32), idx_host.numel(), ctypes.byref(p), lp,
                                         _stream_ptr(stream)), "smdd_step_host")


def smdd_step_ex(plan: int, X: torch.Tensor, U_obs: torch.Tensor, idx: torch.Tensor, alpha: float, flags: int = 0,
                 V: torch.Tensor | None = None, mu: float = 0.0, mute: torch.Tensor | None = None,
                 loss: torch.Tensor | None = None, stream=None, S: torch.Tensor | None = None, t: int = 0,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """N-SGD (flags with SMDD_NESTEROV and a velocity V), Adam (SMDD_ADAM, moments V and S, step count t
    from 1) and/or the causality mute (int32 [nv][nr])."""
    adam = bool(flags & SMDD_ADAM)
    p = smdd_step_ex_params(float(alpha), int(flags), float(mu), int(t) if adam else 0,
                            None if V is None else _dev(V, "V", torch.float32, tuple(X.shape)).value,
                            None if mute is None else _dev(mute, "mute", torch.int32, (X.shape[0], X.shape[1])).value,
                            None if S is None else _dev(S, "S", torch.float32, tuple(X.shape)).value,
                            float(beta1) if adam else 0.0, float(beta2) if adam else 0.0, float(eps) if adam else 0.0, 0)
    lp = ctypes.c_void_p(0) if loss is None else _dev(loss, "loss", torch.float64)
    _check(load_library().smdd_step_ex(ctypes.c_void_p(plan), _dev(X, "X", torch.float32),
                                       _dev(U_obs, "U_obs", torch.float32), _dev(idx, "idx", torch.int32), idx.numel(),
                                       ctypes.byref(p), lp, _stream_ptr(stream)), "smdd_step_ex")


def smdd_lsqr(plan: int, X: torch.Tensor, U_obs: torch.Tensor, n_iter: int, flags: int = 0,
              mute: torch.Tensor | None = None, norms: torch.Tensor | None = None, stream=None) -> None:
    """Full-gradient LSQR on every source (the plan needs nb_max >= ns); X holds the start and the result."""
    mp = ctypes.c_void_p(0) if mute is None else _dev(mute, "mute", torch.int32, (X.shape[0], X.shape[1]))
    npp = ctypes.c_void_p(0) if norms is None else _dev(norms, "norms", torch.float64, (n_iter + 1,))
    _check(load_library().smdd_lsqr(ctypes.c_void_p(plan), _dev(X, "X", torch.float32),
                                    _dev(U_obs, "U_obs", torch.float32), int(n_iter), int(flags), mp, npp,
                                    _stream_ptr(stream)), "smdd_lsqr")


def mdc_plan_set_wait_probe(plan: int, cycles: int) -> None:
    """Failure-path check of the tensor-core kernels' bounded waits (0 = off); see include/smdd.h."""
    _check(load_library().mdc_plan_set_wait_probe(ctypes.c_void_p(plan), int(cycles)), "mdc_plan_set_wait_probe")


def mdc_plan_sync_status(plan: int) -> int:
    return int(load_library().mdc_plan_sync_status(ctypes.c_void_p(plan)))


def mdc_plan_set_profiling(plan: int, enable: bool) -> None:
    _check(load_library().mdc_plan_set_profiling(ctypes.c_void_p(plan), int(bool(enable))), "mdc_plan_set_profiling")


def mdc_plan_stage_times(plan: int, reset: bool = False) -> dict:
    lib = load_library()
    ms = (ctypes.c_double * MDC_NUM_STAGES)()
    n = (ctypes.c_longlong * MDC_NUM_STAGES)()
    _check(lib.mdc_plan_stage_times(ctypes.c_void_p(plan), ms, n, int(reset)), "mdc_plan_stage_times")
    return {lib.mdc_stage_name(s).decode(): (ms[s], n[s]) for s in range(MDC_NUM_STAGES)}


def mdc_plan_launch_count(plan: int) -> int:
    return int(load_library().mdc_plan_launch_count(ctypes.c_void_p(plan)))


def mdc_alu_probe(kind: int, blocks: int, iters: int, sink: torch.Tensor, stream=None) -> float:
    """Launch the FMA throughput probe (kind 0 FP32, 1 FP64) on `stream`; returns its flop count."""
    need = torch.float32 if kind == 0 else torch.float64
    if sink.dtype != need or not sink.is_cuda or sink.numel() < blocks * 256:
        raise MDCError(MDC_ERR_INVALID_ARG, "mdc_alu_probe")
    fl = ctypes.c_double()
    _check(load_library().mdc_alu_probe(kind, blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(fl),
                                        _stream_ptr(stream)), "mdc_alu_probe")
    return fl.value


def alu_peak_tflops(kind: int = 0, iters: int | None = None, repeats: int = 5) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (median of `repeats` timed launches after
    two warm-up launches; CUDA events on the launch stream).  Blocks: 8 per SM (64 warps per SM)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = 8 * sms
    if iters is None:
        iters = 65536 if kind == 0 else 2048
    sink = torch.empty(blocks * 256, device="cuda", dtype=torch.float32 if kind == 0 else torch.float64)
    st = torch.cuda.current_stream()
    for _ in range(2):
        mdc_alu_probe(kind, blocks, iters, sink, st)
    times = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        flops = mdc_alu_probe(kind, blocks, iters, sink, st)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    times.sort()
    return flops / times[len(times) // 2] / 1e12


def _static_shapes(D, X, idx, U, dev_status) -> tuple[int, int, int, int, int]:
    """Shapes of an mdc_forward_static call, checked before anything reaches the library: the entry
    point has no plan to check them against, and a wrong size would make its kernels read or write
    outside the caller's arrays.  Returns (nt, nr, nv, ns, nb)."""
    if D.dim() != 3:
        raise ValueError(f"D must be [ns][nr][nt], got shape {tuple(D.shape)}")
    ns, nr, nt = D.shape
    if idx.dim() != 1 or idx.numel() < 1:
        raise ValueError(f"idx must be a non-empty 1-D tensor, got shape {tuple(idx.shape)}")
    if X.dim() != 3 or tuple(X.shape[1:]) != (nr, nt):
        raise ValueError(f"X has shape {tuple(X.shape)}, expected (nv, {nr}, {nt})")
    nv, nb = X.shape[0], idx.numel()
    if tuple(U.shape) != (nb, nv, nt):
        raise ValueError(f"U has shape {tuple(U.shape)}, expected {(nb, nv, nt)}")
    if dev_status is None or dev_status.numel() != 1:
        raise ValueError("dev_status must be a one-element int32 tensor (index errors are reported there)")
    return nt, nr, nv, ns, nb


def mdc_forward_static(D: torch.Tensor, X: torch.Tensor, idx: torch.Tensor, U: torch.Tensor, scale: float = 1.0,
                       dev_status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Forward MDC through the allocation-free entry point (no plan; intermediates in the library's
    static device scratch).  D [ns][nr][nt], X [nv][nr][nt], idx int32 [nb], U [nb][nv][nt]; dev_status
    a device int32 scalar the caller zeroes, set to 1 when an index lies outside [0, ns)."""
    nt, nr, nv, ns, nb = _static_shapes(D, X, idx, U, dev_status)
    _require_cuda()
    _check(load_library().mdc_forward_static(nt, nr, nv, ns, float(scale), _dev(D, "D", torch.float32),
                                             _dev(X, "X", torch.float32), _dev(idx, "idx", torch.int32), nb,
                                             _dev(U, "U", torch.float32), _dev(dev_status, "dev_status", torch.int32),
                                             _stream_ptr(stream)), "mdc_forward_static")
    return U


def mdc_plan_get_config(plan: int) -> dict:
    c = mdc_config()
    _check(load_library().mdc_plan_get_config(ctypes.c_void_p(plan), ctypes.byref(c)), "mdc_plan_get_config")
    return c.as_dict()


def mdc_plan_set_config(plan: int, fft_variant: int = 0, gemm_fwd: int = MDC_GEMM_SIMT,
                        gemm_adj: int = MDC_GEMM_SIMT, fft_prefetch: int = 0) -> None:
    c = mdc_config(int(fft_variant), int(gemm_fwd), int(gemm_adj), int(fft_prefetch))
    _check(load_library().mdc_plan_set_config(ctypes.c_void_p(plan), ctypes.byref(c)), "mdc_plan_set_config")


def mdc_plan_autotune(plan: int, nb: int, flags: int = 0, reps: int = 5, stream=None) -> dict:
    c = mdc_config()
    _check(load_library().mdc_plan_autotune(ctypes.c_void_p(plan), int(nb), int(flags), int(reps), ctypes.byref(c),
                                            _stream_ptr(stream)), "mdc_plan_autotune")
    return c.as_dict()


class MDCBatch:
    """Many independent problems, whole SGD epochs replayed from one captured CUDA graph.

    members: list of dicts with keys plan (MDCPlan), X, U_obs, perm (int32 [n_perm][ns]), nb, alpha,
    flags (0, SMDD_RECIPROCITY, or SMDD_RECIPROCITY | SMDD_SYMMETRIC for a model that starts symmetric),
    loss (float64 [loss_rows][steps] or None).  The tensors must stay
    alive (and at the same addresses) while the batch lives; this object keeps references to them.
    mode: MDC_BATCH_BRANCHES (members on n_branches graph branches) or MDC_BATCH_QUEUE (waves of
    persistent kernels with device work queues; split-BF16 plans with tensor-core products).
    """

    def __init__(self, members: list, n_branches: int = 8, stream=None, mode: int = MDC_BATCH_BRANCHES):
        _require_cuda()
        lib = load_library()
        arr = (smdd_member * len(members))()
        self._keep = []
        self.steps = []
        for k, m in enumerate(members):
            plan = m["plan"]
            X, U, perm = m["X"], m["U_obs"], m["perm"]
            _dev(X, "X", torch.float32, (plan.nv, plan.nr, plan.nt))
            _dev(U, "U_obs", torch.float32, (plan.ns, plan.nv, plan.nt))
            if perm.dim() != 2 or perm.shape[1] != plan.ns:
                raise ValueError("perm must be [n_perm][ns]")
            _dev(perm, "perm", torch.int32)
            nb = int(m["nb"])
            steps = -(-plan.ns // nb)
            loss = m.get("loss")
            if loss is not None:
                if loss.dim() != 2 or loss.shape[1] != steps:
                    raise ValueError(f"loss must be [loss_rows][{steps}]")
                _dev(loss, "loss", torch.float64)
            arr[k].plan = plan.handle
            arr[k].X = X.data_ptr()
            arr[k].U_obs = U.data_ptr()
            arr[k].perm = perm.data_ptr()
            arr[k].n_perm = perm.shape[0]
            arr[k].nb = nb
            arr[k].alpha = float(m["alpha"])
            arr[k].flags = int(m.get("flags", 0))
            arr[k].loss = 0 if loss is None else loss.data_ptr()
            arr[k].loss_rows = 0 if loss is None else loss.shape[0]
            self._keep.append((plan, X, U, perm, loss))
            self.steps.append(steps)
        h = ctypes.c_void_p()
        _check(lib.mdc_batch_create_ex(ctypes.byref(h), arr, len(members), int(mode), int(n_branches),
                                       _stream_ptr(stream)), "mdc_batch_create_ex")
        self.mode = int(mode)
        self.handle = h.value
        kpe, nbr = ctypes.c_longlong(), ctypes.c_int()
        _check(lib.mdc_batch_info(ctypes.c_void_p(self.handle), ctypes.byref(kpe), ctypes.byref(nbr)), "mdc_batch_info")
        self.kernels_per_epoch, self.n_branches = kpe.value, nbr.value

    def run(self, first_epoch: int, n_epochs: int = 1, stream=None) -> None:
        _check(load_library().mdc_batch_run(ctypes.c_void_p(self.handle), int(first_epoch), int(n_epochs),
                                            _stream_ptr(stream)), "mdc_batch_run")

    def close(self):
        if getattr(self, "handle", None):
            _check(load_library().mdc_batch_destroy(ctypes.c_void_p(self.handle)), "mdc_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------------------
# convenience object
# ------------------------------------------------------------------------------------------------
class MDCPlan:
    """Owns one C plan: D is transformed once at construction; the methods wrap the C calls."""

    def __init__(self, D: torch.Tensor, nv: int, nb_max: int = 0, nfft: int = 0, scale: float = 1.0, stream=None,
                 precision: int = MDC_PREC_FP32):
        self.ns, self.nr, self.nt = D.shape
        self.nv = nv
        self.nb_max = nb_max or self.ns
        self.precision = precision
        self.handle = mdc_plan_create(D, nv, nb_max, nfft, scale, precision, stream)
        self.nfft, self.nf = mdc_plan_info(self.handle)
        self.device = D.device

    def close(self):
        if getattr(self, "handle", None):
            mdc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sigma2_max(self, n_iter: int = 60) -> float:
        return mdc_plan_sigma2_max(self.handle, n_iter)

    def _model(self, X, name="X"):
        _shape(X, name, (self.nv, self.nr, self.nt))

    def _data(self, U, nb, name):
        _shape(U, name, (nb, self.nv, self.nt))

    def forward(self, X: torch.Tensor, idx: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._model(X)
        if out is None:
            out = torch.empty((idx.numel(), self.nv, self.nt), device=X.device, dtype=torch.float32)
        self._data(out, idx.numel(), "out")
        return mdc_forward(self.handle, X, idx, out)

    def adjoint(self, R: torch.Tensor, idx: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._data(R, idx.numel(), "R")
        if out is None:
            out = torch.empty((self.nv, self.nr, self.nt), device=R.device, dtype=torch.float32)
        self._model(out, "out")
        return mdc_adjoint(self.handle, R, idx, out)

    def _step_shapes(self, X, U_obs, idx, flags):
        self._model(X)
        self._data(U_obs, idx.numel() if flags & SMDD_UOBS_GATHERED else self.ns, "U_obs")

    def step(self, X, U_obs, idx, alpha, flags=0, loss=None):
        self._step_shapes(X, U_obs, idx, flags)
        smdd_step(self.handle, X, U_obs, idx, alpha, flags, loss)

    def step_nsgd(self, X, V, U_obs, idx, alpha, mu=0.9, flags=0, mute=None, loss=None):
        """N-SGD step (Nesterov momentum, velocity V) with the optional causality mute."""
        self._step_shapes(X, U_obs, idx, flags)
        smdd_step_ex(self.handle, X, U_obs, idx, alpha, flags | SMDD_NESTEROV, V=V, mu=mu, mute=mute, loss=loss)

    def step_adam(self, X, M, V, U_obs, idx, alpha, t, beta1=0.9, beta2=0.999, eps=1e-8, flags=0, mute=None, loss=None):
        """Adam step t (from 1) with first / second moments M, V and the optional causality mute."""
        self._step_shapes(X, U_obs, idx, flags)
        smdd_step_ex(self.handle, X, U_obs, idx, alpha, flags | SMDD_ADAM, V=M, mute=mute, loss=loss, S=V, t=t,
                     beta1=beta1, beta2=beta2, eps=eps)

    def lsqr(self, X, U_obs, n_iter, flags=0, mute=None, norms=None):
        """Full-gradient LSQR over every source (the plan needs nb_max >= ns); X: start in, solution out."""
        smdd_lsqr(self.handle, X, U_obs, n_iter, flags, mute, norms)

    def sync_status(self) -> int:
        return mdc_plan_sync_status(self.handle)

    def get_config(self) -> dict:
        return mdc_plan_get_config(self.handle)

    def set_config(self, **cfg) -> None:
        cur = self.get_config()
        cur.update(cfg)
        mdc_plan_set_config(self.handle, **cur)

    def set_band(self, nf_active: int) -> None:
        """Only bins f < nf_active take part in the products (0: every bin)."""
        _check(load_library().mdc_plan_set_band(ctypes.c_void_p(self.handle), int(nf_active)), "mdc_plan_set_band")

    def autotune(self, nb: int, flags: int = 0, reps: int = 5) -> dict:
        return mdc_plan_autotune(self.handle, nb, flags, reps)
