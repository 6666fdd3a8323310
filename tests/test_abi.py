"""C-ABI checks that need no GPU: the library builds, loads, and exports every function that
include/*.h declares; the binding refuses to run without a CUDA device (no CPU fallback)."""
import glob
import os
import re

import pytest
import torch

from paper_2202_04486_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:(?:unsigned|long|signed)\s+)*[A-Za-z_]\w*(?:\s+|\s*\*+\s*)([a-z_]\w*)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("mdc_plan_create", "mdc_forward", "mdc_adjoint", "smdd_step", "mdc_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.EXPORTED) <= set(_declared_functions())


def test_status_strings(lib):
    assert binding.status_string(0) == "MDC_OK"
    assert binding.status_string(3) == "MDC_ERR_INDEX_RANGE"
    assert binding.status_string(99) == "MDC_ERR_UNKNOWN"


def test_null_arguments_rejected_without_touching_the_gpu(lib):
    import ctypes
    h = ctypes.c_void_p()
    # null output pointer / null D: host-side validation, nothing launched
    assert lib.mdc_plan_create(None, 8, 2, 2, 2, 0, 0, 1.0, None, 0, None) == binding.MDC_ERR_INVALID_ARG
    assert lib.mdc_plan_create(ctypes.byref(h), 8, 2, 2, 2, 0, 0, 1.0, None, 0, None) == binding.MDC_ERR_INVALID_ARG
    assert lib.mdc_forward(None, None, None, 1, None, None) == binding.MDC_ERR_INVALID_ARG
    assert lib.mdc_plan_destroy(None) == binding.MDC_OK


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_binding_fails_loudly_without_cuda():
    with pytest.raises(RuntimeError):
        binding.mdc_plan_create(torch.zeros(2, 2, 8), 2)


def test_alu_probe_argument_errors_without_launching(lib):
    import ctypes
    d = ctypes.c_double()
    assert lib.mdc_alu_probe(0, 1, 16, None, ctypes.byref(d), None) == binding.MDC_ERR_INVALID_ARG   # no sink
    assert lib.mdc_alu_probe(2, 1, 16, None, None, None) == binding.MDC_ERR_INVALID_ARG              # unknown kind
    assert lib.mdc_alu_probe(0, 1, 24, ctypes.c_void_p(16), None, None) == binding.MDC_ERR_INVALID_ARG  # iters % 16
    assert lib.mdc_alu_probe(0, 0, 16, ctypes.c_void_p(16), None, None) == binding.MDC_ERR_INVALID_ARG  # no blocks


def test_host_step_argument_errors_without_launching(lib):
    assert lib.smdd_step_host(None, None, None, None, 1, None, None, None) == binding.MDC_ERR_INVALID_ARG


def test_forward_static_shapes_checked_before_any_launch():
    """The allocation-free entry point has no plan to check shapes against: the binding rejects a
    mis-shaped array (or a missing status word) with ValueError before the library or a GPU is touched."""
    D = torch.zeros(5, 3, 8)
    X = torch.zeros(4, 3, 8)
    idx = torch.zeros(2, dtype=torch.int32)
    status = torch.zeros(1, dtype=torch.int32)
    bad = [
        dict(U=torch.zeros(2, 4, 7), dev_status=status),     # U too short in time
        dict(U=torch.zeros(3, 4, 8), dev_status=status),     # U rows != idx.numel()
        dict(U=torch.zeros(2, 4, 8), dev_status=None),       # no status word
    ]
    for kw in bad:
        with pytest.raises(ValueError):
            binding.mdc_forward_static(D, X, idx, **kw)
    with pytest.raises(ValueError):
        binding.mdc_forward_static(D, torch.zeros(4, 2, 8), idx, torch.zeros(2, 4, 8), dev_status=status)
    with pytest.raises(ValueError):
        binding.mdc_forward_static(D[0], X, idx, torch.zeros(2, 4, 8), dev_status=status)


def test_forward_static_requires_status_word(lib):
    import ctypes
    p = ctypes.c_void_p(256)   # never dereferenced: the argument check comes first
    assert lib.mdc_forward_static(8, 2, 2, 2, 1.0, p, p, p, 1, p, None, None) == binding.MDC_ERR_INVALID_ARG


def test_profile_driver_fails_loudly_without_cuda():
    """The profiling driver runs the library's steps only: without a GPU it raises instead of falling back."""
    import torch
    from paper_2202_04486_gb300 import profile_step
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        profile_step.main(["--nt", "8", "--nr", "4", "--nv", "4", "--ns", "4", "--nb", "2"])


def test_binding_constants_equal_the_header():
    """Every status, flag, precision, product-kernel and batch-layout constant the binding passes to the
    library has the value include/smdd.h gives it."""
    text = open(os.path.join(ROOT, "include", "smdd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+((?:MDC|SMDD)_[A-Z0-9_]+)\s+(\d+)", text)}
    values.update({m.group(1): int(m.group(2)) for m in re.finditer(r"\b((?:MDC)_[A-Z0-9_]+)\s*=\s*(\d+)", text)})
    names = [n for n in dir(binding) if re.fullmatch(r"(MDC|SMDD)_[A-Z0-9_]+", n)]
    assert len(names) >= 20
    for n in names:
        assert n in values, f"{n} is not declared in include/smdd.h"
        assert getattr(binding, n) == values[n], n
