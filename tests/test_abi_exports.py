"""CPU checks of the C ABI: the library loads and exports every declared entry point."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(cdmpt_[A-Za-z0-9_]+)\s*\(", txt))
    return names


def test_header_declares_boundary():
    d = _declared()
    for name in ("cdmpt_create", "cdmpt_set_H", "cdmpt_solve", "cdmpt_destroy"):
        assert name in d


def test_library_exports_every_declared_symbol(cdmpt_lib):
    import ctypes
    L = ctypes.CDLL(cdmpt_lib.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    assert set(cdmpt_lib.EXPORTS) == _declared()


def test_library_is_built_for_sm103a_only():
    """Every translation unit is compiled with the single sm_103a target (build flags)."""
    from paper_1503_07037_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_and_defaults(cdmpt_lib):
    assert cdmpt_lib.version() == 0x1
    o = cdmpt_lib.default_opts()
    assert o.precision == cdmpt_lib.FP32 and o.cg_maxit > 0 and o.mu_maxit > 0


def test_create_rejects_bad_options(cdmpt_lib):
    o = cdmpt_lib.default_opts()
    o.precision = 17
    with pytest.raises(cdmpt_lib.CdmptError):
        cdmpt_lib.create(o)


def test_no_cpu_fallback_without_gpu(cdmpt_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(cdmpt_lib.CdmptError) as e:
        cdmpt_lib.Handle()
    assert e.value.status == 6   # ERR_CUDA: the library has no host path


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1503_07037_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


@pytest.mark.parametrize("flag", ["fd_exact", "grand_canonical"])
def test_batch_refuses_options_it_does_not_implement(cdmpt_lib, flag):
    """The batched path solves the canonical problem from the linear start only; the host-side
    option check refuses the rest before any device call."""
    with pytest.raises(cdmpt_lib.CdmptError) as e:
        cdmpt_lib.Batch([8, 12], 1, **{flag: 1})
    assert e.value.status == 8   # ERR_UNSUPPORTED


@pytest.mark.parametrize("case", ["fp64", "bf16", "simt", "negative", "nan"])
def test_screening_option_checks(cdmpt_lib, case):
    """screen_tau > 0 needs FP32 storage and a TF32 tensor-core engine; it must be >= 0."""
    import math
    o = cdmpt_lib.default_opts()
    o.screen_tau = 1e-6
    if case == "fp64":
        o.precision = cdmpt_lib.FP64
    elif case == "bf16":
        o.precision = cdmpt_lib.MIXED_BF16
    elif case == "simt":
        o.gemm_engine = cdmpt_lib.GEMM_SIMT
    elif case == "negative":
        o.screen_tau = -1.0
    else:
        o.screen_tau = math.nan
    with pytest.raises(cdmpt_lib.CdmptError) as e:
        cdmpt_lib.create(o)
    assert e.value.status == 1   # ERR_ARG, before any device call
