"""Host-side checks of the C ABI: the library builds, loads, exports every entry point
declared in include/lbve.h, and rejects bad parameters without a GPU."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_12279_gb300 import build, lbve

    build.build()
    return lbve.load()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "lbve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbve_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2009_12279_gb300 import lbve

    so = lbve.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbve_[a-z_0-9]+)", out))
    declared = declared_entry_points()
    assert declared, "no entry points parsed from lbve.h"
    missing = [s for s in declared if s not in exported]
    assert not missing, f"declared but not exported: {missing}"
    assert set(lbve.EXPORTS) == set(declared)
    for s in declared:
        getattr(lib, s)


def test_library_is_built_for_sm_103a():
    from paper_2009_12279_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_default_params_and_memory_estimate(lib):
    from paper_2009_12279_gb300 import lbve

    p = lbve.default_params()
    assert (p.nx, p.ny, p.nz) == (16, 16, 16) and p.pdf_prec == lbve.F32
    p32 = lbve.make_params((512, 512, 512), precision="f32")
    p16 = lbve.make_params((512, 512, 512), precision="f16")
    b32, b16 = lbve.device_bytes(p32), lbve.device_bytes(p16)
    n = 512 ** 3
    # PDFs + stress ping-pong + velocity ping-pong + flags + neighbour masks
    per_cell = 19 * 4 + 12 * 4 + 6 * 4 + 1 + 4
    assert per_cell * n <= b32 <= per_cell * n + 10 ** 7
    assert b16 < b32


@pytest.mark.parametrize("bad", [dict(eta=-1.0), dict(beta=1.0), dict(beta=0.5, lambda_p=0.0),
                                 dict(rho0=0.0), dict(precision=7), dict(block_x=48), dict(fv_terms=16),
                                 dict(fv_terms=-1), dict(giesekus_alpha=-0.1), dict(giesekus_alpha=0.51)])
def test_invalid_parameters_are_rejected_before_any_gpu_work(lib, bad):
    import ctypes as ct

    from paper_2009_12279_gb300 import lbve

    kw = dict(dict(eta=1.0 / 6.0, beta=0.5, lambda_p=100.0, precision="f32"), **bad)
    p = lbve.make_params((8, 8, 8), **kw)
    h = ct.c_void_p()
    rc = lib.lbve_create(ct.byref(p), None, ct.byref(h))
    assert rc == 1 and not h.value
    assert lib.lbve_last_error(None)
    assert lbve.device_bytes(p) == 0


@pytest.mark.parametrize("ok", [dict(fv_terms=4), dict(fv_terms=15), dict(giesekus_alpha=0.5),
                                dict(giesekus_alpha=0.2, fv_terms=9)])
def test_finite_volume_variant_parameters_are_accepted(lib, ok):
    """Variant settings pass validation: the memory estimate (which validates without
    touching a GPU) is that of the plain method."""
    from paper_2009_12279_gb300 import lbve

    base = dict(eta=1.0 / 6.0, beta=0.5, lambda_p=100.0, precision="f32")
    assert lbve.device_bytes(lbve.make_params((8, 8, 8), **base, **ok)) == \
        lbve.device_bytes(lbve.make_params((8, 8, 8), **base)) > 0


def test_status_strings(lib):
    assert lib.lbve_status_string(0) == b"LBVE_OK"
    assert lib.lbve_status_string(4) == b"LBVE_EUNSTABLE"
    assert lib.lbve_status_string(99) == b"LBVE_UNKNOWN"


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2009_12279_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
                assert "lbve_oracle" not in text and "orc_" not in text, f


def test_no_cpu_fallback_without_a_gpu():
    """On a machine without a GPU the product path fails loudly: creating a solve reports
    a CUDA error instead of computing anywhere else."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2009_12279_gb300 import LbveError, Solver

    with pytest.raises(LbveError, match="LBVE_ECUDA|LBVE_ENOMEM"):
        Solver((8, 8, 8), precision="f32", eta=1.0 / 6.0, beta=0.5, lambda_p=100.0)
