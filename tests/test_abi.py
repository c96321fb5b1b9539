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
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbve(?:2d)?_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    from paper_2009_12279_gb300 import lbve

    so = lbve.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbve(?:2d)?_[a-z_0-9]+)", out))
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
                                 dict(fv_terms=-1), dict(giesekus_alpha=-0.1), dict(giesekus_alpha=0.51),
                                 dict(schedule=4), dict(schedule=-1)])
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


def test_binding_constants_match_the_header():
    """The Python binding's constants and parameter struct follow include/lbve.h."""
    import ctypes as ct
    import re

    from paper_2009_12279_gb300 import lbve

    hdr = open(os.path.join(ROOT, "include", "lbve.h")).read()
    defs = {m.group(1): m.group(2) for m in re.finditer(r"^#define (LBVE_\w+) (\S+)", hdr, re.M)}
    pairs = {"LBVE_FV_FLUX": lbve.FV_FLUX, "LBVE_FV_SOURCE": lbve.FV_SOURCE, "LBVE_FV_CTU": lbve.FV_CTU,
             "LBVE_FV_DIVU": lbve.FV_DIVU, "LBVE_SCHED_AUTO": lbve.SCHED_AUTO, "LBVE_SCHED_SPLIT": lbve.SCHED_SPLIT,
             "LBVE_SCHED_FUSED": lbve.SCHED_FUSED, "LBVE_SCHED_PIPELINED": lbve.SCHED_PIPELINED,
             "LBVE_FLAG_FLUID": lbve.FLAG_FLUID,
             "LBVE_FLAG_NOSLIP": lbve.FLAG_NOSLIP, "LBVE_FLAG_WALL0": lbve.FLAG_WALL0,
             "LBVE_FLAG_PARTICLE0": lbve.FLAG_PARTICLE0, "LBVE_LB_CELLS": lbve.LB_CELLS,
             "LBVE_LB_ROWS": lbve.LB_ROWS, "LBVE_FV_TILES": lbve.FV_TILES, "LBVE_FV_PAIRS": lbve.FV_PAIRS}
    for name, value in pairs.items():
        assert int(defs[name]) == value, name
    m = re.search(r"^#define LBVE_NOALLOC_MAX_CELLS \(1 << (\d+)\)", hdr, re.M)
    assert m and 1 << int(m.group(1)) == lbve.NOALLOC_MAX_CELLS
    # lbve_params field order and types, as declared
    body = re.search(r"typedef struct \{(.*?)\} lbve_params;", hdr, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        for nm in names.split(","):
            nm = nm.strip()
            fields.append((re.sub(r"\[.*\]", "", nm), ctype, "[" in nm))
    py = [(f[0], f[1]) for f in lbve.Params._fields_]
    assert [f[0] for f in fields] == [p[0] for p in py]
    for (name, ctype, is_array), (_, pytype) in zip(fields, py):
        base = pytype._type_ if is_array else pytype
        assert base == {"int": ct.c_int, "double": ct.c_double}[ctype], name


def test_noalloc_validates_on_the_host(lib):
    """lbve_step_noalloc rejects, before any CUDA call: the fused schedule (it runs the
    split kernels only), grids beyond its fixed scratch, and NULL buffers."""
    from paper_2009_12279_gb300 import lbve

    fused = lbve.make_params((8, 8, 8), precision="f32", schedule=lbve.SCHED_FUSED)
    with pytest.raises(lbve.LbveError, match="split schedule only"):
        lbve.step_noalloc(fused, 1, 1, 1, 1, nsteps=1)
    big = lbve.make_params((128, 128, 64), precision="f32")
    with pytest.raises(lbve.LbveError, match="LBVE_NOALLOC_MAX_CELLS"):
        lbve.step_noalloc(big, 1, 1, 1, 1, nsteps=1)
    ok = lbve.make_params((8, 8, 8), precision="f32", schedule=lbve.SCHED_SPLIT)
    with pytest.raises(lbve.LbveError, match="NULL"):
        lbve.step_noalloc(ok, 0, 1, 1, 1, nsteps=1)


@pytest.mark.parametrize("bad", [dict(fene_L2=2.0), dict(fene_L2=-1.0), dict(fene_L2=10.0, beta=0.0),
                                 dict(fene_L2=10.0, giesekus_alpha=0.1)])
def test_fene_parameters_are_validated(lib, bad):
    from paper_2009_12279_gb300 import lbve

    kw = dict(dict(eta=1.0 / 6.0, beta=0.5, lambda_p=100.0, precision="f32"), **bad)
    assert lbve.device_bytes(lbve.make_params((8, 8, 8), **kw)) == 0
    assert lbve.device_bytes(lbve.make_params((8, 8, 8), eta=1.0 / 6.0, beta=0.5, lambda_p=100.0, fene_L2=10.0)) > 0
