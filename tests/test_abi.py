"""The C ABI library builds, loads and exports every function include/adagio.h declares.

CPU only: no compute call is made without a GPU.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(adagio_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("adagio_ctx_create", "adagio_ctx_destroy", "adagio_fit", "adagio_embed",
                     "adagio_distortion"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1609_05388_gb300 import build
    lib_path = build.build()
    import ctypes
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads():
    from paper_1609_05388_gb300 import adagio
    assert set(adagio.exported_symbols()) <= set(declared_functions())


def test_ctx_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1609_05388_gb300 import adagio
    with pytest.raises(adagio.AdagioError) as ei:
        adagio.Context(0)
    assert ei.value.code in (adagio.E_CUDA, adagio.E_INVALID_ARG, adagio.E_UNSUPPORTED)


def test_default_opts_without_gpu():
    from paper_1609_05388_gb300 import adagio
    o = adagio.Context.default_opts()
    assert o.s == -1 and o.oversample == 32 and o.precision == adagio.PREC_FP16X3


def test_binding_refuses_to_load_without_the_library(tmp_path):
    """No CPU fallback: without libadagio.so the binding raises on import."""
    import shutil
    import subprocess
    import sys
    pkg = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1609_05388_gb300")
    copy = tmp_path / "paper_1609_05388_gb300"
    shutil.copytree(pkg, copy, ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__", "csrc"))
    r = subprocess.run([sys.executable, "-c", "import paper_1609_05388_gb300.adagio"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "libadagio.so is missing" in r.stderr
