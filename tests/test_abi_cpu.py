"""CPU checks of the boundary: the library builds for sm_103a, loads without a
GPU, and exports exactly the entry points that include/qsd.h declares; the
binding's names follow the header; the library path never touches the oracle."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qsd.h")
PKG = os.path.join(ROOT, "paper_2603_18731_gb300")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qsd_[A-Za-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("qsd_create", "qsd_load_operator", "qsd_build_subspace", "qsd_apply_H",
                 "qsd_lanczos_ground_state", "qsd_subspace_index", "qsd_target_table"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_2603_18731_gb300 import build, lib
    build.build()
    L = ctypes.CDLL(os.path.join(PKG, "libqsd.so"))
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    lib()  # binding signatures resolve


def test_binding_covers_header():
    from paper_2603_18731_gb300 import SIGNATURES
    bound = {n for n, _, _ in SIGNATURES}
    assert bound == set(declared_functions())


def test_create_without_gpu_reports_error():
    import ctypes
    from paper_2603_18731_gb300 import lib
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    rc = lib().qsd_create(0, None, ctypes.byref(h))
    assert rc != 0
    assert lib().qsd_last_error(None)


def test_product_path_does_not_import_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                tree = ast.parse(open(os.path.join(dirpath, f)).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert all(not a.name.startswith("oracle") for a in node.names), f
                    if isinstance(node, ast.ImportFrom):
                        assert not (node.module or "").startswith("oracle"), f
            if f.endswith((".cu", ".cuh", ".cpp", ".h")):
                assert "oracle" not in open(os.path.join(dirpath, f)).read().lower(), f
