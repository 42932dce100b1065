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


STRUCTS = {"qsd_op_info": "OpInfo", "qsd_lanczos_params": "LanczosParams", "qsd_lanczos_info": "LanczosInfo",
           "qsd_lobpcg_params": "LobpcgParams", "qsd_lobpcg_info": "LobpcgInfo", "qsd_trim_info": "TrimInfo",
           "qsd_ramps_info": "RampsInfo", "qsd_server_stats": "ServerStats"}


def header_structs():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(qsd_\w+)\s*;", text, flags=re.S):
        fields = []
        for stmt in body.split(";"):
            m = re.match(r"\s*(?:const\s+)?(\w+)\s+(.*\S)\s*$", stmt, flags=re.S)
            if not m:
                continue
            ctype = m.group(1)
            for decl in m.group(2).split(","):
                d = re.match(r"\s*(\*?)\s*(\w+)\s*(?:\[(\d+)\])?\s*$", decl)
                fields.append((d.group(2), "ptr" if d.group(1) else ctype, int(d.group(3) or 1)))
        out[name] = fields
    return out


def test_binding_structs_match_header():
    """Every ABI struct of the header has a ctypes twin with the same fields,
    in order, of the same types and sizes."""
    import ctypes as C
    import paper_2603_18731_gb300 as q
    ctype_of = {"int32_t": C.c_int32, "int64_t": C.c_int64, "uint64_t": C.c_uint64, "double": C.c_double,
                "ptr": C.c_void_p}
    structs = header_structs()
    assert set(STRUCTS) <= set(structs)
    for cname, pyname in STRUCTS.items():
        py = getattr(q, pyname)._fields_
        hdr = structs[cname]
        assert [f for f, *_ in py] == [f for f, *_ in hdr], cname
        for (fname, pytype), (_, ctype, n) in zip(py, hdr):
            want = ctype_of[ctype] * n if n > 1 else ctype_of[ctype]
            assert C.sizeof(pytype) == C.sizeof(want), (cname, fname)
            if n == 1 and ctype != "ptr":
                assert pytype is want, (cname, fname)


def test_bench_names_every_product_path():
    """bench.py has a name for every product path code of the header."""
    import sys
    codes = {int(v) for v in re.findall(r"#define QSD_PATH_\w+\s+(\d+)", open(HEADER).read())}
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.pop(0)
    assert set(bench.PATH_NAMES) == codes
