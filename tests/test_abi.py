"""The C-ABI library builds for sm_103a, loads, and exports every function
include/sphgb.h declares (no device calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sphgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|size_t|void|int32_t)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_stage_calls():
    names = _declared()
    for required in ("sph_bin_and_sort", "sph_build_neighbors", "sph_density", "sph_forces",
                     "pp_gravity", "integrate_step", "sph_step", "sph_rhs_initial"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1807_08116_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # host-only entry points work without a device
    lib.sph_version.restype = ctypes.c_int
    assert lib.sph_version() == 1
    lib.sph_ctx_workspace_bytes.restype = ctypes.c_size_t
    lib.sph_ctx_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
    small = lib.sph_ctx_workspace_bytes(1000, 12, 100000)
    big = lib.sph_ctx_workspace_bytes(100000, 18, 10000000)
    assert 0 < small < big
    assert lib.sph_ctx_workspace_bytes(-1, 12, 10) == 0
    assert lib.sph_ctx_workspace_bytes(10, 40, 10) == 0


def test_native_binding_refuses_cpu_tensors():
    import pytest
    import torch
    from paper_1807_08116_gb300 import native as nv
    nv.lib()
    with pytest.raises(TypeError):
        nv.pp_gravity(torch.zeros((4, 4)), torch.zeros((4, 4)))


def test_oracle_and_product_share_no_code():
    # the oracle imports / includes nothing from the package, and vice versa
    imp = re.compile(r"^\s*(?:from\s+(\S+)\s+import|import\s+(\S+)|#\s*include\s+[\"<](\S+)[\">])",
                     re.M)

    def imports(path):
        return [x for m in imp.findall(open(path).read()) for x in m if x]

    pkg = os.path.join(ROOT, "paper_1807_08116_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert not any("oracle" in x for x in imports(os.path.join(dirpath, f))), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            bad = [x for x in imports(os.path.join(ROOT, "oracle", f))
                   if "paper_1807_08116_gb300" in x or "sphgb" in x or "csrc" in x]
            assert not bad, (f, bad)
