"""CPU-side checks of the C ABI: libpc.so builds for sm_103a, loads without
a GPU, and exports exactly the functions include/pc.h declares; the Python
binding declares a signature for each of them."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2308_07173_gb300 import _build, pc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "pc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"PC_API\s+[\w\s\*]*?\b(pc_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    return _build.build()


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ("pc_build_target", "pc_knn", "pc_cov", "pc_knn_cov", "pc_sync_status",
                 "pc_batch_plan", "pc_batch_run", "pc_destroy_target", "pc_status_string"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (pc_\w+)$", out, flags=re.M))
    assert set(header_functions()) == exported
    lib = ctypes.CDLL(lib_path)
    for name in header_functions():
        assert getattr(lib, name)


def test_binding_covers_every_declared_symbol():
    assert set(pc.SIGNATURES) == set(header_functions())


def test_no_cuda_needed_for_strings_and_defaults(lib_path):
    pc.load(lib_path)
    assert pc.pc_version().startswith("pc ")
    assert pc.pc_status_string(pc.PC_ERR_K_GT_M) == "k larger than the target size"
    o = pc.pc_default_build_opts()
    assert o.cell_size == 0 and o.occupancy == 12 and o.hash_load == 0.5 and o.max_box_cells == 4096 and o.exhaustive == 1


def test_build_targets_sm_103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
