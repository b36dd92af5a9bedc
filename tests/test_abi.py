"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/dim3.h declares. No compute call is made (no GPU here)."""

import os
import re
import subprocess

import pytest

import paper_2206_04995_gb300 as dim3
from paper_2206_04995_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dim3.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"DIM3_API\s+[\w\s\*]*?\b(dim3_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for need in ("dim3_map", "dim3_partition", "dim3_join_project", "dim3_join_count",
                 "dim3_plan_join_project", "dim3_plan_join_count", "dim3_ctx_create"):
        assert need in syms


def test_library_builds_and_exports_every_declared_symbol():
    lib = libbuild.build()
    assert os.path.exists(lib)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(dim3_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_without_gpu_and_reports_version():
    L = dim3.load()
    assert L.dim3_version() >= 100
    assert isinstance(L.dim3_last_error(), bytes)
    assert dim3.launch_count() >= 0


def test_library_is_built_for_sm103a_only():
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_oracle_in_product_path():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2206_04995_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


@pytest.mark.parametrize("bad", [-1])
def test_bad_arguments_rejected_on_host(bad):
    """Argument errors are reported before any device work (no GPU needed)."""
    import ctypes
    L = dim3.load()
    n = ctypes.c_int64()
    rc = L.dim3_map(None, None, bad, None, None, ctypes.byref(n), None)
    assert rc == dim3.dim3.DIM3_ERR_ARG
    assert L.dim3_last_error()
