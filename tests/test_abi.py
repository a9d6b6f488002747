"""The C-ABI library loads and exports every symbol include/hyrf.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hyrf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hyrf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_stage_calls():
    names = _declared()
    for stage in ("query_fields", "project", "bin_sort", "rasterize", "composite_background"):
        assert f"hyrf_{stage}" in names and f"hyrf_{stage}_backward" in names
    assert "hyrf_loss" in names


def test_library_exports_every_declared_symbol():
    from paper_2509_17083_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2509_17083_gb300 import hyrf as H
    for n in _declared():
        if n.endswith("_workspace_size") or n in ("hyrf_read_status", "hyrf_error_string",
                                                    "hyrf_launch_count"):
            continue
        assert hasattr(H, n), n
