"""The C ABI library builds for sm_103a and exports every entry point that
include/binarize.h declares (no GPU needed: nothing is called)."""
import ctypes
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
        for m in re.finditer(r"\b(?:bz_status|int64_t|int32_t|const char\s*\*)\s*\**\s*(\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for n in ["binarize_sauvola", "binarize_niblack", "binarize_quantile", "window_sums",
              "window_quantile", "binarize_precision_report", "binarize_batch", "bz_server_create",
              "bz_server_submit", "bz_server_wait", "bz_server_cancel", "bz_server_destroy",
              "bz_status_string", "bz_last_fp64_fallbacks", "binarize_wolf", "binarize_feng",
              "binarize_rais", "binarize_nick", "binarize_phansalkar", "global_stats",
              "binarize_precision_report_ext", "binarize_batch_noalloc", "window_minmax",
              "binarize_bernsen", "haar_feature", "binarize_inplace", "bz_inplace_scratch_bytes",
              "binarize_inplace_cols", "bz_inplace_cols_scratch_bytes",
              "binarize_host", "bz_kernels_per_call", "binarize_host_multi", "bz_tile_schedule"]:
        assert n in names, n


def test_library_exports_every_declared_symbol():
    import paper_1905_13038_gb300 as bz
    path = bz.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_status_strings_without_gpu():
    import paper_1905_13038_gb300 as bz
    bz.build()
    assert bz.status_string(0) == "ok"
    assert "overlap" in bz.status_string(2)
