"""The C-ABI library builds, loads and exports every symbol include/rift2.h declares; the
ctypes mirrors of its structs match the C layout; host-side argument checks (no GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rift2.h")


@pytest.fixture(scope="module")
def pkg():
    from paper_2303_00319_gb300 import _build
    _build.build()
    import paper_2303_00319_gb300 as p
    p.lib()
    return p


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rift2_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_exported(pkg):
    lib = pkg.lib()
    decl = declared_functions()
    assert decl, "no declarations parsed"
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(pkg.EXPORTS) == decl


def test_struct_layouts_match_c(tmp_path, pkg):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "rift2.h"
int main(void) {
  printf("%zu %zu\\n", sizeof(rift2_params), offsetof(rift2_params, flags));
  printf("%zu %zu\\n", sizeof(rift2_image), offsetof(rift2_image, pitch));
  printf("%zu %zu %zu\\n", sizeof(rift2_features), offsetof(rift2_features, counts),
         offsetof(rift2_features, debug));
  printf("%zu %zu\\n", sizeof(rift2_matches), offsetof(rift2_matches, count));
  printf("%zu\\n", sizeof(rift2_debug_maps));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = [list(map(int, l.split())) for l in subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.split("\n") if l]
    assert out[0] == [C.sizeof(pkg.Params), pkg.Params.flags.offset]
    assert out[1] == [C.sizeof(pkg.Image), pkg.Image.pitch.offset]
    assert out[2] == [C.sizeof(pkg.FeaturesC), pkg.FeaturesC.counts.offset,
                      pkg.FeaturesC.debug.offset]
    assert out[3] == [C.sizeof(pkg.MatchesC), pkg.MatchesC.count.offset]
    assert out[4] == [C.sizeof(pkg.DebugMaps)]


def test_default_params_match_oracle(pkg):
    import oracle as O
    p = pkg.default_params()
    d = O.DEFAULT
    for name in ("n_scales", "n_orient", "lp_order", "fast_arc", "max_keypoints", "patch", "cells"):
        assert getattr(p, name) == getattr(d, name), name
    for name in ("min_wavelength", "mult", "sigma_onf", "k", "g", "cutoff", "eps", "lp_cutoff",
                 "fast_threshold", "second_ratio"):
        assert abs(getattr(p, name) - getattr(d, name)) <= 1e-7 * max(1.0, abs(getattr(d, name)))
    assert p.flags == 0


def test_status_strings(pkg):
    lib = pkg.lib()
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.rift2_status_str(code)
    assert b"unknown" in lib.rift2_status_str(-99)


def test_host_argument_checks_without_gpu(pkg):
    lib = pkg.lib()
    # NULL out-pointer and unsupported geometry are refused before any device work
    assert lib.rift2_create(None, 0, 0, None) == pkg.E_INVAL
    h = C.c_void_p()
    bad = pkg.default_params(n_orient=8)
    assert lib.rift2_create(C.byref(bad), 0, 0, C.byref(h)) == pkg.E_UNIMPL
    bad = pkg.default_params(mult=0.5)
    assert lib.rift2_create(C.byref(bad), 0, 0, C.byref(h)) == pkg.E_INVAL
    assert lib.rift2_extract(None, 1, None, None, None) == pkg.E_INVAL
    assert lib.rift2_match(None, 1, None, None, None, None) == pkg.E_INVAL
    assert lib.rift2_destroy(None) == pkg.E_INVAL
    assert lib.rift2_launch_count(None) == -1


def test_no_device_is_an_error_not_a_fallback(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    p = pkg.default_params()
    assert pkg.lib().rift2_create(C.byref(p), 0, 0, C.byref(h)) == pkg.E_CUDA
