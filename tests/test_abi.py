"""The C ABI library: it loads, exports every entry point include/tfn.h
declares, and its struct layouts match the Python binding.  No compute calls:
this runs without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tfn.h")


@pytest.fixture(scope="module")
def tfn():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2005_08165_gb300 as tfn
    return tfn


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tfn_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(tfn):
    lib = ctypes.CDLL(tfn.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), f"{name} declared in tfn.h but not exported"
    assert set(names) <= set(tfn.EXPORTED) | {"tfn_stream"}


def test_struct_layouts_match_header(tfn, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "tfn.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(tfn_frame), sizeof(tfn_camera), sizeof(tfn_method),
         offsetof(tfn_frame, cam), offsetof(tfn_frame, normals), offsetof(tfn_frame, mask),
         offsetof(tfn_frame, mask_pitch), offsetof(tfn_method, flags));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = list(map(int, subprocess.check_output([str(exe)]).split()))
    want = [ctypes.sizeof(tfn.tfn_frame), ctypes.sizeof(tfn.tfn_camera), ctypes.sizeof(tfn.tfn_method),
            tfn.tfn_frame.cam.offset, tfn.tfn_frame.normals.offset, tfn.tfn_frame.mask.offset,
            tfn.tfn_frame.mask_pitch.offset, tfn.tfn_method.flags.offset]
    assert got == want


def test_status_strings_and_version(tfn):
    assert tfn.tfn_status_string(tfn.TFN_OK) == b"ok"
    for s in range(10):
        assert tfn.tfn_status_string(s)
    assert b"sm_103a" in tfn.tfn_version()


def test_null_context_is_rejected_without_touching_the_gpu(tfn):
    f = tfn.tfn_frame()
    m = tfn.make_method()
    assert tfn.tfn_normals(None, ctypes.byref(f), ctypes.byref(m), None) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_normals_batch(None, ctypes.byref(f), 1, ctypes.byref(m), None) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_create(None, 0, 0) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_destroy(None) == tfn.TFN_OK


def test_library_links_no_torch(tfn):
    out = subprocess.check_output(["ldd", tfn.LIB_PATH], text=True)
    assert "torch" not in out and "c10" not in out
