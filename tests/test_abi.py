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


STRUCTS = ["tfn_camera", "tfn_frame", "tfn_method", "tfn_server_opts", "tfn_serving_stats"]


def test_struct_layouts_match_header(tfn, tmp_path):
    # size and every field offset of every struct, as the C compiler lays them out
    lines, want = [], []
    for name in STRUCTS:
        cls = getattr(tfn, name)
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        want.append(ctypes.sizeof(cls))
        for field, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {field}));')
            want.append(getattr(cls, field).offset)
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"tfn.h\"\nint main(void) {\n" +
                   "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = list(map(int, subprocess.check_output([str(exe)]).split()))
    assert got == want


def test_status_strings_and_version(tfn):
    assert tfn.tfn_status_string(tfn.TFN_OK) == b"ok"
    for s in range(11):
        assert tfn.tfn_status_string(s) != b"unknown status"
    assert tfn.tfn_status_string(11) == b"unknown status"
    assert b"sm_103a" in tfn.tfn_version()


def test_null_context_is_rejected_without_touching_the_gpu(tfn):
    f = tfn.tfn_frame()
    m = tfn.make_method()
    assert tfn.tfn_normals(None, ctypes.byref(f), ctypes.byref(m), None) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_normals_batch(None, ctypes.byref(f), 1, ctypes.byref(m), None) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_create(None, 0, 0) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_destroy(None) == tfn.TFN_OK


def test_null_handles_of_tuner_and_server_are_rejected(tfn, tmp_path):
    f = tfn.tfn_frame()
    m = tfn.make_method()
    best = ctypes.c_int()
    assert tfn.tfn_autotune(None, ctypes.byref(f), 1, ctypes.byref(m), 1, None, ctypes.byref(best),
                            None) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_tuned_shape(None, 0, ctypes.byref(m), ctypes.byref(best)) == tfn.TFN_ERR_INVALID_ARG
    path = os.fsencode(str(tmp_path / "tune.txt"))
    assert tfn.tfn_tune_cache_save(None, path) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_tune_cache_load(None, path) == tfn.TFN_ERR_INVALID_ARG
    o = tfn.tfn_server_opts()
    h = ctypes.c_void_p(1)
    assert tfn.tfn_server_create(None, ctypes.byref(o), ctypes.byref(h)) == tfn.TFN_ERR_INVALID_ARG
    assert h.value is None  # *srv is cleared on failure
    t = ctypes.c_uint64()
    r = ctypes.c_int()
    assert tfn.tfn_submit(None, ctypes.byref(f), 0, ctypes.byref(t)) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_wait(None, 1, 0, ctypes.byref(r)) == tfn.TFN_ERR_INVALID_ARG
    st = tfn.tfn_serving_stats()
    assert tfn.tfn_server_stats(None, ctypes.byref(st), 0) == tfn.TFN_ERR_INVALID_ARG
    assert tfn.tfn_server_destroy(None) == tfn.TFN_OK


def test_library_links_no_torch(tfn):
    out = subprocess.check_output(["ldd", tfn.LIB_PATH], text=True)
    assert "torch" not in out and "c10" not in out


def test_each_kernel_instance_is_compiled_once(tfn):
    # The kernels are instantiated across translation units (per input kind, and the FD mean's with
    # the error bound apart from the rest): every (kind, filter, Phi, tile shape, NOREF) instance
    # must exist exactly once, and the FD mean, which refines in its own kernel, has no refinement
    # kernel.  Host-side launch stubs name the instances.
    import shutil
    if not shutil.which("nm"):
        pytest.skip("nm not available")
    out = subprocess.check_output(["nm", "-C", tfn.LIB_PATH], text=True)
    stubs = re.findall(r" t void tfn::dev::(normals_kernel|refine_kernel)<([^>]*)>\(tfn::LaunchArgs\)$", out, re.M)
    normals = [tuple(int(x) if x.strip().lstrip("-").isdigit() else x.strip() for x in a.split(","))
               for k, a in stubs if k == "normals_kernel"]
    refiners = [tuple(int(x) for x in a.split(",")) for k, a in stubs if k == "refine_kernel"]
    assert len(normals) == len(set(normals)) and len(refiners) == len(set(refiners))
    kinds, shapes = range(4), range(tfn.tfn_tile_shape_count())
    want = {(k, g, p, c, "false") for k in kinds for g in (0, 1, 2, 3, 4, 5) for p in (0, 1) for c in shapes}
    want |= {(k, 9, 0, c, "false") for k in kinds for c in shapes}  # PlanePCA
    want |= {(1, 0, p, c, "true") for p in (0, 1) for c in shapes}  # FP16 depth, FD, without the bound
    assert set(normals) == want
    assert set(refiners) == {(k, g, p) for k in kinds for g in (0, 1, 2, 3, 4, 5) for p in (0, 1)} - \
        {(k, 0, 0) for k in kinds}
