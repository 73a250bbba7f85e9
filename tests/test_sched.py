"""Host-only scheduling pieces, compiled from the library's own headers with g++: the request server's
ring arena and admission rule (tests/native/sched_test.cpp), and the kernel's item -> frame lookup
(tests/native/items_test.cpp).  No GPU."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ring_arena_and_admission(tmp_path):
    exe = tmp_path / "sched_test"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-Werror",
                           "-I", os.path.join(ROOT, "paper_2005_08165_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "sched_test.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def test_item_to_frame_lookup(tmp_path):
    exe = tmp_path / "items_test"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-Werror",
                           "-I", os.path.join(ROOT, "paper_2005_08165_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "items_test.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
