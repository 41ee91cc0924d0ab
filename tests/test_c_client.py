"""The C ABI from plain C: tests/c_client/cartogram_client.c includes only
include/cartogram.h and links libcartogram.so. On the CPU it is compiled and linked
(no call runs); on the GPU it runs a two-strip cartogram in both precisions."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compile():
    from paper_1802_07625_gb300 import build
    lib = build.build()
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    out = os.path.join(os.path.dirname(lib), "cartogram_client")
    cmd = [gcc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_client", "cartogram_client.c"), "-o", out,
           "-L", os.path.dirname(lib), "-lcartogram", "-Wl,-rpath," + os.path.dirname(lib), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def test_c_client_compiles_and_links_against_the_header_and_library():
    assert os.path.exists(_compile())


@pytest.mark.gpu
def test_c_client_runs_a_cartogram():
    exe = _compile()
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
    assert r.stdout.count("iterations") == 2
