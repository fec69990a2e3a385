"""The C ABI from plain C: tests/c/abi_host.c is compiled as strict C99
against include/glu.h, linked to the library and run (host analysis only,
no GPU).  It checks closed forms (tridiagonal and arrow fill and levels),
the rejection of a malformed input, and glu_order_nd."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_uses_the_abi(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import paper_1908_00204_gb300 as g
    g.build.build()
    lib = os.path.dirname(g.load_library()._name)
    exe = str(tmp_path / "abi_host")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_host.c"), "-L", lib, "-lglu", f"-Wl,-rpath,{lib}", "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
