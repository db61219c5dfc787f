"""The C ABI from plain C: include/hp.h compiles as strict C99 and a C program
linked against libhp.so plans nests and selects levels without a GPU."""
import os
import shutil
import subprocess

import pytest

from paper_2309_01906_gb300 import binding as hb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_compiles_as_c99_and_the_host_entry_points_work():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    hb.lib()   # libhp.so is built
    out_dir = os.path.join(ROOT, "_build", "c_abi")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "c_abi_check")
    lib_dir = os.path.dirname(hb.LIB_PATH)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_check.c"), "-L", lib_dir, "-lhp", "-Wl,-rpath," + lib_dir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.returncode, r.stdout, r.stderr)
