"""The library is usable from plain C: a C99 client compiled against
include/ccladder.h and linked with the shared library runs its host-only calls
(no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_2202_02019_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_plain_c_client(tmp_path):
    lib = _build.build()
    exe = str(tmp_path / "client")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(HERE, "c", "client.c"), "-o", exe, "-L", os.path.dirname(lib),
                        "-lccladder", "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
