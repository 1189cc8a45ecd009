"""The C ABI from a plain C99 program: tests/cpp/abi_c_client.c includes
include/qtask.h alone, links libqtask.so and drives circuit edits, error
reporting and a dry-run update plan (no GPU needed), showing that the
boundary needs neither Python nor PyTorch nor C++."""
import os
import shutil
import subprocess

import pytest

from paper_2210_01076_gb300 import build as qbuild

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.timeout(120)
def test_plain_c_caller(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = qbuild.build()
    pkg = os.path.dirname(lib)
    exe = str(tmp_path / "abi_c_client")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-O1", f"-I{os.path.join(ROOT, 'include')}",
           os.path.join(HERE, "cpp", "abi_c_client.c"), "-o", exe, f"-L{pkg}", "-lqtask", f"-Wl,-rpath,{pkg}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, f"check {r.returncode} failed: {r.stdout}{r.stderr}"
    assert r.stdout.strip() == "ok"
