"""The register-kernel layout planner against a direct application of the
encoded ops, on the host.

tests/cpp/planner_emulator.cpp plans random circuits' passes with
plan_register_layout (relabeled X/SWAP gates and their flip mask, register
renames, layout changes, commuting-op reordering, conditions on physical
bits) and executes the result with the register kernel's op semantics in
binary64 on random tile contents; it must agree with the encoded ops applied
in list order to the logical tile.  Compiled against the built library."""
import os
import shutil
import subprocess

import pytest

from paper_2210_01076_gb300 import build as qbuild

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.timeout(300)
def test_layout_planner_matches_direct_application(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    lib = qbuild.build()
    pkg = os.path.dirname(lib)
    cuda = qbuild._cuda_home()
    exe = str(tmp_path / "planner_emulator")
    cmd = ["g++", "-O1", "-std=c++17", f"-I{os.path.join(ROOT, 'include')}", f"-I{qbuild.CSRC}",
           f"-I{os.path.join(cuda, 'include')}", os.path.join(HERE, "cpp", "planner_emulator.cpp"), "-o", exe,
           f"-L{pkg}", "-lqtask", f"-Wl,-rpath,{pkg}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe, "40"], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK"), r.stdout
