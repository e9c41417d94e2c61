"""The persistent 3-D step schedule, compiled from the library's own host sources
(plan_persistent in tmap.cpp, schedule_segment in step3d.h) and checked on the CPU: for
every combination of plane count, radius, tile columns and resident CTAs (the launch
sizes of two CTAs of 8 warps or four of 4 warps per SM among them), with and without the
in-step z-parts, each (tile column, output plane) is computed by exactly one CTA segment
and the grid never exceeds the resident CTAs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_persistent_schedule_covers_every_unit_once(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("g++ and the CUDA headers are needed to build the check")
    exe = str(tmp_path / "schedule_check")
    csrc = os.path.join(ROOT, "paper_1912_08063_gb300", "csrc")
    cmd = [cxx, "-O2", "-std=c++17", f"-I{CUDA}/include", f"-I{ROOT}/include", f"-I{csrc}",
           os.path.join(ROOT, "tests", "schedule_check.cpp"), os.path.join(csrc, "tmap.cpp"),
           f"-L{CUDA}/lib64", "-lcudart", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=f"{CUDA}/lib64:" + os.environ.get("LD_LIBRARY_PATH", ""))
    out = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) == 8 * 2 * 18 * 6 * 2
