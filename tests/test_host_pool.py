"""The library's host worker pool (the graph preparation's parallel_for / parallel_items): every
block and item runs exactly once, a job posted from inside a job runs inline, jobs posted from
several threads at once all complete, and a forked child starts its own workers.  Host code only:
a small program linked against the built library (tests/host_pool_check.cu)."""
import os
import subprocess

from tests.conftest import ROOT


def test_worker_pool(tmp_path):
    from paper_2605_05330_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "host_pool_check")
    cmd = [build.nvcc()] + build.ARCH + ["-O2", "-std=c++17", "-Xcompiler", "-pthread",
                                         "-I", build.INCLUDE, "-I", build.CSRC,
                                         os.path.join(ROOT, "tests", "host_pool_check.cu"),
                                         "-o", exe, "-L", os.path.dirname(lib), "-lgn",
                                         "-Xlinker", "-rpath=" + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
