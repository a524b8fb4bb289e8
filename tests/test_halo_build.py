"""The halo block builder's host steps on random inputs:
- the 64-colour slice colouring gives the same columns as the general one, and both are proper
  edge colourings of the lanes x banks multigraph (every lane's entries in distinct columns,
  every column's entries in distinct banks, no column at or past the width);
- each send piece's placement equals its greedy rule written out, slot for slot, with every
  value in exactly one slot and padding on a bank its gather leaves free;
- the halo lists match their definition, and every CTA's decoded block, in both exchanges,
  sums each row once over exactly its neighbours' values (own rows, pull lists, the owners'
  send lists), with zero slots everywhere else.
Host code only: a small program that includes the builder's source (tests/halo_build_check.cu)."""
import os
import subprocess

from tests.conftest import ROOT


def test_halo_builder_steps(tmp_path):
    from paper_2605_05330_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "halo_build_check")
    cmd = [build.nvcc()] + build.ARCH + ["-O2", "-std=c++17", "-Xcompiler", "-pthread",
                                         "-I", build.INCLUDE, "-I", build.CSRC,
                                         os.path.join(ROOT, "tests", "halo_build_check.cu"),
                                         "-o", exe, "-L", os.path.dirname(lib), "-lgn",
                                         "-Xlinker", "-rpath=" + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
