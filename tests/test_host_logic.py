"""Host-side launch arithmetic of the library, compiled from its own header
with the host compiler (no GPU): the z-chunk clamp keeps every launch within
the 65535 CTAs that gridDim.y and gridDim.z allow."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1609_09841_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "hermite_impl.h"
int main() {
  const int nzs[] = {1, 2, 7, 16, 65535, 65536, 131071, 300000, 1 << 20};
  const int chunks[] = {-3, 0, 1, 8, 16, 64, 4096};
  for (int nz : nzs)
    for (int zc : chunks) {
      const int r = hermite::clamp_zchunk(nz, zc);
      const long long ctas = ((long long)nz + r - 1) / r;
      std::printf("%d %d %d %lld\n", nz, zc, r, ctas);
    }
  return 0;
}
"""


def test_zchunk_clamp_keeps_launches_within_the_grid_limit(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    src = tmp_path / "clamp.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "clamp"
    subprocess.run([gxx, "-std=c++17", "-I", CSRC, "-I", cuda_inc, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [tuple(int(v) for v in ln.split()) for ln in out if ln.strip()]
    assert len(rows) == 9 * 7
    for nz, zc, r, ctas in rows:
        assert r >= 1 and ctas <= 65535, (nz, zc, r, ctas)
        if zc >= 1 and (nz + zc - 1) // zc <= 65535:
            assert r == zc              # a chunk that already fits is kept
        if zc >= 1:
            assert r >= zc              # never a smaller chunk than asked for
