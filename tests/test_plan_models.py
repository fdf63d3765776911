"""Host-side launch models behind the automatic launch parameters
(`paper_0712_0813_gb300/csrc/ce_plan.h`), compiled with the host compiler and
checked against the choices the GB300 timings fixed (CPU; no GPU needed):

* the z-sweep kernel's automatic z-chunk count, for 8-row tiles at 2 CTAs per SM
  on 152 SMs: the measured best of the autotuner's full tables at 128^3-640^3
  (at 256^3, 4 chunks = 0.84 of a wave, 93.3 us, against the 14 chunks of whole
  waves, 101.6 us) and at 1024^3 the plan that beat the autotuner's (16 chunks,
  5.19 against 5.28 ms);
* the row kernel's item length on one FP32 lattice (304 resident CTAs): the
  measured best among the item lengths timed (96^3: 4, 160^3: 16, 224^3: 48,
  288^3: 96, 2D 2048^2: 16, 2D 16384^2: 128)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0712_0813_gb300", "csrc")

PROGRAM = r'''
#include <cstdio>
#include "ce_plan.h"
int main() {
  using namespace ce::plan;
  // z-chunks: N, columns (N/128 x N/8), CTAs per SM, SMs
  const long long zc[][2] = {{128, 16}, {256, 64}, {384, 144}, {512, 256}, {640, 400}, {1024, 1024}};
  for (auto& c : zc) std::printf("z %lld %d\n", c[0], auto_zchunks(c[0], c[1], 2, 152));
  // row kernel item length: dims, N (FP32: 4 sites per 16 bytes), 304 slots
  const int rl[][2] = {{3, 96}, {3, 160}, {3, 224}, {3, 288}, {2, 2048}, {2, 16384}, {1, 65536}};
  for (auto& c : rl) std::printf("r %d %d %d\n", c[0], c[1], rows_item_length(c[0], c[1], 4, 304));
  return 0;
}
'''


@pytest.fixture(scope="module")
def picks(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("plan")
    src, exe = d / "plan.cpp", d / "plan"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    z, r = {}, {}
    for line in out.splitlines():
        f = line.split()
        if f[0] == "z":
            z[int(f[1])] = int(f[2])
        else:
            r[(int(f[1]), int(f[2]))] = int(f[3])
    return z, r


def test_automatic_zchunks_match_the_measured_best(picks):
    z, _ = picks
    assert z == {128: 19, 256: 4, 384: 6, 512: 8, 640: 12, 1024: 16}


def test_row_kernel_item_length_matches_the_measured_best(picks):
    _, r = picks
    assert r == {(3, 96): 4, (3, 160): 16, (3, 224): 48, (3, 288): 96, (2, 2048): 16, (2, 16384): 128,
                 (1, 65536): 128}
