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
  288^3: 96, 2D 2048^2: 16, 2D 16384^2: 128);
* the chunk length of the column and line-sweep kernels (wave model, 3 blocks
  per SM on 152 SMs): the plans their timings were taken with (383^3: 192 planes,
  345.5 us, where the earlier "two waves of warps" rule took 77 planes, 406 us;
  511^3: 73; 255^3: 29, 115.5 against 132.5 us at 37; 2D 6001^2: 172 rows), and
  that every pick covers the axis with chunks of at least the minimum length."""
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
  // chunk length: N, blocks per chunk, minimum length (456 slots, 5 planes overhead)
  const long long wc[][3] = {{383, 208, 4}, {511, 387, 4}, {255, 97, 4}, {6001, 26, 8}};
  for (auto& c : wc) std::printf("w %lld %d\n", c[0], wave_chunk_length(c[0], c[1], 456, c[2], 5.0));
  // invariants over a grid of cases: chunks of at least min(N, min_len), covering N
  int bad = 0;
  for (long long N = 3; N <= 700; N += 7)
    for (long long b = 1; b <= 1000; b = b * 3 + 1)
      for (long long m : {4LL, 8LL}) {
        const long long len = wave_chunk_length(N, b, 456, m, 5.0), chunks = (N + len - 1) / len;
        if (len < 1 || len > N || (len < m && len != N && N >= m) || chunks * len < N || (chunks - 1) * len >= N) ++bad;
      }
  std::printf("i %d\n", bad);
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
    z, r, w, inv = {}, {}, {}, None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "z":
            z[int(f[1])] = int(f[2])
        elif f[0] == "r":
            r[(int(f[1]), int(f[2]))] = int(f[3])
        elif f[0] == "w":
            w[int(f[1])] = int(f[2])
        else:
            inv = int(f[1])
    return z, r, w, inv


def test_automatic_zchunks_match_the_measured_best(picks):
    z = picks[0]
    assert z == {128: 19, 256: 4, 384: 6, 512: 8, 640: 12, 1024: 16}


def test_row_kernel_item_length_matches_the_measured_best(picks):
    r = picks[1]
    assert r == {(3, 96): 4, (3, 160): 16, (3, 224): 48, (3, 288): 96, (2, 2048): 16, (2, 16384): 128,
                 (1, 65536): 128}


def test_wave_chunk_length_picks_the_timed_plans(picks):
    w, inv = picks[2], picks[3]
    assert w == {383: 192, 511: 73, 255: 29, 6001: 172}
    assert inv == 0
