"""The persistent lateral kernel's split of each frame length, run as host code.

A transform of length N = N1 x N2 runs its N2-point DFTs in the registers of
N1 threads, then N2 DFTs of N1 points spread over the same N1 threads, NI =
ceil(N2 / N1) each, the last one idle where N1 does not divide N2 (384, 640,
768).  Every stage-2 DFT k2 < N2 must be computed exactly once and no thread
may index past the N2 rows.  Column bands are copied in whole tensor-copy boxes
of at most 256 rows.  This compiles a tiny host program with nvcc (no GPU
needed) against the kernel's own header and checks both for every compiled
length.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_08960_gb300", "csrc")
SIZES = (64, 128, 256, 384, 512, 640, 768, 1024)

HARNESS = r"""
#include <cstdio>
#include "ssoct_internal.h"
template <int N, int N1 = ssoct::split_n1(N)> void check(const char* tag) {
  using S = ssoct::Stage2<N, N1>;
  int count[1024] = {0};
  int bad = 0;
  for (int j1 = 0; j1 < S::N1; ++j1)
    for (int i = 0; i < S::NI; ++i)
      if (S::live(i, j1)) {
        const int k2 = j1 + S::N1 * i;
        if (k2 < 0 || k2 >= S::N2) ++bad;
        else ++count[k2];
      }
  int once = 1;
  for (int k = 0; k < S::N2; ++k) once &= count[k] == 1;
  printf("%s %d %d %d %d %d %d %d %d\n", tag, N, S::N1, S::N2, S::NI, S::A, bad, once, ssoct::band_box_rows(N));
}
int main() {
  check<64>("lat"); check<128>("lat"); check<256>("lat"); check<384>("lat"); check<512>("lat");
  check<640>("lat"); check<768>("lat"); check<1024>("lat");
  check<64, ssoct::ra_split_n1(64)>("ra"); check<96, ssoct::ra_split_n1(96)>("ra");
  check<128, ssoct::ra_split_n1(128)>("ra"); check<160, ssoct::ra_split_n1(160)>("ra");
  check<200, ssoct::ra_split_n1(200)>("ra"); check<256, ssoct::ra_split_n1(256)>("ra");
  return 0;
}
"""


@pytest.fixture(scope="module")
def splits(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("split")
    src = d / "s.cu"
    src.write_text(HARNESS)
    exe = d / "s"
    subprocess.check_call([nvcc, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    rows = {"lat": {}, "ra": {}}
    for line in out.splitlines():
        tag, *vals = line.split()
        n, n1, n2, ni, a, bad, once, box = (int(v) for v in vals)
        rows[tag][n] = dict(n1=n1, n2=n2, ni=ni, a=a, bad=bad, once=once, box=box)
    return rows


def test_every_stage2_dft_once(splits):
    assert set(splits["lat"]) == set(SIZES)
    assert set(splits["ra"]) == {64, 96, 128, 160, 200, 256}
    for kind in ("lat", "ra"):
        for n, r in splits[kind].items():
            assert r["n1"] * r["n2"] == n, (kind, n)
            assert r["bad"] == 0 and r["once"] == 1, (kind, n, r)
            assert r["a"] >= r["n2"] and r["a"] >= r["ni"] * r["n1"], (kind, n, r)


def test_a_row_lies_in_one_warp(splits):
    for n, r in splits["lat"].items():
        assert r["n1"] <= 32 and 32 % r["n1"] == 0, (n, r)


def test_mixed_radix_lengths_have_idle_stage2_threads(splits):
    """384 = 16 x 24, 640 = 32 x 20, 768 = 32 x 24: N1 does not divide N2."""
    for n in (384, 640, 768):
        r = splits["lat"][n]
        assert r["n2"] % r["n1"] != 0 and r["ni"] * r["n1"] > r["n2"], (n, r)


def test_first_pass_tiles_have_eight_to_twenty_warps(splits):
    """A first-pass tile runs 32 N1 threads with one loader thread per frame:
    96 = 16 x 6, 160 = 16 x 10, 200 = 20 x 10 give 16 to 20 warps."""
    for n, r in splits["ra"].items():
        assert 8 <= r["n1"] <= 20 and 32 * r["n1"] >= n, (n, r)
    assert (splits["ra"][96]["n1"], splits["ra"][160]["n1"], splits["ra"][200]["n1"]) == (16, 16, 20)


def test_band_boxes_cover_the_column(splits):
    for n, r in splits["lat"].items():
        assert 1 <= r["box"] <= 256 and n % r["box"] == 0, (n, r)
    lat = splits["lat"]
    assert lat[640]["box"] == 160 and lat[768]["box"] == 256 and lat[384]["box"] == 192
