"""The generated in-register DFT codelets, run as host code, against numpy's FFT.

The codelets are __host__ __device__; this compiles a tiny host program with
nvcc (no GPU needed) that applies every codelet to fixed inputs and prints the
results.
"""

import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_08960_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_codelets  # noqa: E402

HARNESS = r"""
#include <cstdio>
#include <cmath>
#include "fft_codelets.cuh"
using namespace ssoct;
template <int N, int S> void one() {
  float2 x[2 * N];
  for (int k = 0; k < 2 * N; ++k) x[k] = make_float2(std::sin(1.3f * k + 0.2f * N), std::cos(0.7f * k * k + S));
  printf("%d %d", N, S);
  for (int k = 0; k < 2 * N; ++k) printf(" %.9g %.9g", x[k].x, x[k].y);
  Dft<N, S>::template run<2, 1>(x);  // odd elements, stride 2: checks ST/OFF handling
  for (int k = 0; k < 2 * N; ++k) printf(" %.9g %.9g", x[k].x, x[k].y);
  printf("\n");
}
int main() {
%BODY%
  return 0;
}
"""


@pytest.fixture(scope="module")
def codelet_output(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("codelets")
    hdr = d / "fft_codelets.cuh"
    gen_codelets.main(str(hdr))
    body = "\n".join(f"  one<{n}, {s}>();" for n in gen_codelets.SIZES for s in (1, -1))
    src = d / "h.cu"
    src.write_text(HARNESS.replace("%BODY%", body))
    exe = d / "h"
    subprocess.check_call([nvcc, "-O1", "-std=c++17", "-I", str(d), str(src), "-o", str(exe)])
    return subprocess.check_output([str(exe)]).decode().strip().splitlines()


def test_codelets_match_dft(codelet_output):
    seen = 0
    for line in codelet_output:
        f = line.split()
        n, s = int(f[0]), int(f[1])
        vals = np.array([float(v) for v in f[2:]]).reshape(2, -1, 2)
        x = vals[0, :, 0] + 1j * vals[0, :, 1]
        got = vals[1, :, 0] + 1j * vals[1, :, 1]
        exp = x.copy()
        j = np.arange(n)
        w = np.exp(s * 2j * np.pi * np.outer(j, j) / n)
        exp[1::2] = w @ x[1::2]
        err = np.max(np.abs(got - exp)) / np.max(np.abs(exp))
        assert err < 4e-7, (n, s, err)
        assert np.array_equal(got[0::2], x[0::2])
        seen += 1
    assert seen == 2 * len(gen_codelets.SIZES)


def test_committed_codelets_match_the_generator(tmp_path):
    """fft_codelets.cuh is written by gen_codelets.py at every build and also
    kept in the tree so the sources read on their own; the committed copy must
    be exactly what the generator writes."""
    out = tmp_path / "fft_codelets.cuh"
    gen_codelets.main(str(out))
    with open(os.path.join(CSRC, "fft_codelets.cuh")) as f:
        committed = f.read()
    assert out.read_text() == committed, "fft_codelets.cuh differs from gen_codelets.py's output: rerun the build"
