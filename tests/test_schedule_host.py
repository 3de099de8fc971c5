"""The lateral kernel's work queue (LateralSchedule), run as host code.

The persistent lateral kernel takes items in ticket order and waits, with a
bounded spin, for the items each one depends on: a column item of frame f needs
every row item of f, and a row item of frame f >= slots reuses the scratch slot
of frame f - slots, so it needs every column item of that frame.  The queue
drains only if every item is handed out exactly once and every dependency has a
lower ticket.  This compiles a tiny host program with nvcc (no GPU needed) that
decodes every ticket of the schedules the library uses and checks both
properties.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_08960_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "ssoct_internal.h"
int main(int argc, char** argv) {
  int nl, nr, nc, lag, slots;
  while (scanf("%d %d %d %d %d", &nl, &nr, &nc, &lag, &slots) == 5) {
    ssoct::LateralSchedule s{nl, nr, nc, lag, slots};
    printf("S %d %d %d %d %d\n", nl, nr, nc, lag, slots);
    for (long long t = 0; t < s.total(); ++t) {
      int kind, f, item;
      s.decode((unsigned)t, kind, f, item);
      printf("%d %d %d\n", kind, f, item);
    }
  }
  return 0;
}
"""

# (frames, row items, column items, lag, slots): the plan's default (lag 2, six
# slots), every autotuner candidate, and the sliding-gate passes over k new
# frames (lag 2 for k >= 3, else k - 1; slots lag + 4)
CASES = [(256, 128, 128, 2, 6), (32, 8, 8, 2, 6), (64, 32, 16, 2, 6)]
CASES += [(256, 128, 128, lag, slots) for lag in (1, 2, 3) for slots in range(lag + 2, 7)]
# the wider candidates of smaller frames (512 x 512: 32 + 32 items per frame,
# 14 slots; 256 x 256: 16 + 16 items, 23 slots; 64 x 64: 2 + 2 items, up to nlambda)
CASES += [(128, 32, 32, lag, slots) for lag in (1, 2, 3, 4, 6, 8, 12) for slots in {lag + 2, lag + 4, 14} if slots >= lag + 2 and slots <= 14]
CASES += [(64, 16, 16, lag, slots) for lag in (1, 2, 4, 8, 16) for slots in {lag + 2, lag + 4, 23} if slots <= 23]
CASES += [(256, 2, 2, lag, slots) for lag in (16, 24, 32) for slots in {lag + 2, lag + 4, 156}]
CASES += [(k, 8, 8, 2 if k >= 3 else k - 1, (2 if k >= 3 else k - 1) + 4) for k in (1, 2, 3, 5, 13, 32)]


@pytest.fixture(scope="module")
def decoded(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("schedule")
    src = d / "s.cu"
    src.write_text(HARNESS)
    exe = d / "s"
    subprocess.check_call([nvcc, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    inp = "\n".join(" ".join(map(str, c)) for c in CASES) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
    runs, cur = {}, None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "S":
            cur = tuple(int(v) for v in f[1:])
            runs[cur] = []
        else:
            runs[cur].append(tuple(int(v) for v in f))
    return runs


def test_every_item_once(decoded):
    for (nl, nr, nc, lag, slots), seq in decoded.items():
        want = {(0, f, i) for f in range(nl) for i in range(nr)} | {(1, f, i) for f in range(nl) for i in range(nc)}
        assert len(seq) == len(want) and set(seq) == want, (nl, nr, nc, lag, slots)


def test_dependencies_have_lower_tickets(decoded):
    for (nl, nr, nc, lag, slots), seq in decoded.items():
        ticket = {item: t for t, item in enumerate(seq)}
        last_row = {f: max(ticket[(0, f, i)] for i in range(nr)) for f in range(nl)}
        last_col = {f: max(ticket[(1, f, i)] for i in range(nc)) for f in range(nl)}
        for (kind, f, i), t in ticket.items():
            if kind == 1:
                assert last_row[f] < t, ("column item before its frame's rows", nl, nr, nc, lag, slots, f, i)
            elif f >= slots:
                assert last_col[f - slots] < t, ("row item before its slot is free", nl, nr, nc, lag, slots, f, i)


def test_row_items_lead_by_the_lag(decoded):
    """Between the columns of frame f and the rows of frame f + lag nothing else
    of a later frame intervenes: the schedule keeps `lag` frames of row items in
    flight, which is what the scratch ring's slots are sized for."""
    for (nl, nr, nc, lag, slots), seq in decoded.items():
        first_col = {}
        for t, (kind, f, i) in enumerate(seq):
            if kind == 1:
                first_col.setdefault(f, t)
        for f, t in first_col.items():
            later_rows = [g for (kind, g, _) in seq[:t] if kind == 0 and g > f + lag]
            assert not later_rows, (nl, nr, nc, lag, slots, f)
