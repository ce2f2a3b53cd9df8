"""The windowed query pass's window decisions (win_cell, win_corner in
gp_query_win.cuh), compiled for the host from the same source and checked
against their definition: a cell belongs to the window when each of its 8
corners lies in the 24^3 vertices of the 3 x 3 x 3 bricks from the window's
lowest corner and in a brick marked present; its corners then land in window
brick ((v - lo) >> 3) (x fastest) at the in-brick slot of v."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "win_cell_host.cu")


@pytest.fixture(scope="module")
def window(tmp_path_factory):
    nvcc = next((c for c in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")) if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("win") / "win_cell_host")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2308_13175_gb300", "csrc"), SRC, "-o", exe],
                   check=True, capture_output=True)

    def run(cases):
        text = "\n".join(" ".join(str(int(v)) for v in c) for c in cases) + "\n"
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
        return [list(map(int, line.split())) for line in out[:len(cases)]]
    return run


def _local(v):
    return ((v[2] & 7) * 8 + (v[1] & 7)) * 8 + (v[0] & 7)


def _expected(lo, present, c):
    corners = [(c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + (k >> 2)) for k in range(8)]
    out = []
    for v in corners:
        r = [v[a] - lo[a] for a in range(3)]
        if any(x < 0 or x >= 24 for x in r):
            return [-1]
        wb = (r[0] >> 3) + 3 * (r[1] >> 3) + 9 * (r[2] >> 3)
        if not (present >> wb) & 1:
            return [-1]
        out += [wb, _local(v)]
    return [out[0]] + out


def test_window_membership_and_corner_slots(window):
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(6000):
        lo = (rng.integers(-2, 30, 3) * 8).tolist()                  # brick-aligned, may be negative
        present = int(rng.integers(0, 1 << 27)) if rng.random() < 0.7 else (1 << 27) - 1
        c = [lo[a] + int(rng.integers(-3, 27)) for a in range(3)]      # around and inside the window
        cases.append(lo + [present] + c)
    # Cells on the window's faces and brick faces, every corner brick present.
    for x in (-1, 0, 7, 8, 15, 16, 22, 23):
        for y in (0, 7, 22):
            cases.append([8, 16, 24, (1 << 27) - 1, 8 + x, 16 + y, 24 + 7])
    got = window(cases)
    n_in = 0
    for case, g in zip(cases, got):
        lo, present, c = case[:3], case[3], case[4:]
        want = _expected(lo, present, c)
        assert g == want, (case, g, want)
        n_in += g[0] >= 0
    assert 1000 < n_in < len(cases) - 1000  # both outcomes well represented
