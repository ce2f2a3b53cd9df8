"""The deterministic sums' exact split of a float32 contribution into two
integers (fix_split in gp_step_device.cuh), compiled for the host from the
same source and checked against exact rational arithmetic: hi 2^40 + lo is
v 2^60 rounded toward zero, |lo| < 2^40, and every v with |v| >= 2^42 or not
finite is refused.  The function is integer arithmetic on the float's bits,
so the host build computes what the device computes."""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "fix_split_host.cu")


def _nvcc():
    for cand in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def fix_split(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fixsplit") / "fix_split_host")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2308_13175_gb300", "csrc"), SRC, "-o", exe],
                   check=True, capture_output=True)

    def run(values):
        bits = [struct.unpack("<I", struct.pack("<f", v))[0] for v in np.asarray(values, np.float32)]
        out = subprocess.run([exe], input="\n".join(f"{b:08x}" for b in bits) + "\n", capture_output=True,
                             text=True, check=True).stdout.split("\n")
        res = []
        for line in out[:len(bits)]:
            ok, hi, lo = line.split()
            res.append((ok == "1", int(hi), int(lo)))
        return res
    return run


def _expected(v):
    """(accepted, v 2^60 rounded toward zero) from the exact value of v."""
    if not np.isfinite(v):
        return False, None
    x = Fraction(float(v))
    if abs(x) >= 2 ** 42:
        return False, None
    t = x * 2 ** 60
    n = t.numerator // t.denominator if t >= 0 else -((-t.numerator) // t.denominator)
    return True, n


def _check(fix_split, values):
    values = np.asarray(values, np.float32)
    for v, (ok, hi, lo) in zip(values, fix_split(values)):
        acc, n = _expected(v)
        assert ok == acc, (float(v), ok)
        if not ok:
            continue
        assert hi * 2 ** 40 + lo == n, (float(v), hi, lo, n)
        assert abs(lo) < 2 ** 40, (float(v), lo)
        assert hi * float(v) >= 0 and lo * float(v) >= 0, (float(v), hi, lo)  # both carry v's sign


def test_boundaries(fix_split):
    below = np.nextafter(np.float32(2.0 ** 42), np.float32(0))
    vals = [0.0, -0.0, 1.0, -1.0, 2.0 ** 42, -(2.0 ** 42), below, -below, 2.0 ** 43, 2.0 ** 45, 3.0e38,
            2.0 ** -20, 2.0 ** -60, 2.0 ** -61, 3 * 2.0 ** -61, 1.4e-45, -1.4e-45, 1.17549435e-38,
            np.inf, -np.inf, np.nan, 1.5 * 2.0 ** 41, 2.0 ** 40 + 2.0 ** 17]
    _check(fix_split, vals)


def test_random_magnitudes(fix_split):
    rng = np.random.default_rng(7)
    mant = rng.uniform(1.0, 2.0, 4000)
    expo = rng.integers(-90, 46, 4000)
    sign = rng.choice([-1.0, 1.0], 4000)
    _check(fix_split, (sign * mant * 2.0 ** expo).astype(np.float32))
