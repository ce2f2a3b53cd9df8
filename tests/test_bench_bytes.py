"""Host-side checks of the benchmark's roofline bookkeeping (no GPU): every
kernel a fitting step can launch has an algorithmic byte count, and the counts
are the arrays each kernel must touch once."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2308_13175_gb300", "csrc")

# Launched by a step of FitStep: sampling (once-per-epoch kernels move no
# per-step data the roofline counts), NN, the step and the update.
STEP_KERNELS = {"k_sample", "k_perm", "k_order_count", "k_order_emit", "k_nn", "k_nn_sorted", "k_count_valid",
                "k_tv", "k_tv_inv", "k_tv_grad", "k_query", "k_adam", "k_tv_adam"}
UNCOUNTED = {"k_order_tiles", "k_emit_slots"}  # a scan of tile counts; a per-epoch gather


def _launched(files):
    names = set()
    for f in files:
        text = open(os.path.join(CSRC, f)).read()
        # launched through GP_KERNEL, or traced by hand with gp_prof_post
        names |= set(re.findall(r'GP_KERNEL\(ctx, "(k_[a-z_0-9]+)"', text))
        names |= set(re.findall(r'gp_prof_post\(ctx, "(k_[a-z_0-9]+)"\)', text))
    return names


def test_every_step_kernel_has_algorithmic_bytes():
    launched = _launched(["gp_sample.cu", "gp_nn.cu", "gp_step.cu"])
    setup = {"k_knn_sigma", "k_normals", "k_emit_pts",   # band set-up, untimed
             "k_nn_count", "k_nn_sorted_count"}           # gp_nn_work's counting launches, outside the step
    assert STEP_KERNELS <= launched
    for name in launched - setup - UNCOUNTED:
        assert bench.alg_bytes(name, 1000, 100, 512, 300) > 0, name


def test_byte_counts_are_the_arrays_touched_once():
    n, J, Vs, Vt = 1000, 100, 512, 300
    assert bench.alg_bytes("k_order_count", n, J, Vs, Vt) == 4 * J          # the epoch's slot of each point
    assert bench.alg_bytes("k_nn", n, J, Vs, Vt) == 36 * n + 16 * J          # q in, record + index out; points
    assert bench.alg_bytes("k_query", n, J, Vs, Vt) == 24 * n + 8 * Vt      # records; D read, grad written
    assert bench.alg_bytes("k_adam", n, J, Vs, Vt) == 28 * Vt               # D, g, m, v read; D, m, v written
    assert bench.alg_bytes("k_tv", n, J, Vs, Vt) == 8 * Vs                  # D read, grad written
    assert bench.alg_bytes("k_tv_inv", n, J, Vs, Vt) == 8 * Vs              # D read, 1/TV written
    assert bench.alg_bytes("k_tv_grad", n, J, Vs, Vt) == 12 * Vs            # D, 1/TV read, grad written
    assert bench.alg_bytes("k_tv_adam", n, J, Vs, Vt) == 4 * Vs + 28 * Vt   # D read; query part, m, v, D
    assert bench.alg_bytes("k_unknown", n, J, Vs, Vt) == 0


def test_nn_roofline_is_fp32_candidate_arithmetic():
    """The nearest-point kernels are rated against the FP32 pipe: 8 flops per
    candidate distance (3 subtractions, 1 multiply, 2 FMAs at 2 flops each)
    against SMs x 128 lanes x 2 flops x the maximum clock."""
    assert bench.NN_FLOPS_PER_CANDIDATE == 8
    peak, kind = bench.fp32_peak_tflops(152)
    assert "derived" in kind
    assert 70.0 < peak < 90.0      # 152 x 128 x 2 x ~2.07 GHz = 80.5 TFLOP/s


def test_band_counts_match_the_oracle_sets():
    """The dense-bitmap counts the CPU baseline extrapolates to equal the
    oracle's band sets."""
    import numpy as np
    from oracle import gridpull as o
    from paper_2308_13175_gb300 import synth
    pts = synth.sphere_cloud(700, 0.4, seed=3)
    for R, M1, M2 in ((32, 2, 2), (32, 1, 3), (16, 0, 0), (16, 2, -1)):
        sets = o.band_sets(pts, R, M1, M2)
        c = bench.band_counts(pts, R, M1, M2)
        assert c["V_tv"] == len(sets["tv"]) and c["V_trainable"] == len(sets["trainable"]), (R, M1, M2)
