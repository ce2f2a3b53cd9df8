"""Benchmark of the GridPull fitting step on GB300.

One step = one pass of the whole hot path over one batch of the epoch's query
pool: gp_sample (Gaussian queries around points in the epoch's random order)
-> gp_nn (exact nearest surface point) -> gp_step (Eq. 8 forward and
hand-written backward, L_TV included) -> gp_update (Adam on the trainable
vertices).  Band construction and sigma are once-per-cloud set-up, untimed.

Default workload: the largest single-GPU configuration, the synthetic indoor
scene (a 10 x 8 x 3 m room plus 60 boxes and cylinders, 10,000,000 points with
N(0, 0.002^2) m noise, normalised to [-1,1]^3), a 1024^3 grid with a band of
cells within 2 voxels of the points stored as 8^3 float32 bricks, a pool of
50,000,000 queries per epoch and batches of 2,097,152 queries.  --workload
selects the single object, the sphere, the superquadrics or the collection.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on all host cores, on a bounded sample of the same workload, instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pull-step queries/sec (fwd+bwd+Adam)"
UNIT = "queries/s"

WORKLOADS = {
    "object": dict(desc="single object: 3 random ellipsoids + torus (R=0.3, r=0.08), 100,000 points + "
                        "N(0,0.001^2) noise; 256^3 grid, band = cells within 2 voxels of a point, 8^3 float32 "
                        "bricks; pool 2,000,000 queries/epoch (q = s_j + sigma_j N(0,I), sigma_j = 50th-NN "
                        "distance); batch 262,144",
                   cloud=lambda: __import__("paper_2308_13175_gb300.synth", fromlist=["x"]).object_cloud(100_000, seed=1),
                   R=256, M1=2, M2=2, Q=2_000_000, B=262_144, lr=1e-3),
    "sphere": dict(desc="single sphere: 5,000 points on a radius-0.5 sphere; dense 64^3 grid; 50,000 queries "
                        "(10 per point), full batch",
                   cloud=lambda: __import__("paper_2308_13175_gb300.synth", fromlist=["x"]).sphere_cloud(5000, 0.5, 0),
                   R=64, M1=-1, M2=-1, Q=50_000, B=50_000, lr=1e-3, init="sphere_noise"),
    "scene": dict(desc="indoor scene: 10 x 8 x 3 m room (floor, ceiling, 4 walls) + 60 boxes / cylinders, "
                       "10,000,000 points + N(0, 0.002 m^2) noise, normalised to [-1,1]^3; 1024^3 grid, band of "
                       "8^3 float32 bricks; pool 50,000,000 queries/epoch, batch 2,097,152",
                  cloud=lambda: __import__("paper_2308_13175_gb300.synth", fromlist=["x"]).room_cloud(10_000_000, seed=2),
                  R=1024, M1=2, M2=2, Q=50_000_000, B=2_097_152, lr=1e-3),
    "superquadric": dict(desc="large object: union of 10 superquadrics (exponents U[0.3,3]), 2,000,000 points + "
                              "N(0,0.001^2) noise; 512^3 grid, band of 8^3 float32 bricks; pool 20,000,000 "
                              "queries/epoch, batch 4,194,304",
                         cloud=lambda: __import__("paper_2308_13175_gb300.synth", fromlist=["x"]).superquadric_cloud(2_000_000, seed=4),
                         R=512, M1=2, M2=2, Q=20_000_000, B=4_194_304, lr=1e-3),
    "collection": dict(desc="batched fitting: 64 shapes, each a union of 1-5 ellipsoids / boxes / tori, point "
                            "counts log-uniform in [5,000, 500,000], grids drawn from {128, 256, 512}^3 with a "
                            "2-voxel band of 8^3 float32 bricks; pool 10 queries per point, batch = pool / 8 per "
                            "shape; all shapes in one launch per stage, the step replayed as a CUDA graph",
                       R=0, M1=2, M2=2, lr=1e-3, n_shapes=64, q_per_point=10, batches_per_epoch=8),
}

# Algorithmic bytes per launch of each kernel: every array the kernel must
# touch, once (re-reads, padding and frozen slots are overhead, not counted).
# n = queries in the launch, J = points, Vs = stored slots, Vt = trainable
# vertices.
def alg_bytes(name, n, J, Vs, Vt):
    return {
        "k_sample": 32 * n,
        "k_perm": 8 * J,
        "k_order_count": 4 * J,
        "k_order_emit": 20 * J + 32 * n,
        "k_nn": 36 * n + 16 * J,
        "k_nn_sorted": 36 * n + 16 * J,
        "k_count_valid": 24 * n,
        "k_tv": 8 * Vs,
        # the two-pass L_TV of gp_step: D read and 1/TV written; D and 1/TV
        # read and the gradient written
        "k_tv_inv": 8 * Vs,
        "k_tv_grad": 12 * Vs,
        "k_query": 24 * n + 8 * Vt,
        "k_adam": 28 * Vt,
        # the fused L_TV + Adam sweep: values read for the stencil; per trainable
        # vertex the query part read and reset, m, v read, value, m, v written
        "k_tv_adam": 4 * Vs + 28 * Vt,
    }.get(name, 0)


# The nearest-point kernels are bound by issue and SIMT divergence in their
# float32 distance arithmetic, not by bytes: their roofline is the FP32 pipe,
# in the flops of the candidate distances they evaluate (counted by
# gp_nn_work): per candidate 3 subtractions, 1 multiply and 2 FMAs = 8 flops
# (FMA = 2).  Peak: 152 SMs x 128 FP32 lanes x 2 flops x the maximum SM clock.
NN_KERNELS = ("k_nn", "k_nn_sorted")
NN_FLOPS_PER_CANDIDATE = 8
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(num_sms: int):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
        kind = "derived: SMs x 128 FP32 lanes x 2 x measured max SM clock"
    except Exception:
        mhz, kind = 2070.0, "derived: SMs x 128 FP32 lanes x 2 x nominal max SM clock 2070 MHz"
    return num_sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, kind


def fwd_bwd_adam(per_kernel: dict, names, queries_per_step: float, V_trainable: int, peak: float) -> dict:
    """The forward + backward + Adam part of the step alone (gp_step +
    gp_update: the L_TV sweep, the fused query kernel, Adam), from the traced
    per-kernel times: its query rate and its roofline against the algorithmic
    bytes 24 B + 36 V_trainable per step (the record; D read and gradient write
    plus Adam's 7 accesses per trainable vertex)."""
    t_us = sum(per_kernel[n]["avg_us"] * per_kernel[n]["launches"] for n in names if n in per_kernel)
    steps = max(per_kernel[n]["launches"] for n in names if n in per_kernel)
    t_us /= steps
    by = 24.0 * queries_per_step + 36.0 * V_trainable
    gbs = by / (t_us * 1e-6) / 1e9
    return {"value": queries_per_step / (t_us * 1e-6), "unit": UNIT, "us_per_step": round(t_us, 2),
            "kernels": [n for n in names if n in per_kernel], "alg_bytes_per_step": int(by),
            "achieved_gbs": round(gbs, 1), "peak_gbs": peak, "frac": round(gbs / peak, 4)}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the dominant kernel from one ncu capture of the current kernel code
# (summaries in profiles/), by workload; a kernel changed since its capture
# must be dropped from here.
NCU_TRAFFIC = {
    # profiles/k_nn_sorted_scene_1024.md: mean of three full-size launches.
    ("scene", "k_nn_sorted"): 1_138_243_072,
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# -------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and throttle reasons sampled by nvidia-smi (read-only query)
    every 50 ms during the timed region.  The GPU is selected by its UUID (a
    local index can name another GPU when CUDA_VISIBLE_DEVICES remaps
    devices), and nvidia-smi's output is read line by line from a pipe by a
    reader thread, so no sample is lost in a file buffer when it is stopped."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local: int):
        self.local = local
        self.proc = None
        self.rows = []
        self.thread = None
        self.error = None

    def _gpu_id(self):
        try:
            import torch
            u = str(torch.cuda.get_device_properties(self.local).uuid)
            return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            if vis:
                return vis.split(",")[self.local].strip()
            return str(self.local)

    def start(self):
        import shutil
        import threading
        cmd = ["nvidia-smi", f"--id={self._gpu_id()}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if shutil.which("stdbuf"):
            cmd = ["stdbuf", "-oL"] + cmd
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, bufsize=1)
        except Exception as e:
            self.proc, self.error = None, f"nvidia-smi: {e}"
            return

        def reader():
            for line in self.proc.stdout:
                if line.strip():
                    self.rows.append(line.strip().split(","))
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        time.sleep(0.3)  # nvidia-smi's first sample

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "error": self.error or "nvidia-smi unavailable"}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        err = ""
        try:
            err = (self.proc.stderr.read() or "").strip()
        except Exception:
            pass
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        out = {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "reasons": sorted(reasons), "samples": len(sm)}
        if not sm:
            out["error"] = "no clock sample during the timed region" + (f": {err[:200]}" if err else "")
            print("bench: WARNING: " + out["error"], file=sys.stderr)
        return out


# ---------------------------------------------------------------- helpers
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, world: int, op: str) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def reduce_max(x: float, world: int) -> float:
    return _reduce(x, world, "max")


def reduce_sum(x: float, world: int) -> float:
    return _reduce(x, world, "sum")


def replica_rate(units: float, ms: float, world: int) -> float:
    """Whole-job rate of N independent replicas: the units every rank
    processed over the slowest rank's time (weak scaling)."""
    return reduce_sum(float(units), world) / (reduce_max(float(ms), world) / 1e3)


# -------------------------------------------------- oracle CPU baseline
def band_counts(pts: np.ndarray, R: int, M1: int, M2: int) -> dict:
    """|T| and the trainable-vertex count of the band (the oracle's
    dense-bitmap form of its band sets): the sizes the CPU baseline
    extrapolates to."""
    from oracle import gridpull as o
    sets = o.band_vertex_sets_bitmap(pts, R, M1, M2)
    return {"V_tv": int(len(sets["tv"])), "V_trainable": int(len(sets["trainable"]))}


def oracle_baseline(pts, wl, counts, budget_s: float, steps: int = 1, seed: int = 0):
    """The FP64 oracle's step on all host cores, timed on a bounded sample of
    the workload and extrapolated to a full batch.

    Per step the four phases run on every core (oracle.parallel): brute-force
    NN of n_nn queries, the sampler plus the query terms with their gradient for
    n_q queries (s = the source point, values on a band-sparse store of the
    analytic initial sphere), L_TV of n_tv TV vertices and Adam on n_ad
    vertices.  Each phase's wall time over its units gives its time per unit;
    a full step is B (t_nn + t_q) + |T| t_tv + V_trainable t_adam.  Sample
    sizes are calibrated so that the timed phases of all steps take about
    budget_s seconds.  Set-up (the cloud on disk, sigma of the sampled points,
    the sparse stores) is untimed."""
    from oracle import gridpull as o
    from oracle.parallel import OraclePool
    R, M1, B = wl["R"], wl["M1"], wl["B"]
    J = len(pts)
    h = 2.0 / R
    centre = 0.5 * (pts.min(0) + pts.max(0)).astype(np.float64)
    init = lambda keys: np.linalg.norm(-1.0 + h * o.key_to_vertex(keys, R) - centre, axis=1) - 2 * h
    occ = o.occupied_cells(pts, R)
    tmp = tempfile.mkdtemp(prefix="gp_oracle_")
    pts_path = os.path.join(tmp, "points.npy")
    np.save(pts_path, np.ascontiguousarray(pts, np.float32))
    occ_path = os.path.join(tmp, "occ.npy")
    np.save(occ_path, occ)
    pool = OraclePool(pts_path)
    C = pool.cores
    rng = np.random.default_rng(seed + 11)
    weights = (1.0, 1.0, 0.005)
    tree = None

    def sigma_of(idx):
        """sigma_j of the sampled points (set-up, untimed): the k-d tree of
        scipy where it is installed (the 51st distance counting the point
        itself is the 50th to another point), else the oracle's brute force."""
        nonlocal tree
        try:
            from scipy.spatial import cKDTree
        except Exception:
            return o.knn_sigma(pts, 50, idx=idx)
        if tree is None:
            tree = cKDTree(np.asarray(pts, np.float64))
        d, _ = tree.query(np.asarray(pts[idx], np.float64), k=min(51, J))
        return d[:, -1] if J > 1 else np.zeros(len(idx))
    try:
        def make_terms(n, tag):
            """Chunks of n sampled queries (pool positions of epoch 0)."""
            pos = (np.arange(n, dtype=np.int64) * 7919 + 12345) % max(wl.get("Q", B), 1)
            j = o.point_permutation(J, seed, 0, pos % J)
            uj = np.unique(j)
            sig = np.zeros(J)
            sig[uj] = sigma_of(uj)
            q, _ = o.sample_queries(pts, sig, seed, 0, pos)
            q = q.astype(np.float32)
            items, qs = [], []
            for k, sl in enumerate(np.array_split(np.arange(n), C)):
                cq, lq, _ = o.cell_and_local(q[sl], R)
                cq = np.clip(cq, 0, R - 1)
                cs, ls, _ = o.cell_and_local(pts[j[sl]], R)
                cs, _ = o.clamp_cell(cs, ls, R)
                keys = np.unique(np.concatenate([o.vertex_key(c + d, R) for c in (cq, cs) for d in o.CORNERS]))
                pth = os.path.join(tmp, f"terms_{tag}_{k}.npz")
                ju = np.unique(j[sl])
                np.savez(pth, pos=pos[sl], j=j[sl], sig_idx=ju, sig_val=sig[ju], keys=keys, vals=init(keys))
                items.append((pth, occ_path, R, M1, weights, seed))
                qs.append(q[sl])
            return items, qs

        def make_nn(qs, n, tag):
            allq = np.concatenate(qs)[:n]
            paths = []
            for k, part in enumerate(np.array_split(allq, C)):
                pth = os.path.join(tmp, f"nn_{tag}_{k}.npy")
                np.save(pth, part)
                paths.append(pth)
            return paths

        def make_tv(n, tag):
            cells = occ[rng.integers(0, len(occ), size=max(1, n // 8 + 1))]
            tv = np.unique(np.concatenate([o.vertex_key(o.key_to_cell(cells, R) + d, R) for d in o.CORNERS]))[:n]
            items = []
            for k, part in enumerate(np.array_split(tv, C)):
                nb, ok = o.axis_neighbours(part, R)
                keys = np.unique(np.concatenate([part, nb[ok]]))
                pth = os.path.join(tmp, f"tv_{tag}_{k}.npz")
                np.savez(pth, tv=part, keys=keys, vals=init(keys))
                items.append((pth, R, counts["V_tv"]))
            return items, len(tv)

        def make_adam(n, tag):
            items = []
            for k in range(C):
                m = n // C
                pth = os.path.join(tmp, f"adam_{tag}_{k}.npz")
                np.savez(pth, d=rng.normal(size=m), g=rng.normal(size=m), m=rng.normal(size=m) * 1e-3,
                         v=rng.random(m) * 1e-6)
                items.append((pth, wl["lr"]))
            return items, m * C

        # Calibration: a small sample of each phase.
        n0 = 2 * C
        ti, qs = make_terms(64 * C, "cal")
        t_q = pool.terms(ti) / (64 * C)
        t_nn = pool.nn(make_nn(qs, n0, "cal")) / n0
        tvi, ntv = make_tv(4096 * C, "cal")
        t_tv = pool.tv(tvi) / ntv
        adi, nad = make_adam(65536 * C, "cal")
        t_ad = pool.adam(adi) / nad
        # Size each phase to a quarter of the per-step budget.
        per = budget_s / max(1, steps) / 4.0
        n_nn = int(max(C, min(64 * C, per / max(t_nn, 1e-9))))
        n_q = int(max(C, min(8192 * C, per / max(t_q, 1e-9))))
        n_tv = int(max(C, min(1 << 20, per / max(t_tv, 1e-9))))
        n_ad = int(max(C, min(1 << 22, per / max(t_ad, 1e-9))))
        ti, qs = make_terms(n_q, "run")
        nni = make_nn(qs, n_nn, "run")
        tvi, n_tv = make_tv(n_tv, "run")
        adi, n_ad = make_adam(n_ad, "run")
        step_s = []
        for _ in range(max(1, steps)):
            a = pool.nn(nni) / n_nn
            b = pool.terms(ti) / n_q
            c = pool.tv(tvi) / n_tv
            d = pool.adam(adi) / n_ad
            step_s.append(B * (a + b) + counts["V_tv"] * c + counts["V_trainable"] * d)
            parts = {"nn_s": B * a, "query_terms_s": B * b, "tv_s": counts["V_tv"] * c,
                     "adam_s": counts["V_trainable"] * d}
        t_step = float(np.median(step_s))
        sample = (f"per step on {C} cores: brute-force NN of {n_nn} queries over all {J} points, sampler + query terms "
                  f"and gradient of {n_q} queries (band-sparse values), L_TV of {n_tv} TV vertices, Adam on {n_ad} "
                  f"vertices; extrapolated to B = {B}, |T| = {counts['V_tv']}, V_trainable = {counts['V_trainable']}")
        return {"value": B / t_step, "unit": UNIT, "cores": C, "kind": "oracle", "sample": sample,
                "step_s": t_step, "parts_s": {k: round(v, 3) for k, v in parts.items()}, "steps": len(step_s)}
    finally:
        pool.close()
        import shutil
        shutil.rmtree(tmp, ignore_errors=True)


def run_reference(args, world, rank):
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    pts = wl["cloud"]()
    t_start = time.perf_counter()
    counts = band_counts(pts, wl["R"], wl["M1"], wl["M2"])
    # The W + K steps' timed phases take about 120 s of wall time in all.
    cpu = oracle_baseline(pts, wl, counts, budget_s=120.0, steps=args.steps + args.warmup)
    elapsed = time.perf_counter() - t_start
    rate = cpu["value"]
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wl["B"] / rate,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": wl["desc"], "host_seconds": round(elapsed, 1)},
           "cpu_baseline": cpu,
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------- our arm
def query_form_times(gb, ctx, band, fit, tuned, workload, reps):
    """The query kernel's time (CUDA events of the library's tracing, µs per
    launch) in every form and launch shape gp_band_autotune chooses among, on
    step 0's batch; the band's choice is restored afterwards."""
    import torch
    from paper_2308_13175_gb300.fit import PAPER_WEIGHTS
    epoch, first, count = fit.batch_of(0)
    cands = [(f, r, b) for f in (gb.GP_QUERY_DIRECT, gb.GP_QUERY_WINDOW) for r in (1, 2) for b in (2, 3, 4)]
    cands += [(gb.GP_QUERY_WINDOW_STAGED, r, 2) for r in (1, 2)]
    names = {gb.GP_QUERY_DIRECT: "direct", gb.GP_QUERY_WINDOW: "window", gb.GP_QUERY_WINDOW_STAGED: "window_staged"}
    out = []
    for f, r, b in cands:
        gb.gp_band_set_query_form(band, f)
        gb.gp_band_set_query_tiles(band, r, b)
        for _ in range(2):
            gb.gp_step(band, fit.rec, count, fit.grad, fit.loss, PAPER_WEIGHTS, nvalid=fit.nvalid)
        torch.cuda.synchronize()
        gb.gp_profile(ctx, True)
        for _ in range(reps):
            gb.gp_step(band, fit.rec, count, fit.grad, fit.loss, PAPER_WEIGHTS, nvalid=fit.nvalid)
        prof = gb.gp_profile_read(ctx)
        gb.gp_profile(ctx, False)
        n, ms = prof["k_query"]
        out.append({"form": names[f], "records_per_thread": r, "blocks_per_sm": b,
                    "us_per_launch": round(1000.0 * ms / n, 2)})
    gb.gp_band_set_query_form(band, tuned["form"])
    gb.gp_band_set_query_tiles(band, tuned["records_per_thread"], tuned["blocks_per_sm"])
    gb.gp_band_check(band)
    return {"workload": workload, "records": count, "autotuned": tuned, "query_forms": out}


def run_ours(args, world, rank, local):
    import torch
    from paper_2308_13175_gb300 import binding as gb
    from paper_2308_13175_gb300 import build as gbuild
    from paper_2308_13175_gb300.fit import FitStep, PAPER_WEIGHTS

    if not os.path.exists(gb.lib_path()):
        gbuild.build()
    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload]
    pts = wl["cloud"]()
    R = wl["R"]
    ctx = gb.gp_create(local)
    band = gb.gp_build_band(ctx, torch.from_numpy(pts).cuda(), R, wl["M1"], wl["M2"], 50, nn_grid=args.nn_grid,
                            deterministic=args.deterministic)
    if wl.get("init") == "sphere_noise":
        # The single-sphere configuration's initial field: |x| - 0.5 plus
        # N(0, 0.01) noise (variance 0.01, std 0.1).
        gb.gp_band_init_sphere(band, (0.0, 0.0, 0.0), 0.5, 0.1, seed=0)
    else:
        c = 0.5 * (pts.min(0) + pts.max(0))
        gb.gp_band_init_sphere(band, c, 2.0 * 2.0 / R, 0.0, seed=0)
    fit = FitStep(band, wl["Q"], wl["B"], seed=rank, weights=PAPER_WEIGHTS, lr=wl["lr"],
                  deterministic=args.deterministic)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    info = band.info

    def timed_steps(first_t, K, profile=False):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        queries = 0
        for k in range(K):
            t = first_t + k
            flush.fill_(float(k))          # L2 flush outside the timed events
            starts[k].record(stream)
            fit.run(t)
            ends[k].record(stream)
            queries += fit.batch_of(t)[2]
        torch.cuda.synchronize()
        ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        return ms, queries

    tuned = fit.autotune(0)
    if args.query_forms:
        print(json.dumps(query_form_times(gb, ctx, band, fit, tuned, args.workload, max(args.steps, 1))))
        return

    def pipelined_steps(first_t, K):
        """K steps as one region, each next batch's draw overlapped with the
        current step (FitStep.run_pipelined); no flush between steps."""
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        queries = sum(fit.batch_of(first_t + k)[2] for k in range(K))
        e0.record(stream)
        fit.run_pipelined(first_t, K)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), queries

    for t in range(args.warmup):
        fit.run(t)
    fit.run_pipelined(args.warmup, 2)
    torch.cuda.synchronize()
    t0 = args.warmup + 2
    # The headline region: the pipelined steps when the step's working set
    # (values, moments, gradient, records, points) is larger than L2, so that
    # no flush is needed between steps; otherwise the sequential steps with an
    # L2 flush between them.
    l2 = int(getattr(torch.cuda.get_device_properties(local), "L2_cache_size", 129 * 2 ** 20))
    working_set = 16 * info["V_stored"] + 24 * wl["B"] + 16 * info["J"]
    pipelined_headline = working_set > l2 and not args.no_pipeline
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = gb.gp_launch_count(ctx)
    if pipelined_headline:
        t_ms, queries = pipelined_steps(t0, args.steps)
    else:
        ms, queries = timed_steps(t0, args.steps)
        t_ms = sum(ms)
    launches = gb.gp_launch_count(ctx) - launches0
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_max = reduce_max(t_ms, world)
    q_total = reduce_sum(float(queries), world)
    value = q_total / (t_max / 1e3)
    t_next = t0 + args.steps
    # The other form, for comparison.
    if pipelined_headline:
        ms_o, q_o = timed_steps(t_next, args.steps)
        other = {"form": "sequential (L2 flushed between steps)", "value": q_o / (sum(ms_o) / 1e3),
                 "ms_per_step": sum(ms_o) / args.steps}
    else:
        pm, q_o = pipelined_steps(t_next, args.steps)
        other = {"form": "pipelined (no flush)", "value": q_o / (pm / 1e3), "ms_per_step": pm / args.steps}
    t_next += args.steps

    # Per-kernel durations: sequential steps again with the library's
    # CUDA-event tracing on (events on the launching stream).
    gb.gp_profile(ctx, True)
    ms_prof, q_prof = timed_steps(t_next, args.steps)
    gb.gp_profile(ctx, False)
    t_next += args.steps
    kern = gb.gp_profile_read(ctx)
    peak, peak_kind = peaks()
    J, Vs, Vt = info["J"], info["V_stored"], info["V_trainable"]
    per_kernel = {}
    for name, (cnt, tot) in kern.items():
        per_step_n = q_prof / args.steps
        by = alg_bytes(name, per_step_n, J, Vs, Vt)
        avg_ms = tot / cnt
        per_kernel[name] = {"launches": cnt, "avg_us": round(1e3 * avg_ms, 2),
                            "share": round(tot / max(sum(v[1] for v in kern.values()), 1e-12), 4),
                            "alg_bytes": int(by), "gbs": round(by / (avg_ms / 1e3) / 1e9, 1) if by else None}
    fba = fwd_bwd_adam(per_kernel, ("k_count_valid", "k_tv", "k_tv_inv", "k_tv_grad", "k_query", "k_adam", "k_tv_adam"),
                       q_prof / args.steps,
                       Vt, peak)
    dom = max(kern.items(), key=lambda kv: kv[1][1])[0]
    dk = per_kernel[dom]
    nn_work = None
    nn_name = next((k for k in NN_KERNELS if k in per_kernel), None)
    if nn_name is not None:
        # Candidate distances of one launch, counted on the batches of the
        # next two steps (the same search, the counting variant of the kernel).
        cands = []
        for t in (t_next, t_next + 1):
            epoch, first, count = fit.batch_of(t)
            gb.gp_sample(band, fit.seed, epoch, fit.Q, first, count, fit.q, fit.src, spatial=True)
            nn_tmp = torch.empty(count, dtype=torch.int32, device="cuda")
            cands.append(gb.gp_nn_work(band, fit.q[:count], nn_tmp, hint=fit.src[:count]) / count)
        per_q = float(np.mean(cands))
        nk = per_kernel[nn_name]
        q_launch = q_prof / nk["launches"]
        tfl = per_q * q_launch * NN_FLOPS_PER_CANDIDATE / (nk["avg_us"] * 1e-6) / 1e12
        fp32_peak, fp32_kind = fp32_peak_tflops(torch.cuda.get_device_properties(local).multi_processor_count)
        nn_work = {"kernel": nn_name, "candidates_per_query": round(per_q, 2),
                   "candidates_per_s": per_q * q_launch / (nk["avg_us"] * 1e-6), "fp32_tflops": round(tfl, 3),
                   "fp32_peak_tflops": round(fp32_peak, 2), "frac": round(tfl / fp32_peak, 4),
                   "peak_kind": fp32_kind}
    if dom in NN_KERNELS and nn_work is not None:
        roofline = {"bound": "alu", "kernel": dom, "achieved": nn_work["fp32_tflops"],
                    "peak": nn_work["fp32_peak_tflops"], "unit": "TFLOP/s", "frac": nn_work["frac"],
                    "traffic": NCU_TRAFFIC.get((args.workload, dom)), "peak_kind": nn_work["peak_kind"],
                    "work": f"{NN_FLOPS_PER_CANDIDATE} FP32 flops per candidate distance, "
                            f"{nn_work['candidates_per_query']} candidates per query (gp_nn_work)"}
    else:
        achieved = dk["gbs"] or 0.0
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "traffic": NCU_TRAFFIC.get((args.workload, dom)), "peak_kind": peak_kind}

    # Mesh extraction of the band as the steps left it (outside the timed
    # region): marching cubes over the optimised cells, each kernel traced.
    # Algorithmic bytes per launch: every active brick's 512 values and 16
    # trainable-mask words once (the +1 apron re-reads are overhead), plus the
    # 36-byte triangles the emit pass writes.
    mesh = None
    if rank == 0 and not args.deterministic and not args.no_mesh:
        # A field worth meshing: every stored vertex gets its exact distance
        # to the cloud (gp_nn on the vertex positions) less half a cell, whose
        # zero set is a thin closed sheet around the points - the shape a
        # fitted band takes, where the steps above have barely moved the
        # initial sphere.
        ijk, _, fl = gb.gp_band_export(band)
        inside = (fl & 4) != 0
        vq = (-1.0 + (2.0 / R) * ijk.to(torch.float32)).contiguous()
        del ijk
        vnn = torch.empty(vq.shape[0], dtype=torch.int32, device="cuda")
        gb.gp_nn(band, vq, vnn, None)
        pts_t = torch.from_numpy(pts).cuda()
        dist = torch.linalg.norm(vq - pts_t[vnn.clamp(min=0).long()], dim=1) - 0.5 * (2.0 / R)
        gb.gp_band_set_values(band, torch.where(inside, dist, torch.zeros_like(dist)).contiguous())
        del vq, vnn, dist, pts_t, inside, fl
        gb.gp_mesh_extract(band, 0.0, with_cells=False)  # warm-up
        gb.gp_profile(ctx, True)
        t_host = time.perf_counter()
        runs = 5
        for _ in range(runs):
            tri, _ = gb.gp_mesh_extract(band, 0.0, with_cells=False)
        torch.cuda.synchronize()
        t_host = (time.perf_counter() - t_host) / runs
        gb.gp_profile(ctx, False)
        mk = gb.gp_profile_read(ctx)
        T = int(tri.shape[0])
        nact = info["n_active_bricks"]
        mesh = {"triangles": T, "active_bricks": nact, "ms_per_call_host": round(1e3 * t_host, 3), "kernels": {}}
        for name in ("k_mesh_count", "k_mesh_emit", "k_mesh_count_w", "k_mesh_emit_w"):
            if name not in mk:
                continue
            cnt, tot = mk[name]
            by = nact * (512 * 4 + 64) + (36 * T if name.startswith("k_mesh_emit") else 4 * nact)
            avg_s = tot / cnt / 1e3
            mesh["kernels"][name] = {"launches": cnt, "avg_us": round(1e6 * avg_s, 2), "alg_bytes": int(by),
                                     "gbs": round(by / avg_s / 1e9, 1), "frac": round(by / avg_s / 1e9 / peak, 4)}
        # Metrics of that mesh against the input cloud (Sec. 4: CD_L1, CD_L2,
        # HD, F; no reference normals, so no NC): quadrature, the two bands'
        # cell lists, the two nearest-point passes and their reductions.
        from paper_2308_13175_gb300 import metrics as gmetrics
        if T > 0:
            pts_dev = torch.from_numpy(pts).cuda()
            gmetrics.surface_metrics(ctx, tri, pts_dev, None)  # warm-up
            gb.gp_profile(ctx, True)
            t_host = time.perf_counter()
            res = gmetrics.surface_metrics(ctx, tri, pts_dev, None)
            torch.cuda.synchronize()
            t_host = time.perf_counter() - t_host
            gb.gp_profile(ctx, False)
            ek = gb.gp_profile_read(ctx)
            mesh["metrics"] = {"cd_l1": res["cd_l1"], "cd_l2": res["cd_l2"], "hd": res["hd"],
                               "fscore": {str(k): v for k, v in res["fscore"].items()},
                               "mesh_points": res["points"], "reference_points": int(len(pts)),
                               "ms_host": round(1e3 * t_host, 3),
                               "kernels_us": {k: round(1e3 * v[1] / v[0], 2) for k, v in ek.items()}}
            del pts_dev
        del tri

    # End to end through the public API on the headline's kind of batch: the
    # queries and source points of NH steps are drawn by the device sampler
    # (the spatially ordered batches the headline steps on) and kept in pinned
    # host memory before timing.  In the timed region every step copies its
    # batch from the host, runs gp_nn (seeded) and the descent (FitStep's
    # form) and copies its loss back to pinned host memory.  Where the
    # headline is pipelined (working set larger than L2) the copy of batch
    # k + 2 and the search of batch k + 1 run on two more streams while step k
    # descends, as FitStep.run_pipelined overlaps its draws; otherwise the
    # steps run in turn with an L2 flush before each, the next copy
    # overlapped.  The K steps are timed as one region.
    B = wl["B"]
    K = args.steps
    NH = min(K, 8)  # distinct host batches, reused in turn
    t_e2e = t_next
    t_next += K
    hq = torch.empty((NH, B, 3), dtype=torch.float32).pin_memory()
    hsrc = torch.empty((NH, B), dtype=torch.int32).pin_memory()
    counts_h = []
    for k in range(NH):
        epoch, first, count = fit.batch_of(t_e2e + k)
        gb.gp_sample(band, fit.seed, epoch, fit.Q, first, count, fit.q, fit.src, spatial=True)
        hq[k, :count].copy_(fit.q[:count])
        hsrc[k, :count].copy_(fit.src[:count])
        counts_h.append(count)
    torch.cuda.synchronize()
    hloss = torch.empty((K, 8), dtype=torch.float32).pin_memory()
    dq = [torch.empty((B, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    dsrc = [torch.empty(B, dtype=torch.int32, device="cuda") for _ in range(2)]
    copy_stream, search_stream = torch.cuda.Stream(), torch.cuda.Stream()
    _, hi_prio = torch.cuda.Stream.priority_range()
    step_stream = torch.cuda.Stream(priority=hi_prio) if pipelined_headline else stream
    if not pipelined_headline:
        search_stream = stream
    side_streams = []
    for st_ in (copy_stream, search_stream, step_stream):
        if st_.cuda_stream != stream.cuda_stream and all(st_.cuda_stream != o.cuda_stream for o in side_streams):
            side_streams.append(st_)
    copied = [torch.cuda.Event() for _ in range(2)]
    searched = [torch.cuda.Event() for _ in range(2)]
    stepped = [torch.cuda.Event() for _ in range(2)]
    queried = [torch.cuda.Event() for _ in range(2)]

    def e2e_copy(k):
        b = k % 2
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(searched[b])  # the search of step k - 2 has read dq[b]
            dq[b].copy_(hq[k % NH], non_blocking=True)
            dsrc[b].copy_(hsrc[k % NH], non_blocking=True)
            copied[b].record(copy_stream)

    def e2e_search(k, after=None):
        b, n = k % 2, counts_h[k % NH]
        with torch.cuda.stream(search_stream):
            search_stream.wait_event(copied[b])
            if after is not None:
                search_stream.wait_event(after)  # the previous step's gp_step is done (so is step k - 2)
            elif k >= 2:
                search_stream.wait_event(stepped[b])  # step k - 2 has read buffer b's records
            gb.gp_nn(band, dq[b][:n], None, fit.bufs[b]["rec"], hint=dsrc[b][:n], nvalid_out=fit.bufs[b]["nvalid"])
            searched[b].record(search_stream)

    barrier(world)
    torch.cuda.synchronize()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for st_ in side_streams:
        st_.wait_stream(stream)
    e2e_q = 0
    e2e_copy(0)
    if K > 1:
        e2e_copy(1)
    if pipelined_headline:
        e2e_search(0)
    # As FitStep.run_pipelined: with the separate descent the next search
    # waits for the current gp_step and overlaps its Adam update; with the
    # fused one it is issued beside the whole descent.
    overlap_all = fit.fused
    for k in range(K):
        b, n = k % 2, counts_h[k % NH]
        if pipelined_headline:
            if overlap_all and k + 1 < K:
                e2e_search(k + 1)
        else:
            flush.fill_(float(k))
            e2e_search(k)
        if k + 2 < K:
            e2e_copy(k + 2)
        with torch.cuda.stream(step_stream):
            step_stream.wait_event(searched[b])
            if fit.fused:
                fit._descend(t_e2e + k, fit.bufs[b], n)
            else:
                buf = fit.bufs[b]
                gb.gp_step(band, buf["rec"], n, fit.grad, fit.loss, fit.weights, nvalid=buf["nvalid"], flags=fit.flags)
                queried[b].record(step_stream)
                gb.gp_update(band, fit.grad, fit.lr_at(t_e2e + k), t_e2e + k + 1)
            hloss[k].copy_(fit.loss, non_blocking=True)
            stepped[b].record(step_stream)
        if pipelined_headline and not overlap_all and k + 1 < K:
            e2e_search(k + 1, after=queried[b])
        e2e_q += n
    for st_ in side_streams:
        stream.wait_stream(st_)
    e_end.record(stream)
    e_end.synchronize()
    e2e_ms = reduce_max(e_start.elapsed_time(e_end), world)
    e2e_value = reduce_sum(float(e2e_q), world) / (e2e_ms / 1e3)
    loss_final = float(hloss[K - 1][gb.GP_LOSS_TOTAL])

    # Plain PyTorch autograd on the same GPU and the same records: Eq. 8 in torch
    # ops (index gathers), loss.backward(), torch.optim.Adam with the frozen
    # vertices masked; beside it our gp_step + gp_update on those records.
    torch_cmp = None
    if not args.no_torch:
        from paper_2308_13175_gb300.torch_reference import from_band
        ts = from_band(band, device="cuda", dtype=torch.float32)
        Dt = gb.gp_band_values(band)[0].clone().requires_grad_(True)
        opt = torch.optim.Adam([Dt], lr=wl["lr"])
        while fit.batch_of(t_next)[2] != B:  # a full batch of the epoch
            t_next += 1
        fit._draw(t_next, fit.bufs[0])
        t_next += 1
        rec = fit.bufs[0]["rec"].clone()
        nv = fit.bufs[0]["nvalid"].clone()
        for _ in range(3):
            ts.step(Dt, opt, rec, PAPER_WEIGHTS)
        Kt = max(3, min(args.steps, 10))
        t_ms, o_ms = [], []
        for k in range(Kt):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ts.step(Dt, opt, rec, PAPER_WEIGHTS)
            e1.record(stream)
            torch.cuda.synchronize()
            t_ms.append(e0.elapsed_time(e1))
            flush.fill_(float(k))
            e0.record(stream)
            gb.gp_step_update(band, rec, B, fit.loss, wl["lr"], t_next + k + 1, PAPER_WEIGHTS, nvalid=nv,
                              flags=fit.flags)
            e1.record(stream)
            torch.cuda.synchronize()
            o_ms.append(e0.elapsed_time(e1))
        tq = B / (float(np.median(t_ms)) / 1e3)
        oq = B / (float(np.median(o_ms)) / 1e3)
        torch_cmp = {"value": tq, "unit": UNIT, "scope": f"loss + backward + Adam over the same {B} step records",
                     "ours_same_scope": oq, "speedup_same_scope": oq / tq, "speedup_full_step": value / tq,
                     "torch_ms": float(np.median(t_ms)), "ours_ms": float(np.median(o_ms))}
        del ts, Dt, opt

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        counts = {"V_tv": info["V_tv"], "V_trainable": Vt}
        cpu = oracle_baseline(pts, wl, counts, budget_s=args.cpu_budget, steps=1)
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": wl["desc"], "parallelism": f"replicas x{world}", "nn_grid": info["nn_grid"],
                          "timed": ("K pipelined steps as one region (each next batch's sampling and nearest "
                                    "points on a second stream)" if pipelined_headline else
                                    "K sequential steps, CUDA events around each"),
                          "l2": (f"inputs larger than L2: working set {working_set / 2**20:.0f} MiB > L2 "
                                 f"{l2 / 2**20:.0f} MiB, no flush" if pipelined_headline else
                                 "flushed between timed steps (256 MB write outside the step events)"),
                          "V_stored": Vs, "V_trainable": Vt, "V_tv": info["V_tv"], "J": J,
                          "gradient_sum": "deterministic two-word fixed point" if args.deterministic
                          else "float atomics",
                          "query_tiles": tuned,
                          "brick": 8},
               "roofline": roofline, "cpu_baseline": cpu,
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16 * B, "d2h_bytes_per_step": 32,
                       "path": ("host batches (the device sampler's spatially ordered queries and their "
                                "source points, drawn before timing) -> H2D copy -> gp_nn (seeded) -> " +
                                ("gp_step_update" if fit.fused else "gp_step + gp_update") +
                                " -> loss to host; " +
                                (("copy of step k + 2 and search of step k + 1 on two more streams while step k "
                                  "descends" if fit.fused else
                                  "copy of step k + 2 on a second stream; search of step k + 1 on a third once step "
                                  "k's gp_step is done, beside its gp_update") if pipelined_headline else
                                 "steps in turn, L2 flush before each, next copy on a second stream") +
                                "; K steps timed as one region")},
               "gpu_launches": int(launches), "clocks": clk, "kernels": per_kernel, "fwd_bwd_adam": fba,
               "nn_work": nn_work, "other_form": other,
               "mesh": mesh,
               "torch_autograd": torch_cmp,
               "loss_last": loss_final}
        print(json.dumps(out), flush=True)
    gb.gp_band_check(band)


# ------------------------------------------------- many clouds at once
def run_collection(args, world, rank, local):
    """The batched form: every shape of the collection stepped together by
    gp_multi_step, autotuned, captured once as a CUDA graph and replayed."""
    import torch
    from paper_2308_13175_gb300 import binding as gb
    from paper_2308_13175_gb300 import build as gbuild
    from paper_2308_13175_gb300 import synth
    from paper_2308_13175_gb300.fit import PAPER_WEIGHTS

    if not os.path.exists(gb.lib_path()):
        gbuild.build()
    torch.cuda.set_device(local)
    wl = WORKLOADS["collection"]
    shapes = synth.shape_collection(wl["n_shapes"], seed=3)
    ctx = gb.gp_create(local)
    bands, Qs, Bs = [], [], []
    for pts, R in shapes:
        band = gb.gp_build_band(ctx, torch.from_numpy(pts).cuda(), R, wl["M1"], wl["M2"], 50)
        c = 0.5 * (pts.min(0) + pts.max(0))
        gb.gp_band_init_sphere(band, c, 2.0 * 2.0 / R, 0.0, seed=0)
        bands.append(band)
        Q = wl["q_per_point"] * len(pts)
        Qs.append(Q)
        Bs.append(-(-Q // wl["batches_per_epoch"]))
    multi = gb.gp_multi_create(ctx, bands, Qs, Bs, seed=rank, spatial=True, deterministic=args.deterministic)
    n = len(bands)
    loss = torch.zeros(8 * n, dtype=torch.float32, device="cuda")
    tune = gb.gp_multi_autotune(multi, PAPER_WEIGHTS)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def queries_at(t):
        tot = 0
        for Q, B in zip(Qs, Bs):
            nb = -(-Q // B)
            first = (t % nb) * B
            tot += min(B, Q - first)
        return tot

    def step():
        gb.gp_multi_step(multi, loss, PAPER_WEIGHTS, lr=wl["lr"])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = gb.gp_launch_count(ctx)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    per_step_launches = gb.gp_launch_count(ctx) - launches0
    t0 = args.warmup
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    queries = 0
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        graph.replay()
        ends[k].record(stream)
        queries += queries_at(t0 + k)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    t_max = reduce_max(t_ms, world)
    value = reduce_sum(float(queries), world) / (t_max / 1e3)
    t_next = t0 + args.steps

    # Per-kernel durations: eager steps with the library's event tracing on.
    Kp = min(args.steps, 20)
    gb.gp_profile(ctx, True)
    q_prof = 0
    for k in range(Kp):
        flush.fill_(float(k))
        step()
        q_prof += queries_at(t_next + k)
    torch.cuda.synchronize()
    gb.gp_profile(ctx, False)
    t_next += Kp
    kern = gb.gp_profile_read(ctx)
    peak, peak_kind = peaks()
    J = sum(len(p) for p, _ in shapes)
    Vs = sum(b.V_stored for b in bands)
    Vt = sum(b.info["V_trainable"] for b in bands)
    per_kernel = {}
    tot_all = max(sum(v[1] for v in kern.values()), 1e-12)
    for name, (cnt, tot) in kern.items():
        by = alg_bytes(name.replace("k_m_", "k_"), q_prof / Kp, J, Vs, Vt)
        if name == "k_m_perm":
            by = 8 * J / wl["batches_per_epoch"]  # an epoch's order, once per epoch
        avg_ms = tot / cnt
        per_kernel[name] = {"launches": cnt, "avg_us": round(1e3 * avg_ms, 2), "share": round(tot / tot_all, 4),
                            "alg_bytes": int(by), "gbs": round(by / (avg_ms / 1e3) / 1e9, 1) if by else None}
    fba = fwd_bwd_adam(per_kernel, ("k_m_tv", "k_m_query", "k_m_adam", "k_m_finish"), q_prof / Kp, Vt, peak)
    dom = max(kern.items(), key=lambda kv: kv[1][1])[0]
    # The search's candidate distances: k_m_nn walks each record's ball as
    # gp_nn does (same seeds, same walk), so gp_nn_work on every cloud's
    # records of the last step counts them.
    cand, nrec = 0, 0
    for k, band in enumerate(bands):
        rec_k, src_k, _ = gb.gp_multi_buffers(multi, k)
        sel = src_k >= 0
        qk = rec_k[sel][:, :3].contiguous()
        if len(qk) == 0:
            continue
        nn_tmp = torch.empty(len(qk), dtype=torch.int32, device="cuda")
        cand += gb.gp_nn_work(band, qk, nn_tmp, hint=src_k[sel].contiguous())
        nrec += len(qk)
    nn_work = None
    if nrec > 0 and "k_m_nn" in per_kernel:
        per_q = cand / nrec
        nk = per_kernel["k_m_nn"]
        tfl = per_q * (q_prof / Kp) * NN_FLOPS_PER_CANDIDATE / (nk["avg_us"] * 1e-6) / 1e12
        fp32_peak, fp32_kind = fp32_peak_tflops(torch.cuda.get_device_properties(local).multi_processor_count)
        nn_work = {"kernel": "k_m_nn", "candidates_per_query": round(per_q, 2),
                   "candidates_per_s": per_q * (q_prof / Kp) / (nk["avg_us"] * 1e-6), "fp32_tflops": round(tfl, 3),
                   "fp32_peak_tflops": round(fp32_peak, 2), "frac": round(tfl / fp32_peak, 4),
                   "peak_kind": fp32_kind}
    if dom == "k_m_nn" and nn_work is not None:
        roofline = {"bound": "alu", "kernel": dom, "achieved": nn_work["fp32_tflops"],
                    "peak": nn_work["fp32_peak_tflops"], "unit": "TFLOP/s", "frac": nn_work["frac"], "traffic": None,
                    "peak_kind": nn_work["peak_kind"],
                    "work": f"{NN_FLOPS_PER_CANDIDATE} FP32 flops per candidate distance, "
                            f"{nn_work['candidates_per_query']} candidates per query (gp_nn_work)"}
    else:
        achieved = per_kernel[dom]["gbs"] or 0.0
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind}

    # End to end through the public call: gp_multi_step from Python (no graph)
    # and the n x 8 loss slots read back to the host every step.
    hloss = torch.empty(8 * n, dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms, e2e_q = 0.0, 0
    Ke = min(args.steps, 50)
    for k in range(Ke):
        flush.fill_(float(k))
        e0.record(stream)
        step()
        hloss.copy_(loss, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_q += queries_at(t_next + k)
    e2e_ms = reduce_max(e2e_ms, world)
    e2e_value = reduce_sum(float(e2e_q), world) / (e2e_ms / 1e3)
    info = gb.gp_multi_get_info(multi)
    if rank == 0:
        Jk = [len(p) for p, _ in shapes]
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": wl["desc"], "parallelism": f"replicas x{world}", "shapes": n,
                          "J_total": J, "J_min": min(Jk), "J_max": max(Jk), "records_per_step": info["total_B"],
                          "V_stored": Vs, "V_trainable": Vt, "autotuned": {k: tune[k] for k in (
                              "records_per_tile", "blocks_per_sm_nn", "blocks_per_sm_tv", "blocks_per_sm_query")},
                          "l2": "flushed between timed steps (256 MB write outside the step events)",
                          "timed": "CUDA graph replays of one captured gp_multi_step",
                          "gradient_sum": "deterministic two-word fixed point" if args.deterministic
                          else "float atomics"},
               "roofline": roofline, "cpu_baseline": None,
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 32 * n},
               "gpu_launches": int(per_step_launches * args.steps), "clocks": clk, "kernels": per_kernel,
               "fwd_bwd_adam": fba, "nn_work": nn_work,
               "error_bits": info["error_bits"],
               "loss_last_mean": float(hloss.view(n, 8)[:, gb.GP_LOSS_TOTAL].mean())}
        print(json.dumps(out), flush=True)
    del graph
    multi.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scene", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of timed oracle work (all host cores) for the line's cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-torch", action="store_true", help="skip the plain PyTorch autograd comparison")
    ap.add_argument("--nn-grid", type=int, default=0, help="cells per axis of the point cell list (0 = automatic)")
    ap.add_argument("--no-mesh", action="store_true", help="skip the surface-extraction and metrics leg")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="time the sequential steps (L2 flushed between them) as the headline")
    ap.add_argument("--deterministic", action="store_true",
                    help="bit-reproducible gradient sums (fixed point) instead of float atomics")
    ap.add_argument("--query-forms", action="store_true",
                    help="print the query kernel's time in every form and launch shape the autotuner chooses among "
                         "(--steps launches each) instead of the bench line")
    ap.add_argument("--m1", type=int, default=None, help="override the pull bandwidth M1 (-1 = all grids)")
    ap.add_argument("--m2", type=int, default=None, help="override the TV bandwidth M2 (-1 = all grids)")
    args = ap.parse_args()
    if args.impl == "reference" and args.workload == "collection":
        ap.error("the oracle arm times the single-cloud workloads")
    if args.m1 is not None or args.m2 is not None:
        if args.workload == "collection":
            ap.error("--m1/--m2 apply to the single-cloud workloads")
        wl = dict(WORKLOADS[args.workload])
        wl["M1"] = wl["M1"] if args.m1 is None else args.m1
        wl["M2"] = wl["M2"] if args.m2 is None else args.m2
        name = lambda m: "all grids" if m < 0 else str(m)
        wl["desc"] += f"; bands overridden: M1 = {name(wl['M1'])}, M2 = {name(wl['M2'])}"
        WORKLOADS[args.workload] = wl
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "collection":
        run_collection(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
