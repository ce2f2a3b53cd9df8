"""The fitting step strung from the C ABI calls (Sec. 3 and Sec. 4 "Details").

``FitStep.run(t)`` performs step t of the fit over one batch of the epoch's
query pool: gp_sample (Gaussian queries around points visited in the epoch's
random order, emitted grouped by source point in the cloud's cell order) -> gp_nn (NN(q), step records; each search seeded with the
query's own source point) -> gp_step (Eq. 8 forward and
hand-written backward) -> gp_update (Adam).  All device buffers are allocated
once here; the calls themselves never allocate."""
from __future__ import annotations

import math

import torch

from . import binding as gb

# Sec. 4 "Details": alpha, beta, gamma of Eq. 8.
PAPER_WEIGHTS = (1.0, 1.0, 0.005)


class FitStep:
    def __init__(self, band: gb.Band, Q: int, B: int, seed: int = 0, weights=PAPER_WEIGHTS, lr: float = 1e-3,
                 lr_decay: float = 1.0, lr_every: int = 0, deterministic: bool = False):
        self.band = band
        self.Q, self.B = int(Q), int(min(B, Q))
        self.seed = int(seed)
        self.weights = tuple(float(w) for w in weights)
        self.lr, self.lr_decay, self.lr_every = float(lr), float(lr_decay), int(lr_every)
        self.flags = gb.GP_STEP_DETERMINISTIC if deterministic else 0
        self.batches_per_epoch = math.ceil(self.Q / self.B)
        dev = torch.device("cuda", band.ctx.device)
        self.q = torch.empty((self.B, 3), dtype=torch.float32, device=dev)
        self.src = torch.empty(self.B, dtype=torch.int32, device=dev)
        self.rec = torch.empty((self.B, 6), dtype=torch.float32, device=dev)
        self.grad = torch.empty(band.V_stored, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(8, dtype=torch.float32, device=dev)
        self.nvalid = torch.zeros(1, dtype=torch.int32, device=dev)

    def batch_of(self, t: int):
        epoch, b = divmod(int(t), self.batches_per_epoch)
        first = b * self.B
        return epoch, first, min(self.B, self.Q - first)

    def lr_at(self, t: int) -> float:
        if self.lr_every > 0:
            return self.lr * self.lr_decay ** (t // self.lr_every)
        return self.lr

    def autotune(self, t: int = 0) -> dict:
        """Draws step t's batch and its nearest points and lets gp_band_autotune
        choose the fused step kernel's tile size and blocks per SM on it
        (set-up: call before timing or graph capture).  Returns the choice."""
        band = self.band
        epoch, first, count = self.batch_of(t)
        gb.gp_sample(band, self.seed, epoch, self.Q, first, count, self.q, self.src, spatial=True)
        gb.gp_nn(band, self.q[:count], None, self.rec, hint=self.src[:count], nvalid_out=self.nvalid)
        return gb.gp_band_autotune(band, self.rec, count, self.weights, nvalid=self.nvalid)

    def run(self, t: int):
        """Step t (0-based); returns the loss buffer (device, 8 floats)."""
        band = self.band
        epoch, first, count = self.batch_of(t)
        gb.gp_sample(band, self.seed, epoch, self.Q, first, count, self.q, self.src, spatial=True)
        gb.gp_nn(band, self.q[:count], None, self.rec, hint=self.src[:count], nvalid_out=self.nvalid)
        gb.gp_step(band, self.rec, count, self.grad, self.loss, self.weights, nvalid=self.nvalid, flags=self.flags)
        gb.gp_update(band, self.grad, self.lr_at(t), t + 1)
        return self.loss


def fit_cloud(ctx: gb.Context, points, R: int = 256, M1: int = 3, M2: int = 14, iters: int = 1600,
              batch: int = 50_000, queries_per_point: int = 10, lr_voxels: float = 1.0, lr_decay: float = 0.3,
              lr_every: int = 400, weights=PAPER_WEIGHTS, init_radius_voxels: float = 2.0, knn_k: int = 50,
              seed: int = 0, deterministic: bool = False):
    """The whole fit of Sec. 3 with the defaults of Sec. 4 "Details": build the
    band of `points` ((J, 3) float32 on the device, in [-1, 1]^3), start from a
    sphere of init_radius_voxels cells about the cloud's bounding-box centre,
    and run `iters` steps of FitStep (a pool of queries_per_point queries per
    point, re-drawn every epoch; Adam at lr_voxels * h, times lr_decay every
    lr_every steps).  Returns (band, fit): the band holds the fitted values,
    fit.loss the last step's loss slots."""
    band = gb.gp_build_band(ctx, points, R, M1, M2, knn_k, deterministic=deterministic)
    lo = points.min(dim=0).values.cpu().numpy()
    hi = points.max(dim=0).values.cpu().numpy()
    h = 2.0 / R
    gb.gp_band_init_sphere(band, 0.5 * (lo + hi), init_radius_voxels * h, 0.0, seed=seed)
    fit = FitStep(band, Q=queries_per_point * band.info["J"], B=batch, seed=seed, weights=weights,
                  lr=lr_voxels * h, lr_decay=lr_decay, lr_every=lr_every, deterministic=deterministic)
    for t in range(iters):
        fit.run(t)
    return band, fit


def reconstruct(ctx: gb.Context, points, iso: float = 0.0, **fit_args):
    """fit_cloud, then marching cubes over the optimised cells at level iso.
    Returns (triangles (T, 3, 3) float32 on the device, band)."""
    band, _ = fit_cloud(ctx, points, **fit_args)
    tri, _ = gb.gp_mesh_extract(band, iso, with_cells=False)
    return tri, band
