"""The fitting step strung from the C ABI calls (Sec. 3 and Sec. 4 "Details").

``FitStep.run(t)`` performs step t of the fit over one batch of the epoch's
query pool: gp_sample (Gaussian queries around points visited in the epoch's
random order, emitted grouped by source point in the cloud's cell order) ->
gp_nn (NN(q), step records; each search seeded with the query's own source
point) -> gp_step (Eq. 8 forward and hand-written backward) -> gp_update
(Adam).  ``FitStep.run_pipelined(t0, K)`` runs K such steps with each next
batch's sampling and nearest points overlapped on a second stream.  All
device buffers are allocated once here; the calls themselves never
allocate."""
from __future__ import annotations

import math

import torch

from . import binding as gb

# Sec. 4 "Details": alpha, beta, gamma of Eq. 8.
PAPER_WEIGHTS = (1.0, 1.0, 0.005)


class FitStep:
    def __init__(self, band: gb.Band, Q: int, B: int, seed: int = 0, weights=PAPER_WEIGHTS, lr: float = 1e-3,
                 lr_decay: float = 1.0, lr_every: int = 0, deterministic: bool = False, fused=None):
        self.band = band
        self.Q, self.B = int(Q), int(min(B, Q))
        self.seed = int(seed)
        self.weights = tuple(float(w) for w in weights)
        self.lr, self.lr_decay, self.lr_every = float(lr), float(lr_decay), int(lr_every)
        self.flags = gb.GP_STEP_DETERMINISTIC if deterministic else 0
        # fused: gp_step_update (no gradient array); else gp_step then gp_update.
        # Default: fused for the deterministic sums (its sweep folds them in at
        # no extra pass; measured 1.6x faster there), separate otherwise (the
        # two forms measured within 5% of each other).
        self.fused = bool(deterministic) if fused is None else bool(fused)
        self.batches_per_epoch = math.ceil(self.Q / self.B)
        dev = torch.device("cuda", band.ctx.device)
        self.device = dev
        # Two sets of per-batch buffers: the pipelined form fills one while the
        # step reads the other; run(t) uses the first.
        self.bufs = [{"q": torch.empty((self.B, 3), dtype=torch.float32, device=dev),
                      "src": torch.empty(self.B, dtype=torch.int32, device=dev),
                      "rec": torch.empty((self.B, 6), dtype=torch.float32, device=dev),
                      "nvalid": torch.zeros(1, dtype=torch.int32, device=dev)} for _ in range(2)]
        self.q, self.src = self.bufs[0]["q"], self.bufs[0]["src"]
        self.rec, self.nvalid = self.bufs[0]["rec"], self.bufs[0]["nvalid"]
        self.grad = torch.empty(band.V_stored, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(8, dtype=torch.float32, device=dev)
        self._streams = None

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

    def _draw(self, t: int, buf: dict):
        """Sampling and nearest points of step t's batch into buf (neither
        reads the grid values)."""
        epoch, first, count = self.batch_of(t)
        gb.gp_sample(self.band, self.seed, epoch, self.Q, first, count, buf["q"], buf["src"], spatial=True)
        gb.gp_nn(self.band, buf["q"][:count], None, buf["rec"], hint=buf["src"][:count], nvalid_out=buf["nvalid"])
        return count

    def _descend(self, t: int, buf: dict, count: int):
        """Eq. 8 forward and backward on buf's records, then Adam."""
        if self.fused:
            gb.gp_step_update(self.band, buf["rec"], count, self.loss, self.lr_at(t), t + 1, self.weights,
                              nvalid=buf["nvalid"], flags=self.flags)
            return
        gb.gp_step(self.band, buf["rec"], count, self.grad, self.loss, self.weights, nvalid=buf["nvalid"],
                   flags=self.flags)
        gb.gp_update(self.band, self.grad, self.lr_at(t), t + 1)

    def run(self, t: int):
        """Step t (0-based); returns the loss buffer (device, 8 floats)."""
        count = self._draw(t, self.bufs[0])
        self._descend(t, self.bufs[0], count)
        return self.loss

    def run_pipelined(self, t0: int, K: int):
        """Steps t0 .. t0 + K - 1, the same as run(t0), ..., run(t0 + K - 1),
        with each next batch's sampling and nearest points on a second stream
        overlapping part of the current step on a third: the draw does not read
        the grid values, so only the record buffers need ordering (two of
        them, alternating).  With the separate descent (gp_step, then
        gp_update) the next draw starts once the current gp_step is done and
        overlaps its Adam update: measured on the 10M-point scene, letting it
        overlap gp_step's L_TV passes and query pass too made the step slower
        than running everything in turn (the search and those passes contend
        for L2), while overlapping Adam only made it faster.  With the fused
        descent (gp_step_update, whose sweep holds every SM) the draw is
        issued beside the whole descent.  The calling stream waits for
        everything before this returns (asynchronously, as every call here).
        Returns the loss buffer of the last step."""
        if K <= 0:
            return self.loss
        if self._streams is None:
            lo, hi = torch.cuda.Stream.priority_range()
            self._streams = (torch.cuda.Stream(self.device), torch.cuda.Stream(self.device, priority=hi))
            self._events = [[torch.cuda.Event() for _ in range(2)] for _ in range(3)]
        sa, sb = self._streams
        drawn, stepped, queried = self._events
        cur = torch.cuda.current_stream(self.device)
        sa.wait_stream(cur)
        sb.wait_stream(cur)
        counts = {}

        def draw(t, after=None):
            p = t % 2
            with torch.cuda.stream(sa):
                if after is not None:
                    sa.wait_event(after)
                elif t - 2 >= t0:
                    sa.wait_event(stepped[p])  # step t - 2 has read buffer p
                counts[t] = self._draw(t, self.bufs[p])
                drawn[p].record(sa)

        def descend(t):
            p = t % 2
            buf = self.bufs[p]
            with torch.cuda.stream(sb):
                sb.wait_event(drawn[p])
                if self.fused:
                    self._descend(t, buf, counts[t])
                else:
                    gb.gp_step(self.band, buf["rec"], counts[t], self.grad, self.loss, self.weights,
                               nvalid=buf["nvalid"], flags=self.flags)
                    queried[p].record(sb)  # buffer p's records are read; step t - 1 is done
                    gb.gp_update(self.band, self.grad, self.lr_at(t), t + 1)
                stepped[p].record(sb)

        draw(t0)
        for t in range(t0, t0 + K):
            if self.fused:
                if t + 1 < t0 + K:
                    draw(t + 1)
                descend(t)
            else:
                descend(t)
                if t + 1 < t0 + K:
                    draw(t + 1, after=queried[t % 2])
        cur.wait_stream(sa)
        cur.wait_stream(sb)
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
