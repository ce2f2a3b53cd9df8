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

    def run(self, t: int):
        """Step t (0-based); returns the loss buffer (device, 8 floats)."""
        band = self.band
        epoch, first, count = self.batch_of(t)
        gb.gp_sample(band, self.seed, epoch, self.Q, first, count, self.q, self.src, spatial=True)
        gb.gp_nn(band, self.q[:count], None, self.rec, hint=self.src[:count], nvalid_out=self.nvalid)
        gb.gp_step(band, self.rec, count, self.grad, self.loss, self.weights, nvalid=self.nvalid, flags=self.flags)
        gb.gp_update(band, self.grad, self.lr_at(t), t + 1)
        return self.loss
