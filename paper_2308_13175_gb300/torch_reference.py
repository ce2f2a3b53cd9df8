"""The same step written in plain PyTorch ops with autograd.

This is the comparison form: the loss of Eq. 8 (Eq. 3-7 inside) over a set of
step records, differentiated by ``loss.backward()`` and optimised by
``torch.optim.Adam``, on the same band values.  It is what one would write
without custom kernels; the benchmark times it beside the CUDA path on the same
GPU, and the tests use it (in float64) as an independent derivation of the
gradient.  It is not called by the library's own path.

Storage follows the band: a flat value vector indexed by slot, with
``slot_keys`` giving the vertex key i + (R+1)(j + (R+1)k) of each slot (or a
negative number for padding slots).  A dense grid is the special case
slot_keys = arange((R+1)^3).
"""
from __future__ import annotations

import torch

CORNERS = [(k & 1, (k >> 1) & 1, (k >> 2) & 1) for k in range(8)]


class TorchStep:
    """Loss of Eq. 8 on a band, in torch ops (autograd-differentiable in the values)."""

    def __init__(self, R: int, slot_keys, tv_mask, train_mask, pull_cell_mask, device="cpu",
                 dtype=torch.float64):
        self.R = int(R)
        self.device = torch.device(device)
        self.dtype = dtype
        n1 = self.R + 1
        keys = torch.as_tensor(slot_keys, dtype=torch.int64, device=self.device)
        self.V = keys.numel()
        self.slot_of = torch.full((n1 ** 3,), -1, dtype=torch.int64, device=self.device)
        ok = keys >= 0
        self.slot_of[keys[ok]] = torch.nonzero(ok).flatten()
        self.pull = torch.as_tensor(pull_cell_mask, dtype=torch.bool, device=self.device)
        self.train = torch.as_tensor(train_mask, dtype=torch.bool, device=self.device)
        tv_slots = torch.nonzero(torch.as_tensor(tv_mask, dtype=torch.bool, device=self.device)).flatten()
        tv_keys = keys[tv_slots]
        ijk = torch.stack([tv_keys % n1, (tv_keys // n1) % n1, tv_keys // (n1 * n1)], dim=1)
        offs = torch.tensor([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]],
                            device=self.device)
        nb = ijk[:, None, :] + offs[None]
        inside = ((nb >= 0) & (nb <= self.R)).all(dim=2)
        nbk = nb.clamp(0, self.R)
        nbk = nbk[..., 0] + n1 * (nbk[..., 1] + n1 * nbk[..., 2])
        self.tv_slots = tv_slots
        self.tv_nbr = torch.where(inside, self.slot_of[nbk], torch.zeros_like(nbk))
        self.tv_in = inside & (self.slot_of[nbk] >= 0)
        self.n_tv = tv_slots.numel()

    # -- pieces ---------------------------------------------------------------
    def _cells(self, x):
        t = (x.to(self.dtype) + 1.0) * (self.R / 2.0)
        c = torch.floor(t)
        return c.to(torch.int64), t - c

    def _interp(self, D, cell, local):
        n1 = self.R + 1
        wx = torch.stack([1 - local[:, 0], local[:, 0]], 1)
        wy = torch.stack([1 - local[:, 1], local[:, 1]], 1)
        wz = torch.stack([1 - local[:, 2], local[:, 2]], 1)
        f = 0.0
        g = 0.0
        for dx, dy, dz in CORNERS:
            key = (cell[:, 0] + dx) + n1 * ((cell[:, 1] + dy) + n1 * (cell[:, 2] + dz))
            d = D[self.slot_of[key].clamp(min=0)]
            sx, sy, sz = (1.0 if dx else -1.0), (1.0 if dy else -1.0), (1.0 if dz else -1.0)
            f = f + wx[:, dx] * wy[:, dy] * wz[:, dz] * d
            g = g + torch.stack([sx * wy[:, dy] * wz[:, dz], wx[:, dx] * sy * wz[:, dz],
                                 wx[:, dx] * wy[:, dy] * sz], 1) * d[:, None]
        return f, g * (self.R / 2.0)

    @staticmethod
    def _unit(g):
        return g / torch.clamp(torch.linalg.vector_norm(g, dim=1, keepdim=True), min=1e-12)

    def loss(self, D, rec, weights=(1.0, 1.0, 0.005), tv: bool = True):
        """Returns (L, parts dict).  D: values (V,), rec: (B, 6) records."""
        alpha, beta, gamma = weights
        R = self.R
        q = rec[:, :3].to(self.dtype)
        s = rec[:, 3:].to(self.dtype)
        cq, lq = self._cells(rec[:, :3])
        cs, ls = self._cells(rec[:, 3:])
        inside = ((cq >= 0) & (cq <= R - 1)).all(dim=1)
        cs_c = cs.clamp(0, R - 1)
        ls = ls + (cs - cs_c).to(self.dtype)
        cq_c = cq.clamp(0, R - 1)
        pull_q = self.pull[cq_c[:, 0] + R * (cq_c[:, 1] + R * cq_c[:, 2])]
        pull_s = self.pull[cs_c[:, 0] + R * (cs_c[:, 1] + R * cs_c[:, 2])]
        valid = inside & pull_q & pull_s
        f, g = self._interp(D, cq_c[valid], lq[valid])
        fs, gs = self._interp(D, cs_c[valid], ls[valid])
        n = self._unit(g)
        ns = self._unit(gs)
        r = (q[valid] - s[valid]) - f[:, None] * n
        l_pull = torch.linalg.vector_norm(r, dim=1)
        l_grad = 1.0 - (n * ns).sum(1)
        l_surf = fs.abs()
        bv = int(valid.sum())
        den = max(bv, 1)
        parts = {"l_pull": l_pull.sum() / den, "l_grad": l_grad.sum() / den, "l_surf": l_surf.sum() / den,
                 "Bv": bv}
        L = parts["l_pull"] + beta * parts["l_surf"] + gamma * parts["l_grad"]
        if tv and self.n_tv:
            di = D[self.tv_slots][:, None]
            diff = torch.where(self.tv_in, di - D[self.tv_nbr], torch.zeros_like(di))
            tvv = torch.sqrt((diff * diff).sum(1))
            parts["l_tv"] = tvv.mean()
            L = L + alpha * parts["l_tv"]
        else:
            parts["l_tv"] = torch.zeros((), dtype=self.dtype, device=self.device)
        parts["loss"] = L
        return L, parts

    def step(self, D, opt, rec, weights=(1.0, 1.0, 0.005)):
        """One fitting step: loss, backward, freeze non-trainable, Adam."""
        opt.zero_grad(set_to_none=False)
        L, _ = self.loss(D, rec, weights)
        L.backward()
        D.grad.mul_(self.train.to(D.grad.dtype))
        opt.step()
        return L.detach()


def from_band(band, device="cuda", dtype=torch.float32) -> TorchStep:
    """TorchStep over a library band (through its export)."""
    from . import binding as gb
    ijk, _, fl = gb.gp_band_export(band)
    R = band.info["R"]
    n1 = R + 1
    ijk = ijk.to(torch.int64)
    exists = (fl & 4) != 0
    keys = torch.where(exists, ijk[:, 0] + n1 * (ijk[:, 1] + n1 * ijk[:, 2]), torch.full_like(ijk[:, 0], -1))
    pull = torch.zeros(R ** 3, dtype=torch.bool, device=device)
    pv = ijk[exists & ((fl & 8) != 0)]
    pull[pv[:, 0] + R * (pv[:, 1] + R * pv[:, 2])] = True
    return TorchStep(R, keys, (fl & 1) != 0, (fl & 2) != 0, pull, device=device, dtype=dtype)
