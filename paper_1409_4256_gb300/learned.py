"""Learned rotation proposal: train the MLP on dense-EMC responsibilities and
turn its top-M logits into candidate sets for the sparse Maximize.

Every numerical step runs in libemc (emc_features, emc_mlp_train_step,
emc_mlp_forward, emc_topm, emc_targets_from_scores); this module only holds
the parameters (torch device tensors), draws the seeded initial weights and
mini-batch order, and loops.
"""
from __future__ import annotations

import math

import numpy as np

from . import emc

SEED_MLP_INIT = 1006
SEED_SPLIT = 1007
HIDDEN = 512


class Proposal:
    """The MLP of the learned proposal (FP32 master weights on the device)."""

    def __init__(self, n_out: int, device="cuda", seed: int = SEED_MLP_INIT):
        import torch
        self.torch = torch
        self.n_out = int(n_out)
        self.ld_out = (self.n_out + 63) // 64 * 64
        self.device = torch.device(device)
        n = emc.mlp_param_count(self.n_out)
        rng = np.random.Generator(np.random.PCG64(seed))
        p = np.zeros(n, dtype=np.float32)
        o = 0
        for fan_out, ld in ((HIDDEN, HIDDEN),) * 3 + ((self.n_out, self.ld_out),):
            W = rng.normal(0.0, math.sqrt(2.0 / HIDDEN), size=(HIDDEN, fan_out))
            blk = np.zeros((HIDDEN, ld), dtype=np.float32)
            blk[:, :fan_out] = W
            p[o:o + HIDDEN * ld] = blk.ravel()
            o += HIDDEN * ld + ld  # weights, then a zero bias
        assert o == n
        self.params = torch.as_tensor(p, device=self.device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0

    def train(self, feat, tidx, tprob, rows: np.ndarray, epochs: int = 8, batch: int = 512,
              lr: float = 1e-3, seed: int = SEED_SPLIT, stream=None):
        """Adam over mini-batches of the frames `rows`; returns the mean loss
        of each epoch."""
        torch = self.torch
        R = tprob.shape[1]
        work = torch.empty(emc.mlp_work_size(self.n_out, batch), dtype=torch.uint8,
                           device=self.device)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        rng = np.random.Generator(np.random.PCG64(seed + 1))
        hist = []
        for _ in range(epochs):
            order = rows[rng.permutation(len(rows))]
            loss.zero_()
            nb = 0
            for s in range(0, len(order) - batch + 1, batch):
                idx = torch.as_tensor(order[s:s + batch], device=self.device)
                X = feat.index_select(0, idx).contiguous()
                ti = tidx.index_select(0, idx).contiguous()
                tp = tprob.index_select(0, idx).contiguous()
                self.step += 1
                emc.mlp_train_step(self.n_out, self.params, self.grads, self.m, self.v, self.step,
                                   lr, X, ti, tp, batch, R, work, loss, stream)
                nb += 1
            hist.append(float(loss.item()) / max(nb, 1))
        return hist

    def logits(self, feat, batch: int = 2048, stream=None):
        torch = self.torch
        n = feat.shape[0]
        out = torch.empty((n, self.ld_out), dtype=torch.float32, device=self.device)
        work = torch.empty(emc.mlp_work_size(self.n_out, batch), dtype=torch.uint8,
                           device=self.device)
        for s in range(0, n, batch):
            b = min(batch, n - s)
            emc.mlp_forward(self.n_out, self.params, feat[s:s + b], b, work, out[s:s + b], stream)
        return out

    def propose(self, feat, M: int, n_frames: int, batch: int = 2048, first=None, stream=None):
        """Top-M rotations per frame: int32 [n_frames, M]. With `first`
        (int32 [n_frames, R], e.g. the top R of the last dense E-step), each set
        is those R followed by the network's best rotations not among them."""
        torch = self.torch
        if first is not None:
            net = self.propose(feat, M, n_frames, batch, stream=stream)
            return emc.merge_candidates(first, net, M, stream=stream)
        cand = torch.empty((n_frames, M), dtype=torch.int32, device=self.device)
        work = torch.empty(emc.mlp_work_size(self.n_out, batch), dtype=torch.uint8,
                           device=self.device)
        z = torch.empty((batch, self.ld_out), dtype=torch.float32, device=self.device)
        for s in range(0, n_frames, batch):
            b = min(batch, n_frames - s)
            emc.mlp_forward(self.n_out, self.params, feat[s:s + b], b, work, z, stream)
            emc.topm(z, b, self.n_out, self.ld_out, M, cand[s:s + b], stream)
        return cand


def split_rows(n_data: int, held_out: float = 0.1, seed: int = SEED_SPLIT):
    """Seeded train / held-out split of the frame indices."""
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(n_data)
    n_test = int(round(held_out * n_data))
    return np.sort(perm[n_test:]), np.sort(perm[:n_test])
