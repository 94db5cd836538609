"""Learned RANSAC proposal (not part of the paper's method).

A small network (8 -> 64 -> 64 -> 1) scores each matched pair's chance of being
an inlier; RANSAC draws its first hypotheses in proportion to the score and
falls back to uniform sampling when a standard stop bound is not met, so the
inlier set is always judged by every match.  Labels come from plain RANSAC's
final inliers.  Every numerical step runs in liblp's kernels
(lp_mlp_features, lp_mlp_forward, lp_mlp_train_step, lp_ransac_prior); this
module only moves tensors between those calls and shuffles minibatches.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import lp


@dataclass
class PairMatches:
    """Compacted matches of one pair and their features, on the device."""
    pts: torch.Tensor      # (M_cap, 4) float32: xA, yA, xB, yB (first M rows used)
    rows: torch.Tensor     # (M_cap,) int32: A row of each pair
    d_M: torch.Tensor      # (1,) int32: M
    feat: torch.Tensor     # (M_cap, 8) float32
    M_cap: int

    @property
    def M(self) -> int:
        return int(self.d_M.item())


def pair_matches(ctx: lp.Context, fa: lp.Features, fb: lp.Features, stream=None) -> PairMatches:
    """lp_match + lp_compact + lp_mlp_features for one pair of described images."""
    m, d1, d2 = lp.match(ctx, fa, fb, stream)
    NA = fa.desc.shape[0]
    cap = max(NA, 1)
    pts = torch.zeros((cap, 4), dtype=torch.float32, device="cuda")
    rows = torch.zeros(cap, dtype=torch.int32, device="cuda")
    dM = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.lp_compact(fa.kp, fa.W, fb.kp, fb.W, m, NA, pts, rows, dM, stream)
    feat = torch.zeros((cap, 8), dtype=torch.float32, device="cuda")
    ctx.lp_mlp_features(fa.kp, fa.ori, fa.H, fa.W, fb.kp, fb.ori, fb.H, fb.W, m, d1, d2, rows, dM, NA, feat, stream)
    return PairMatches(pts, rows, dM, feat, NA)


def images_matches(ctx: lp.Context, A, B, stream=None) -> PairMatches:
    return pair_matches(ctx, lp.features(ctx, A, stream), lp.features(ctx, B, stream), stream)


def plain_labels(ctx: lp.Context, pm: PairMatches, pair_id: int = 0, stream=None) -> torch.Tensor:
    """uint8 (M_cap,) final inlier mask of plain (uniform) RANSAC: the labels."""
    _, inl, _, _ = lp.ransac(ctx, pm.pts, pair_id, pm.d_M, stream)
    return inl


def collect(ctx: lp.Context, pairs, pair_id0: int = 0) -> tuple[torch.Tensor, torch.Tensor]:
    """Labelled features of an iterable of (A, B) images: (N, 8) float32, (N,) uint8."""
    feats, labels = [], []
    for k, (A, B) in enumerate(pairs):
        pm = images_matches(ctx, A, B)
        y = plain_labels(ctx, pm, pair_id0 + k)
        M = pm.M
        feats.append(pm.feat[:M])
        labels.append(y[:M])
    return torch.cat(feats).contiguous(), torch.cat(labels).contiguous()


def train(mlp: lp.Mlp, feat: torch.Tensor, label: torch.Tensor, epochs: int = 4, batch: int = 4096,
          lr: float = 1e-3, seed: int = 0) -> list[float]:
    """Adam on the mean BCE-with-logits loss, shuffled minibatches.  Returns
    the loss of every minibatch (read back once, at the end)."""
    N = feat.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    nb = (N + batch - 1) // batch
    losses = torch.zeros(epochs * nb, dtype=torch.float32, device="cuda")
    k = 0
    for _ in range(epochs):
        perm = torch.randperm(N, generator=g, device="cuda")
        for b in range(0, N, batch):
            idx = perm[b:b + batch]
            f = feat.index_select(0, idx).contiguous()
            y = label.index_select(0, idx).contiguous()
            mlp.lp_mlp_train_step(f, y, idx.numel(), lr, losses[k:k + 1])
            k += 1
    return losses.cpu().tolist()


@dataclass
class GuidedResult:
    H: np.ndarray
    inliers: np.ndarray
    n_in: int
    best_t: int
    iters: int
    counts: list[int]


def guided_ransac(ctx: lp.Context, mlp: lp.Mlp, pm: PairMatches, guided_iters: int = 64, pair_id: int = 0,
                  want_counts: bool = False, stream=None) -> GuidedResult:
    cap = pm.M_cap if pm.M_cap > 0 else 1
    prob = torch.zeros(cap, dtype=torch.float32, device="cuda")
    mlp.lp_mlp_forward(pm.feat, pm.M_cap, pm.d_M, prob, None, stream)
    H = torch.zeros(9, dtype=torch.float64, device="cuda")
    inl = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    bt = torch.zeros(1, dtype=torch.int32, device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.lp_ransac_prior(pm.pts, pm.M_cap, pm.d_M, prob, guided_iters, pair_id, H, inl, n, bt, it, stream)
    counts = ctx.lp_diag_last_ransac_counts(guided_iters + ctx.cfg.ransac_iters) if want_counts else []
    M = pm.M
    return GuidedResult(H.cpu().numpy().reshape(3, 3), inl[:M].cpu().numpy(), int(n.item()), int(bt.item()),
                        int(it.item()), counts)


def iterations_to_reach(counts, target: int) -> int:
    """1 + the first hypothesis whose FP32 inlier count reaches target (len + 1 if none)."""
    for t, c in enumerate(counts):
        if c >= target:
            return t + 1
    return len(counts) + 1
