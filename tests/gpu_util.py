"""Helpers shared by the GPU parity tests: run liblp stages on numpy inputs.

Everything here goes through the C ABI (paper_2405_08578_gb300.lp); the oracle
is imported by the tests themselves.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_2405_08578_gb300 import lp


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def detect(ctx, img):
    """(kp uint32, gray uint8 HxW) from lp_detect on a gray or RGB numpy image."""
    buf, pitch = lp.pitched_device(img)
    H, W = img.shape[:2]
    ch = 3 if img.ndim == 3 else 1
    K = lp.lp_num_keypoints(H, W, ctx.Ls)
    kp = torch.full((max(K, 1),), -1, dtype=torch.int32, device="cuda")
    gray = torch.zeros(H * W + 16, dtype=torch.uint8, device="cuda") if ch == 3 else None
    ctx.lp_detect(buf, H, W, pitch, ch, kp, gray)
    g = host(gray)[:H * W].reshape(H, W) if ch == 3 else None
    return host(kp)[:K].astype(np.uint32), g


def describe(ctx, gray, kp, bf16=False):
    H, W = gray.shape
    buf, pitch = lp.pitched_device(gray)
    K = len(kp)
    k = dev(kp.astype(np.int64).astype(np.int32))
    ori = torch.zeros(max(K, 1), dtype=torch.uint8, device="cuda")
    desc = torch.zeros((max(K, 1), 128), dtype=torch.float32, device="cuda")
    d16 = torch.zeros((max(K, 1), 128), dtype=torch.bfloat16, device="cuda") if bf16 else None
    valid = torch.zeros(max(K, 1), dtype=torch.uint8, device="cuda")
    ctx.lp_describe(buf, H, W, pitch, k, K, ori, desc, d16, valid)
    out = (host(ori)[:K], host(desc)[:K], host(valid)[:K])
    if bf16:
        out = out + (host(d16.float())[:K],)
    return out


def match(ctx, dA, vA, dB, vB):
    NA, NB = len(dA), len(dB)
    A = dev(np.asarray(dA, np.float32))
    B = dev(np.asarray(dB, np.float32)) if NB else torch.zeros((1, 128), device="cuda")
    A16 = A.to(torch.bfloat16)
    B16 = B.to(torch.bfloat16)
    va = dev(np.asarray(vA, np.uint8))
    vb = dev(np.asarray(vB, np.uint8)) if NB else torch.zeros(1, dtype=torch.uint8, device="cuda")
    m = torch.zeros(max(NA, 1), dtype=torch.int32, device="cuda")
    d1 = torch.zeros(max(NA, 1), dtype=torch.float32, device="cuda")
    d2 = torch.zeros(max(NA, 1), dtype=torch.float32, device="cuda")
    ctx.lp_match(A, A16, va, NA, B, B16, vb, NB, m, d1, d2)
    return host(m)[:NA], host(d1)[:NA], host(d2)[:NA]


def compact(ctx, kpA, WA, kpB, WB, m):
    NA = len(m)
    pts = torch.zeros((max(NA, 1), 4), dtype=torch.float32, device="cuda")
    rows = torch.zeros(max(NA, 1), dtype=torch.int32, device="cuda")
    dM = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.lp_compact(dev(kpA.astype(np.int64).astype(np.int32)), WA, dev(kpB.astype(np.int64).astype(np.int32)), WB,
                   dev(np.asarray(m, np.int32)), NA, pts, rows, dM)
    M = int(host(dM)[0])
    return host(pts)[:M], host(rows)[:M]


def ransac(ctx, pts, pair_id=0, use_dM=True):
    pts = np.asarray(pts, np.float32).reshape(-1, 4)
    M = len(pts)
    p = dev(pts) if M else torch.zeros((1, 4), device="cuda")
    dM = dev(np.array([M], np.int32)) if use_dM else None
    H = torch.zeros(9, dtype=torch.float64, device="cuda")
    inl = torch.zeros(max(M, 1), dtype=torch.uint8, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    bt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.lp_ransac(p, M, dM, pair_id, H, inl, n, bt)
    return dict(H=host(H).reshape(3, 3), inliers=host(inl)[:M], n_in=int(host(n)[0]), best_t=int(host(bt)[0]))


def stitch(ctx, A, B, pair_id=0):
    bA, pA = lp.pitched_device(A)
    bB, pB = lp.pitched_device(B)
    ch = 3 if A.ndim == 3 else 1
    H = torch.zeros(9, dtype=torch.float64, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    M = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.lp_stitch_pair(bA, A.shape[0], A.shape[1], pA, bB, B.shape[0], B.shape[1], pB, ch, pair_id, H, n, M)
    return host(H).reshape(3, 3), int(host(n)[0]), int(host(M)[0])


def proj(H, p):
    q = np.c_[p, np.ones(len(p))] @ np.asarray(H).T
    return q[:, :2] / q[:, 2:]
