"""Benchmark: image pairs/s of the LP-SIFT hot path (detect -> describe ->
match -> RANSAC) on one 2688x1600 RGB pair per step, L = {16, 32, 64, 128}.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lp|reference]
                [--precision fp32|bf16]

One JSON line on rank 0.  `value` times K steps with the inputs resident in
HBM (L2 flushed between steps, outside the timed events); `e2e` times the
public host-buffer call lp_stitch_pairs_host over the K steps' pairs (H2D of
both images of every pair from pinned memory, D2H of every pair's H, inlier
and match count), and beside it one lp_stitch_pair_host call per pair.  `--impl reference` times the CPU oracle on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H_IMG, W_IMG = 1600, 2688
LS = (16, 32, 64, 128)
WORKLOAD = "pair_2688x1600_rgb"
METRIC = "image pairs/s at 2688x1600 (detect->RANSAC)"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


class L2Flush:
    """Evicts the 129 MB L2 between timed steps: writes a 256 MB buffer, then
    reads it back, so the next step starts with clean lines that hold none of
    its data (a write alone leaves the L2 full of dirty lines whose write-back
    would be charged to the next timed kernel)."""

    def __init__(self, nbytes: int = 256 << 20):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.acc = torch.zeros((), dtype=torch.int64, device="cuda")

    def __call__(self):
        import torch
        self.buf.zero_()
        torch.sum(self.buf.view(torch.int32), 0, dtype=torch.int64, out=self.acc)


# ----------------------------------------------------------------------------- CPU oracle sample
def oracle_pair_seconds(pair, rows_sample=1500, desc_sample=15000, seed=0, M=3000):
    """Single-thread FP64 oracle time for one pair, from a bounded sample:
    intensity + peaks in full, orientation+description of `desc_sample`
    random points per image (scaled to all K), matching of `rows_sample`
    random rows against all of B (scaled to all rows), RANSAC in full on the
    oracle's own matches of the sampled rows replicated to the full count."""
    import oracle
    rng = np.random.default_rng(seed)
    t = {}
    t0 = time.perf_counter()
    ga, gb = oracle.gray(pair.A), oracle.gray(pair.B)
    ka, kb = oracle.detect(ga, LS), oracle.detect(gb, LS)
    t["detect"] = time.perf_counter() - t0
    _, ws = oracle.keypoint_scales(H_IMG, W_IMG, LS)
    K = len(ka)
    t_desc = 0.0
    descs = []
    for g, kp in ((ga, ka), (gb, kb)):
        sel = np.sort(rng.choice(K, desc_sample, replace=False))
        t0 = time.perf_counter()
        o = oracle.orient(g, kp[sel], ws[sel])
        d, v = oracle.describe(g, kp[sel], ws[sel], o)
        t_desc += (time.perf_counter() - t0) * K / desc_sample
        descs.append((d, v))
    t["describe"] = t_desc
    # matching: sampled rows of A against a full-size B (sampled descriptors tiled to K rows)
    dA, vA = descs[0]
    dB = np.tile(descs[1][0], (K // desc_sample + 1, 1))[:K]
    vB = np.tile(descs[1][1], K // desc_sample + 1)[:K]
    t0 = time.perf_counter()
    oracle.match(dA[:rows_sample], vA[:rows_sample], dB, vB, rows=np.arange(rows_sample))
    t["match"] = (time.perf_counter() - t0) * K / rows_sample
    # RANSAC on a synthetic match set of the size the GPU path produces
    pa = rng.uniform(0, W_IMG, (M, 2)).round()
    pb = pa + np.array([800.0, 20.0]) + rng.normal(0, 0.5, (M, 2))
    pb[M // 2:] = rng.uniform(0, W_IMG, (M - M // 2, 2)).round()
    t0 = time.perf_counter()
    oracle.ransac(np.c_[pa, pb], T=1000, thresh=3.0, seed=0)
    t["ransac"] = time.perf_counter() - t0
    total = sum(t.values())
    sample = (f"full intensity+peaks of both images; orientation+descriptors of {desc_sample} random points per "
              f"image scaled to K={K}; {rows_sample} query rows x {K} candidates scaled to {K} rows; RANSAC 1000 "
              f"iterations on {M} matches")
    return total, t, sample


# ----------------------------------------------------------------------------- GPU arm
# DRAM bytes (read + write) of one launch of the distance kernel on this
# workload, from one ncu capture, valid only for the kernel source it was taken
# on (file SHA-1).
PROFILED_TRAFFIC = {
    "k_match_tc.cu": ("d06d4a49ea64a19a641e36e26566ae90b93a11b6", 44.02e6),
}


def profiled_traffic(src):
    import hashlib
    rec = PROFILED_TRAFFIC.get(src)
    if rec is None:
        return None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2405_08578_gb300", "csrc", src)
    with open(path, "rb") as f:
        return rec[1] if hashlib.sha1(f.read()).hexdigest() == rec[0] else None


def run_lp(args, rank, world):
    import torch
    import torch.distributed as dist

    from paper_2405_08578_gb300 import lp, synth

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    prec = lp.PREC_BF16 if args.precision == "bf16" else lp.PREC_FP32
    ctx = lp.Context(Ls=LS, precision=prec)
    pair = synth.pair_2688x1600(seed=rank)
    s = torch.cuda.current_stream()
    bA, pA = lp.pitched_device(pair.A)
    bB, pB = lp.pitched_device(pair.B)
    K = lp.lp_num_keypoints(H_IMG, W_IMG, LS)
    bf = prec == lp.PREC_BF16
    mk = lambda *shape, dt: torch.empty(*shape, dtype=dt, device="cuda")  # noqa: E731
    kpA, kpB = mk(K, dt=torch.int32), mk(K, dt=torch.int32)
    gA, gB = mk(H_IMG * W_IMG + 16, dt=torch.uint8), mk(H_IMG * W_IMG + 16, dt=torch.uint8)
    oA, oB = mk(K, dt=torch.uint8), mk(K, dt=torch.uint8)
    dA, dB = mk(K, 128, dt=torch.float32), mk(K, 128, dt=torch.float32)
    hA = mk(K, 128, dt=torch.bfloat16) if bf else None
    hB = mk(K, 128, dt=torch.bfloat16) if bf else None
    vA, vB = mk(K, dt=torch.uint8), mk(K, dt=torch.uint8)
    m, d1, d2 = mk(K, dt=torch.int32), mk(K, dt=torch.float32), mk(K, dt=torch.float32)
    pts, dM = mk(K, 4, dt=torch.float32), mk(1, dt=torch.int32)
    Hd, inl, nin = mk(9, dt=torch.float64), mk(K, dt=torch.uint8), mk(1, dt=torch.int32)
    flush = L2Flush()

    def step(ev=None):
        if ev:
            ev[0].record(s)
        ctx.lp_detect(bA, H_IMG, W_IMG, pA, 3, kpA, gA)
        ctx.lp_detect(bB, H_IMG, W_IMG, pB, 3, kpB, gB)
        ctx.lp_describe(gA, H_IMG, W_IMG, W_IMG, kpA, K, oA, dA, hA, vA)
        ctx.lp_describe(gB, H_IMG, W_IMG, W_IMG, kpB, K, oB, dB, hB, vB)
        if ev:
            ev[1].record(s)
        ctx.lp_match(dA, hA, vA, K, dB, hB, vB, K, m, d1, d2)
        if ev:
            ev[2].record(s)
        ctx.lp_compact(kpA, W_IMG, kpB, W_IMG, m, K, pts, None, dM)
        ctx.lp_ransac(pts, K, dM, rank, Hd, inl, nin)
        if ev:
            ev[3].record(s)

    # stage breakdown: the same pipeline call by call (detect, describe,
    # match, compact + RANSAC), each stage bracketed by events
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for i in range(args.steps):
        flush()
        step(evs[i])
    torch.cuda.synchronize()
    per = [[a.elapsed_time(b) for a, b in zip(e[:-1], e[1:])] for e in evs]
    t_match = sum(p[1] for p in per) / 1e3 / args.steps

    # the timed steps: one lp_stitch_pair per step (the whole path in one
    # call; image B is detected and described beside image A)
    Hs = mk(9, dt=torch.float64)
    ns = mk(1, dt=torch.int32)
    Ms = mk(1, dt=torch.int32)

    def pair_step():
        ctx.lp_stitch_pair(bA, H_IMG, W_IMG, pA, bB, H_IMG, W_IMG, pB, 3, rank, Hs, ns, Ms)

    for _ in range(args.warmup):
        pair_step()
    torch.cuda.synchronize()
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.lp_set_profiling(True)
    kern_ms = []
    with ClockSampler(dev) as clk:
        for i in range(args.steps):
            flush()
            pev[i][0].record(s)
            pair_step()
            pev[i][1].record(s)
            kern_ms.append(ctx.lp_diag_last_match_kernel_ms())   # events around the distance kernel
        torch.cuda.synchronize()
    ctx.lp_set_profiling(False)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_steps = sum(a.elapsed_time(b) for a, b in pev) / 1e3
    assert int(ns.item()) == int(nin.item()) and int(Ms.item()) == int(dM.item())
    stages = {"stage_calls_ms_per_pair": sum(sum(p) for p in per) / args.steps,
              "detect_describe_ms": 1e3 * sum(p[0] for p in per) / 1e3 / args.steps,
              "match_ms": 1e3 * t_match, "compact_ransac_ms": 1e3 * sum(p[2] for p in per) / 1e3 / args.steps}
    n_in = int(nin.item())
    M = int(dM.item())
    assert ctx.lp_sync_status() == 0
    rescans = ctx.lp_diag_last_rescans()

    # end to end through the public host-buffer call
    hostA = torch.from_numpy(np.ascontiguousarray(lp.pitched_device(pair.A)[0].cpu().numpy())).pin_memory()
    hostB = torch.from_numpy(np.ascontiguousarray(lp.pitched_device(pair.B)[0].cpu().numpy())).pin_memory()
    for _ in range(max(1, args.warmup // 2)):
        ctx.lp_stitch_pair_host(hostA, H_IMG, W_IMG, pA, hostB, H_IMG, W_IMG, pB, 3, rank)
    torch.cuda.synchronize()
    e2e_one = 0.0
    for i in range(args.steps):
        flush()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        ctx.lp_stitch_pair_host(hostA, H_IMG, W_IMG, pA, hostB, H_IMG, W_IMG, pB, 3, rank)
        b.record(s)
        b.synchronize()
        e2e_one += a.elapsed_time(b) / 1e3
    # the streamed form: all K steps in one lp_stitch_pairs_host call, every
    # step's two images copied from pinned host memory (pair q + 1's copies
    # beside pair q's computation) and every step's H, n_in and M read back
    stream_pairs = [(hostA, H_IMG, W_IMG, pA, hostB, H_IMG, W_IMG, pB)] * args.steps
    ctx.lp_stitch_pairs_host(stream_pairs[:2], 3, pair_id0=rank)
    flush()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    Hs_, ns_, Ms_ = ctx.lp_stitch_pairs_host(stream_pairs, 3, pair_id0=rank)
    b.record(s)
    b.synchronize()
    e2e_t = a.elapsed_time(b) / 1e3
    assert int(ns_[0]) == n_in and int(Ms_[0]) == M

    t_kern = sum(kern_ms) / 1e3 / args.steps
    tt = torch.tensor([t_steps, e2e_t, t_match, t_kern, e2e_one], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t_steps, e2e_t, t_match, t_kern, e2e_one = tt.tolist()
    return dict(t_steps=t_steps, e2e_t=e2e_t, e2e_one=e2e_one, t_match=t_match, t_kern=t_kern, stages=stages,
                clocks=clk.summary(), n_in=n_in, M=M,
                K=K, pair=pair, h2d=int(hostA.numel() + hostB.numel()), bf=bf, rescans=rescans)


def fp32_form_and_batch(args, rank):
    """Side measurements on the same GPU: the plain FP32 form of the same pair
    (the comparison the metric names) and the nine-tile batch (36 pairs, one
    lp_stitch_pairs call replayed as a CUDA graph)."""
    import torch

    from paper_2405_08578_gb300 import lp, synth
    out = {}
    s = torch.cuda.current_stream()
    flush = L2Flush()
    pair = synth.pair_2688x1600(seed=rank)
    ctx = lp.Context(Ls=LS, precision=lp.PREC_FP32)
    bA, pA = lp.pitched_device(pair.A)
    bB, pB = lp.pitched_device(pair.B)
    H = torch.zeros(9, dtype=torch.float64, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    M = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        ctx.lp_stitch_pair(bA, H_IMG, W_IMG, pA, bB, H_IMG, W_IMG, pB, 3, rank, H, n, M)
    torch.cuda.synchronize()
    k = max(3, args.steps // 3)
    t = 0.0
    for _ in range(k):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        ctx.lp_stitch_pair(bA, H_IMG, W_IMG, pA, bB, H_IMG, W_IMG, pB, 3, rank, H, n, M)
        b.record(s)
        torch.cuda.synchronize()
        t += a.elapsed_time(b) / 1e3
    out["fp32_form_pairs_per_s"] = k / t
    out["fp32_form_inliers"] = int(n.item())
    H32 = H.clone()
    del ctx
    # the E4M3 form of the same pair: its pairs/s, the distance passes' time
    # and rate against the FP8 dense peak (the measured BF16 peak x 2, the
    # nominal ratio), the rows its filter could not certify, equality with FP32
    ctx = lp.Context(Ls=LS, precision=lp.PREC_FP8)
    ctx.lp_set_profiling(True)
    for _ in range(2):
        ctx.lp_stitch_pair(bA, H_IMG, W_IMG, pA, bB, H_IMG, W_IMG, pB, 3, rank, H, n, M)
    torch.cuda.synchronize()
    t, tk = 0.0, 0.0
    for _ in range(k):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        ctx.lp_stitch_pair(bA, H_IMG, W_IMG, pA, bB, H_IMG, W_IMG, pB, 3, rank, H, n, M)
        b.record(s)
        torch.cuda.synchronize()
        t += a.elapsed_time(b) / 1e3
        tk += ctx.lp_diag_last_match_kernel_ms() / 1e3
    Kp = lp.lp_num_keypoints(H_IMG, W_IMG, LS)
    pk = peaks()[0]
    out["fp8_form"] = {"pairs_per_s": k / t, "distance_passes_ms": 1e3 * tk / k,
                       "distance_tflops_useful": 2.0 * Kp * Kp * 128 / (tk / k) / 1e12,
                       "frac_of_fp8_peak": 2.0 * Kp * Kp * 128 / (tk / k) / 1e12 / (2 * pk["bf16_tflops"]),
                       "fp8_peak_tflops": 2 * pk["bf16_tflops"], "fp8_peak_kind": "measured BF16 burst x 2 (nominal ratio)",
                       "rescanned_rows": int(ctx.lp_diag_last_rescans()), "rows": int(Kp),
                       "H_equals_fp32_form": bool(torch.equal(H, H32))}
    ctx.lp_set_profiling(False)
    del ctx
    bt = synth.batch_3x3(seed=1)
    ctx = lp.Context(Ls=LS, precision=lp.PREC_BF16)
    bufs = [lp.pitched_device(im) for im in bt.images]
    images = [(tb, H_IMG, W_IMG, pb, 3) for (tb, pb) in bufs]
    HM = torch.zeros((36, 9), dtype=torch.float64, device="cuda")
    ni = torch.zeros(36, dtype=torch.int32, device="cuda")
    va = torch.zeros(36, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ctx.lp_stitch_pairs(images, HM, ni, va)
    torch.cuda.synchronize()
    t = 0.0
    for _ in range(k):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        ctx.lp_stitch_pairs(images, HM, ni, va)
        b.record(s)
        torch.cuda.synchronize()
        t += a.elapsed_time(b) / 1e3
    out["batch_3x3"] = {"images": 9, "pairs": 36, "pairs_per_s": 36 * k / t, "ms_per_batch": 1e3 * t / k,
                        "valid_pairs": int(va.sum().item()), "graph": True}
    # the same batch through the plain FP32 form (FP32 SIMT distances): the
    # comparison the metric names, on identical work
    ctx32 = lp.Context(Ls=LS, precision=lp.PREC_FP32)
    HM32 = torch.zeros((36, 9), dtype=torch.float64, device="cuda")
    ni32 = torch.zeros(36, dtype=torch.int32, device="cuda")
    va32 = torch.zeros(36, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        ctx32.lp_stitch_pairs(images, HM32, ni32, va32)
    torch.cuda.synchronize()
    k32 = max(3, k // 2)
    t32 = 0.0
    for _ in range(k32):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        ctx32.lp_stitch_pairs(images, HM32, ni32, va32)
        b.record(s)
        torch.cuda.synchronize()
        t32 += a.elapsed_time(b) / 1e3
    ref = {"pairs_per_s": 36 * k32 / t32, "bf16_pairs_per_s": 36 * k / t,
           "HM": HM32.cpu().numpy().reshape(36, 3, 3), "n_in": ni32.cpu().numpy()}
    out["batch_3x3_fp32"] = {"pairs_per_s": ref["pairs_per_s"], "ms_per_batch": 1e3 * t32 / k32,
                             "valid_pairs": int(va32.sum().item()),
                             "bf16_equals_fp32": bool(torch.equal(HM, HM32) and torch.equal(ni, ni32))}
    del ctx32
    out["mosaic_3x3"] = mosaic(bt, images, ctx, HM, va, flush, k)
    out["detect_3x3"] = detect_batch(ctx, images, flush, k)
    out["table2"] = table2(flush)
    out["uneven_64"] = uneven_64(flush, max(3, k // 2))
    out["fp8_census"] = fp8_census()
    out["describe"] = describe_rate(flush)
    if args.train_pairs > 0:
        out["learned_proposal"] = learned_proposal(args, bt, images, ctx, HM, ni, va, flush, k, ref)
    return out


def mosaic(bt, images, ctx, HM, va, flush, k):
    """Sec. 4 on the nine-tile batch: the reference rounds over H_M (host) and
    the canvas warp (device), timed after the batch's H_M."""
    import torch

    from paper_2405_08578_gb300 import lp, shard
    pairs = shard.all_pairs(9)
    HMh, vh = HM.cpu().numpy(), va.cpu().numpy()
    t0 = time.perf_counter()
    plan = lp.lp_mosaic_plan(9, pairs, HMh, vh, [(H_IMG, W_IMG)] * 9)
    plan_ms = 1e3 * (time.perf_counter() - t0)
    ch, cw = plan["canvas"]
    pitch = (cw * 3 + 15) // 16 * 16
    canvas = torch.empty((ch, pitch), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    for _ in range(2):
        ctx.lp_mosaic_render(images, plan["G"], plan["round"], canvas, cw, ch, pitch)
    torch.cuda.synchronize()
    t = 0.0
    for _ in range(k):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        ctx.lp_mosaic_render(images, plan["G"], plan["round"], canvas, cw, ch, pitch)
        e1.record(s)
        torch.cuda.synchronize()
        t += e0.elapsed_time(e1) / 1e3
    placed = int((plan["round"] >= 0).sum())
    # each tile against the reference it was placed through, on their true overlap
    gy, gx = np.mgrid[0:H_IMG:64, 0:W_IMG:64]
    grid = np.c_[gx.ravel(), gy.ravel(), np.ones(gx.size)]
    err = 0.0
    for j, r in enumerate(plan["ref"]):
        if r < 0 or r == j:
            continue
        q = grid @ bt.H[(j, r)].T
        q = q[:, :2] / q[:, 2:]
        inside = (q[:, 0] >= 0) & (q[:, 0] <= W_IMG - 1) & (q[:, 1] >= 0) & (q[:, 1] <= H_IMG - 1)
        a = grid[inside] @ plan["G"][j].T
        b = np.c_[q[inside], np.ones(inside.sum())] @ plan["G"][r].T
        if len(a):
            err = max(err, float(np.abs(a[:, :2] / a[:, 2:] - b[:, :2] / b[:, 2:]).max()))
    bytes_alg = ch * cw * 3 + placed * H_IMG * W_IMG * 3
    return {"placed": placed, "rounds": int(plan["round"].max()) + 1, "canvas": [ch, cw], "plan_ms": round(plan_ms, 3),
            "placement_err_px": round(err, 2),
            "render_ms": 1e3 * t / k, "render_GBps_algorithmic": bytes_alg / (t / k) / 1e9}


def detect_batch(ctx, images, flush, k):
    """Sec. 2.1-2.2 on the nine RGB tiles: one lp_detect_batch against nine
    lp_detect calls.  Algorithmic bytes as the detect stage's work is counted:
    the RGB read once plus the 4-byte keys written; the intensity image that
    the describe stage reads (1 byte per pixel) is written as well and is
    reported separately, as the kernel's whole DRAM traffic.  Device time: after
    the L2 flush the stream spins for about 0.2 ms (torch.cuda._sleep) while
    the host enqueues the timed call, so the events bracket the launch alone
    and not the host's argument marshalling."""
    import torch

    from paper_2405_08578_gb300 import lp
    s = torch.cuda.current_stream()
    K = lp.lp_num_keypoints(H_IMG, W_IMG, LS)
    kps = [torch.empty(K, dtype=torch.int32, device="cuda") for _ in images]
    grays = [torch.empty(H_IMG * W_IMG + 16, dtype=torch.uint8, device="cuda") for _ in images]
    nbytes = len(images) * (H_IMG * W_IMG * 3 + 4 * K)
    nbytes_all = nbytes + len(images) * H_IMG * W_IMG

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        t = 0.0
        for _ in range(k):
            flush()
            torch.cuda._sleep(400_000)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) / 1e3
        return t / k

    tb = timed(lambda: ctx.lp_detect_batch(images, kps, grays))
    ts = timed(lambda: [ctx.lp_detect(t, h, w, p, ch, kp, g) for (t, h, w, p, ch), kp, g in zip(images, kps, grays)])
    pk = peaks()[0]
    return {"images": len(images), "algorithmic_MB": nbytes / 1e6,
            "bytes_model": "H*W*3 RGB read + 4*K keys written per image",
            "batch_ms": 1e3 * tb, "batch_GBps": nbytes / tb / 1e9, "batch_frac_hbm": nbytes / tb / 1e9 / pk["hbm_gbs"],
            "with_intensity_write_MB": nbytes_all / 1e6, "with_intensity_write_GBps": nbytes_all / tb / 1e9,
            "with_intensity_write_frac_hbm": nbytes_all / tb / 1e9 / pk["hbm_gbs"],
            "one_by_one_ms": 1e3 * ts, "one_by_one_GBps": nbytes / ts / 1e9}


# Table 2 stitching times of LP-SIFT (MATLAB on an i9-12900 CPU, detection to
# stitching), for context beside the per-pair device times below
TABLE2_PAPER_S = {"mountain": 1.16, "street_view": 2.05, "terrain": 4.47, "building": 2.03,
                  "campus_translation": 4.49, "campus_rotation": 4.58}


def table2(flush, k=10):
    """Per-pair device time of lp_stitch_pair (BF16) on stand-ins for Table 2's
    LP-SIFT rows: the printed sizes and window-size sets."""
    import torch

    from paper_2405_08578_gb300 import lp, synth
    out = {}
    s = torch.cuda.current_stream()
    for name in sorted(synth.TABLE2):
        p, Ls = synth.table2_pair(name)
        h, w = p.A.shape
        bA, pA = lp.pitched_device(p.A)
        bB, pB = lp.pitched_device(p.B)
        H = torch.zeros(9, dtype=torch.float64, device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        M = torch.zeros(1, dtype=torch.int32, device="cuda")
        row = {"W": w, "H": h, "Ls": list(Ls), "K_per_image": lp.lp_num_keypoints(h, w, Ls),
               "paper_matlab_s": TABLE2_PAPER_S[name]}
        for model, tag in ((lp.MODEL_HOMOGRAPHY, ""), (lp.MODEL_RIGID, "_rigid")):
            ctx = lp.Context(Ls=Ls, precision=lp.PREC_BF16, model=model)
            for _ in range(3):
                ctx.lp_stitch_pair(bA, h, w, pA, bB, h, w, pB, 1, 0, H, n, M)
            torch.cuda.synchronize()
            t = 0.0
            for _ in range(k):
                flush()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                ctx.lp_stitch_pair(bA, h, w, pA, bB, h, w, pB, 1, 0, H, n, M)
                e1.record(s)
                torch.cuda.synchronize()
                t += e0.elapsed_time(e1)
            row["ms_per_pair" + tag] = round(t / k, 4)
            row["inliers" + tag] = int(n.item())
            row["matches"] = int(M.item())
        out[name] = row
    return out


def _training_pair(seed: int):
    """One seeded 640x480 training pair (runs in a spawned worker process)."""
    from paper_2405_08578_gb300 import synth
    p = synth.pair_640x480_random(seed)
    return p.A, p.B


def training_pairs(seeds):
    """The training pairs in seed order, generated on the host's cores by a
    spawned process pool (no CUDA state is inherited) and streamed to the
    caller as they are ready."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    seeds = list(seeds)
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        yield from ex.map(_training_pair, seeds, chunksize=8)


def describe_rate(flush, k=10):
    """lp_describe on both images of the 2688x1600 pair, L2 flushed before
    each timed call: ms per image and samples per ns, where a point of region
    size w_s (Eq. 3-4) takes (4 w_s + 1)^2 orientation samples, (4 w_s + 2)^2
    turned-grid interpolations and 16 w_s^2 descriptor samples."""
    import torch

    from paper_2405_08578_gb300 import lp, synth
    pair = synth.pair_2688x1600(seed=0)
    ctx = lp.Context(Ls=LS, precision=lp.PREC_BF16)
    K = lp.lp_num_keypoints(H_IMG, W_IMG, LS)
    outs = []
    for im in (pair.A, pair.B):
        buf, pitch = lp.pitched_device(im)
        kp = torch.empty(K, dtype=torch.int32, device="cuda")
        g = torch.empty(H_IMG * W_IMG + 16, dtype=torch.uint8, device="cuda")
        ctx.lp_detect(buf, H_IMG, W_IMG, pitch, 3, kp, g)
        outs.append((g, kp, torch.empty(K, dtype=torch.uint8, device="cuda"),
                     torch.empty((K, 128), device="cuda"), torch.empty((K, 128), dtype=torch.bfloat16, device="cuda"),
                     torch.empty(K, dtype=torch.uint8, device="cuda")))
    s = torch.cuda.current_stream()

    def run():
        for (g, kp, o, d, d16, v) in outs:
            ctx.lp_describe(g, H_IMG, W_IMG, W_IMG, kp, K, o, d, d16, v)

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    t = []
    for _ in range(k):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        run()
        e1.record(s)
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1) / 2)
    t.sort()
    ms = t[len(t) // 2]
    # Eq. 3-4 with the default beta0 (the largest that keeps 4 w_s <= L):
    # w_s = round(beta0 sqrt(L Lmax) ), 2 (H/L)(W/L) points at scale L
    beta0 = math.sqrt(min(LS) / max(LS)) / 4
    samples = 0
    for L in LS:
        w = max(1, int(math.floor(beta0 * math.sqrt(L * max(LS)) + 0.5)))
        samples += 2 * (H_IMG // L) * (W_IMG // L) * ((4 * w + 1) ** 2 + (4 * w + 2) ** 2 + 16 * w * w)
    # the describe stage's work model: 16 w_s^2 descriptor samples per point
    # (4 w_s x 4 w_s region, Eq. 3-4) at about 70 FP32 operations each
    # (bilinear taps, gradient, direction, magnitude, binning); peak: 152 SMs x
    # 128 FP32 lanes x 2 (FMA) x the maximum SM clock
    desc_samples = 0
    for L in LS:
        w = max(1, int(math.floor(beta0 * math.sqrt(L * max(LS)) + 0.5)))
        desc_samples += 2 * (H_IMG // L) * (W_IMG // L) * 16 * w * w
    pk = peaks()[0]
    alu_peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = desc_samples * 70 / (ms * 1e-3) / 1e12
    return {"ms_per_image": ms, "points_per_image": int(K), "samples_per_image": samples,
            "samples_per_ns": samples / (ms * 1e6),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak, "work": f"{desc_samples} descriptor samples x 70 FP32 operations",
                         "note": "the kernels are bound by instruction issue (no pipe saturated; "
                                 "profiles/k_describe_pair_2688x1600.md): most of their work is integer, table and "
                                 "shared-memory work that this FP32 operation count leaves out"}}


def fp8_census(chunk=4096, margin=5e-3, capacity=192):
    """How many columns per row a certified low-precision filter must keep on
    the 2688x1600 pair, for BF16 (the built matcher's operands) and for E4M3
    with per-descriptor scaling (max entry -> 448).  For unit descriptors the
    estimate v~ = 1 - 2 a~.b~ of v = |b|^2 - 2 a.b is within
    delta(v) = c + k (1 + eps - v), k = 2u + u^2 (u = 2^-8 for BF16, 2^-4 for
    E4M3).  The window of a row is every column with v~ <= x + delta(x), x its
    exact second-best plus the certification margin (the smallest x any first
    pass could give).  Analysis only: plain torch matmuls, TF32 off."""
    import torch

    from paper_2405_08578_gb300 import lp, synth
    pair = synth.pair_2688x1600(seed=0)
    ctx = lp.Context(Ls=LS, precision=lp.PREC_BF16)
    fa, fb = lp.features(ctx, pair.A), lp.features(ctx, pair.B)
    A = fa.desc[fa.valid.bool()].float()
    B = fb.desc[fb.valid.bool()].float()
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    nb = (B * B).sum(1)

    def e4m3(X):
        s = 448.0 / X.abs().amax(1, keepdim=True).clamp_min(1e-30)
        return (X * s).to(torch.float8_e4m3fn).float(), s

    A8, sa = e4m3(A)
    B8, sb = e4m3(B)
    A16, B16 = A.bfloat16().float(), B.bfloat16().float()
    eps, c = 5e-5, 2e-4
    counts = {"bf16": [], "e4m3": []}
    for r0 in range(0, A.shape[0], chunk):
        a = A[r0:r0 + chunk]
        v = nb[None, :] - 2.0 * (a @ B.T)
        x = v.topk(2, dim=1, largest=False).values[:, 1:2] + margin
        for name, u, vt in (("bf16", 2.0 ** -8, 1.0 - 2.0 * (A16[r0:r0 + chunk] @ B16.T)),
                            ("e4m3", 2.0 ** -4, 1.0 - 2.0 * ((A8[r0:r0 + chunk] @ B8.T) / (sa[r0:r0 + chunk] * sb.T)))):
            k = 2 * u + u * u
            top = x + c + k * (1.0 + eps - x).clamp_min(0.0)
            counts[name].append((vt <= top).sum(1))
        del v
    torch.backends.cuda.matmul.allow_tf32 = tf32
    out = {"rows": int(A.shape[0]), "columns": int(B.shape[0]), "margin": margin, "list_capacity": capacity}
    for name, cs in counts.items():
        cs = torch.cat(cs).float()
        out[name] = {"mean": float(cs.mean()), "median": float(cs.median()),
                     "p99": float(cs.quantile(0.99)), "max": float(cs.max()),
                     "rows_over_capacity": int((cs > capacity).sum())}
    return out


def _uneven_pair(spec):
    """One pair of the uneven workload (runs in a spawned worker process)."""
    from paper_2405_08578_gb300 import synth
    p = synth.make_pair(*spec)
    return p.A, p.B, p.H


def _grid_dev(Ha, Hb, h, w, Href=None, step=32):
    """Largest distance (px) between Ha and Hb images of a grid of A's pixels
    that Href (default Ha) maps inside a w x h image B."""
    ys, xs = np.mgrid[0:h:step, 0:w:step]
    x = np.c_[xs.ravel(), ys.ravel(), np.ones(xs.size)]
    r = x @ np.asarray(Ha if Href is None else Href).T
    r = r[:, :2] / r[:, 2:]
    inside = (r[:, 0] >= 0) & (r[:, 0] < w) & (r[:, 1] >= 0) & (r[:, 1] < h)
    a = x[inside] @ np.asarray(Ha).T
    b = x[inside] @ np.asarray(Hb).T
    return float(np.abs(a[:, :2] / a[:, 2:] - b[:, :2] / b[:, 2:]).max(initial=0.0)), int(inside.sum())


def uneven_64(flush, k):
    """The 64-pair uneven workload (long sides U[480, 4096], aspect U[4/3,
    16/9], gray, L = {16, 32, 64, 128}) as one lp_stitch_pairs call with an
    explicit pair list, BF16 with and without the matcher's autotuner: pairs/s
    of each, the tuning table and the error against each pair's true
    homography."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import torch

    from paper_2405_08578_gb300 import lp, synth
    specs = synth.uneven_pair_specs(64, seed=2)
    t0 = time.time()
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        pairs = list(ex.map(_uneven_pair, specs))
    gen_s = time.time() - t0
    images, plist = [], []
    for q, (A, B, _) in enumerate(pairs):
        for im in (A, B):
            buf, pitch = lp.pitched_device(im)
            images.append((buf, im.shape[0], im.shape[1], pitch, 1))
        plist.append((2 * q, 2 * q + 1))
    s = torch.cuda.current_stream()
    res = {}
    for tuned in (False, True):
        ctx = lp.Context(Ls=LS, precision=lp.PREC_BF16)
        ctx.lp_set_autotune(tuned)
        HM = torch.zeros((64, 9), dtype=torch.float64, device="cuda")
        ni = torch.zeros(64, dtype=torch.int32, device="cuda")
        va = torch.zeros(64, dtype=torch.uint8, device="cuda")
        for _ in range(3):
            ctx.lp_stitch_pairs(images, HM, ni, va, pairs=plist)
        torch.cuda.synchronize()
        t = 0.0
        for _ in range(k):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            ctx.lp_stitch_pairs(images, HM, ni, va, pairs=plist)
            e1.record(s)
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) / 1e3
        assert ctx.lp_sync_status() == 0
        res[tuned] = dict(pps=64 * k / t, HM=HM.cpu().numpy().reshape(64, 3, 3), ni=ni.cpu().numpy(),
                          va=va.cpu().numpy(), table=ctx.lp_autotune_table() if tuned else [])
        del ctx
    out = {"pairs": 64, "images": 128, "long_side_px": [min(sp[1] for sp in specs), max(sp[1] for sp in specs)],
           "generate_s": round(gen_s, 1), "pairs_per_s_builtin_tiles": res[False]["pps"],
           "pairs_per_s_autotuned": res[True]["pps"], "autotune_table": res[True]["table"],
           "tuned_equals_builtin": bool(np.array_equal(res[True]["HM"], res[False]["HM"]) and
                                        np.array_equal(res[True]["ni"], res[False]["ni"])),
           "valid_pairs": int(res[True]["va"].sum())}
    # error against each pair's true homography over the true overlap
    dev_t = [_grid_dev(res[True]["HM"][q], pairs[q][2], pairs[q][0].shape[0], pairs[q][0].shape[1])[0]
             for q in range(64) if res[True]["va"][q]]
    out["truth_error_px"] = {"median": float(np.median(dev_t)) if dev_t else None,
                             "max": float(np.max(dev_t)) if dev_t else None}
    return out


def learned_proposal(args, bt, images, ctx, HM, ni, va, flush, k, ref=None):
    """Train the inlier-probability network on seeded 640x480 pairs labelled by
    plain RANSAC, then run the nine-tile batch with it guiding RANSAC: the
    iterations each pair needs to reach plain RANSAC's best count, whether the
    inlier sets agree, and the batch's pairs/s with the network attached."""
    import torch

    from paper_2405_08578_gb300 import lp, proposal, synth
    t0 = time.time()
    ctx_t = lp.Context(Ls=synth.PAIR_640x480_LS)
    seeds = range(1000, 1000 + args.train_pairs)
    feat, label = proposal.collect(ctx_t, training_pairs(seeds))
    collect_s = time.time() - t0
    net = lp.Mlp(seed=0)
    # about 100 passes over 4096-match minibatches per 100k matches, at least 4 epochs
    epochs = max(4, min(20, int(2.0e6 / max(1, feat.shape[0]))))
    t1 = time.time()
    losses = proposal.train(net, feat, label, epochs=epochs, batch=4096, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.time() - t1
    Tg, T = 64, ctx.cfg.ransac_iters
    feats = [lp.features(ctx, im) for im in bt.images]
    reach_u, reach_g, stopped, same, nvalid, q = [], [], 0, 0, 0, 0
    inl_pts = {}          # pair -> plain RANSAC's inlier points (xA, yA)
    dev_inl = 0.0         # guided vs plain H on plain's inliers, px
    pms = []
    for a in range(9):
        for b in range(a + 1, 9):
            pm = proposal.pair_matches(ctx, feats[a], feats[b])
            pms.append(pm)
            H_u, inl_u, n_u, _ = lp.ransac(ctx, pm.pts, q, pm.d_M)
            cu = ctx.lp_diag_last_ransac_counts(T)
            g = proposal.guided_ransac(ctx, net, pm, Tg, q, want_counts=True)
            q += 1
            if int(n_u.item()) < ctx.cfg.min_inliers:
                continue
            nvalid += 1
            sel = inl_u[:pm.M].cpu().numpy().astype(bool)
            pa = pm.pts[:pm.M, :2].cpu().numpy().astype(np.float64)[sel]
            inl_pts[q - 1] = pa
            hu = H_u.cpu().numpy().reshape(3, 3)
            x = np.c_[pa, np.ones(len(pa))]
            pu, pg = x @ hu.T, x @ g.H.T
            dev_inl = max(dev_inl, float(np.abs(pu[:, :2] / pu[:, 2:] - pg[:, :2] / pg[:, 2:]).max(initial=0.0)))
            target = max(cu)
            reach_u.append(proposal.iterations_to_reach(cu, target))
            reach_g.append(proposal.iterations_to_reach(g.counts[:Tg], target) if g.iters == Tg
                           else Tg + proposal.iterations_to_reach(g.counts[Tg:], target))
            stopped += g.iters == Tg
            same += bool(np.array_equal(g.inliers, inl_u[:pm.M].cpu().numpy()))
    # the RANSAC stage alone, pair after pair (no matching beside it): plain
    # lp_ransac against the proposal's forward pass + guided RANSAC
    s = torch.cuda.current_stream()

    def stage(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for qq, pm in enumerate(pms):
            fn(qq, pm)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    Hs_ = torch.zeros(9, dtype=torch.float64, device="cuda")
    ns_ = torch.zeros(1, dtype=torch.int32, device="cuda")
    inl_ = torch.zeros(max(pm.M_cap for pm in pms), dtype=torch.uint8, device="cuda")
    prob_ = torch.zeros(max(pm.M_cap for pm in pms), dtype=torch.float32, device="cuda")

    def plain(qq, pm):
        ctx.lp_ransac(pm.pts, pm.M_cap, pm.d_M, qq, Hs_, inl_, ns_, None)

    def guided(qq, pm):
        net.lp_mlp_forward(pm.feat, pm.M_cap, pm.d_M, prob_, None)
        ctx.lp_ransac_prior(pm.pts, pm.M_cap, pm.d_M, prob_, Tg, qq, Hs_, inl_, ns_, None, None)

    for fn in (plain, guided):
        stage(fn)
    ms_plain = min(stage(plain) for _ in range(3))
    ms_guided = min(stage(guided) for _ in range(3))
    ctx.lp_set_proposal(net, Tg)
    for _ in range(3):
        ctx.lp_stitch_pairs(images, HM, ni, va)
    torch.cuda.synchronize()
    t = 0.0
    for _ in range(k):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        ctx.lp_stitch_pairs(images, HM, ni, va)
        e1.record(s)
        torch.cuda.synchronize()
        t += e0.elapsed_time(e1) / 1e3
    ctx.lp_set_proposal(None)
    pps = 36 * k / t
    out = {"train_pairs": args.train_pairs, "train_matches": int(feat.shape[0]),
           "inlier_label_frac": float(label.float().mean().item()), "loss_first": losses[0], "loss_last": losses[-1],
           "epochs": epochs, "collect_s": round(collect_s, 1), "train_s": round(train_s, 1), "guided_iters": Tg,
           "valid_pairs": nvalid,
           "mean_iters_to_plain_best": {"uniform": float(np.mean(reach_u)) if reach_u else None,
                                        "guided": float(np.mean(reach_g)) if reach_g else None},
           "guided_stopped": stopped, "identical_inlier_sets": same,
           "max_reprojection_px_on_plain_inliers": dev_inl,
           "ransac_stage_ms_36_pairs": {"plain": ms_plain, "learned": ms_guided,
                                        "note": "pair after pair, nothing beside it; learned = forward pass + "
                                                "guided RANSAC with uniform fallback"},
           "batch_pairs_per_s": pps, "batch_valid_pairs": int(va.sum().item())}
    if ref is not None:
        # the same 36 pairs through the plain FP32 form: the metric's comparison
        hm = HM.cpu().numpy().reshape(36, 3, 3)
        n_l = ni.cpu().numpy()
        same_n = int((n_l == ref["n_in"]).sum())
        # both homographies on the FP32 form's valid pairs, at plain RANSAC's inlier points
        dev = 0.0
        for p_, pa in inl_pts.items():
            x = np.c_[pa, np.ones(len(pa))]
            a, b_ = x @ ref["HM"][p_].T, x @ hm[p_].T
            dev = max(dev, float(np.abs(b_[:, :2] / b_[:, 2:] - a[:, :2] / a[:, 2:]).max(initial=0.0)))
        out["vs_fp32_batch"] = {"fp32_batch_pairs_per_s": ref["pairs_per_s"],
                                "bf16_batch_pairs_per_s": ref["bf16_pairs_per_s"],
                                "bf16_learned_batch_pairs_per_s": pps,
                                "speedup_bf16_learned_vs_fp32": pps / ref["pairs_per_s"],
                                "speedup_bf16_vs_fp32": ref["bf16_pairs_per_s"] / ref["pairs_per_s"],
                                "learned_vs_plain_bf16": pps / ref["bf16_pairs_per_s"],
                                "pairs_with_equal_inlier_count": same_n,
                                "max_reprojection_px_on_inliers": dev}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lp", choices=["lp", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP32-form and 3x3-batch side measurements")
    ap.add_argument("--train-pairs", type=int, default=2000,
                    help="640x480 pairs that train the learned RANSAC proposal (0 skips it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        from paper_2405_08578_gb300 import synth
        pair = synth.pair_2688x1600(0)
        secs, walls = [], []
        for i in range(args.warmup + args.steps):
            w0 = time.perf_counter()
            tot, parts, sample = oracle_pair_seconds(pair, rows_sample=200, desc_sample=3000, seed=i)
            if i >= args.warmup:
                secs.append(tot)
                walls.append(time.perf_counter() - w0)
        # a step runs a bounded sample, pairs_per_step of one pair's work: the
        # sample's wall time over the whole pair's time scaled from it
        pps = [w / t for w, t in zip(walls, secs)]
        v = sum(pps) / sum(walls)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
                "pairs_per_step": sum(pps) / len(pps),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD, "H": H_IMG, "W": W_IMG, "Ls": list(LS),
                                                "flush": "n/a (CPU)",
                                                "timing": "sample-scaled: each step runs a bounded sample of the "
                                                          "pair (see cpu_baseline.sample), pairs_per_step of one "
                                                          "pair's work; ms_per_step is the step's measured wall "
                                                          "time, value the pairs/s this implies "
                                                          f"({1e3 * sum(secs) / len(secs):.0f} ms per whole pair, "
                                                          "scaled from the sample, not measured in full)"},
                "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
    r = run_lp(args, rank, world)
    if rank != 0:
        dist.destroy_process_group()
        return
    pk, pk_kind = peaks()
    K = r["K"]
    flops = 2.0 * K * K * 128
    if r["bf"]:
        roof = {"bound": "tensor", "achieved": flops / r["t_kern"] / 1e12, "peak": pk["bf16_tflops"],
                "unit": "TFLOP/s", "kernel": "k_match_tc pass 1 + k_row_threshold + k_match_tc pass 2",
                "launch_ms": 1e3 * r["t_kern"], "stage_tflops": flops / r["t_match"] / 1e12,
                "note": "achieved counts the useful 2*NA*NB*128 flops; the tensor pipe also runs pass 1 on a "
                        "third of the tiles; traffic is the DRAM bytes of both passes from one ncu capture"}
    else:
        sm_max = pk.get("sm_max_mhz", 2070.0)
        fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / r["t_kern"] / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                "kernel": "k_match_fp32_main", "launch_ms": 1e3 * r["t_kern"]}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = profiled_traffic("k_match_tc.cu" if r["bf"] else "k_match_fp32.cu")
    roof["peak_source"] = f"{pk_kind}" if r["bf"] else "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"
    value = world * args.steps / r["t_steps"]
    # our kernels per step (BF16 form): detect 2, describe 6, match 9 (two row
    # norms, pass 1, threshold, pass 2, re-rank, re-scan, re-scan merge,
    # finish), compact 2, RANSAC 9 (hypotheses, score, recount, argmax, three
    # refit sums, solve, final); FP32 form: match 4 (two row norms, main,
    # finish) and the rest as BF16
    # liblp kernels one lp_stitch_pair launches: detect 1; describe 4 per image
    # (two per-point-CTA scales, two warp-per-point scales); BF16 match 9 (two
    # row-norm launches, pass 1, thresholds, pass 2, re-rank, re-scan, merge,
    # finish) or FP32 match 4 (row norms x 2, distances, finish); compaction 2;
    # RANSAC 4 (hypotheses, score, recount, argmax); refit 5
    launches_per_step = 29 if r["bf"] else 24
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * r["t_steps"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if r["bf"] else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H_IMG, "W": W_IMG, "Ls": list(LS), "K_per_image": K,
                       "precision": args.precision, "flush": "L2 flushed between timed steps: a 256 MB buffer written, then read (L2 left holding clean, unrelated lines)",
                       "timed_call": "lp_stitch_pair, one per pair (detect, describe, match, compact, RANSAC); "
                                     "the *_ms stage figures come from the per-stage calls",
                       "matches": r["M"], "inliers": r["n_in"], "rescanned_rows": r["rescans"], "Mpix_per_s": value * 2 * H_IMG * W_IMG / 1e6,
                       **r["stages"]},
            "roofline": roof,
            "e2e": {"value": world * args.steps / r["e2e_t"], "unit": "pairs/s", "h2d_bytes_per_step": r["h2d"],
                    "d2h_bytes_per_step": 9 * 8 + 2 * 4,
                    "call": "lp_stitch_pairs_host over the K steps' pairs (copies of the next pair beside the "
                            "current pair's computation)",
                    "one_call_per_pair": world * args.steps / r["e2e_one"]},
            "gpu_launches": launches_per_step * args.steps, "clocks": r["clocks"]}
    if not args.no_extras:
        extra = fp32_form_and_batch(args, rank)
        line["config"]["fp32_form_pairs_per_s"] = extra["fp32_form_pairs_per_s"]
        line["config"]["speedup_vs_fp32_form"] = value / world / extra["fp32_form_pairs_per_s"]
        line["config"]["fp32_form_inliers"] = extra["fp32_form_inliers"]
        line["config"]["fp8_form"] = extra["fp8_form"]
        line["config"]["batch_3x3"] = extra["batch_3x3"]
        line["config"]["batch_3x3_fp32"] = extra["batch_3x3_fp32"]
        line["config"]["uneven_64"] = extra["uneven_64"]
        line["config"]["fp8_census"] = extra["fp8_census"]
        line["config"]["describe"] = extra["describe"]
        line["config"]["mosaic_3x3"] = extra["mosaic_3x3"]
        line["config"]["table2"] = extra["table2"]
        line["config"]["detect_3x3"] = extra["detect_3x3"]
        if "learned_proposal" in extra:
            line["config"]["learned_proposal"] = extra["learned_proposal"]
    if world == 1 and not args.no_cpu_baseline:
        tot, parts, sample = oracle_pair_seconds(r["pair"], M=max(r["M"], 4))
        line["cpu_baseline"] = {"value": 1.0 / tot, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                                "sample": sample, "seconds_per_pair": tot,
                                "parts_s": {k: round(v, 3) for k, v in parts.items()}, "host_cores": os.cpu_count()}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
