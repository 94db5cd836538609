"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/lp.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2405_08578_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^LP_API[^;(]*?\b(lp_\w+)\s*\(", txt, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = set(declared_symbols())
    for n in ("lp_detect", "lp_describe", "lp_match", "lp_ransac", "lp_stitch_pair", "lp_create", "lp_destroy"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points():
    from paper_2405_08578_gb300 import lp
    assert lp.lp_num_keypoints(480, 640, [8, 16, 32]) == 12600
    assert lp.lp_num_keypoints(1600, 2688, [16, 32, 64, 128]) == 44604
    assert lp.lp_num_keypoints(10, 10, [1]) == -1
    c = lp.config(Ls=(8, 16, 32))
    assert c.nL == 3 and abs(c.ratio - 0.8) < 1e-7 and c.ransac_iters == 1000


def test_binding_refuses_host_tensors():
    torch = pytest.importorskip("torch")
    from paper_2405_08578_gb300 import lp
    with pytest.raises(ValueError):
        lp._ptr(torch.zeros(4))


def test_num_keypoints_equals_oracle_over_a_sweep():
    # the library's host scale table against the oracle's count: every full
    # window of every scale contributes its maximum and its minimum
    import numpy as np
    import oracle
    from paper_2405_08578_gb300 import lp
    rng = np.random.default_rng(11)
    sets = [(8, 16, 32), (16, 32, 64, 128), (32, 40), (100, 128), (256, 512), (5, 7, 12), (3,), (64, 160)]
    for _ in range(60):
        H, W = (int(v) for v in rng.integers(1, 3000, size=2))
        Ls = sets[int(rng.integers(len(sets)))]
        want = oracle.num_keypoints(H, W, Ls)
        got = lp.lp_num_keypoints(H, W, list(Ls))
        assert got == want, (H, W, Ls)
