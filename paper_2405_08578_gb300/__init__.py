"""LP-SIFT hot path on GB300 (sm_103a): C-ABI library liblp + thin binding.

Stages (paper Sec. 2): multiscale local-peak detection, orientation and
128-d description, Eq. 6 nearest-neighbour matching with the ratio test, and
RANSAC homography estimation; Sec. 4's all-pairs matrix H_M on top.
"""
from . import build  # noqa: F401
