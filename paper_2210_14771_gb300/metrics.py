"""Evaluation of content-area estimates (Sec. 2.3, Eq. 4-6).

The Hausdorff distance between the edge points of the true and the inferred
content areas, scaled to a 1920x1080 frame (Eq. 6), and the miss / bad-miss
rates at 15 px and 25 px.  Host-side numpy; used by the tests and the
benchmark's accuracy report, not by the estimation path.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

D_REF = math.hypot(1920.0, 1080.0)  # diagonal of a 1920x1080 frame
MISS_PX, BAD_MISS_PX = 15.0, 25.0


def content_mask(H: int, W: int, circle) -> np.ndarray:
    """Disc intersected with the rectangle (pixel centres at integer indices);
    the whole rectangle when `circle` is None."""
    if circle is None:
        return np.ones((H, W), bool)
    cx, cy, r = (float(v) for v in circle)
    ys = np.arange(H, dtype=np.float64)[:, None]
    xs = np.arange(W, dtype=np.float64)[None, :]
    return (xs - cx) ** 2 + (ys - cy) ** 2 <= r * r


def edge_points(mask: np.ndarray) -> np.ndarray:
    """(n, 2) array of (x, y) of content pixels with a 4-neighbour that is not
    content or lies outside the frame."""
    m = np.asarray(mask, bool)
    p = np.pad(m, 1, constant_values=False)
    inner = p[:-2, 1:-1] & p[2:, 1:-1] & p[1:-1, :-2] & p[1:-1, 2:]
    ys, xs = np.nonzero(m & ~inner)
    return np.stack([xs, ys], axis=1).astype(np.float64)


def hausdorff(mask_a: np.ndarray, mask_b: np.ndarray) -> float:
    """H(A, B) = max(h(A, B), h(B, A)), h(A, B) = max_a min_b |a - b| (Eq. 4-5)."""
    A, B = edge_points(mask_a), edge_points(mask_b)
    if len(A) == 0 and len(B) == 0:
        return 0.0
    if len(A) == 0 or len(B) == 0:
        return math.inf
    hab = cKDTree(B).query(A)[0].max()
    hba = cKDTree(A).query(B)[0].max()
    return float(max(hab, hba))


def normalised_hausdorff(mask_a, mask_b) -> float:
    """NH = (d / d_I) H (Eq. 6)."""
    H, W = np.shape(mask_a)
    return hausdorff(mask_a, mask_b) * D_REF / math.hypot(W, H)


def gt_mask(gt: dict, H: int, W: int) -> np.ndarray:
    if not gt["valid"]:
        return content_mask(H, W, None)
    return content_mask(H, W, (gt["cx"], gt["cy"], gt["r"]))


def summarise(nh_values) -> dict:
    v = np.asarray(list(nh_values), np.float64)
    if v.size == 0:
        return dict(mean_nh=None, miss_pct=None, bad_miss_pct=None, n=0)
    return dict(mean_nh=float(v.mean()), miss_pct=float(100.0 * (v > MISS_PX).mean()),
                bad_miss_pct=float(100.0 * (v > BAD_MISS_PX).mean()), n=int(v.size))
