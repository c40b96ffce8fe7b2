"""Seeded synthetic endoscopic frames with a known content-area circle.

The paper's datasets (CholecECA, RobustECA, PseudoECA; Sec. 2.1) are not
available, so frames are drawn from a generator shaped like the footage the
paper describes (Sec. 1.1-1.3, Fig. 1-3): a bright, textured circular
projection over a dark, slightly noisy border, joined by a 2-pixel edge ramp,
in the three regimes of Fig. 1 (clipped circle, full circle, no border) plus
hard cases (saturated blobs, dark tissue touching the edge, vignetting).

This module only draws inputs and their ground truth.  It contains none of the
estimation method, and both the CUDA path and the CPU oracle are fed from it.
Every frame is a pure function of (seed, index, H, W, geometry).
"""
from __future__ import annotations

import math

import numpy as np

GEOMETRIES = ("centred", "clipped", "full", "none", "hard")

# Mix of the 1080p workload: 40 % clipped, 30 % full circle, 20 % no border,
# 10 % hard cases, assigned by frame index modulo 10.
_MIX10 = ("clipped",) * 4 + ("full",) * 3 + ("none",) * 2 + ("hard",)


def geometry_of(mix: str, idx: int) -> str:
    if mix == "centred":
        return "centred"
    if mix == "mixed":
        return _MIX10[idx % 10]
    if mix in GEOMETRIES:
        return mix
    raise ValueError(mix)


def frame_key(seed: int, idx: int) -> int:
    """Key of frame `idx` of stream/batch `seed` (feeds the RANSAC draws)."""
    return ((seed & 0xFFFFFFFF) << 32) | (idx & 0xFFFFFFFF)


def _cubic_weights(n_out: int, n_grid: int) -> np.ndarray:
    """(n_out, n_grid) matrix of Catmull-Rom weights (bicubic upsampling)."""
    u = (np.arange(n_out, dtype=np.float64) + 0.5) * n_grid / n_out - 0.5
    i0 = np.floor(u).astype(np.int64)
    t = u - i0
    w = np.zeros((n_out, n_grid))
    taps = (
        (-1, ((-0.5 * t + 1.0) * t - 0.5) * t),
        (0, (1.5 * t - 2.5) * t * t + 1.0),
        (1, ((-1.5 * t + 2.0) * t + 0.5) * t),
        (2, (0.5 * t - 0.5) * t * t),
    )
    rows = np.arange(n_out)
    for off, wt in taps:
        idx = np.clip(i0 + off, 0, n_grid - 1)
        np.add.at(w, (rows, idx), wt)
    return w.astype(np.float32)


def _texture(rng, H, W, grid=8, sigma=25.0) -> np.ndarray:
    g = rng.standard_normal((grid, grid)).astype(np.float32)
    t = _cubic_weights(H, grid) @ g @ _cubic_weights(W, grid).T
    sd = float(t.std()) or 1.0
    return t * (sigma / sd)


def _draw_circle(rng, kind, H, W):
    c0x, c0y = (W - 1) / 2.0, (H - 1) / 2.0
    if kind == "centred":
        cx = c0x + rng.uniform(-0.1, 0.1) * W
        cy = c0y + rng.uniform(-0.1, 0.1) * H
        r = rng.uniform(0.45, 0.60) * W
    elif kind == "clipped":
        cx = c0x + rng.uniform(-0.1, 0.1) * W
        cy = c0y + rng.uniform(-0.1, 0.1) * H
        r = rng.uniform(0.5, 0.7) * W
    elif kind == "full":
        r = rng.uniform(0.25, 0.45) * H
        lo_x, hi_x = max(r + 2, c0x - 0.1 * W), min(W - 3 - r, c0x + 0.1 * W)
        lo_y, hi_y = max(r + 2, c0y - 0.1 * H), min(H - 3 - r, c0y + 0.1 * H)
        cx = rng.uniform(lo_x, hi_x) if hi_x > lo_x else c0x
        cy = rng.uniform(lo_y, hi_y) if hi_y > lo_y else c0y
    else:
        raise ValueError(kind)
    return float(cx), float(cy), float(r)


def gt_valid(cx, cy, r, H, W) -> bool:
    """The circle bounds the content area iff some pixel centre lies outside
    it; otherwise the content area is the whole rectangle."""
    corners = ((0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1))
    return any(math.hypot(x - cx, y - cy) > r for x, y in corners)


def frame(seed: int, idx: int, H: int, W: int, geometry: str = "centred"):
    """One RGB uint8 frame (H, W, 3) and its ground truth dict."""
    rng = np.random.default_rng([seed & 0xFFFFFFFF, idx & 0xFFFFFFFF, H, W])
    kind = geometry
    base = kind
    if kind == "hard":
        base = "clipped" if rng.uniform() < 0.5 else "full"

    # interior: per-frame mean 80-200 with a mild per-channel tint, low-frequency
    # texture (sigma 25) and a little pixel noise
    mean = rng.uniform(80, 200)
    tint = rng.uniform(-15, 15, size=3)
    gains = rng.uniform(0.8, 1.2, size=3)
    tex = _texture(rng, H, W)
    noise_in = rng.standard_normal((H, W, 3), dtype=np.float32) * 2.0
    interior = (mean + tint[None, None, :]).astype(np.float32) + tex[:, :, None] * gains[None, None, :].astype(np.float32) + noise_in

    # border: level 0-15 plus pixel noise sigma 3
    level = rng.uniform(0, 15)
    border = level + rng.standard_normal((H, W, 3), dtype=np.float32) * 3.0

    if base == "none":
        img = interior
        gt = dict(cx=0.0, cy=0.0, r=0.0, valid=False, kind=kind)
    else:
        cx, cy, r = _draw_circle(rng, base, H, W)
        ys = np.arange(H, dtype=np.float32)[:, None]
        xs = np.arange(W, dtype=np.float32)[None, :]
        d = np.sqrt((xs - np.float32(cx)) ** 2 + (ys - np.float32(cy)) ** 2)
        if kind == "hard":
            # radial vignetting I * (1 - 0.5 (d/r)^2) inside the projection
            vig = 1.0 - 0.5 * np.minimum(d / np.float32(r), 1.0) ** 2
            interior = interior * vig[:, :, None]
            # dark tissue patches (10-30) touching the circle edge
            for _ in range(int(rng.integers(1, 3))):
                ang = rng.uniform(0, 2 * math.pi)
                pr = rng.uniform(0.08, 0.2) * min(H, W)
                px, py = cx + r * math.cos(ang), cy + r * math.sin(ang)
                dp = np.sqrt((xs - np.float32(px)) ** 2 + (ys - np.float32(py)) ** 2)
                beta = np.clip((pr + 1 - dp) / 2, 0, 1)[:, :, None]
                interior = interior * (1 - beta) + rng.uniform(10, 30) * beta
            # saturated specular blobs (255, radius 5-30)
            for _ in range(int(rng.integers(1, 5))):
                ang = rng.uniform(0, 2 * math.pi)
                rad = r * math.sqrt(rng.uniform(0.0, 0.9))
                px, py = cx + rad * math.cos(ang), cy + rad * math.sin(ang)
                br = rng.uniform(5, 30)
                dp = np.sqrt((xs - np.float32(px)) ** 2 + (ys - np.float32(py)) ** 2)
                beta = np.clip((br + 1 - dp) / 2, 0, 1)[:, :, None]
                interior = interior * (1 - beta) + 255.0 * beta
        # 2-pixel linear edge ramp between projection and border
        a = np.clip((np.float32(r) + 1.0 - d) / 2.0, 0.0, 1.0)[:, :, None]
        img = interior * a + border * (1.0 - a)
        gt = dict(cx=cx, cy=cy, r=r, valid=gt_valid(cx, cy, r, H, W), kind=kind)
    out = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    return out, gt


def batch(seed: int, n: int, H: int, W: int, mix: str = "centred"):
    """n frames (n, H, W, 3), their ground truths and frame keys."""
    frames = np.empty((n, H, W, 3), np.uint8)
    gts, keys = [], []
    for i in range(n):
        frames[i], gt = frame(seed, i, H, W, geometry_of(mix, i))
        gts.append(gt)
        keys.append(frame_key(seed, i))
    return frames, gts, keys


# Resolutions of the mixed-resolution workload (25 % each).
MIXED_RESOLUTIONS = ((576, 720), (1024, 1280), (1080, 1920), (2160, 3840))


def _frame_job(args):
    seed, idx, H, W, geometry = args
    return frame(seed, idx, H, W, geometry)


def mixed_batch(seed: int, n: int, unique: int | None = None, workers: int = 0,
                resolutions=MIXED_RESOLUTIONS, mix: str = "mixed"):
    """The mixed-resolution workload: frame i has resolution
    resolutions[i % len(resolutions)] and the geometry of the 1080p mix.

    With `unique` < n, only the first `unique` frames are drawn and frame i
    repeats the content of frame i % unique (same resolution when `unique` is
    a multiple of the resolution count) under its own frame key, so that the
    RANSAC draws still differ.  `workers` > 1 draws in that many spawned
    processes.  Returns (list of (H, W, 3) arrays, ground truths, keys)."""
    nres = len(resolutions)
    u = n if unique is None else max(1, min(unique, n))
    if u < n and u % nres:
        raise ValueError("unique must be a multiple of the resolution count")
    jobs = [(seed, i, resolutions[i % nres][0], resolutions[i % nres][1], geometry_of(mix, i))
            for i in range(u)]
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            drawn = list(ex.map(_frame_job, jobs, chunksize=1))
    else:
        drawn = [_frame_job(j) for j in jobs]
    frames = [drawn[i % u][0] for i in range(n)]
    gts = [drawn[i % u][1] for i in range(n)]
    keys = [frame_key(seed, i) for i in range(n)]
    return frames, gts, keys


_GRAMS = {}


def _grams(H, W):
    """Bicubic weights of both axes with their Gram matrices and column sums."""
    if (H, W) not in _GRAMS:
        wy, wx = _cubic_weights(H, 8), _cubic_weights(W, 8)
        y64, x64 = wy.astype(np.float64), wx.astype(np.float64)
        _GRAMS[(H, W)] = (wy, wx, y64.T @ y64, x64.T @ x64, y64.sum(0), x64.sum(0))
    return _GRAMS[(H, W)]


def _render_strip(seed: int, idx: int, H: int, W: int, geometry: str, half_rows: int):
    """Rows y - half_rows .. y + half_rows (clamped into the frame) of a scene
    drawn like `frame` (same geometry classes and appearance); only those rows
    are rendered.  Returns (pixels (2 half_rows + 1, W, 3) uint8, y, the
    frame rows, the circle (cx, cy, r) or None, its ground-truth validity)."""
    rng = np.random.default_rng([0x57A1, seed & 0xFFFFFFFF, idx & 0xFFFFFFFF, H, W])
    kind = geometry_of(geometry, idx) if geometry == "mixed" else geometry
    base = kind
    if kind == "hard":
        base = "clipped" if rng.uniform() < 0.5 else "full"
    y = int(rng.integers(1, H - 1))
    rows = np.clip(np.arange(y - half_rows, y + half_rows + 1), 0, H - 1)
    n = len(rows)
    ys = rows.astype(np.float32)
    mean = rng.uniform(80, 200)
    tint = rng.uniform(-15, 15, size=3)
    gains = rng.uniform(0.8, 1.2, size=3)
    g = rng.standard_normal((8, 8)).astype(np.float32)
    wy, wx, gy, gx, sy, sx = _grams(H, W)
    tex = wy[rows] @ g @ wx.T
    # standard deviation of the whole frame's texture, from 8x8 Gram matrices
    g64 = g.astype(np.float64)
    m1 = float(sy @ g64 @ sx) / (H * W)
    m2 = float(np.trace(g64.T @ gy @ g64 @ gx)) / (H * W)
    sd = math.sqrt(max(m2 - m1 * m1, 0.0)) or 1.0
    tex = tex * np.float32(25.0 / sd)
    noise_in = rng.standard_normal((n, W, 3), dtype=np.float32) * 2.0
    interior = (mean + tint[None, None, :]).astype(np.float32) + \
        tex[:, :, None] * gains[None, None, :].astype(np.float32) + noise_in
    level = rng.uniform(0, 15)
    border = level + rng.standard_normal((n, W, 3), dtype=np.float32) * 3.0
    circle, valid = None, False
    if base == "none":
        img = interior
    else:
        cx, cy, r = _draw_circle(rng, base, H, W)
        circle, valid = (cx, cy, r), gt_valid(cx, cy, r, H, W)
        xs = np.arange(W, dtype=np.float32)[None, :]
        d = np.sqrt((xs - np.float32(cx)) ** 2 + (ys[:, None] - np.float32(cy)) ** 2)
        if kind == "hard":
            vig = 1.0 - 0.5 * np.minimum(d / np.float32(r), 1.0) ** 2
            interior = interior * vig[:, :, None]
            for _ in range(int(rng.integers(1, 3))):
                ang = rng.uniform(0, 2 * math.pi)
                pr = rng.uniform(0.08, 0.2) * min(H, W)
                px, py = cx + r * math.cos(ang), cy + r * math.sin(ang)
                dp = np.sqrt((xs - np.float32(px)) ** 2 + (ys[:, None] - np.float32(py)) ** 2)
                beta = np.clip((pr + 1 - dp) / 2, 0, 1)[:, :, None]
                interior = interior * (1 - beta) + rng.uniform(10, 30) * beta
            for _ in range(int(rng.integers(1, 5))):
                ang = rng.uniform(0, 2 * math.pi)
                rad = r * math.sqrt(rng.uniform(0.0, 0.9))
                px, py = cx + rad * math.cos(ang), cy + rad * math.sin(ang)
                br = rng.uniform(5, 30)
                dp = np.sqrt((xs - np.float32(px)) ** 2 + (ys[:, None] - np.float32(py)) ** 2)
                beta = np.clip((br + 1 - dp) / 2, 0, 1)[:, :, None]
                interior = interior * (1 - beta) + 255.0 * beta
        a = np.clip((np.float32(r) + 1.0 - d) / 2.0, 0.0, 1.0)[:, :, None]
        img = interior * a + border * (1.0 - a)
    out = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    return out, y, rows.astype(np.int32), circle, valid


def training_strip(seed: int, idx: int, H: int, W: int, geometry: str = "mixed"):
    """One labelled training strip: rows y-1, y, y+1 (3, W, 3) of a scene drawn
    like `frame` (same geometry classes and appearance), its middle row y and
    per-column labels: 1 within 2 px of a crossing of the true circle with
    row y, else 0.  Only the three rows are rendered."""
    out, y, _, circle, _ = _render_strip(seed, idx, H, W, geometry, 1)
    labels = np.zeros(W, np.uint8)
    if circle is not None:
        cx, cy, r = circle
        dy = y - cy
        if abs(dy) <= r:
            h = math.sqrt(r * r - dy * dy)
            for xc in (cx - h, cx + h):
                lo, hi = int(math.ceil(xc - 2.0)), int(math.floor(xc + 2.0))
                lo, hi = max(lo, 0), min(hi, W - 1)
                if lo <= hi:
                    labels[lo:hi + 1] = 1
    return out, y, labels


def soft_targets(circle, valid: bool, W: int, y: int, sigma: float = 3.0) -> np.ndarray:
    """Soft edge targets of row y (the paper blurs its edge map with a Gaussian
    of sigma 3): exp(-d^2 / (2 sigma^2)), d the distance of pixel (x, y) to
    the true circle; zero when the circle does not bound the content area."""
    if circle is None or not valid:
        return np.zeros(W, np.float32)
    cx, cy, r = circle
    d = np.abs(np.hypot(np.arange(W, dtype=np.float64) - cx, float(y) - cy) - r)
    return np.exp(-d * d / (2.0 * sigma * sigma)).astype(np.float32)


def training_strip7(seed: int, idx: int, H: int, W: int, geometry: str = "mixed",
                    sigma: float = 3.0):
    """One training strip of the paper's 2-D scorer: rows y-3 .. y+3 (clamped
    into the frame) (7, W, 3), their frame rows (7,) and the soft targets of
    the middle row (W,) float32."""
    out, y, rows, circle, valid = _render_strip(seed, idx, H, W, geometry, 3)
    return out, rows, soft_targets(circle, valid, W, y, sigma)


def _strip7_job(args):
    seed, i0, i1, H, W, geometry = args
    n = i1 - i0
    s = np.empty((n, 7, W, 3), np.uint8)
    rows = np.empty((n, 7), np.int32)
    tg = np.empty((n, W), np.float32)
    for k in range(n):
        s[k], rows[k], tg[k] = training_strip7(seed, i0 + k, H, W, geometry)
    return s, rows, tg


def training_strips7(seed: int, n: int, H: int = 1080, W: int = 1920, geometry: str = "mixed",
                     workers: int = 0):
    """n training strips of the 2-D scorer: (strips (n, 7, W, 3) uint8, frame
    rows (n, 7) int32, soft targets (n, W) float32)."""
    chunk = 256
    jobs = [(seed, i, min(n, i + chunk), H, W, geometry) for i in range(0, n, chunk)]
    if workers > 1 and len(jobs) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_strip7_job, jobs))
    else:
        parts = [_strip7_job(j) for j in jobs]
    if not parts:
        return (np.empty((0, 7, W, 3), np.uint8), np.empty((0, 7), np.int32),
                np.empty((0, W), np.float32))
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]))


def _strip_job(args):
    seed, i0, i1, H, W, geometry = args
    n = i1 - i0
    s = np.empty((n, 3, W, 3), np.uint8)
    ys = np.empty(n, np.int32)
    lab = np.empty((n, W), np.uint8)
    for k in range(n):
        s[k], ys[k], lab[k] = training_strip(seed, i0 + k, H, W, geometry)
    return s, ys, lab


def training_strips(seed: int, n: int, H: int = 1080, W: int = 1920, geometry: str = "mixed",
                    workers: int = 0):
    """n labelled strips: (strips (n, 3, W, 3) uint8, ys (n,) int32, labels (n, W) uint8)."""
    chunk = 256
    jobs = [(seed, i, min(n, i + chunk), H, W, geometry) for i in range(0, n, chunk)]
    if workers > 1 and len(jobs) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_strip_job, jobs))
    else:
        parts = [_strip_job(j) for j in jobs]
    if not parts:
        return (np.empty((0, 3, W, 3), np.uint8), np.empty(0, np.int32), np.empty((0, W), np.uint8))
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]))


class VideoStream:
    """A synthetic endoscopic video stream: its frames are windows of a larger
    scene that drift by at most 2 px per frame (the scope moving), with a
    scope change -- a new scene -- with probability 1 % per frame, and arrive
    as a Poisson process of `fps` frames per second.  Only `bank` distinct
    frames are rendered; frame k shows frame k mod bank of the walk, so the
    stream can be served for any length with bounded memory (the walk is a
    there-and-back path, so consecutive frames stay within 2 px)."""

    MARGIN = 48

    def __init__(self, seed: int, sid: int, H: int, W: int, fps: float, bank: int = 8,
                 geometry: str | None = None):
        self.seed, self.sid, self.H, self.W, self.fps = seed, sid, H, W, fps
        rng = np.random.default_rng([0x5E7, seed & 0xFFFFFFFF, sid])
        geo = geometry or ("centred", "clipped", "full", "hard")[sid % 4]
        M = self.MARGIN
        scenes, k = [], 0
        half = max(1, bank // 2)
        offs, which = [], []
        ox = oy = 0
        for i in range(half):
            if i == 0 or rng.uniform() < 0.01:
                scenes.append(frame(seed, (sid << 16) | k, H + 2 * M, W + 2 * M, geo))
                k += 1
                ox = oy = 0
            else:
                ox = int(np.clip(ox + rng.integers(-2, 3), -M + 2, M - 2))
                oy = int(np.clip(oy + rng.integers(-2, 3), -M + 2, M - 2))
            offs.append((ox, oy))
            which.append(len(scenes) - 1)
        path = list(range(half)) + list(range(half - 1, -1, -1))   # there and back
        self.frames, self.gts = [], []
        for j in path[:bank]:
            img, gt = scenes[which[j]]
            ox, oy = offs[j]
            x0, y0 = M + ox, M + oy
            self.frames.append(np.ascontiguousarray(img[y0:y0 + H, x0:x0 + W]))
            g = dict(gt)
            if g["kind"] != "none":
                g["cx"] -= x0
                g["cy"] -= y0
                g["valid"] = gt_valid(g["cx"], g["cy"], g["r"], H, W)
            self.gts.append(g)
        self._rng = np.random.default_rng([0xA77, seed & 0xFFFFFFFF, sid])

    def arrivals(self, n: int) -> np.ndarray:
        """Arrival times (s, from 0) of the first n frames."""
        return np.cumsum(self._rng.exponential(1.0 / self.fps, size=n))

    def frame(self, k: int):
        return self.frames[k % len(self.frames)], self.gts[k % len(self.gts)]

    def key(self, k: int) -> int:
        return frame_key((self.seed << 8) | self.sid, k)


SERVING_RESOLUTIONS = MIXED_RESOLUTIONS


def _stream_job(args):
    seed, sid, H, W, fps, bank = args
    return VideoStream(seed, sid, H, W, fps, bank)


def video_streams(seed: int, n: int, resolutions=SERVING_RESOLUTIONS, bank: int = 8,
                  workers: int = 0):
    """n streams with resolutions drawn from `resolutions` and rates U[30, 60] fps."""
    rng = np.random.default_rng([0x57E, seed & 0xFFFFFFFF])
    jobs = []
    for sid in range(n):
        H, W = resolutions[int(rng.integers(0, len(resolutions)))]
        jobs.append((seed, sid, H, W, float(rng.uniform(30.0, 60.0)), bank))
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_stream_job, jobs))
    return [_stream_job(j) for j in jobs]
