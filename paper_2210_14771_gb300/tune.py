"""Autotuning of the parameters that change results: strip count N,
candidates per strip K and RANSAC hypotheses.

The launch shapes that leave results unchanged are tuned inside the library
(ca_tune).  N, K and the hypothesis count trade accuracy for speed, so they
are chosen here, on a labelled calibration batch, among the settings whose
accuracy against the ground truth (normalised Hausdorff distance of Sec. 2.3)
is no worse than that of a reference setting: the fastest such setting wins.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import metrics


@dataclass
class Trial:
    N: int
    K: int
    NH: int
    ms: float            # mean time per call of the tuned launch configuration
    mean_nh: float       # mean normalised Hausdorff distance (px, Eq. 6)
    miss_pct: float      # NH > 15 px
    launch: dict = field(default_factory=dict)   # ca_tune outcome
    nh: np.ndarray = field(default_factory=lambda: np.zeros(0))   # per calibration frame
    by_class: dict = field(default_factory=dict)  # metrics.summarise per geometry class


def no_worse(t: Trial, ref: Trial) -> bool:
    """t is not measurably less accurate than ref on the same frames: its
    mean per-frame excess of normalised Hausdorff distance over ref is at most
    two standard errors of that paired difference (so frame-level noise does
    not decide), and it misses no more frames (NH > 15 px)."""
    if len(t.nh) == 0 or len(t.nh) != len(ref.nh):
        return t.mean_nh <= ref.mean_nh + 1e-9 and t.miss_pct <= ref.miss_pct + 1e-9
    d = np.asarray(t.nh, np.float64) - np.asarray(ref.nh, np.float64)
    se = float(d.std(ddof=1) / np.sqrt(len(d))) if len(d) > 1 else 0.0
    misses = int((np.asarray(t.nh) > 15).sum()), int((np.asarray(ref.nh) > 15).sum())
    return float(d.mean()) <= 2.0 * se + 1e-9 and misses[0] <= misses[1]


def choose(trials, ref):
    """The fastest trial that is no worse than trial `ref` (ties in time go to
    the more accurate one)."""
    ok = [t for t in trials if no_worse(t, ref)]
    if not ok:
        return ref
    return min(ok, key=lambda t: (t.ms, t.mean_nh))


def accuracy(results, masks, gts):
    """Per-frame normalised Hausdorff distances of masks (list of (H, W) uint8
    arrays) against the truth, their summary and the summary per geometry
    class."""
    nh = np.array([metrics.normalised_hausdorff(m.astype(bool), metrics.gt_mask(g, *m.shape))
                   for m, g in zip(masks, gts)])
    by = {}
    for v, g in zip(nh, gts):
        by.setdefault(g.get("kind", "?"), []).append(float(v))
    return nh, metrics.summarise(nh), {k: metrics.summarise(v) for k, v in sorted(by.items())}


def calibration_subset(gts, n):
    """Up to n frame indices taking the geometry classes in turn (so that no
    class dominates the accuracy a trial is judged by)."""
    by = {}
    for i, g in enumerate(gts):
        by.setdefault(g.get("kind", "?"), []).append(i)
    out, k = [], 0
    while len(out) < n and any(k < len(v) for v in by.values()):
        for v in by.values():
            if k < len(v) and len(out) < n:
                out.append(v[k])
        k += 1
    return sorted(out)


def sweep(ca, frames, gts, keys, strips=(16, 32, 64), hyps=(512, 1024, 4096), cands=(2,),
          ref=(32, 2, 1024), **fixed):
    """Runs every (N, K, NH) on the calibration batch (a list of (H, W, 3)
    uint8 CUDA tensors with ground truths `gts`), tuning the launch shape of
    each.  Returns (trials, reference trial, chosen trial)."""
    import torch

    from . import api
    masks = [torch.empty(f.shape[:2], dtype=torch.uint8, device=f.device) for f in frames]
    combos = sorted({(n, k, h) for n in strips for k in cands for h in hyps} | {tuple(ref)})
    trials = []
    for N, K, NH in combos:
        if N * K > 256:
            continue
        p = api.params(n_strips=N, cands_per_strip=K, n_hyps=NH, **fixed)
        t = ca.tune(frames, p, keys=keys, masks=masks)
        res, _ = ca.estimate(frames, p, keys=keys, masks=masks)
        ca.sync()
        host = [m.cpu().numpy() for m in masks]
        nh, summ, by = accuracy(api.results_numpy(res), host, gts)
        trials.append(Trial(N, K, NH, float(t["ms"]), summ["mean_nh"], summ["miss_pct"], t, nh,
                            by))
    ref_t = next(t for t in trials if (t.N, t.K, t.NH) == tuple(ref))
    return trials, ref_t, choose(trials, ref_t)


def as_dict(t: Trial, ref: Trial | None = None) -> dict:
    d = {"N": t.N, "K": t.K, "NH": t.NH, "ms": t.ms, "mean_nh": t.mean_nh,
         "miss_pct": t.miss_pct, "by_class": t.by_class,
         "launch": {k: t.launch.get(k) for k in ("batch_mode", "hyp_threads", "wave_frames",
                                                  "fit_lag", "mask_lag")}}
    if ref is not None:
        d["no_worse_than_reference"] = bool(no_worse(t, ref))
    return d


__all__ = ["Trial", "no_worse", "choose", "accuracy", "calibration_subset", "sweep", "as_dict",
           "np"]
