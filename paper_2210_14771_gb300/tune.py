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


def choose(trials, ref):
    """The fastest trial whose mean NH and miss rate are both no worse than
    those of trial `ref` (ties in time go to the more accurate one)."""
    ok = [t for t in trials if t.mean_nh <= ref.mean_nh + 1e-9 and t.miss_pct <= ref.miss_pct + 1e-9]
    if not ok:
        return ref
    return min(ok, key=lambda t: (t.ms, t.mean_nh))


def accuracy(results, masks, gts):
    """Mean NH and miss rate of masks (list of (H, W) uint8 arrays) vs truth."""
    nh = [metrics.normalised_hausdorff(m.astype(bool), metrics.gt_mask(g, *m.shape))
          for m, g in zip(masks, gts)]
    s = metrics.summarise(nh)
    return s["mean_nh"], s["miss_pct"]


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
        mean_nh, miss = accuracy(api.results_numpy(res), host, gts)
        trials.append(Trial(N, K, NH, float(t["ms"]), mean_nh, miss, t))
    ref_t = next(t for t in trials if (t.N, t.K, t.NH) == tuple(ref))
    return trials, ref_t, choose(trials, ref_t)


def as_dict(t: Trial) -> dict:
    return {"N": t.N, "K": t.K, "NH": t.NH, "ms": t.ms, "mean_nh": t.mean_nh,
            "miss_pct": t.miss_pct, "launch": {k: t.launch.get(k) for k in
                                               ("batch_mode", "hyp_threads", "wave_frames")}}


__all__ = ["Trial", "choose", "accuracy", "sweep", "as_dict", "np"]
