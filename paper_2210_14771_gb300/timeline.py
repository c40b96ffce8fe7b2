"""Timeline of the fused kernel (ca_set_trace): when each work item of a
fused call was taken, released by its dependencies and finished.

    python -m paper_2210_14771_gb300.timeline [--T 1 2 4 8] [--waves 16 32 64]
    python -m paper_2210_14771_gb300.timeline --staged [--T 2]

runs the 64-frame 1080p batch (N=32, K=2, 1024 hypotheses) once per launch
shape and prints, per phase, when its items ran and how long they waited
and worked; the CUDA-event time of the same call is printed beside it.
With --staged it times the staged launch (k_strips, k_fit, k_mask) per
hypothesis split instead, with no trace: three warm-up calls, then ten
timed ones (a fixed launch sequence for profilers).
"""
from __future__ import annotations

import argparse

import numpy as np

PHASES = ("strips", "fit", "mask")


def summarise(tr) -> dict:
    """Per-phase statistics of one traced call (times in microseconds from
    the first item taken)."""
    t0 = int(tr["t_grab"].min())
    span = (int(tr["t_end"].max()) - t0) / 1e3
    out = {"span_us": span, "items": int(len(tr)), "ctas": int(len(np.unique(tr["cta"])))}
    for k, name in enumerate(PHASES):
        m = tr["phase"] == k
        if not m.any():
            continue
        g = (tr["t_grab"][m].astype(np.int64) - t0) / 1e3
        r = (tr["t_ready"][m].astype(np.int64) - t0) / 1e3
        e = (tr["t_end"][m].astype(np.int64) - t0) / 1e3
        out[name] = {"n": int(m.sum()), "first_us": float(g.min()), "last_us": float(e.max()),
                     "wait_us": float((r - g).mean()), "work_us": float((e - r).mean()),
                     "work_p90_us": float(np.percentile(e - r, 90)),
                     "cta_us": float((e - g).sum())}
    return out


def occupancy(tr, bin_us: float = 5.0) -> dict:
    """Mean number of items of each phase in progress per time bin."""
    t0 = int(tr["t_grab"].min())
    span = (int(tr["t_end"].max()) - t0) / 1e3
    nb = int(span // bin_us) + 1
    out = {}
    for k, name in enumerate(PHASES):
        m = tr["phase"] == k
        occ = np.zeros(nb)
        for a, b in zip((tr["t_grab"][m].astype(np.int64) - t0) / 1e3,
                        (tr["t_end"][m].astype(np.int64) - t0) / 1e3):
            for i in range(int(a // bin_us), int(b // bin_us) + 1):
                lo, hi = max(a, i * bin_us), min(b, (i + 1) * bin_us)
                if hi > lo:
                    occ[i] += (hi - lo) / bin_us
        out[name] = occ
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--T", type=int, nargs="+", default=[1, 2, 4, 8])
    ap.add_argument("--waves", type=int, nargs="+", default=[16, 32, 64])
    ap.add_argument("--bins", action="store_true", help="print items in progress per 5 us")
    ap.add_argument("--staged", action="store_true", help="time the staged launch instead")
    a = ap.parse_args()
    from . import synth
    frames, _, keys = synth.batch(1, 64, 1080, 1920, "mixed")
    import torch
    from .build import build
    build()
    from . import api
    ca = api.ContentArea(0)
    dev = torch.device("cuda", 0)
    fr = torch.from_numpy(frames).to(dev)
    masks = torch.empty((64, 1080, 1920), dtype=torch.uint8, device=dev)
    res = api.new_results(64, dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.staged:
        for T in a.T:
            p = api.params(n_strips=32, cands_per_strip=2, n_hyps=1024, batch_mode=1,
                           hyp_threads=T)
            for _ in range(3):
                ca.estimate(fr, p, keys=keys, masks=masks, results=res)
            e0.record()
            for _ in range(10):
                ca.estimate(fr, p, keys=keys, masks=masks, results=res)
            e1.record()
            torch.cuda.synchronize()
            print("staged T=%d  %.1f us per call (events)" % (T, e0.elapsed_time(e1) / 10 * 1e3),
                  flush=True)
        ca.close()
        return
    for T in a.T:
        for wave in a.waves:
            p = api.params(n_strips=32, cands_per_strip=2, n_hyps=1024, batch_mode=2,
                           hyp_threads=T, wave_frames=wave)
            for _ in range(3):
                ca.estimate(fr, p, keys=keys, masks=masks, results=res)
            e0.record()
            for _ in range(10):
                ca.estimate(fr, p, keys=keys, masks=masks, results=res)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 10
            ca.set_trace(True)
            ca.estimate(fr, p, keys=keys, masks=masks, results=res)
            tr = ca.dump_trace()
            ca.set_trace(False)
            s = summarise(tr)
            line = "T=%d wave=%2d  %.1f us per call (events)  span %.1f us  %d items  %d CTAs" % (
                T, wave, ms * 1e3, s["span_us"], s["items"], s["ctas"])
            for name in PHASES:
                if name in s:
                    q = s[name]
                    line += " | %s %d [%.1f..%.1f] wait %.2f work %.2f (p90 %.2f)" % (
                        name, q["n"], q["first_us"], q["last_us"], q["wait_us"], q["work_us"],
                        q["work_p90_us"])
            print(line, flush=True)
            if a.bins:
                for name, occ in occupancy(tr).items():
                    print("    %-6s" % name, " ".join("%4d" % v for v in occ), flush=True)
    ca.close()


if __name__ == "__main__":
    main()
