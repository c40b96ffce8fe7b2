"""Shared helpers of the tests (not collected as tests)."""
import math

import numpy as np

ORACLE_KEYS = ("n_strips", "cands_per_strip", "n_hyps", "refine_iters", "alpha", "t_g",
               "t_theta_deg", "t_iota", "t_ps", "t_cs", "t_px", "t_ri", "r_min", "r_max",
               "d_max", "sup_px", "hyp_mode", "score_norm", "sobel_norm", "seed")


def both_params(orc, **kw):
    """Matching (library, oracle) parameter structs."""
    from paper_2210_14771_gb300 import api
    lp = api.params(**kw)
    op = orc.params(**{k: v for k, v in kw.items() if k in ORACLE_KEYS})
    return lp, op


def f32_bits(a):
    return np.asarray(a, np.float32).view(np.uint32)


def same_f32(a, b):
    return np.array_equal(f32_bits(a), f32_bits(b))


def inliers_f32(X, Y, c, t_ri):
    """Inlier predicate of the method: max(r-t,0)^2 <= |p-c|^2 <= (r+t)^2 in
    binary32, each operation rounded (numpy float32 does not fuse)."""
    f = np.float32
    X = np.asarray(X, np.float32)
    Y = np.asarray(Y, np.float32)
    r = f(c[2])
    lo = max(f(r - f(t_ri)), f(0.0))
    hi = f(r + f(t_ri))
    dx = X - f(c[0])
    dy = Y - f(c[1])
    d2 = dx * dx + dy * dy
    return (d2 >= f(lo * lo)) & (d2 <= f(hi * hi))


def coope_fit64(X, Y):
    """Binary64 least-squares circle of the linear Coope system (numpy lstsq)."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    A = np.stack([X, Y, np.ones_like(X)], 1)
    b = -(X * X + Y * Y)
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    cx, cy = -sol[0] / 2, -sol[1] / 2
    return cx, cy, math.sqrt(max(cx * cx + cy * cy - sol[2], 0.0))


def replay_last_fit_set(orc, X, Y, triple, refine_iters, t_ri):
    """Follow the refit schedule of Sec. 2.2.5 with the oracle's circle pieces
    and return the point set the final circle was fitted to (or None if the
    circle is the circumcircle itself)."""
    t = sorted(int(v) for v in triple)
    c = orc.circumcircle((X[t[0]], Y[t[0]]), (X[t[1]], Y[t[1]]), (X[t[2]], Y[t[2]]))
    if c is None:
        return None, None
    last = None
    for _ in range(refine_iters):
        m = inliers_f32(X, Y, c, t_ri)
        f = orc.ls_fit(np.asarray(X)[m], np.asarray(Y)[m])
        if f is None:
            break
        c, last = f, m
    return last, c
