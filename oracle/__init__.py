"""ctypes view of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  The CUDA library never does, and nothing here is
shared with it.  See ``ca_oracle.h`` for what each function computes and the
paper passage it follows.
"""
import ctypes as C

import numpy as np

from .build import build

_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("n_strips", C.c_int32), ("cands_per_strip", C.c_int32),
        ("n_hyps", C.c_int32), ("refine_iters", C.c_int32),
        ("alpha", C.c_float), ("t_g", C.c_float), ("t_theta_deg", C.c_float),
        ("t_iota", C.c_float), ("t_ps", C.c_float), ("t_cs", C.c_float),
        ("t_px", C.c_float), ("t_ri", C.c_float), ("r_min", C.c_float),
        ("r_max", C.c_float), ("d_max", C.c_float),
        ("sup_px", C.c_int32), ("hyp_mode", C.c_int32), ("score_norm", C.c_int32),
        ("sobel_norm", C.c_int32), ("seed", C.c_uint64),
    ]


class OrcResult(C.Structure):
    _fields_ = [("cx", C.c_float), ("cy", C.c_float), ("r", C.c_float),
                ("score", C.c_float), ("valid", C.c_int32), ("n_inliers", C.c_int32)]


class OrcSmoothParams(C.Structure):
    _fields_ = [("gamma", C.c_float), ("jump", C.c_float), ("t_hold", C.c_float),
                ("pad", C.c_int32)]


class OrcDebug(C.Structure):
    _fields_ = [
        ("cand_cap", C.c_int32), ("n_cands", C.POINTER(C.c_int32)),
        ("cand_x", C.POINTER(C.c_int16)), ("cand_y", C.POINTER(C.c_int16)),
        ("cand_s", C.POINTER(C.c_uint16)),
        ("hyp_cap", C.c_int32), ("n_hyps", C.POINTER(C.c_int32)),
        ("triple", C.POINTER(C.c_int32)), ("hyp_n_inl", C.POINTER(C.c_int32)),
        ("hyp_score", C.POINTER(C.c_uint32)), ("hyp_pass", C.POINTER(C.c_int32)),
        ("hyp_circle", C.POINTER(C.c_float)), ("best_h", C.POINTER(C.c_int32)),
        ("best_inl", C.POINTER(C.c_uint8)),
    ]


LUT_G, LUT_T, LUT_I = 5772, 8193, 256
HYP_RANDOM, HYP_EXHAUSTIVE = 0, 1
NORM_2N, NORM_NK, NORM_RAW, NORM_CIRCLE = 0, 1, 2, 3


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.orc_params_default.argtypes = [P(OrcParams)]
        L.orc_strip_rows.argtypes = [C.c_int, C.c_int, C.c_float, C.c_void_p]
        L.orc_build_luts.argtypes = [P(OrcParams), C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_luma.argtypes = [C.c_int] * 3
        L.orc_strip_scores.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_int,
                                       P(OrcParams), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p]
        L.orc_score_exact.argtypes = [C.c_int] * 5 + [P(OrcParams)]
        L.orc_score_exact.restype = C.c_double
        L.orc_candidates.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, P(OrcParams),
                                     C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_candidates_centre.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64,
                                            P(OrcParams), C.c_int32, C.c_int32, C.c_int,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_prior_centre2.argtypes = [C.c_float, C.c_float, C.c_int, C.c_int, C.c_void_p]
        L.orc_prior_centre2.restype = None
        L.orc_smooth.argtypes = [P(OrcResult), C.c_int, P(OrcSmoothParams), C.c_void_p,
                                 P(OrcResult)]
        L.orc_smooth.restype = None
        L.orc_sc2_offsets.argtypes = [C.c_void_p]
        L.orc_sc2_offsets.restype = None
        L.orc_sc2_strip.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_int, C.c_void_p,
                                    C.c_void_p]
        L.orc_sc2_strip.restype = None
        L.orc_sc2_features.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.orc_sc2_features.restype = None
        L.orc_sc2_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                      C.c_void_p]
        L.orc_sc2_forward_mode.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                           C.c_int, C.c_void_p]
        L.orc_sc2_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                        C.c_double, C.c_void_p, C.c_void_p]
        L.orc_sc2_loss_grad.restype = C.c_double
        L.orc_sc2_targets.argtypes = [C.c_float, C.c_float, C.c_float, C.c_int, C.c_int, C.c_int,
                                      C.c_double, C.c_void_p]
        L.orc_sc2_targets.restype = None
        L.orc_circle_strips.argtypes = [C.c_void_p, C.c_int, C.c_float, C.c_float, C.c_float]
        L.orc_circle_strips.restype = C.c_int
        L.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_triple.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int, C.c_void_p]
        L.orc_triple_exhaustive.argtypes = [C.c_int64, C.c_int, C.c_void_p]
        L.orc_circumcircle.argtypes = [C.c_int] * 6 + [C.c_void_p]
        L.orc_rn_ratio.argtypes = [C.c_int64, C.c_int64]
        L.orc_rn_ratio.restype = C.c_float
        L.orc_ls_fit.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.orc_i128_to_f32.argtypes = [C.c_int64, C.c_uint64]
        L.orc_i128_to_f32.restype = C.c_float
        L.orc_estimate.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_uint64,
                                   P(OrcParams), P(OrcResult), P(OrcDebug)]
        L.orc_mask.argtypes = [P(OrcResult), C.c_int, C.c_int, C.c_void_p]
        L.orc_learned_candidates.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64,
                                             P(OrcParams), C.c_void_p, C.c_int, C.c_int,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_fit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int, C.c_int,
                              C.c_uint64, P(OrcParams), P(OrcResult), P(OrcDebug)]
        L.orc_fit_prior.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int,
                                    C.c_int, C.c_uint64, P(OrcParams), C.c_void_p, P(OrcResult),
                                    P(OrcDebug)]
        L.orc_bf16.argtypes = [C.c_float]
        L.orc_bf16.restype = C.c_float
        L.orc_sc_offsets.argtypes = [C.c_void_p]
        L.orc_sc_features.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
        L.orc_sc_forward.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                     C.c_void_p, C.c_void_p]
        L.orc_sc_loss_grad.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                       C.c_float, C.c_void_p, C.c_int, C.c_void_p]
        L.orc_sc_loss_grad.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def params(**kw) -> OrcParams:
    p = OrcParams()
    lib().orc_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def strip_rows(H, N, alpha=8.0):
    out = np.zeros(N, np.int32)
    if lib().orc_strip_rows(H, N, alpha, _ptr(out)) != 0:
        raise ValueError("bad strip arguments")
    return out


def luts(p=None):
    p = p or params()
    g = np.zeros(LUT_G, np.uint16)
    t = np.zeros(LUT_T, np.uint16)
    i = np.zeros(LUT_I, np.uint16)
    lib().orc_build_luts(C.byref(p), _ptr(g), _ptr(t), _ptr(i))
    return g, t, i


def luma(r, g, b):
    return lib().orc_luma(int(r), int(g), int(b))


def _frame(frame):
    f = np.ascontiguousarray(frame, dtype=np.uint8)
    assert f.ndim == 3 and f.shape[2] == 3
    return f


def strip_scores(frame, row, p=None):
    f = _frame(frame)
    H, W = f.shape[:2]
    p = p or params()
    s = np.zeros(W, np.uint16)
    gx = np.zeros(W, np.int32)
    gy = np.zeros(W, np.int32)
    io = np.zeros(W, np.uint8)
    if lib().orc_strip_scores(_ptr(f), H, W, W * 3, row, C.byref(p), _ptr(s), _ptr(gx),
                              _ptr(gy), _ptr(io)) != 0:
        raise ValueError("bad strip row")
    return s, gx, gy, io


def score_exact(gx, gy, cx2, cy2, iota, p=None):
    p = p or params()
    return lib().orc_score_exact(int(gx), int(gy), int(cx2), int(cy2), int(iota), C.byref(p))


def learned_candidates(frame, learned, fallback, p=None):
    """Candidates from learned Q15 pixel scores (N x W), with or without the
    handcrafted fallback of unsure half-strips."""
    f = _frame(frame)
    H, W = f.shape[:2]
    p = p or params()
    lq = np.ascontiguousarray(learned, np.uint16)
    assert lq.shape == (p.n_strips, W)
    cap = p.n_strips * p.cands_per_strip
    xs = np.zeros(cap, np.int16)
    ys = np.zeros(cap, np.int16)
    ss = np.zeros(cap, np.uint16)
    M = C.c_int32(0)
    if lib().orc_learned_candidates(_ptr(f), H, W, W * 3, C.byref(p), _ptr(lq),
                                    1 if fallback else 0, cap, _ptr(xs), _ptr(ys), _ptr(ss),
                                    C.byref(M)) != 0:
        raise ValueError("bad candidate arguments")
    m = M.value
    return xs[:m].copy(), ys[:m].copy(), ss[:m].copy()


def sc_q15(logits):
    """Learned Q15 score of logits: round(32768 sigmoid(l))."""
    l = np.asarray(logits, np.float64)
    return np.floor(32768.0 / (1.0 + np.exp(-l)) + 0.5).astype(np.uint16)


def candidates(frame, p=None, centre2=None):
    """Candidates of a frame (Sec. 2.2.3-2.2.5); centre2 = the doubled
    integer centre (C2x, C2y) of the angle term, default the image centre."""
    f = _frame(frame)
    H, W = f.shape[:2]
    p = p or params()
    cap = p.n_strips * p.cands_per_strip
    xs = np.zeros(cap, np.int16)
    ys = np.zeros(cap, np.int16)
    ss = np.zeros(cap, np.uint16)
    M = C.c_int32(0)
    if centre2 is None:
        rc = lib().orc_candidates(_ptr(f), H, W, W * 3, C.byref(p), cap, _ptr(xs), _ptr(ys),
                                  _ptr(ss), C.byref(M))
    else:
        rc = lib().orc_candidates_centre(_ptr(f), H, W, W * 3, C.byref(p), int(centre2[0]),
                                         int(centre2[1]), cap, _ptr(xs), _ptr(ys), _ptr(ss),
                                         C.byref(M))
    if rc != 0:
        raise ValueError("bad candidate arguments")
    m = M.value
    return xs[:m].copy(), ys[:m].copy(), ss[:m].copy()


def prior_centre2(cx, cy, H, W):
    """Doubled integer centre of a prior circle centre (orc_prior_centre2)."""
    out = np.zeros(2, np.int32)
    lib().orc_prior_centre2(C.c_float(cx), C.c_float(cy), H, W, _ptr(out))
    return int(out[0]), int(out[1])


def philox(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def triple(seed, frame_key, h, M):
    out = np.zeros(3, np.int32)
    lib().orc_triple(seed, frame_key, h, M, _ptr(out))
    return out


def triple_exhaustive(h, M):
    out = np.zeros(3, np.int32)
    lib().orc_triple_exhaustive(h, M, _ptr(out))
    return out


def rn_ratio(num, den):
    """The binary32 value nearest to num / den (ties to even)."""
    return np.float32(lib().orc_rn_ratio(int(num), int(den)))


def circumcircle(a, b, c):
    out = np.zeros(3, np.float32)
    ok = lib().orc_circumcircle(int(a[0]), int(a[1]), int(b[0]), int(b[1]), int(c[0]),
                                int(c[1]), _ptr(out))
    return out if ok else None


def ls_fit(X, Y):
    X = np.ascontiguousarray(X, np.int32)
    Y = np.ascontiguousarray(Y, np.int32)
    out = np.zeros(3, np.float32)
    ok = lib().orc_ls_fit(_ptr(X), _ptr(Y), len(X), _ptr(out))
    return out if ok else None


def i128_to_f32(v: int) -> np.float32:
    v &= (1 << 128) - 1
    hi = v >> 64
    if hi >= 1 << 63:
        hi -= 1 << 64
    return np.float32(lib().orc_i128_to_f32(hi, v & ((1 << 64) - 1)))


def estimate_tracked(frame, frame_key, p, prior, prior_centre=False):
    """Whole pipeline with the previous circle (cx, cy, r) as an extra
    hypothesis, or None for none; with prior_centre, the angle term of the
    candidate scores also points at the previous circle's centre."""
    H, W = np.shape(frame)[:2]
    c2 = prior_centre2(prior[0], prior[1], H, W) if (prior_centre and prior is not None) else None
    xs, ys, ss = candidates(frame, p, c2)
    return fit(xs, ys, ss, H, W, frame_key, p, prior)


def estimate(frame, frame_key=0, p=None, debug=False, hyp_cap=None):
    """Run the whole pipeline on one frame.  Returns (result dict, debug dict)."""
    f = _frame(frame)
    H, W = f.shape[:2]
    p = p or params()
    res = OrcResult()
    dbg = None
    d = {}
    if debug:
        cap = p.n_strips * p.cands_per_strip
        if hyp_cap is None:
            hyp_cap = p.n_hyps if p.hyp_mode == HYP_RANDOM else cap * (cap - 1) * (cap - 2) // 6
        d = dict(n_cands=np.zeros(1, np.int32), cand_x=np.zeros(cap, np.int16),
                 cand_y=np.zeros(cap, np.int16), cand_s=np.zeros(cap, np.uint16),
                 n_hyps=np.zeros(1, np.int32), triple=np.zeros(3 * hyp_cap, np.int32),
                 hyp_n_inl=np.zeros(hyp_cap, np.int32), hyp_score=np.zeros(hyp_cap, np.uint32),
                 hyp_pass=np.zeros(hyp_cap, np.int32),
                 hyp_circle=np.zeros(3 * hyp_cap, np.float32),
                 best_h=np.zeros(1, np.int32), best_inl=np.zeros(cap, np.uint8))
        dbg = OrcDebug()
        dbg.cand_cap = cap
        dbg.hyp_cap = hyp_cap
        for k, a in d.items():
            setattr(dbg, k, a.ctypes.data_as(dict(OrcDebug._fields_)[k]))
    rc = lib().orc_estimate(_ptr(f), H, W, W * 3, frame_key, C.byref(p), C.byref(res),
                            C.byref(dbg) if dbg is not None else None)
    if rc != 0:
        raise ValueError("bad estimate arguments")
    out = dict(cx=res.cx, cy=res.cy, r=res.r, score=res.score, valid=res.valid,
               n_inliers=res.n_inliers)
    if debug:
        M = int(d["n_cands"][0])
        nh = min(int(d["n_hyps"][0]), hyp_cap)
        d = dict(M=M, cand_x=d["cand_x"][:M], cand_y=d["cand_y"][:M], cand_s=d["cand_s"][:M],
                 n_hyps=int(d["n_hyps"][0]), triple=d["triple"][:3 * nh].reshape(nh, 3),
                 hyp_n_inl=d["hyp_n_inl"][:nh], hyp_score=d["hyp_score"][:nh],
                 hyp_pass=d["hyp_pass"][:nh], hyp_circle=d["hyp_circle"][:3 * nh].reshape(nh, 3),
                 best_h=int(d["best_h"][0]), best_inl=d["best_inl"][:M].astype(bool))
    return out, d


def mask(result, H, W):
    res = OrcResult(result["cx"], result["cy"], result["r"], result["score"],
                    result["valid"], result["n_inliers"])
    out = np.zeros((H, W), np.uint8)
    lib().orc_mask(C.byref(res), H, W, _ptr(out))
    return out


def fit(xs, ys, ss, H, W, frame_key=0, p=None, prior=None):
    """Sec. 2.2.5 on a given candidate list (pixel x, y and Q15 scores); with
    `prior` (cx, cy, r) the previous circle is one more hypothesis."""
    p = p or params()
    xs = np.ascontiguousarray(xs, np.int16)
    ys = np.ascontiguousarray(ys, np.int16)
    ss = np.ascontiguousarray(ss, np.uint16)
    res = OrcResult()
    pr = np.ascontiguousarray(prior, np.float32) if prior is not None else None
    if lib().orc_fit_prior(_ptr(xs), _ptr(ys), _ptr(ss), len(xs), H, W, frame_key, C.byref(p),
                           _ptr(pr) if pr is not None else None, C.byref(res), None) != 0:
        raise ValueError("bad fit arguments")
    return dict(cx=res.cx, cy=res.cy, r=res.r, score=res.score, valid=res.valid,
                n_inliers=res.n_inliers)


# ------------------------------------------------------- learned scorer --
SC_CIN, SC_CH, SC_K, SC_NPARAM = 14, 32, 7, 17601
SC_EXACT, SC_MIXED = 0, 1


def bf16(v):
    return np.float32(lib().orc_bf16(float(v)))


def sc_offsets():
    out = np.zeros(8, np.int32)
    lib().orc_sc_offsets(_ptr(out))
    return dict(zip(("W1", "b1", "W2", "b2", "W3", "b3", "wh", "bh"), (int(v) for v in out)))


def _strip(rgb3):
    s = np.ascontiguousarray(rgb3, np.uint8)
    assert s.ndim == 3 and s.shape[0] == 3 and s.shape[2] == 3
    return s


def sc_features(rgb3, y, H, mixed=True):
    s = _strip(rgb3)
    W = s.shape[1]
    out = np.zeros((W, SC_CIN), np.float64)
    lib().orc_sc_features(_ptr(s), W, int(y), int(H), 1 if mixed else 0, _ptr(out))
    return out


def sc_forward(rgb3, y, H, prm, mode=SC_MIXED, acts=False):
    """Logits (W,) of one strip; with acts=True also (features, a1, a2, a3)."""
    s = _strip(rgb3)
    W = s.shape[1]
    prm = np.ascontiguousarray(prm, np.float32)
    assert prm.size == SC_NPARAM
    lg = np.zeros(W, np.float64)
    ac = np.zeros(W * SC_CIN + 3 * W * SC_CH, np.float64) if acts else None
    if lib().orc_sc_forward(_ptr(s), W, int(y), int(H), _ptr(prm), mode, _ptr(lg),
                            _ptr(ac) if acts else None) != 0:
        raise ValueError("bad scorer arguments")
    if not acts:
        return lg
    f = ac[:W * SC_CIN].reshape(W, SC_CIN)
    a = [ac[W * SC_CIN + l * W * SC_CH: W * SC_CIN + (l + 1) * W * SC_CH].reshape(W, SC_CH)
         for l in range(3)]
    return lg, (f, *a)


def sc_loss_grad(rgb3, y, H, labels, prm, pos_weight=1.0, mode=SC_MIXED):
    """(loss, gradient) of one strip: summed weighted cross-entropy."""
    s = _strip(rgb3)
    W = s.shape[1]
    prm = np.ascontiguousarray(prm, np.float32)
    lab = np.ascontiguousarray(labels, np.uint8)
    assert lab.size == W and prm.size == SC_NPARAM
    g = np.zeros(SC_NPARAM, np.float64)
    loss = lib().orc_sc_loss_grad(_ptr(s), W, int(y), int(H), _ptr(lab), float(pos_weight),
                                  _ptr(prm), mode, _ptr(g))
    return loss, g


def smooth_chain(results, W, gamma, jump, t_hold, state=None):
    """orc_smooth over one stream's results in order (dicts or 6-tuples
    cx, cy, r, score, valid, n_inliers); returns (smoothed dicts, state)."""
    sp = OrcSmoothParams(gamma, jump, t_hold, 0)
    st = np.zeros(4, np.float32) if state is None else np.asarray(state, np.float32).copy()
    out = []
    for r in results:
        if isinstance(r, dict):
            r = (r["cx"], r["cy"], r["r"], r["score"], r["valid"], r["n_inliers"])
        cur = OrcResult(*[float(v) for v in r[:4]], int(r[4]), int(r[5]))
        o = OrcResult()
        lib().orc_smooth(C.byref(cur), int(W), C.byref(sp), _ptr(st), C.byref(o))
        out.append(dict(cx=o.cx, cy=o.cy, r=o.r, score=o.score, valid=o.valid,
                        n_inliers=o.n_inliers))
    return out, st


# ---- the paper's 2-D learned scorer (ca_scorer2d_oracle.c)
SC2_NPARAM = 6209


def sc2_offsets():
    o = np.zeros(8, np.int32)
    lib().orc_sc2_offsets(_ptr(o))
    keys = ("W1", "b1", "W2", "b2", "W3", "b3", "wh", "bh")
    return {k: int(v) for k, v in zip(keys, o)}


def sc2_strip(frame, y):
    """(rgb7 (7, W, 3) uint8, rows (7,) int32) of the strip centred on row y."""
    f = _frame(frame)
    H, W = f.shape[:2]
    rgb7 = np.zeros((7, W, 3), np.uint8)
    rows = np.zeros(7, np.int32)
    lib().orc_sc2_strip(_ptr(f), H, W, W * 3, int(y), _ptr(rgb7), _ptr(rows))
    return rgb7, rows


def sc2_features(rgb7, rows, H):
    rgb7 = np.ascontiguousarray(rgb7, np.uint8)
    W = rgb7.shape[1]
    feat = np.zeros((7, W, 5), np.float64)
    lib().orc_sc2_features(_ptr(rgb7), _ptr(np.ascontiguousarray(rows, np.int32)), W, H,
                           _ptr(feat))
    return feat


def sc2_forward(rgb7, rows, H, params, mixed=False):
    rgb7 = np.ascontiguousarray(rgb7, np.uint8)
    W = rgb7.shape[1]
    prm = np.ascontiguousarray(params, np.float32)
    assert prm.size == SC2_NPARAM
    out = np.zeros(W, np.float64)
    if lib().orc_sc2_forward_mode(_ptr(rgb7), _ptr(np.ascontiguousarray(rows, np.int32)), W, H,
                                  _ptr(prm), 1 if mixed else 0, _ptr(out)) != 0:
        raise ValueError("bad scorer arguments")
    return out


def sc2_loss_grad(rgb7, rows, H, targets, params, pos_weight=1.0):
    rgb7 = np.ascontiguousarray(rgb7, np.uint8)
    W = rgb7.shape[1]
    prm = np.ascontiguousarray(params, np.float32)
    t = np.ascontiguousarray(targets, np.float64)
    g = np.zeros(SC2_NPARAM, np.float64)
    loss = lib().orc_sc2_loss_grad(_ptr(rgb7), _ptr(np.ascontiguousarray(rows, np.int32)), W, H,
                                   _ptr(t), float(pos_weight), _ptr(prm), _ptr(g))
    return loss, g


def circle_strips(rows, cy, r, t_ri):
    """Strips whose row is within r + t_ri of the circle's centre row (binary32)."""
    rw = np.ascontiguousarray(rows, np.int32)
    return int(lib().orc_circle_strips(_ptr(rw), len(rw), float(cy), float(r), float(t_ri)))


def sc2_targets(cx, cy, r, valid, W, y, sigma=3.0):
    t = np.zeros(W, np.float64)
    lib().orc_sc2_targets(float(cx), float(cy), float(r), int(valid), int(W), int(y),
                          float(sigma), _ptr(t))
    return t
