"""Python view of libca: same calls as include/ca.h, argument marshalling only.

PyTorch supplies device memory and streams; every step of the estimation runs
in the library's CUDA kernels.  There is no CPU fallback: without the built
library or a GPU these functions raise.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N

RESULT_DTYPE = np.dtype([("cx", "<f4"), ("cy", "<f4"), ("r", "<f4"), ("score", "<f4"),
                         ("valid", "<i4"), ("n_inliers", "<i4")])
SLOT_DTYPE = np.dtype([("x", "<i2"), ("y", "<i2"), ("s", "<u2"), ("kept", "<u2")])
TRACE_DTYPE = np.dtype([("t_grab", "<u8"), ("t_ready", "<u8"), ("t_end", "<u8"),
                        ("phase", "<i4"), ("sm", "<i4"), ("cta", "<i4")])
HYP_DTYPE = np.dtype([("i0", "<i4"), ("i1", "<i4"), ("i2", "<i4"), ("n_inl", "<i4"),
                      ("S", "<u4"), ("pass", "<i4"), ("cx", "<f4"), ("cy", "<f4"),
                      ("r", "<f4")])


def params(**kw) -> N.CaParams:
    """ca_params with the paper's defaults (Appendix A), overridden by kw."""
    p = N.CaParams()
    N.lib().ca_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _stream_ptr(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return C.c_void_p(s.cuda_stream)


def results_numpy(res: torch.Tensor) -> np.ndarray:
    """(B, 6) float32 result tensor (any device) -> structured numpy array."""
    return res.detach().cpu().contiguous().numpy().view(RESULT_DTYPE).reshape(-1)


def new_results(B: int, device) -> torch.Tensor:
    return torch.zeros((B, 6), dtype=torch.float32, device=device)


def estimate_static(frames: torch.Tensor, p=None, keys=None, masks=None, results=None,
                    stream=None):
    """ca_estimate_static: the estimate of a uniform batch without any device
    allocation by the library (for callers that cannot allocate; see ca.h).
    `results` and `masks` must be preallocated by the caller (or None for no
    masks); frames (B, H, W, 3) uint8 CUDA, B <= 256."""
    p = p or params()
    B, H, W, _ = frames.shape
    assert frames.dtype == torch.uint8 and frames.is_cuda and frames.is_contiguous()
    assert results is not None and results.shape == (B, 6)
    karr = (C.c_uint64 * max(B, 1))(*(keys if keys is not None else range(B)))
    N.check(N.lib().ca_estimate_static(
        C.c_void_p(frames.data_ptr()), B, H, W, karr, C.byref(p),
        C.c_void_p(results.data_ptr()),
        C.c_void_p(masks.data_ptr()) if masks is not None else None,
        _stream_ptr(stream, frames.device)))
    return results, masks


class ContentArea:
    """One libca handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = torch.device("cuda", device)
        h = C.c_void_p()
        N.check(N.lib().ca_create(C.byref(h), device))
        self._h = h
        self._plans = []

    def close(self):
        for pl in getattr(self, "_plans", []):
            pl.close()
        self._plans = []
        if getattr(self, "_h", None):
            N.lib().ca_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        N.check(st, self._h)

    # ------------------------------------------------------------ estimate --
    def estimate(self, frames, p=None, keys=None, masks=None, results=None, stream=None):
        """Content area of a batch (Sec. 2.2).

        frames: uint8 CUDA tensor (B, H, W, 3), or a list of (H, W, 3) tensors
        of any sizes.  keys: frame keys (defaults 0..B-1).  masks: None, True
        (allocate), a (B, H, W) uint8 tensor, or a list of (H, W) tensors.
        Returns (results (B, 6) float32 tensor, masks or None); queued on
        `stream` (default: the current stream).
        """
        p = p or params()
        st = _stream_ptr(stream, self.device)
        if masks is False:
            masks = None
        if isinstance(frames, torch.Tensor):
            B, H, W, _ = frames.shape
            assert frames.dtype == torch.uint8 and frames.is_cuda and frames.is_contiguous()
            if masks is True:
                masks = torch.empty((B, H, W), dtype=torch.uint8, device=frames.device)
            if results is None:
                results = new_results(B, frames.device)
            karr = (C.c_uint64 * B)(*(keys if keys is not None else range(B)))
            self._check(N.lib().ca_estimate_uniform(
                self._h, C.c_void_p(frames.data_ptr()), B, H, W, karr, C.byref(p),
                C.c_void_p(results.data_ptr()),
                C.c_void_p(masks.data_ptr()) if masks is not None else None, st))
            return results, masks
        arr, B, masks, results = self._descriptors(frames, keys, masks, results)
        self._check(N.lib().ca_estimate(self._h, arr, B, C.byref(p),
                                        C.c_void_p(results.data_ptr()), st))
        return results, masks

    def _descriptors(self, frames, keys, masks, results):
        """ca_frame array for a list of (H, W, 3) uint8 CUDA tensors."""
        frames = list(frames)
        B = len(frames)
        if masks is True:
            masks = [torch.empty(f.shape[:2], dtype=torch.uint8, device=f.device) for f in frames]
        if results is None:
            results = new_results(B, self.device)
        arr = (N.CaFrame * max(B, 1))()
        for i, f in enumerate(frames):
            assert f.dtype == torch.uint8 and f.is_cuda and f.dim() == 3 and f.shape[2] == 3
            assert f.stride(2) == 1 and f.stride(1) == 3
            arr[i].rgb_dev = f.data_ptr()
            arr[i].mask_dev = (masks[i].data_ptr() if masks is not None and masks[i] is not None
                               else None)
            arr[i].H, arr[i].W = int(f.shape[0]), int(f.shape[1])
            arr[i].pitch = int(f.stride(0))
            arr[i].frame_key = int(keys[i]) if keys is not None else i
        return arr, B, masks, results

    # ------------------------------------------------------------ batching --
    def tune(self, frames, p=None, keys=None, masks=None, results=None, stream=None) -> dict:
        """ca_tune: time the result-preserving launch configurations on this
        batch (list of (H, W, 3) tensors) and remember the fastest."""
        p = p or params()
        if isinstance(frames, torch.Tensor):
            frames = list(frames)
            if isinstance(masks, torch.Tensor):
                masks = list(masks)
        arr, B, masks, results = self._descriptors(frames, keys, masks, results)
        t = N.CaTuning()
        self._check(N.lib().ca_tune(self._h, arr, B, C.byref(p), C.c_void_p(results.data_ptr()),
                                    _stream_ptr(stream, self.device), C.byref(t)))
        return {k: getattr(t, k) for k, _ in N.CaTuning._fields_}

    def plan(self, frames, p=None, keys=None, masks=None, results=None) -> "Plan":
        """ca_plan_create: capture the estimate of this batch in a CUDA graph."""
        p = p or params()
        if isinstance(frames, torch.Tensor):
            frames = list(frames)
            if isinstance(masks, torch.Tensor):
                masks = list(masks)
        arr, B, masks, results = self._descriptors(frames, keys, masks, results)
        h = C.c_void_p()
        self._check(N.lib().ca_plan_create(self._h, arr, B, C.byref(p),
                                           C.c_void_p(results.data_ptr()), C.byref(h)))
        pl = Plan(self, h, frames, masks, results)
        self._plans.append(pl)
        return pl

    def mask(self, results: torch.Tensor, sizes, masks=None, stream=None):
        """Content-area masks of results (Sec. 1.1): sizes = [(H, W), ...]."""
        B = len(sizes)
        if masks is None:
            masks = [torch.empty(s, dtype=torch.uint8, device=results.device) for s in sizes]
        Hs = (C.c_int32 * B)(*[int(s[0]) for s in sizes])
        Ws = (C.c_int32 * B)(*[int(s[1]) for s in sizes])
        ptrs = (C.c_void_p * B)(*[m.data_ptr() for m in masks])
        self._check(N.lib().ca_mask(self._h, C.c_void_p(results.data_ptr()), B, Hs, Ws, ptrs,
                                    _stream_ptr(stream, self.device)))
        return masks

    def run_host(self, frames: np.ndarray, p=None, keys=None, want_masks=True):
        """End-to-end call on host buffers (copies in, estimates, copies out)."""
        p = p or params()
        frames = np.ascontiguousarray(frames, np.uint8)
        B, H, W, _ = frames.shape
        res = np.zeros(B, RESULT_DTYPE)
        masks = np.empty((B, H, W), np.uint8) if want_masks else None
        karr = (C.c_uint64 * B)(*(keys if keys is not None else range(B)))
        self._check(N.lib().ca_run_host(
            self._h, frames.ctypes.data_as(C.c_void_p), B, H, W, karr, C.byref(p),
            res.ctypes.data_as(C.c_void_p),
            masks.ctypes.data_as(C.c_void_p) if masks is not None else None))
        return res, masks

    def run_host_ptr(self, frames_ptr: int, B, H, W, keys_arr, p, res_ptr: int, masks_ptr):
        """ca_run_host on raw host pointers (pinned buffers of the caller)."""
        self._check(N.lib().ca_run_host(self._h, C.c_void_p(frames_ptr), B, H, W, keys_arr,
                                        C.byref(p), C.c_void_p(res_ptr),
                                        C.c_void_p(masks_ptr) if masks_ptr else None))

    def run_host_zero_copy_ptr(self, frames_ptr: int, B, H, W, keys_arr, p, res_ptr: int,
                               masks_ptr):
        """ca_run_host_zero_copy on page-locked host buffers of the caller."""
        self._check(N.lib().ca_run_host_zero_copy(self._h, C.c_void_p(frames_ptr), B, H, W,
                                                  keys_arr, C.byref(p), C.c_void_p(res_ptr),
                                                  C.c_void_p(masks_ptr) if masks_ptr else None))

    # ---------------------------------------- the paper's 2-D scorer --
    @staticmethod
    def _strip7_args(strips7, rows):
        assert strips7.dtype == torch.uint8 and strips7.is_cuda and strips7.is_contiguous()
        assert strips7.dim() == 4 and strips7.shape[1] == 7 and strips7.shape[3] == 3
        n, W = int(strips7.shape[0]), int(strips7.shape[2])
        assert rows.dtype == torch.int32 and rows.is_cuda and rows.is_contiguous()
        assert rows.shape == (n, 7)
        return n, W

    def scorer2d_forward(self, strips7: torch.Tensor, rows: torch.Tensor, H: int,
                         params: torch.Tensor | None = None, stream=None, scores=False):
        """ca_scorer2d_forward: logits (n, W) of the middle rows of n strips
        (n, 7, W, 3) uint8 with their frame rows (n, 7) int32, all on the
        device; params: CA_SCORER2D_NPARAM float32 on the device, or None for
        the handle's parameters.  scores=True also returns the Q15 scores."""
        n, W = self._strip7_args(strips7, rows)
        if params is not None:
            assert params.dtype == torch.float32 and params.is_cuda
            assert params.numel() == N.CA_SCORER2D_NPARAM
            params = params.contiguous()
        out = torch.empty((n, W), dtype=torch.float32, device=strips7.device)
        sc = torch.empty((n, W), dtype=torch.int16, device=strips7.device) if scores else None
        self._check(N.lib().ca_scorer2d_forward(
            self._h, C.c_void_p(strips7.data_ptr()), C.c_void_p(rows.data_ptr()), n, W, H,
            C.c_void_p(params.data_ptr()) if params is not None else None,
            C.c_void_p(out.data_ptr()), C.c_void_p(sc.data_ptr()) if sc is not None else None,
            _stream_ptr(stream, strips7.device)))
        return (out, sc) if scores else out

    def scorer2d_init(self, seed: int = 0):
        self._check(N.lib().ca_scorer2d_init(self._h, seed))

    def scorer2d_set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, np.float32)
        self._check(N.lib().ca_scorer2d_set_params(self._h, p.ctypes.data_as(C.c_void_p), p.size))

    def scorer2d_get_params(self) -> np.ndarray:
        p = np.zeros(N.CA_SCORER2D_NPARAM, np.float32)
        self._check(N.lib().ca_scorer2d_get_params(self._h, p.ctypes.data_as(C.c_void_p), p.size))
        return p

    def scorer2d_save(self, path: str):
        self._check(N.lib().ca_scorer2d_save(self._h, path.encode()))

    def scorer2d_load(self, path: str):
        self._check(N.lib().ca_scorer2d_load(self._h, path.encode()))

    def scorer2d_step(self, strips7, rows, targets, H: int, idx=None, lr=0.0, momentum=0.9,
                      pos_weight=1.0, apply=False, want_grads=True, clip_norm=0.0):
        """One training step of the 2-D network on soft targets (n, W) float32;
        returns (summed loss, summed gradient or None)."""
        n, W = self._strip7_args(strips7, rows)
        assert targets.dtype == torch.float32 and targets.is_cuda and targets.shape == (n, W)
        if idx is not None:
            assert idx.dtype == torch.int32 and idx.is_cuda
            n = int(idx.numel())
        tp = N.CaTrainParams(lr, momentum, pos_weight, 1 if apply else 0, clip_norm,
                             N.CA_LR_CONSTANT)
        loss = C.c_float(0.0)
        g = np.zeros(N.CA_SCORER2D_NPARAM, np.float32) if want_grads else None
        self._check(N.lib().ca_scorer2d_step(
            self._h, C.c_void_p(strips7.data_ptr()), C.c_void_p(rows.data_ptr()),
            C.c_void_p(targets.data_ptr()), C.c_void_p(idx.data_ptr()) if idx is not None else None,
            n, W, H, C.byref(tp), C.byref(loss),
            g.ctypes.data_as(C.c_void_p) if g is not None else None))
        return float(loss.value), g

    def scorer2d_train(self, strips7, rows, targets, H: int, epochs=1, batch=64, seed=0, lr=0.05,
                       momentum=0.9, pos_weight=1.0, clip_norm=1.0, schedule="cosine"):
        """ca_scorer2d_train; returns the mean loss per column of each epoch."""
        n, W = self._strip7_args(strips7, rows)
        assert targets.dtype == torch.float32 and targets.shape == (n, W)
        sched = {"constant": N.CA_LR_CONSTANT, "cosine": N.CA_LR_COSINE}[schedule]
        tp = N.CaTrainParams(lr, momentum, pos_weight, 1, clip_norm, sched)
        out = np.zeros(max(epochs, 1), np.float32)
        self._check(N.lib().ca_scorer2d_train(
            self._h, C.c_void_p(strips7.data_ptr()), C.c_void_p(rows.data_ptr()),
            C.c_void_p(targets.data_ptr()), n, W, H, C.byref(tp), epochs, batch, seed,
            out.ctypes.data_as(C.c_void_p)))
        return out[:epochs]

    def smooth_tracked(self, res: torch.Tensor, widths, track, state: torch.Tensor, gamma: float,
                       jump: float, t_hold: float, out: torch.Tensor | None = None, stream=None):
        """ca_smooth_tracked: (B, 6) results (device) of frames of the given
        widths on the given tracks -> smoothed results (device); state is the
        (n_tracks, 4) float32 device state, updated."""
        B = int(res.shape[0])
        assert res.is_cuda and res.dtype == torch.float32 and res.shape == (B, 6)
        assert state.is_cuda and state.dtype == torch.float32 and state.shape[1] == 4
        out = res if out is None else out
        sp = N.CaSmoothParams(gamma, jump, t_hold, 0)
        W = (C.c_int32 * max(B, 1))(*[int(w) for w in widths])
        T = (C.c_int32 * max(B, 1))(*[int(t) for t in track])
        self._check(N.lib().ca_smooth_tracked(self._h, C.c_void_p(res.data_ptr()), B, W, T,
                                              int(state.shape[0]), C.byref(sp),
                                              C.c_void_p(state.data_ptr()),
                                              C.c_void_p(out.data_ptr()),
                                              _stream_ptr(stream, self.device)))
        return out

    def sync(self, stream=None):
        self._check(N.lib().ca_sync(self._h, _stream_ptr(stream, self.device)))

    def launch_count(self) -> int:
        return int(N.lib().ca_launch_count(self._h))

    def set_timing(self, on: bool):
        self._check(N.lib().ca_set_timing(self._h, 1 if on else 0))

    def set_trace(self, on: bool):
        """ca_set_trace: record the timeline of later fused calls."""
        self._check(N.lib().ca_set_trace(self._h, 1 if on else 0))

    def dump_trace(self):
        """Timeline of the last traced fused call: a structured array with one
        record per work item (t_grab, t_ready, t_end in ns; phase 0 strips,
        1 fit, 2 mask; sm; cta), in item order."""
        hdr = self._dump(N.CA_DUMP_TRACE, 0, None, 8)   # the header sizes the buffer
        n = int(hdr[:4].view(np.int32)[0])
        raw = self._dump(N.CA_DUMP_TRACE, 0, None, 8 + 32 * n)
        w = raw[8:8 + 32 * n].view(np.uint64).reshape(n, 4)
        out = np.zeros(n, dtype=TRACE_DTYPE)
        out["t_grab"], out["t_ready"], out["t_end"] = w[:, 0], w[:, 1], w[:, 2]
        out["phase"] = (w[:, 3] >> np.uint64(48)).astype(np.int32)
        out["sm"] = ((w[:, 3] >> np.uint64(32)) & np.uint64(0xFFFF)).astype(np.int32)
        out["cta"] = (w[:, 3] & np.uint64(0xFFFFFFFF)).astype(np.int32)
        return out

    def kernel_times(self):
        """{kernel: (total ms, launches)} since the last read (CUDA events)."""
        ms = (C.c_double * 5)()
        cnt = (C.c_int32 * 5)()
        self._check(N.lib().ca_kernel_times(self._h, ms, cnt))
        names = ("strips", "fit", "mask", "fused", "scorer")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(names)}

    # ------------------------------------------------------ learned scorer --
    def scorer_init(self, seed: int = 0):
        self._check(N.lib().ca_scorer_init(self._h, seed))

    def scorer_set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, np.float32)
        self._check(N.lib().ca_scorer_set_params(self._h, p.ctypes.data_as(C.c_void_p), p.size))

    def scorer_get_params(self) -> np.ndarray:
        p = np.zeros(N.CA_SCORER_NPARAM, np.float32)
        self._check(N.lib().ca_scorer_get_params(self._h, p.ctypes.data_as(C.c_void_p), p.size))
        return p

    def scorer_save(self, path: str):
        self._check(N.lib().ca_scorer_save(self._h, path.encode()))

    def scorer_load(self, path: str):
        self._check(N.lib().ca_scorer_load(self._h, path.encode()))

    @staticmethod
    def _strip_args(strips, ys):
        assert strips.dtype == torch.uint8 and strips.is_cuda and strips.is_contiguous()
        assert strips.dim() == 4 and strips.shape[1] == 3 and strips.shape[3] == 3
        assert ys.dtype == torch.int32 and ys.is_cuda and ys.is_contiguous()
        return int(strips.shape[0]), int(strips.shape[2])

    def scorer_forward(self, strips, ys, H: int, stream=None):
        """Logits and Q15 scores (n, W) of stand-alone strips (n, 3, W, 3)."""
        n, W = self._strip_args(strips, ys)
        logits = torch.empty((n, W), dtype=torch.float32, device=strips.device)
        scores = torch.empty((n, W), dtype=torch.int16, device=strips.device)
        self._check(N.lib().ca_scorer_forward(
            self._h, C.c_void_p(strips.data_ptr()), C.c_void_p(ys.data_ptr()), n, W, H,
            C.c_void_p(logits.data_ptr()), C.c_void_p(scores.data_ptr()),
            _stream_ptr(stream, strips.device)))
        return logits, scores

    def scorer_step(self, strips, ys, labels, H: int, idx=None, lr=0.0, momentum=0.9,
                    pos_weight=1.0, apply=False, want_grads=True, clip_norm=0.0):
        """One training step; returns (summed loss, summed gradient or None)."""
        n, W = self._strip_args(strips, ys)
        if idx is not None:
            assert idx.dtype == torch.int32 and idx.is_cuda
            n = int(idx.numel())
        tp = N.CaTrainParams(lr, momentum, pos_weight, 1 if apply else 0, clip_norm,
                             N.CA_LR_CONSTANT)
        loss = C.c_float(0.0)
        g = np.zeros(N.CA_SCORER_NPARAM, np.float32) if want_grads else None
        self._check(N.lib().ca_scorer_step(
            self._h, C.c_void_p(strips.data_ptr()), C.c_void_p(ys.data_ptr()),
            C.c_void_p(labels.data_ptr()), C.c_void_p(idx.data_ptr()) if idx is not None else None,
            n, W, H, C.byref(tp), C.byref(loss),
            g.ctypes.data_as(C.c_void_p) if g is not None else None))
        return float(loss.value), g

    def scorer_train(self, strips, ys, labels, H: int, epochs=1, batch=64, seed=0, lr=0.05,
                     momentum=0.9, pos_weight=20.0, clip_norm=1.0, schedule="cosine"):
        """ca_scorer_train; returns the mean loss per column of each epoch.
        schedule: "cosine" (warm-up, then cosine decay of lr) or "constant"."""
        n, W = self._strip_args(strips, ys)
        assert labels.dtype == torch.uint8 and labels.shape == (n, W)
        sched = {"constant": N.CA_LR_CONSTANT, "cosine": N.CA_LR_COSINE}[schedule]
        tp = N.CaTrainParams(lr, momentum, pos_weight, 1, clip_norm, sched)
        out = np.zeros(max(epochs, 1), np.float32)
        self._check(N.lib().ca_scorer_train(
            self._h, C.c_void_p(strips.data_ptr()), C.c_void_p(ys.data_ptr()),
            C.c_void_p(labels.data_ptr()), n, W, H, C.byref(tp), epochs, batch, seed,
            out.ctypes.data_as(C.c_void_p)))
        return out[:epochs]

    def dump_learned(self, frame: int, n_strips: int, W: int):
        """Learned Q15 scores (N, W) of one frame of the last call."""
        raw = self._dump(N.CA_DUMP_LEARNED, frame, None, 2 * n_strips * W)
        return raw.view(np.uint16).reshape(n_strips, W)

    # --------------------------------------------------------------- debug --
    def set_debug(self, level: int):
        self._check(N.lib().ca_set_debug(self._h, level))

    def set_wait_limit(self, ns: int):
        self._check(N.lib().ca_set_wait_limit(self._h, ns))

    def _dump(self, what, frame, p, nbytes):
        buf = np.zeros(nbytes, np.uint8)
        written = C.c_size_t(0)
        self._check(N.lib().ca_debug_dump(self._h, what, frame, C.byref(p) if p else None,
                                          buf.ctypes.data_as(C.c_void_p), nbytes,
                                          C.byref(written)))
        return buf[:written.value]

    def dump_candidates(self, frame: int):
        """Candidate slots of one frame of the last call (debug level >= 1)."""
        raw = self._dump(N.CA_DUMP_CANDIDATES, frame, None, 8 + 8 * 256)
        M, n = (int(v) for v in raw[:8].view(np.int32))
        slots = raw[8:8 + 8 * n].view(SLOT_DTYPE)
        kept = slots[slots["kept"] == 1]
        return dict(M=M, slots=slots, x=kept["x"].copy(), y=kept["y"].copy(), s=kept["s"].copy())

    def dump_hypotheses(self, frame: int, max_hyps: int = 1 << 20):
        """Per-hypothesis records of one frame of the last call (debug level 2)."""
        nbytes = 4 + HYP_DTYPE.itemsize * max_hyps
        raw = self._dump(N.CA_DUMP_HYPOTHESES, frame, None, nbytes)
        nh = int(raw[:4].view(np.int32)[0])
        return raw[4:4 + HYP_DTYPE.itemsize * nh].view(HYP_DTYPE)

    def tables(self, p, H: int):
        """The library's own s_g / s_theta / s_iota tables and Eq. 1 rows."""
        nb = 2 * (N.LUT_G + N.LUT_T + N.LUT_I) + 4 * p.n_strips
        raw = self._dump(N.CA_DUMP_TABLES, H, p, nb)
        u16 = raw[:2 * (N.LUT_G + N.LUT_T + N.LUT_I)].view(np.uint16)
        rows = raw[2 * (N.LUT_G + N.LUT_T + N.LUT_I):].view(np.int32)
        return (u16[:N.LUT_G], u16[N.LUT_G:N.LUT_G + N.LUT_T], u16[N.LUT_G + N.LUT_T:], rows)


class Plan:
    """A captured estimate (ca_plan): `launch()` replays one CUDA graph.  Holds
    references to the frames, masks and results it was captured with."""

    def __init__(self, owner: ContentArea, h, frames, masks, results):
        self.owner, self._h = owner, h
        self.frames, self.masks, self.results = frames, masks, results

    def launch(self, stream=None):
        self.owner._check(N.lib().ca_plan_launch(self._h, _stream_ptr(stream, self.owner.device)))
        return self.results, self.masks

    def close(self):
        if getattr(self, "_h", None):
            N.lib().ca_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
