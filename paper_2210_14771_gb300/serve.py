"""Python view of the serving API of libca (ca_server_*), and a load driver
that feeds it synthetic video streams.  Marshalling and bookkeeping only:
admission, batching and estimation run in the library."""
from __future__ import annotations

import ctypes as C
import time

import numpy as np
import torch

from . import _native as N
from .api import ContentArea, params as make_params


class Server:
    def __init__(self, ca: ContentArea, p=None, mem_budget: int = 4 << 30, max_streams: int = 32,
                 max_batch: int = 64, track: bool = True, want_masks: bool = False,
                 smooth=None, zero_copy: bool = False):
        """smooth: None, or (gamma, jump, t_hold) of ca_smooth_tracked applied to
        each stream's results (and masks) before they are returned.
        zero_copy: frames (page-locked) are read in place by the kernels,
        never copied to the device."""
        self.ca = ca
        cfg = N.CaServerConfig()
        cfg.params = p or make_params()
        cfg.mem_budget = mem_budget
        cfg.max_streams = max_streams
        cfg.max_batch = max_batch
        cfg.track = 1 if track else 0
        cfg.want_masks = 1 if want_masks else 0
        cfg.zero_copy = 1 if zero_copy else 0
        if smooth is not None:
            cfg.smooth = 1
            cfg.smooth_params = N.CaSmoothParams(float(smooth[0]), float(smooth[1]),
                                                 float(smooth[2]), 0)
        h = C.c_void_p()
        ca._check(N.lib().ca_server_create(ca._h, C.byref(cfg), C.byref(h)))
        self._h = h
        self._out = (N.CaServerResult * 1024)()

    @staticmethod
    def now() -> float:
        return float(N.lib().ca_server_now())

    def submit(self, sid: int, frame: torch.Tensor | np.ndarray, key: int, t_arrival: float,
               mask_host=None):
        """Ticket, or None when the memory budget refuses the frame."""
        if isinstance(frame, torch.Tensor):
            assert frame.device.type == "cpu" and frame.is_contiguous() and frame.dtype == torch.uint8
            ptr = frame.data_ptr()
        else:
            assert frame.flags["C_CONTIGUOUS"] and frame.dtype == np.uint8
            ptr = frame.ctypes.data
        H, W = int(frame.shape[0]), int(frame.shape[1])
        t = C.c_uint64(0)
        st = N.lib().ca_server_submit(self._h, sid, C.c_void_p(ptr), H, W, key, t_arrival,
                                      C.c_void_p(mask_host) if mask_host else None, C.byref(t))
        if st == N.CA_ERR_ADMISSION:
            return None
        self.ca._check(st)
        return int(t.value)

    def submit_batch(self, items):
        """items: list of (sid, frame, key, t_arrival) in admission order.
        One library call; returns the tickets of the admitted prefix (the
        budget refused the rest)."""
        n = len(items)
        if n == 0:
            return []
        reqs = (N.CaServerRequest * n)()
        for i, (sid, frame, key, t_arr) in enumerate(items):
            q = reqs[i]
            if isinstance(frame, torch.Tensor):
                q.frame_host = frame.data_ptr()
            else:
                q.frame_host = frame.ctypes.data
            q.frame_key = key
            q.t_arrival = t_arr
            q.stream_id = sid
            q.H, q.W = int(frame.shape[0]), int(frame.shape[1])
        tickets = (C.c_uint64 * n)()
        got = C.c_int(0)
        st = N.lib().ca_server_submit_batch(self._h, reqs, n, tickets, C.byref(got))
        if st != N.CA_ERR_ADMISSION:
            self.ca._check(st)
        return [int(tickets[i]) for i in range(got.value)]

    def poll(self, wait: bool = False):
        n = C.c_int(0)
        self.ca._check(N.lib().ca_server_poll(self._h, 1 if wait else 0, self._out, 1024,
                                              C.byref(n)))
        out = []
        for i in range(n.value):
            r = self._out[i]
            out.append(dict(ticket=r.ticket, sid=r.stream_id, key=r.frame_key, status=r.status,
                            result=(r.result.cx, r.result.cy, r.result.r, r.result.score,
                                    r.result.valid, r.result.n_inliers),
                            t_arrival=r.t_arrival, t_submit=r.t_submit, t_launch=r.t_launch,
                            t_done=r.t_done))
        return out

    def stats(self):
        used = C.c_size_t(0)
        pend = C.c_int32(0)
        infl = C.c_int32(0)
        self.ca._check(N.lib().ca_server_stats(self._h, C.byref(used), C.byref(pend),
                                               C.byref(infl)))
        return dict(bytes_in_use=used.value, pending=pend.value, launches_in_flight=infl.value)

    def close(self):
        if getattr(self, "_h", None):
            N.lib().ca_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pinned_banks(streams):
    """Each stream's frame bank in pinned host memory (the server copies from it)."""
    return [[torch.from_numpy(f).pin_memory() for f in s.frames] for s in streams]


def run_load(server: Server, streams, banks, n_frames: int, realtime: bool = True,
             sids=None, batched: bool = True):
    """Feeds n_frames of each stream (all, or the ids in `sids`) to the server.
    realtime: frames are submitted at their Poisson arrival times; else all
    arrive at once (saturation).  batched: every frame that has arrived is
    submitted by one ca_server_submit_batch call per loop (in arrival order),
    else one ca_server_submit call per frame.  Returns per-frame records
    (stream, index, result, latency) and the wall time."""
    sids = list(range(len(streams))) if sids is None else list(sids)
    arr = {s: (streams[s].arrivals(n_frames) if realtime else np.zeros(n_frames)) for s in sids}
    nxt = {s: 0 for s in sids}
    ticket_of = {}
    records = []
    t0 = server.now()
    total = n_frames * len(sids)
    while len(records) < total:
        now = server.now() - t0
        progressed = False
        if batched:
            due = []
            for s in sids:
                k = nxt[s]
                while k < n_frames and arr[s][k] <= now:
                    due.append((float(arr[s][k]), s, k))
                    k += 1
            due.sort(key=lambda d: d[0])   # stable: each stream's frames stay in order
            items = [(s, banks[s][k % len(banks[s])], streams[s].key(k), t0 + a)
                     for a, s, k in due]
            for (a, s, k), t in zip(due, server.submit_batch(items)):
                ticket_of[t] = (s, k)
                nxt[s] = k + 1
                progressed = True
        else:
            for s in sids:
                while nxt[s] < n_frames and arr[s][nxt[s]] <= now:
                    k = nxt[s]
                    fr = banks[s][k % len(banks[s])]
                    t = server.submit(s, fr, streams[s].key(k), t0 + float(arr[s][k]))
                    if t is None:   # budget full: retry after the next poll
                        break
                    ticket_of[t] = (s, k)
                    nxt[s] += 1
                    progressed = True
        done = server.poll(wait=False)
        for d in done:
            s, k = ticket_of.pop(d["ticket"])
            d.update(stream=s, index=k, latency=d["t_done"] - d["t_arrival"])
            records.append(d)
        if not done and not progressed:
            pending = sum(n_frames - nxt[s] for s in sids)
            if pending and not ticket_of:
                nx = min(arr[s][nxt[s]] for s in sids if nxt[s] < n_frames)
                time.sleep(max(0.0, min(0.002, nx - (server.now() - t0))))
            elif ticket_of:
                server_done = server.poll(wait=True)
                for d in server_done:
                    s, k = ticket_of.pop(d["ticket"])
                    d.update(stream=s, index=k, latency=d["t_done"] - d["t_arrival"])
                    records.append(d)
    return records, server.now() - t0


def summarise(records, wall):
    """Throughput and latency (arrival to result) of a run, with the latency
    split into its parts: arrival to submission (the feeding loop),
    submission to launch (queued for a batch slot) and launch to result (GPU
    work and collection)."""
    lat = np.array([r["latency"] for r in records]) * 1e3
    part = {
        "feed": np.array([r["t_submit"] - r["t_arrival"] for r in records]) * 1e3,
        "queue": np.array([r["t_launch"] - r["t_submit"] for r in records]) * 1e3,
        "gpu": np.array([r["t_done"] - r["t_launch"] for r in records]) * 1e3,
    }
    out = {"frames": len(records), "seconds": wall, "frames_per_s": len(records) / wall,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "max_ms": float(lat.max()), "over_10ms": int((lat > 10.0).sum())}
    for k, v in part.items():
        out["p99_%s_ms" % k] = float(np.percentile(v, 99))
    return out
