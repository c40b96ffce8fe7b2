"""Tracked estimation and the serving loop on the GPU.

The tracked call must equal the oracle's tracked fit (the previous circle of
the stream as one more hypothesis) bit for bit along a whole stream; the
server must give every frame the result it gets when its stream is served
alone, whatever the mix, batch sizes and admission refusals around it.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2210_14771_gb300 import synth

from _helpers import both_params, same_f32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL = ((240, 320), (288, 360), (480, 640))


@pytest.fixture(scope="module")
def ca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_14771_gb300.build import build
    build()
    from paper_2210_14771_gb300 import api
    h = api.ContentArea(0)
    yield h
    h.close()


@pytest.fixture(scope="module")
def streams():
    return synth.video_streams(5, 6, resolutions=SMALL, bank=6)


def _oracle_chain(orc, stream, n, op, prior_centre=False):
    out, prior = [], None
    for k in range(n):
        f, _ = stream.frame(k)
        r = orc.estimate_tracked(f, stream.key(k), op, prior, prior_centre)
        out.append(r)
        prior = (r["cx"], r["cy"], r["r"]) if r["valid"] else None
    return out


def _same(g, o):
    return (all(same_f32(g[i], o[k]) for i, k in enumerate(("cx", "cy", "r", "score")))
            and int(g[4]) == o["valid"] and int(g[5]) == o["n_inliers"])


def test_tracked_estimate_matches_oracle(ca, orc, streams):
    from paper_2210_14771_gb300 import _native as N, api
    lp, op = both_params(orc, n_strips=16, cands_per_strip=2, n_hyps=64, seed=4)
    n = 6
    want = [_oracle_chain(orc, s, n, op) for s in streams]
    state = torch.zeros((len(streams), 6), dtype=torch.float32, device="cuda")
    for k in range(n):
        ts = [torch.from_numpy(s.frame(k)[0]).cuda() for s in streams]
        arr, B, _, res = ca._descriptors(ts, [s.key(k) for s in streams], None, None)
        track = (C.c_int32 * B)(*range(B))
        ca._check(N.lib().ca_estimate_tracked(ca._h, arr, B, C.byref(lp),
                                              C.c_void_p(state.data_ptr()), track, B,
                                              C.c_void_p(res.data_ptr()),
                                              api._stream_ptr(None, ca.device)))
        ca.sync()
        g = api.results_numpy(res)
        for i in range(B):
            assert _same(tuple(g[i]), want[i][k]), (i, k, g[i], want[i][k])


@pytest.mark.parametrize("mode", [1, 2])
def test_prior_guided_tracked_estimate_matches_oracle(ca, orc, streams, mode):
    """prior_centre: the angle term of each frame points at its stream's
    previous circle; bit for bit the oracle's chain, staged and fused, and
    different from the chain without it (the option is not ignored)."""
    from paper_2210_14771_gb300 import _native as N, api
    lp, op = both_params(orc, n_strips=16, cands_per_strip=2, n_hyps=64, seed=4, batch_mode=mode)
    lp.prior_centre = 1
    n = 6
    want = [_oracle_chain(orc, s, n, op, True) for s in streams]
    plain = [_oracle_chain(orc, s, n, op, False) for s in streams]
    assert want != plain
    state = torch.zeros((len(streams), 6), dtype=torch.float32, device="cuda")
    for k in range(n):
        ts = [torch.from_numpy(s.frame(k)[0]).cuda() for s in streams]
        arr, B, _, res = ca._descriptors(ts, [s.key(k) for s in streams], None, None)
        track = (C.c_int32 * B)(*range(B))
        ca._check(N.lib().ca_estimate_tracked(ca._h, arr, B, C.byref(lp),
                                              C.c_void_p(state.data_ptr()), track, B,
                                              C.c_void_p(res.data_ptr()),
                                              api._stream_ptr(None, ca.device)))
        ca.sync()
        g = api.results_numpy(res)
        for i in range(B):
            assert _same(tuple(g[i]), want[i][k]), (i, k, g[i], want[i][k])


def test_prior_centre_argument_check(ca):
    from paper_2210_14771_gb300 import _native as N, api
    t = torch.zeros((1, 64, 96, 3), dtype=torch.uint8, device="cuda")
    for kw in (dict(prior_centre=2), dict(reserved=1)):
        with pytest.raises(N.CaError) as e:
            ca.estimate(t, api.params(**kw))
        assert e.value.status == 1


def _serve(ca, streams, banks, n, sids, max_batch, budget, p):
    from paper_2210_14771_gb300 import serve
    srv = serve.Server(ca, p, mem_budget=budget, max_streams=len(streams), max_batch=max_batch)
    recs, _ = serve.run_load(srv, streams, banks, n, realtime=False, sids=sids)
    srv.close()
    return {(r["stream"], r["index"]): r["result"] for r in recs}


def test_server_result_same_alone_and_in_the_mix(ca, orc, streams):
    from paper_2210_14771_gb300 import api, serve
    lp, op = both_params(orc, n_strips=16, cands_per_strip=2, n_hyps=64, seed=4)
    banks = serve.pinned_banks(streams)
    n = 8
    mix = _serve(ca, streams, banks, n, None, 4, 1 << 30, lp)
    # a budget of about two frames forces admission refusals and retries
    tight = _serve(ca, streams, banks, n, None, 3, 2 * 480 * 640 * 3 + 4096, lp)
    assert mix == tight
    for s in range(len(streams)):
        alone = _serve(ca, streams, banks, n, [s], 64, 1 << 28, lp)
        assert all(alone[(s, k)] == mix[(s, k)] for k in range(n)), s
    want = _oracle_chain(orc, streams[2], n, op)
    assert all(_same(mix[(2, k)], want[k]) for k in range(n))
    del api


def test_zero_copy_server_reads_frames_in_place(ca, orc, streams):
    """With zero_copy the frames stay in page-locked host memory (the kernels
    read their strip rows over the host link) and masks go straight into
    page-locked host buffers: every result equals the copying server's and
    the oracle's tracked chain bit for bit, every mask equals the oracle's
    mask of that result, and the pool holds nothing but device masks."""
    from paper_2210_14771_gb300 import serve
    lp, op = both_params(orc, n_strips=16, cands_per_strip=2, n_hyps=64, seed=4)
    banks = serve.pinned_banks(streams)
    n = 8
    copied = _serve(ca, streams, banks, n, None, 4, 1 << 30, lp)
    srv = serve.Server(ca, lp, mem_budget=4096, max_streams=len(streams), max_batch=4,
                       zero_copy=True)
    recs, _ = serve.run_load(srv, streams, banks, n, realtime=False)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()
    zc = {(r["stream"], r["index"]): r["result"] for r in recs}
    assert zc == copied
    want = _oracle_chain(orc, streams[1], n, op)
    assert all(_same(zc[(1, k)], want[k]) for k in range(n))
    # masks into page-locked host buffers, one stream, frame by frame
    s = streams[3]
    srv = serve.Server(ca, lp, mem_budget=4096, max_streams=len(streams), want_masks=True,
                       zero_copy=True)
    masks = [torch.zeros((s.H, s.W), dtype=torch.uint8).pin_memory() for _ in range(n)]
    got = {}
    for k in range(n):
        t = srv.submit(3, banks[3][k % len(banks[3])], s.key(k), srv.now(),
                       mask_host=masks[k].data_ptr())
        assert t is not None
        for d in srv.poll(wait=True):
            got[d["ticket"]] = (k, d)
    srv.close()
    want = _oracle_chain(orc, s, n, op)
    for k, d in got.values():
        assert d["status"] == 0 and _same(d["result"], want[k])
        assert np.array_equal(masks[k].numpy(), orc.mask(want[k], s.H, s.W)), k


def test_zero_copy_server_refuses_pageable_frames(ca, streams):
    from paper_2210_14771_gb300 import _native as N, serve
    srv = serve.Server(ca, None, mem_budget=4096, max_streams=2, zero_copy=True)
    f = np.ascontiguousarray(streams[0].frames[0])      # pageable numpy memory
    with pytest.raises(N.CaError) as e:
        srv.submit(0, f, 1, srv.now())
    assert e.value.status == 1
    with pytest.raises(N.CaError) as e:
        srv.submit_batch([(0, f, 1, srv.now())])
    assert e.value.status == 1 and srv.stats()["pending"] == 0
    srv.close()


def test_failed_launch_is_requeued_and_served_in_order(ca, orc, streams):
    """A launch whose estimate fails on the host (an injected CA_ERR_OOM)
    queues nothing: poll reports the error, the frames go back to the front
    of the queue, and later polls serve every stream in order with the
    results of an undisturbed run."""
    from paper_2210_14771_gb300 import _native as N, serve
    lp, op = both_params(orc, n_strips=16, cands_per_strip=2, n_hyps=64, seed=4)
    banks = serve.pinned_banks(streams)
    n = 4
    clean = _serve(ca, streams, banks, n, None, 3, 1 << 30, lp)
    srv = serve.Server(ca, lp, mem_budget=1 << 30, max_streams=len(streams), max_batch=3)
    tickets = {}
    items = [(s, banks[s][k % len(banks[s])], streams[s].key(k), srv.now())
             for k in range(n) for s in range(len(streams))]
    for (s, _, _, _), t in zip(items, srv.submit_batch(items)):
        tickets[t] = s
    assert len(tickets) == n * len(streams)
    ca._check(N.lib().ca_inject_failure(ca._h, 1, N.CA_ERR_OOM))   # the second launch fails
    with pytest.raises(N.CaError) as e:
        srv.poll(wait=False)
    assert e.value.status == N.CA_ERR_OOM
    assert srv.stats()["pending"] == n * len(streams) - 3       # only the first launch left
    done = []
    while len(done) < n * len(streams):
        done += srv.poll(wait=True)
    srv.close()
    order = {}
    for d in sorted(done, key=lambda d: d["ticket"]):
        assert d["status"] == 0
        order.setdefault(d["sid"], []).append(d)
    for sid, ds in order.items():
        for k, d in enumerate(ds):
            assert d["key"] == streams[sid].key(k)
            assert d["result"] == clean[(sid, k)], (sid, k)


def test_admission_refuses_beyond_the_budget(ca, streams):
    from paper_2210_14771_gb300 import serve
    s = streams[0]
    fb = s.H * s.W * 3
    srv = serve.Server(ca, None, mem_budget=2 * ((fb + 255) // 256 * 256), max_streams=6)
    f = torch.from_numpy(s.frames[0]).pin_memory()
    t0 = srv.submit(0, f, 1, srv.now())
    t1 = srv.submit(1, f, 2, srv.now())
    assert t0 is not None and t1 is not None
    assert srv.submit(2, f, 3, srv.now()) is None          # budget full
    got = []
    while len(got) < 2:
        got += srv.poll(wait=True)
    assert srv.stats()["bytes_in_use"] == 0
    assert srv.submit(2, f, 3, srv.now()) is not None      # admitted once memory is free
    while not srv.poll(wait=True):
        pass
    srv.close()


def test_realtime_serving_latency(ca, streams):
    """Poisson arrivals at 30-60 fps per stream: every frame is served and the
    tail latency stays far below a frame interval."""
    from paper_2210_14771_gb300 import api, serve
    p = api.params(n_strips=32, cands_per_strip=2, n_hyps=1024)
    srv = serve.Server(ca, p, mem_budget=1 << 30, max_streams=len(streams))
    banks = serve.pinned_banks(streams)
    recs, wall = serve.run_load(srv, streams, banks, 15, realtime=True)
    srv.close()
    st = serve.summarise(recs, wall)
    print("serving:", st)
    assert st["frames"] == 15 * len(streams)
    assert st["p99_ms"] < 20.0


def _results_tensor(rows):
    from paper_2210_14771_gb300 import api
    a = np.zeros(len(rows), dtype=api.RESULT_DTYPE)
    for i, r in enumerate(rows):
        a[i] = tuple(r)
    return torch.from_numpy(a.view(np.float32).reshape(len(rows), 6).copy()).cuda()


def test_smooth_tracked_matches_oracle(ca, orc):
    """ca_smooth_tracked on random result sequences of 6 tracks over 40 calls
    (random subsets of tracks per call, random widths and validity, scene
    jumps): every output and the final states equal the oracle's
    orc_smooth applied to each track's sequence, bit for bit."""
    from paper_2210_14771_gb300 import api
    rng = np.random.default_rng(21)
    n_tracks, gamma, jump, t_hold = 6, 0.8, 0.05, 0.06
    widths = [int(w) for w in rng.choice([640, 720, 1280, 1920], n_tracks)]
    state = torch.zeros((n_tracks, 4), dtype=torch.float32, device="cuda")
    seqs = {t: [] for t in range(n_tracks)}
    got = {t: [] for t in range(n_tracks)}
    centre = rng.uniform(100, 500, (n_tracks, 3))
    for _ in range(40):
        tracks = [int(t) for t in rng.permutation(n_tracks)[:rng.integers(1, n_tracks + 1)]]
        rows = []
        for t in tracks:
            if rng.random() < 0.1:                     # a new scene
                centre[t] = rng.uniform(100, 500, 3)
            c = centre[t] + rng.normal(0, 2.0, 3)
            valid = int(rng.random() < 0.8)
            rows.append((np.float32(c[0]), np.float32(c[1]), np.float32(c[2]),
                         np.float32(rng.uniform(0.05, 1.0)) if valid else np.float32(0),
                         valid, int(rng.integers(3, 60)) if valid else 0))
        res = _results_tensor(rows)
        out = ca.smooth_tracked(res, [widths[t] for t in tracks], tracks, state, gamma, jump,
                                t_hold, out=torch.empty_like(res))
        g = api.results_numpy(out)
        for i, t in enumerate(tracks):
            seqs[t].append(rows[i])
            got[t].append(tuple(g[i]))
    for t in range(n_tracks):
        want, st = orc.smooth_chain(seqs[t], widths[t], gamma, jump, t_hold)
        for a, b in zip(got[t], want):
            assert _same(a, b), (t, a, b)
        assert np.array_equal(state[t].cpu().numpy().view(np.uint32), st.view(np.uint32)), t


def test_server_smoothing_matches_the_oracle_chain(ca, orc, streams):
    """Served with smoothing: each frame's result is the oracle's tracked
    estimate of the stream smoothed by orc_smooth, bit for bit, alone or in
    the mix."""
    from paper_2210_14771_gb300 import serve
    lp, op = both_params(orc, n_strips=16, cands_per_strip=2, n_hyps=64, seed=4)
    banks = serve.pinned_banks(streams)
    n, sm = 8, (0.75, 0.05, 0.06)
    srv = serve.Server(ca, lp, mem_budget=1 << 30, max_streams=len(streams), max_batch=4,
                       smooth=sm, want_masks=True)
    recs, _ = serve.run_load(srv, streams, banks, n, realtime=False)
    srv.close()
    got = {(r["stream"], r["index"]): r["result"] for r in recs}
    for s_id, s in enumerate(streams):
        raw = _oracle_chain(orc, s, n, op)
        want, _ = orc.smooth_chain(raw, s.W, *sm)
        for k in range(n):
            assert _same(got[(s_id, k)], want[k]), (s_id, k, got[(s_id, k)], want[k])


def test_smooth_argument_errors(ca):
    from paper_2210_14771_gb300 import _native as N
    res = _results_tensor([(1.0, 2.0, 3.0, 0.5, 1, 4)] * 2)
    state = torch.zeros((2, 4), dtype=torch.float32, device="cuda")
    for kw, tr in ((dict(gamma=1.0), [0, 1]), (dict(gamma=0.5, jump=-1.0), [0, 1]),
                   (dict(gamma=0.5), [0, 0]), (dict(gamma=0.5), [0, 2])):
        args = dict(gamma=0.5, jump=0.05, t_hold=0.06)
        args.update(kw)
        with pytest.raises(N.CaError) as e:
            ca.smooth_tracked(res, [64, 64], tr, state, **args)
        assert e.value.status == 1, (kw, tr)
