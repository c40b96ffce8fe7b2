"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: candidates (x, y, score), hypothesis triples, per-hypothesis inlier
counts, score sums, filter flags and circles, the result records and the mask
bytes.  The circle is also checked against a binary64 least-squares fit of the
point set it was fitted to, within 1e-3 px.
"""
import numpy as np
import pytest

from paper_2210_14771_gb300 import metrics, synth

from _helpers import both_params, coope_fit64, f32_bits, replay_last_fit_set, same_f32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def _gpu_batch(ca, frames, keys, lp, debug=0, masks=True):
    from paper_2210_14771_gb300 import api
    ca.set_debug(debug)
    if isinstance(frames, np.ndarray):
        t = torch.from_numpy(frames).cuda()
        res, m = ca.estimate(t, lp, keys=keys, masks=masks)
        torch.cuda.synchronize()
        return api.results_numpy(res), (m.cpu().numpy() if m is not None else None)
    ts = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in frames]
    res, m = ca.estimate(ts, lp, keys=keys, masks=masks)
    torch.cuda.synchronize()
    return api.results_numpy(res), ([x.cpu().numpy() for x in m] if m is not None else None)


def _compare_frame(orc, ca, b, frame, key, lp, op, gres, gmask, detail):
    ores, od = orc.estimate(frame, key, op, debug=detail)
    for k in ("cx", "cy", "r", "score"):
        assert same_f32(gres[k][b], ores[k]), (b, k, gres[b], ores)
    assert int(gres["valid"][b]) == ores["valid"] and int(gres["n_inliers"][b]) == ores["n_inliers"]
    if gmask is not None:
        H, W = frame.shape[:2]
        om = orc.mask(ores, H, W)
        assert np.array_equal(gmask, om), (b, int((gmask != om).sum()))
    if detail:
        gc = ca.dump_candidates(b)
        assert gc["M"] == od["M"], (b, gc["M"], od["M"])
        assert np.array_equal(gc["x"], od["cand_x"]) and np.array_equal(gc["y"], od["cand_y"])
        assert np.array_equal(gc["s"], od["cand_s"])
        gh = ca.dump_hypotheses(b)
        assert len(gh) == od["n_hyps"]
        tri = np.stack([gh["i0"], gh["i1"], gh["i2"]], 1)
        assert np.array_equal(tri, od["triple"])
        assert np.array_equal(gh["n_inl"], od["hyp_n_inl"])
        assert np.array_equal(gh["S"], od["hyp_score"])
        assert np.array_equal(gh["pass"], od["hyp_pass"])
        circ = np.stack([gh["cx"], gh["cy"], gh["r"]], 1)
        assert np.array_equal(f32_bits(circ), f32_bits(od["hyp_circle"]))
    return ores, od


def test_parity_640x480_every_intermediate(ca, orc):
    """8 frames 640x480 (N=16, K=4, 256 hypotheses): every intermediate value."""
    frames, gts, keys = synth.batch(0, 8, 480, 640, "centred")
    lp, op = both_params(orc, n_strips=16, cands_per_strip=4, n_hyps=256)
    gres, gmask = _gpu_batch(ca, frames, keys, lp, debug=2)
    for b in range(8):
        _compare_frame(orc, ca, b, frames[b], keys[b], lp, op, gres, gmask[b], True)
    assert gres["valid"].all()


@pytest.mark.parametrize("K,NH,sup", [(2, 300, 8), (6, 513, 3), (4, 1, 0)])
def test_parity_ragged_mixed_sizes(ca, orc, K, NH, sup):
    """Odd and tiny sizes in one call (vector and byte paths, ragged halves,
    ragged hypothesis tiles), frames with row padding (pitch > 3W)."""
    sizes = [(250, 333), (97, 131), (3, 8), (17, 9), (64, 64), (121, 200), (480, 640), (33, 47)]
    frames, keys = [], []
    for i, (H, W) in enumerate(sizes):
        f, _ = synth.frame(40 + K, i, H, W, "centred" if i % 2 else "full" if min(H, W) > 40 else "centred")
        frames.append(f)
        keys.append(1000 + i)
    lp, op = both_params(orc, n_strips=12, cands_per_strip=K, n_hyps=NH, sup_px=sup, seed=77)
    gres, gmask = _gpu_batch(ca, frames, keys, lp, debug=2)
    for b, f in enumerate(frames):
        _compare_frame(orc, ca, b, f, keys[b], lp, op, gres, gmask[b], True)
    # padded rows: the same frames inside wider buffers
    padded = []
    for f in frames:
        H, W, _ = f.shape
        buf = np.zeros((H, W + 5, 3), np.uint8)
        buf[:, :W] = f
        padded.append(torch.from_numpy(buf).cuda()[:, :W])
    from paper_2210_14771_gb300 import api
    ca.set_debug(0)
    res, _ = ca.estimate(padded, lp, keys=keys, masks=None)
    torch.cuda.synchronize()
    pres = api.results_numpy(res)
    assert np.array_equal(pres.view(np.uint8), gres.view(np.uint8))


def test_parity_exhaustive_mode(ca, orc):
    lp, op = both_params(orc, n_strips=6, cands_per_strip=2, hyp_mode=1)
    frames, _, keys = synth.batch(21, 6, 120, 160, "centred")
    gres, gmask = _gpu_batch(ca, frames, keys, lp, debug=2)
    for b in range(len(frames)):
        _compare_frame(orc, ca, b, frames[b], keys[b], lp, op, gres, gmask[b], True)


@pytest.fixture(scope="module")
def hd_batch():
    """The full 1080p workload: 64 frames, geometry mix, seed 1."""
    return synth.batch(1, 64, 1080, 1920, "mixed")


def test_parity_1080p_full_workload(ca, orc, hd_batch):
    """64 x 1920x1080, N=32, K=2, 1024 hypotheses, in the launch configuration
    the benchmark times: results and masks of every frame, candidates and
    hypotheses of a sample."""
    frames, gts, keys = hd_batch
    lp, op = both_params(orc, n_strips=32, cands_per_strip=2, n_hyps=1024)
    gres, gmask = _gpu_batch(ca, frames, keys, lp, debug=2)
    for b in range(64):
        _compare_frame(orc, ca, b, frames[b], keys[b], lp, op, gres, gmask[b], b % 9 == 0)
    # accuracy against the generator's ground truth (Sec. 2.3) on the regimes the
    # strip layout of Eq. 1 targets.  Clipped circles whose only border is one
    # corner just outside the circle are the failure mode the paper reports
    # (Sec. 4): a miss at 15 px but never a bad miss at 25 px.
    for kind, bar, miss in (("clipped", 5.0, 10.0), ("none", 0.0, 0.0)):
        nh = [metrics.normalised_hausdorff(gmask[b].astype(bool), metrics.gt_mask(gts[b], 1080, 1920))
              for b in range(64) if gts[b]["kind"] == kind]
        s = metrics.summarise(nh)
        assert s["bad_miss_pct"] == 0.0 and s["miss_pct"] <= miss and s["mean_nh"] <= bar, (kind, s)


def test_circle_within_1e3_px_of_fp64_fit(ca, orc, hd_batch):
    """The reported circle equals a binary64 least-squares fit of the point set
    it was fitted to within 1e-3 px (Sec. 2.2.5 least-squares refit)."""
    frames, _, keys = hd_batch
    lp, op = both_params(orc, n_strips=32, cands_per_strip=2, n_hyps=1024)
    gres, _ = _gpu_batch(ca, frames[:16], keys[:16], lp, debug=2, masks=False)
    checked = 0
    for b in range(16):
        if not gres["valid"][b]:
            continue
        gc = ca.dump_candidates(b)
        gh = ca.dump_hypotheses(b)
        H, W = frames[b].shape[:2]
        X = gc["x"].astype(np.int64) - W // 2
        Y = gc["y"].astype(np.int64) - H // 2
        ok = gh["pass"] == 1
        best = int(np.flatnonzero(ok & (gh["S"] == gh["S"][ok].max()))[0])
        last, c = replay_last_fit_set(orc, X, Y, (gh["i0"][best], gh["i1"][best], gh["i2"][best]),
                                      3, 3.0)
        assert last is not None
        assert same_f32(c, [gh["cx"][best], gh["cy"][best], gh["r"][best]])
        cx, cy, r = coope_fit64(X[last], Y[last])
        assert abs(cx + W // 2 - gres["cx"][b]) <= 1e-3
        assert abs(cy + H // 2 - gres["cy"][b]) <= 1e-3
        assert abs(r - gres["r"][b]) <= 1e-3
        checked += 1
    assert checked >= 8


def test_batch_position_invariance(ca, orc, hd_batch):
    """A frame's result is the same alone and anywhere in a batch."""
    frames, _, keys = hd_batch
    lp, _ = both_params(orc, n_strips=32, cands_per_strip=2, n_hyps=1024)
    full, _ = _gpu_batch(ca, frames[:20], keys[:20], lp, masks=False)
    for b in (0, 7, 19):
        alone, _ = _gpu_batch(ca, frames[b:b + 1], keys[b:b + 1], lp, masks=False)
        assert alone.view(np.uint8).tobytes() == full[b:b + 1].view(np.uint8).tobytes()
    perm = [19, 3, 11, 0]
    sub, _ = _gpu_batch(ca, [frames[i] for i in perm], [keys[i] for i in perm], lp, masks=False)
    for j, i in enumerate(perm):
        assert sub[j:j + 1].view(np.uint8).tobytes() == full[i:i + 1].view(np.uint8).tobytes()


def test_mask_call_and_host_path_agree(ca, orc, hd_batch):
    """ca_mask on the results, and ca_run_host on host buffers, reproduce the
    masks and results of ca_estimate."""
    frames, _, keys = hd_batch
    lp, _ = both_params(orc, n_strips=32, cands_per_strip=2, n_hyps=1024)
    t = torch.from_numpy(frames[:6]).cuda()
    ca.set_debug(0)
    res, masks = ca.estimate(t, lp, keys=keys[:6], masks=True)
    m2 = ca.mask(res, [(1080, 1920)] * 6)
    torch.cuda.synchronize()
    for i in range(6):
        assert torch.equal(masks[i], m2[i])
    hres, hmasks = ca.run_host(frames[:6], lp, keys=keys[:6])
    from paper_2210_14771_gb300 import _native as N, api
    assert hres.view(np.uint8).tobytes() == api.results_numpy(res).view(np.uint8).tobytes()
    assert np.array_equal(hmasks, masks.cpu().numpy())
    # zero-copy: kernels read the frames from and write the masks to
    # page-locked host memory; same results and masks
    import ctypes as C
    hf = torch.from_numpy(np.ascontiguousarray(frames[:6])).pin_memory()
    hm = torch.zeros((6, 1080, 1920), dtype=torch.uint8).pin_memory()
    hr = torch.zeros((6, 6), dtype=torch.float32).pin_memory()
    karr = (C.c_uint64 * 6)(*keys[:6])
    ca.run_host_zero_copy_ptr(hf.data_ptr(), 6, 1080, 1920, karr, lp, hr.data_ptr(), hm.data_ptr())
    assert hr.numpy().tobytes() == api.results_numpy(res).tobytes()
    assert np.array_equal(hm.numpy(), masks.cpu().numpy())
    pageable = np.ascontiguousarray(frames[:6])
    with pytest.raises(N.CaError):
        ca.run_host_zero_copy_ptr(pageable.ctypes.data, 6, 1080, 1920, karr, lp, hr.data_ptr(),
                                  None)


def test_full_rectangle_and_empty_inputs(ca, orc):
    frames, gts, keys = synth.batch(9, 3, 240, 320, "none")
    lp, op = both_params(orc, n_strips=16)
    gres, gmask = _gpu_batch(ca, frames, keys, lp)
    assert not gres["valid"].any() and all(m.all() for m in gmask)
    for b in range(3):
        _compare_frame(orc, ca, b, frames[b], keys[b], lp, op, gres, gmask[b], False)
    flat = np.full((2, 64, 96, 3), 40, np.uint8)   # no gradient: no candidates at all
    gres, gmask = _gpu_batch(ca, flat, [0, 1], lp)
    assert not gres["valid"].any() and gmask.all()
    res, m = ca.estimate(torch.empty((0, 64, 96, 3), dtype=torch.uint8, device="cuda"), lp)
    assert res.shape[0] == 0


def test_argument_errors(ca, orc):
    from paper_2210_14771_gb300 import api
    from paper_2210_14771_gb300._native import CaError
    t = torch.zeros((1, 64, 96, 3), dtype=torch.uint8, device="cuda")
    for kw in (dict(n_strips=0), dict(cands_per_strip=3), dict(n_strips=200, cands_per_strip=4),
               dict(n_hyps=0), dict(sobel_norm=3), dict(t_g=0.0), dict(t_ps=float("nan"))):
        with pytest.raises(CaError) as e:
            ca.estimate(t, api.params(**kw))
        assert e.value.status == 1, kw
    with pytest.raises(CaError):
        ca.estimate(torch.zeros((1, 2, 96, 3), dtype=torch.uint8, device="cuda"), api.params())
    with pytest.raises(CaError):
        ca.estimate(torch.zeros((1, 64, 5000, 3), dtype=torch.uint8, device="cuda"), api.params())
    with pytest.raises(CaError) as e:
        ca.estimate(t, api.params(scorer_mode=1))
    assert e.value.status == 5
    ca.sync()   # the context is healthy after rejected calls


@pytest.mark.parametrize("T", [1, 2, 4, 8])
def test_hypothesis_split_invariance(ca, orc, T):
    """Splitting each hypothesis over 1, 2, 4 or 8 threads changes nothing."""
    frames, _, keys = synth.batch(12, 6, 480, 640, "centred")
    lp, op = both_params(orc, n_strips=16, cands_per_strip=4, n_hyps=300, hyp_threads=T)
    gres, gmask = _gpu_batch(ca, frames, keys, lp, debug=2)
    for b in range(len(frames)):
        _compare_frame(orc, ca, b, frames[b], keys[b], lp, op, gres, gmask[b], True)


@pytest.mark.parametrize("norm", [0, 1, 2, 3])
def test_parity_score_normalisers(ca, orc, hd_batch, norm):
    """Every reading of the t_cs divisor (2N, N K, none, and the default
    circle normaliser, which counts each frame's strips within r + t_ri of
    the best circle's centre row): results and masks equal the oracle's on
    16 frames of the 1080p mix, in both launch modes."""
    frames, _, keys = hd_batch
    for mode in (1, 2):
        lp, op = both_params(orc, n_strips=32, cands_per_strip=2, n_hyps=256, score_norm=norm,
                             batch_mode=mode)
        gres, gmask = _gpu_batch(ca, frames[:16], keys[:16], lp)
        for b in range(16):
            _compare_frame(orc, ca, b, frames[b], keys[b], lp, op, gres, gmask[b], False)


@pytest.mark.parametrize("K", [2, 4])
def test_parity_zero_thresholds(ca, orc, K):
    """t_ps = 0 and t_px = 0 keep zero-score picks (flat runs, image edges):
    the pruned scans must still pick exactly the oracle's pixels."""
    frames = []
    rng = np.random.default_rng(3)
    for i, (H, W) in enumerate([(64, 96), (40, 72), (33, 50)]):
        f, _ = synth.frame(60, i, H, W, "centred")
        f = f.copy()
        f[: H // 3] = 20                            # flat rows: every score 0
        f[:, : W // 4] = rng.integers(0, 3, size=(H, W // 4, 3))
        frames.append(f)
    keys = [5, 6, 7]
    lp, op = both_params(orc, n_strips=8, cands_per_strip=K, n_hyps=200, t_ps=0.0, t_px=0.0,
                         t_cs=0.0)
    gres, gmask = _gpu_batch(ca, frames, keys, lp, debug=2)
    for b, f in enumerate(frames):
        _compare_frame(orc, ca, b, f, keys[b], lp, op, gres, gmask[b], True)
