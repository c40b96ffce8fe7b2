"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, inverse functions, brute force on tiny inputs, published known-answer
vectors, exact rational arithmetic, library routines used as a step, and the
ground truth of synthetic frames.  None of them needs a GPU.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2210_14771_gb300 import metrics, synth

# ------------------------------------------------------------ Eq. 1 strips --


@pytest.mark.parametrize("H,N", [(480, 16), (1080, 32), (576, 64), (2160, 16), (7, 5)])
def test_strip_rows_floor_via_inverse_logistic(orc, H, N):
    """rows[i] = floor(h_i) with h_i from Eq. 1, checked through the inverse of
    the logistic map: i(h) = (N-1)/2 + (N/alpha) ln(h / (H - h))."""
    alpha = 8.0
    rows = orc.strip_rows(H, N, alpha)

    def i_of(h):
        if h <= 0:
            return -math.inf
        if h >= H:
            return math.inf
        return (N - 1) / 2 + (N / alpha) * math.log(h / (H - h))

    for i, r in enumerate(rows):
        r = int(r)
        if 1 < r < H - 2:   # unclamped rows
            assert i_of(r) <= i + 1e-9 and i < i_of(r + 1) + 1e-9, (i, r)
        else:
            assert r in (1, H - 2)


def test_strip_rows_symmetric_and_monotone(orc):
    """h_i + h_{N-1-i} = H, so floor(h_i) + floor(h_{N-1-i}) = H - 1 when h_i
    is not an integer; rows increase with i and favour the top and bottom."""
    H, N = 480, 16
    rows = orc.strip_rows(H, N, 8.0).astype(int)
    assert all(rows[i] + rows[N - 1 - i] == H - 1 for i in range(N))
    assert all(np.diff(rows) >= 0)
    gaps = np.diff(rows)
    assert gaps[0] < gaps[N // 2 - 1] and gaps[-1] < gaps[N // 2 - 1]


def test_strip_rows_alpha_zero_all_middle(orc):
    """alpha = 0 puts every strip at H/2 (logistic(0) = 1/2)."""
    assert set(orc.strip_rows(481, 9, 0.0).tolist()) == {240}
    assert set(orc.strip_rows(480, 8, 0.0).tolist()) == {240}


# ------------------------------------------------------------- luma, Sobel --


def test_luma_closed_forms(orc):
    for v in range(256):   # weights sum to 256: grey maps to itself
        assert orc.luma(v, v, v) == v
    assert orc.luma(255, 0, 0) == 77 and orc.luma(0, 255, 0) == 149
    assert orc.luma(0, 0, 255) == 29 and orc.luma(0, 0, 0) == 0


def _grey(img2d):
    return np.repeat(np.asarray(img2d, np.uint8)[:, :, None], 3, axis=2)


def test_sobel_step_and_ramp(orc):
    H, W = 9, 20
    a, b, s = 10, 110, 8           # vertical step: columns < s are a, >= s are b
    img = np.full((H, W), a)
    img[:, s:] = b
    _, gx, gy, _ = orc.strip_scores(_grey(img), 4, orc.params())
    expect = np.zeros(W, int)
    expect[s - 1] = expect[s] = 4 * (b - a)
    assert gx.tolist() == expect.tolist() and not gy.any()
    # horizontal step below the middle row: gy = 4 (b - a) on interior columns
    img = np.full((H, W), a)
    img[5:, :] = b
    _, gx, gy, _ = orc.strip_scores(_grey(img), 4, orc.params())
    assert not gx.any()
    assert gy[1:-1].tolist() == [4 * (b - a)] * (W - 2) and gy[0] == gy[-1] == 0
    # linear ramp Y = 3x: gx = 8 * 3 on interior columns
    img = np.tile(np.arange(W) * 3, (H, 1))
    _, gx, gy, _ = orc.strip_scores(_grey(img), 4, orc.params())
    assert gx[1:-1].tolist() == [24] * (W - 2) and not gy.any()


def test_preceding_max_brute_force(orc):
    rng = np.random.default_rng(5)
    for W in (8, 9, 31, 64):
        img = rng.integers(0, 256, size=(3, W))
        _, _, _, iota = orc.strip_scores(_grey(img), 1, orc.params())
        mid = img[1]
        hw = W // 2
        for x in range(W):
            if x < hw:
                ref = max(mid[:x]) if x > 0 else 0
            else:
                ref = max(mid[x + 1:]) if x < W - 1 else 0
            assert iota[x] == ref, (W, x)


# ---------------------------------------------------------- Eq. 2-3 scores --

def _tanh_via_exp(x):
    e = math.e ** (2 * x)
    return (e - 1) / (e + 1)


def test_lut_special_values(orc):
    g, t, i = orc.luts(orc.params())
    assert g[0] == 0 and all(np.diff(g.astype(int)) >= 0) and g[-1] == 32768
    assert g[80] == round(32768 * _tanh_via_exp(1.0))          # |g| = t_g = 20
    assert t[-1] == 32768 and t[0] == 0                         # theta = 0 / 180 deg
    assert all(np.diff(t.astype(int)) >= 0)
    # bin q covers the signed squared cosine u in [q/4096 - 1, (q+1)/4096 - 1):
    # q = 6144 starts at u = 0.5, i.e. theta = 45 degrees; q = 7168 at 30 degrees
    for q in (6144, 7168, 4096, 1000):
        def theta(u):
            c = math.copysign(math.sqrt(abs(u)), u)
            return math.degrees(math.acos(max(-1.0, min(1.0, c))))
        lo = 1 - _tanh_via_exp(theta(q / 4096 - 1) / 30)
        hi = 1 - _tanh_via_exp(theta((q + 1) / 4096 - 1) / 30)
        assert round(32768 * lo) <= t[q] <= round(32768 * hi), q
    assert i[0] == 32768 and i[25] == round(32768 * (1 - _tanh_via_exp(1.0)))
    assert all(np.diff(i.astype(int)) <= 0)


def test_quantised_score_close_to_eq2(orc):
    """The table-driven Q15 score stays within the quantisation bound of the
    double-precision score of Eq. 2-3 on every pixel of real strips."""
    p = orc.params()
    f, _ = synth.frame(3, 0, 480, 640, "centred")
    rows = orc.strip_rows(480, 16, 8.0)
    worst = 0.0
    for y in rows[::3]:
        s, gx, gy, iota = orc.strip_scores(f, int(y), p)
        for x in range(0, 640, 3):
            ref = orc.score_exact(gx[x], gy[x], 639 - 2 * x, 479 - 2 * int(y), iota[x], p)
            worst = max(worst, abs(s[x] / 32768.0 - ref))
    # |g| steps of 1/4 (<= 0.25/t_g); squared-cosine bins of 1/4096 span at most
    # 0.9 degrees (near 0 and 90 degrees), i.e. <= tanh(0.9/30) in s_theta; rounding
    assert worst <= 0.25 / 20 + math.tanh(0.9 / 30) + 1e-3, worst


def test_score_direction_reading(orc):
    """A dark-to-bright edge towards the image centre scores high; the same
    edge facing away from the centre scores near zero (Eq. 2, s_theta)."""
    H, W = 9, 64
    img = np.full((H, W), 5)
    img[:, 10:] = 150          # left border dark, content bright: faces the centre
    s, *_ = orc.strip_scores(_grey(img), 4, orc.params())
    assert s[9] > 16000
    img = np.full((H, W), 150)
    img[:, 10:] = 5            # bright outside, dark inside: gradient points away
    s, *_ = orc.strip_scores(_grey(img), 4, orc.params())
    assert s.max() < 400


# ---------------------------------------------------------- candidates --


def test_candidates_greedy_brute_force(orc):
    """Top-K/2 with suppression equals a greedy pass over all pixels of the
    half sorted by (score, outwardness), skipping suppressed ones."""
    rng = np.random.default_rng(11)
    for trial in range(30):
        H, W = 12, int(rng.integers(12, 41))
        K = int(rng.choice([2, 4, 6]))
        sup = int(rng.integers(0, 5))
        img = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
        p = orc.params(n_strips=2, cands_per_strip=K, sup_px=sup, t_px=1.0, t_ps=0.0)
        xs, ys, ss = orc.candidates(img, p)
        rows = orc.strip_rows(H, 2, p.alpha)
        ref = []
        for y in rows:
            s, *_ = orc.strip_scores(img, int(y), p)
            for half in (0, 1):
                xr = range(W // 2, W) if half else range(0, W // 2)
                order = sorted(xr, key=lambda x: (int(s[x]), x if half else -x), reverse=True)
                picks = []
                for x in order:
                    if len(picks) == K // 2:
                        break
                    if all(abs(x - q) > sup for q in picks):
                        picks.append(x)
                for x in picks:
                    if 1 <= x <= W - 2 and 1 <= y <= H - 2:
                        ref.append((x, int(y), int(s[x])))
        assert list(zip(xs.tolist(), ys.tolist(), ss.tolist())) == ref, trial


def test_candidates_on_true_circle(orc):
    """On clean synthetic frames the kept candidates lie on the true edge."""
    for i in range(4):
        f, gt = synth.frame(0, i, 480, 640, "centred")
        xs, ys, _ = orc.candidates(f, orc.params(n_strips=16, cands_per_strip=2))
        d = np.hypot(xs - gt["cx"], ys - gt["cy"]) - gt["r"]
        assert len(xs) >= 8 and np.mean(np.abs(d) <= 3.0) >= 0.9, d


def test_candidate_filter_t_ps_and_t_px(orc):
    """Points within t_px of the edge or scoring below t_ps are dropped."""
    H, W = 9, 40
    img = np.full((H, W), 5)
    img[:, 2:] = 150                    # edge at x = 1..2, closer than t_px = 3
    xs, *_ = orc.candidates(_grey(img), orc.params(n_strips=1, t_px=3.0))
    assert 1 not in xs.tolist() and 2 not in xs.tolist()
    flat = np.full((H, W, 3), 90, np.uint8)   # no gradient: every score is 0
    xs, *_ = orc.candidates(flat, orc.params(n_strips=3))
    assert len(xs) == 0


# --------------------------------------------------------------- Philox --


def _kat():
    path = __file__.replace("test_oracle_pins.py", "golden/philox4x32_10_kat.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            v = [int(t, 16) for t in line.split()]
            yield v[:4], v[4:6], v[6:]


def test_philox_known_answers(orc):
    for ctr, key, out in _kat():
        assert orc.philox(ctr, key).tolist() == out


def test_triples_distinct_and_uniform(orc):
    M, n = 5, 30000
    counts = {}
    for h in range(n):
        t = tuple(orc.triple(123, 456, h, M).tolist())
        assert len(set(t)) == 3 and all(0 <= v < M for v in t)
        counts[t] = counts.get(t, 0) + 1
    assert len(counts) == M * (M - 1) * (M - 2)
    e = n / len(counts)
    chi2 = sum((c - e) ** 2 / e for c in counts.values())
    assert chi2 < 110    # 59 dof: p ~ 1e-4 upper tail


def test_exhaustive_triples_lexicographic(orc):
    M = 7
    ref = list(itertools.combinations(range(M), 3))
    got = [tuple(orc.triple_exhaustive(h, M).tolist()) for h in range(len(ref))]
    assert got == ref


# --------------------------------------------------------- circle maths --


def test_circumcircle_closed_forms(orc):
    c = orc.circumcircle((0, 0), (2, 0), (0, 2))
    assert c.tolist() == [1.0, 1.0, np.float32(math.sqrt(2))]
    c = orc.circumcircle((5, 0), (-3, 4), (0, -5))
    assert c.tolist() == [0.0, 0.0, 5.0]
    c = orc.circumcircle((305, 200), (297, 204), (300, 195))
    assert c.tolist() == [300.0, 200.0, 5.0]
    assert orc.circumcircle((0, 0), (1, 1), (5, 5)) is None


def _nearest_f32(fr):
    """The binary32 value nearest to the rational fr, ties to even (from the
    exact distances of the candidates around a first estimate)."""
    f = np.float32(float(fr))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    best = None
    for c in cands:
        d = abs(Fraction(float(c)) - fr)
        even = int(np.array(c, np.float32).view(np.uint32)) & 1 == 0
        if best is None or d < best[0] or (d == best[0] and even):
            best = (d, c)
    return np.float32(best[1])


def test_rn_ratio_is_the_nearest_binary32(orc):
    """The circumcentre quotient: the binary32 value nearest to an integer
    ratio, against exact rational rounding -- random ratios over the operand
    range of 4096-pixel frames, both signs, and exact halfway cases (both
    tie directions)."""
    rng = np.random.default_rng(11)
    cases = [(1, 3), (-1, 3), (2, 3), (10, -7), (1 << 37, 3), (3, 1 << 37), (0, 5)]
    for _ in range(3000):
        den = int(rng.integers(1, 1 << int(rng.integers(1, 36))))
        num = int(rng.integers(-(1 << int(rng.integers(1, 37))), 1 << 36))
        cases.append((num, den if rng.random() < 0.5 else -den))
    for k in range(3):
        # (2 m + 1) / 2 with m of 24 bits: halfway between two binary32 values
        m = (1 << 23) + 12345 + k
        cases += [(2 * m + 1, 2), (2 * m + 3, 2), (-(2 * m + 1), 2)]
    for num, den in cases:
        got = orc.rn_ratio(num, den)
        want = _nearest_f32(Fraction(num, den))
        bits = lambda v: int(np.array(v, np.float32).view(np.uint32))
        assert bits(got) == bits(want) or (num == 0 and got == 0), (num, den, got, want)


def test_circumcircle_vs_exact_bisectors(orc):
    """Against the exact rational intersection of two perpendicular bisectors:
    the centre is its nearest binary32 point, bit for bit."""
    rng = np.random.default_rng(2)
    for _ in range(300):
        a, b, c = rng.integers(-1900, 1900, size=(3, 2)).tolist()
        out = orc.circumcircle(a, b, c)
        # |p-a|^2 = |p-b|^2 and |p-a|^2 = |p-c|^2 -> 2x2 linear system
        m11, m12 = 2 * (b[0] - a[0]), 2 * (b[1] - a[1])
        m21, m22 = 2 * (c[0] - a[0]), 2 * (c[1] - a[1])
        r1 = b[0] ** 2 + b[1] ** 2 - a[0] ** 2 - a[1] ** 2
        r2 = c[0] ** 2 + c[1] ** 2 - a[0] ** 2 - a[1] ** 2
        det = m11 * m22 - m12 * m21
        if det == 0:
            assert out is None
            continue
        px = Fraction(r1 * m22 - r2 * m12, det)
        py = Fraction(m11 * r2 - m21 * r1, det)
        r = math.sqrt(float((px - a[0]) ** 2 + (py - a[1]) ** 2))
        assert out[0] == _nearest_f32(px) and out[1] == _nearest_f32(py), (a, b, c, out, px, py)
        tol = 4e-7 * max(1.0, abs(float(px)), abs(float(py)))
        assert abs(out[2] - r) <= 4e-7 * max(1.0, r) + 2 * tol


def _lattice_points(R2):
    pts = []
    R = int(math.isqrt(R2))
    for x in range(-R, R + 1):
        y2 = R2 - x * x
        y = math.isqrt(y2)
        if y * y == y2:
            pts += [(x, y)] + ([(x, -y)] if y else [])
    return pts


@pytest.mark.parametrize("R2,off", [(25, (300, 200)), (625, (-700, 13)), (4225, (0, 0)),
                                    (4225, (901, -512))])
def test_ls_fit_exact_on_lattice_circles(orc, R2, off):
    pts = _lattice_points(R2)
    X = [p[0] + off[0] for p in pts]
    Y = [p[1] + off[1] for p in pts]
    c = orc.ls_fit(X, Y)
    # numerator and denominator are rounded to binary32 before the quotient,
    # so the exact rational answer is met to within two units in the last place
    for got, want in zip(c.tolist(), [off[0], off[1], math.sqrt(R2)]):
        assert abs(got - want) <= 2.5 * np.spacing(np.float32(max(abs(want), 1.0))), (got, want)
    # any three or more lattice points of an arc also give the exact circle
    arc = [p for p in pts if p[1] > 0][:5]
    c = orc.ls_fit([p[0] + off[0] for p in arc], [p[1] + off[1] for p in arc])
    assert abs(c[0] - off[0]) < 1e-3 and abs(c[1] - off[1]) < 1e-3


def test_ls_fit_vs_lstsq(orc):
    """Noisy points: the oracle equals the binary64 least-squares solution of
    the Coope linear system (numpy lstsq) to binary32 precision."""
    rng = np.random.default_rng(9)
    for trial in range(100):
        n = int(rng.integers(3, 200))
        cx, cy = rng.uniform(-400, 400, 2)
        r = rng.uniform(50, 1500)
        t = rng.uniform(0, rng.uniform(0.3, 2 * math.pi), n)
        X = np.rint(cx + r * np.cos(t) + rng.normal(0, 2, n)).astype(np.int64)
        Y = np.rint(cy + r * np.sin(t) + rng.normal(0, 2, n)).astype(np.int64)
        keep = (np.abs(X) <= 1920) & (np.abs(Y) <= 1080)
        X, Y = X[keep], Y[keep]
        if len(X) < 3:
            continue
        out = orc.ls_fit(X, Y)
        A = np.stack([X, Y, np.ones(len(X))], 1).astype(np.float64)
        b = -(X.astype(np.float64) ** 2 + Y.astype(np.float64) ** 2)
        sol, *_ = np.linalg.lstsq(A, b, rcond=None)
        ecx, ecy = -sol[0] / 2, -sol[1] / 2
        er = math.sqrt(ecx * ecx + ecy * ecy - sol[2])
        scale = max(1.0, abs(ecx), abs(ecy), er)
        cond = np.linalg.cond(A)
        tol = 1e-6 * scale + 1e-13 * cond * scale
        assert abs(out[0] - ecx) <= tol and abs(out[1] - ecy) <= tol, (trial, out, ecx, ecy)
        assert abs(out[2] - er) <= 2 * tol, (trial, out[2], er)


def test_ls_fit_degenerate(orc):
    assert orc.ls_fit([0, 1], [0, 1]) is None
    assert orc.ls_fit([0, 10, 20, 30], [5, 5, 5, 5]) is None     # collinear


def _nearest_f32(v: int) -> float:
    f = np.float32(float(v))
    best = None
    for c in (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))):
        d = abs(Fraction(float(c)) - v)
        even = (np.frombuffer(np.float32(c).tobytes(), np.uint32)[0] & 1) == 0
        key = (d, not even)
        if best is None or key < best[0]:
            best = (key, c)
    return float(best[1])


def test_i128_to_f32_correct_rounding(orc):
    rng = np.random.default_rng(4)
    vals = [0, 1, -1, 2 ** 24 + 1, 2 ** 24 + 3, -(2 ** 100) - 12345, (2 ** 64) + (2 ** 40) + 1]
    for _ in range(500):
        bits = int(rng.integers(1, 110))
        v = int(rng.integers(0, 2 ** 62)) << max(0, bits - 62)
        v += int(rng.integers(0, 2 ** 20))
        vals.append(v if rng.uniform() < 0.5 else -v)
    for v in vals:
        assert float(orc.i128_to_f32(v)) == _nearest_f32(v), v


# ------------------------------------------------------- whole pipeline --


def test_estimate_matches_ground_truth(orc):
    p = orc.params(n_strips=16, cands_per_strip=4, n_hyps=256)
    nh = []
    for i in range(8):
        f, gt = synth.frame(0, i, 480, 640, "centred")
        res, _ = orc.estimate(f, synth.frame_key(0, i), p)
        assert res["valid"] == 1
        m = orc.mask(res, 480, 640).astype(bool)
        nh.append(metrics.normalised_hausdorff(m, metrics.gt_mask(gt, 480, 640)))
    s = metrics.summarise(nh)
    assert s["mean_nh"] < 6.0 and s["miss_pct"] == 0.0, nh


def test_circle_strips_by_hand(orc):
    """The circle normaliser counts the strips whose row lies within r + t_ri
    of the centre row, boundary included, each strip once even when rows
    repeat."""
    rows = [10, 20, 30, 40, 50]
    assert orc.circle_strips(rows, 30.0, 10.0, 3.0) == 3          # |dy| <= 13: 20, 30, 40
    assert orc.circle_strips(rows, 30.0, 7.0, 3.0) == 3           # |dy| = 10 counts
    assert orc.circle_strips(rows, 30.0, 6.5, 3.0) == 1           # only the centre row
    assert orc.circle_strips(rows, 35.0, 4.5, 0.0) == 0           # between rows
    assert orc.circle_strips(rows, 35.5, 5.5, 0.0) == 2           # 30 and 40, 5.5 away
    assert orc.circle_strips([1, 1, 1, 2], 1.0, 0.5, 0.0) == 3    # repeated rows count each
    assert orc.circle_strips(rows, 0.0, 1000.0, 3.0) == 5


@pytest.mark.parametrize("K", [2, 4])
def test_circle_normaliser_score_by_hand(orc, K):
    """Candidates at full score on a circle crossing known strips: the best
    circle is that circle, its score is n_inliers / (K n) with n the strips
    within r + t_ri of its centre row, and t_cs just below / above that
    fraction accepts / rejects it; the 2N reading divides by 2N instead."""
    H, W, N = 480, 640, 16
    rows = orc.strip_rows(H, N)
    cx, cy, r = 320.0, 240.0, 100.0
    xs, ys = [], []
    for y in rows:
        dy = float(y) - cy
        if abs(dy) < r:
            h = (r * r - dy * dy) ** 0.5
            xs += [int(round(cx - h)), int(round(cx + h))]
            ys += [int(y), int(y)]
    xs, ys = np.array(xs), np.array(ys)
    ss = np.full(len(xs), 32768, np.uint16)
    p = orc.params(n_strips=N, cands_per_strip=K, n_hyps=256, score_norm=orc.NORM_CIRCLE,
                   t_cs=0.0, t_ri=3.0)
    res = orc.fit(xs, ys, ss, H, W, 5, p)
    assert res["valid"] == 1 and abs(res["cx"] - cx) < 1 and abs(res["r"] - r) < 1
    n = orc.circle_strips(rows, res["cy"], res["r"], 3.0)
    n_by_hand = int(sum(abs(float(y) - res["cy"]) <= res["r"] + 3.0 for y in rows))
    assert n == n_by_hand and 0 < n < N
    frac = res["n_inliers"] / (K * n)
    assert res["score"] == pytest.approx(frac, rel=1e-6)
    for t, want in ((frac * 0.999, 1), (frac * 1.001, 0)):
        p.t_cs = t
        assert orc.fit(xs, ys, ss, H, W, 5, p)["valid"] == want, t
    p.score_norm = orc.NORM_2N
    p.t_cs = 0.0
    assert orc.fit(xs, ys, ss, H, W, 5, p)["score"] == pytest.approx(
        res["n_inliers"] / (2 * N), rel=1e-6)


def test_mixed_geometry_1080p_accuracy(orc):
    """1080p geometry mix (N=32): clipped circles and border-free frames are
    recovered (no miss at 15 px, Sec. 2.3); every full circle located to
    within 3 px is accepted (the default circle normaliser) and is no miss."""
    p = orc.params(n_strips=32, cands_per_strip=2, n_hyps=1024)
    by = {}
    for i in range(20):
        kind = synth.geometry_of("mixed", i)
        f, gt = synth.frame(1, i, 1080, 1920, kind)
        res, _ = orc.estimate(f, synth.frame_key(1, i), p)
        m = orc.mask(res, 1080, 1920).astype(bool)
        nh = metrics.normalised_hausdorff(m, metrics.gt_mask(gt, 1080, 1920))
        by.setdefault(kind, []).append((nh, res, gt))
    assert metrics.summarise(v[0] for v in by["clipped"])["bad_miss_pct"] == 0.0
    assert all(v[0] == 0.0 for v in by["none"])
    located = 0
    for nh, res, gt in by["full"]:
        if abs(res["cx"] - gt["cx"]) < 3 and abs(res["cy"] - gt["cy"]) < 3 and \
                abs(res["r"] - gt["r"]) < 3:
            located += 1
            assert res["valid"] and nh < 15, (res, gt, nh)
    assert located >= len(by["full"]) - 1


def test_full_rectangle_frames_invalid(orc):
    for i in range(3):
        f, gt = synth.frame(7, i, 480, 640, "none")
        assert not gt["valid"]
        res, _ = orc.estimate(f, i, orc.params(n_strips=16, n_hyps=256))
        assert res["valid"] == 0
        assert orc.mask(res, 480, 640).all()


def test_random_equals_exhaustive_on_tiny_inputs(orc):
    """With 4096 random draws over at most C(12,3) = 220 triples every triple is
    drawn (P(miss) < 1e-6); the best score and validity then equal those of the
    exhaustive search, and so does the circle when the best score is unique."""
    checked = 0
    for i in range(12):
        f, _ = synth.frame(21, i, 120, 160, "centred")
        pe = orc.params(n_strips=6, cands_per_strip=2, hyp_mode=orc.HYP_EXHAUSTIVE)
        pr = orc.params(n_strips=6, cands_per_strip=2, n_hyps=4096)
        re_, de = orc.estimate(f, i, pe, debug=True)
        rr, dr = orc.estimate(f, i, pr, debug=True)
        if de["M"] < 3:
            continue
        checked += 1
        se = de["hyp_score"][de["hyp_pass"] == 1]
        sr = dr["hyp_score"][dr["hyp_pass"] == 1]
        assert (se.max() if len(se) else -1) == (sr.max() if len(sr) else -1)
        assert re_["valid"] == rr["valid"]
        if len(se) and (se == se.max()).sum() == 1:
            assert (re_["cx"], re_["cy"], re_["r"]) == (rr["cx"], rr["cy"], rr["r"])
        # every random hypothesis equals the exhaustive one of the same set
        index = {t: h for h, t in enumerate(itertools.combinations(range(de["M"]), 3))}
        for h in range(0, 4096, 37):
            he = index[tuple(sorted(dr["triple"][h].tolist()))]
            assert dr["hyp_score"][h] == de["hyp_score"][he]
            assert dr["hyp_circle"][h].tolist() == de["hyp_circle"][he].tolist()
    assert checked >= 8


def test_horizontal_flip_equivariance(orc):
    p = orc.params(n_strips=16, cands_per_strip=4, hyp_mode=orc.HYP_EXHAUSTIVE)
    for i in range(3):
        f, _ = synth.frame(5, i, 96, 128, "centred")
        W = f.shape[1]
        r1, d1 = orc.estimate(f, 0, p, debug=True)
        r2, d2 = orc.estimate(f[:, ::-1], 0, p, debug=True)
        a = sorted(zip(d1["cand_x"].tolist(), d1["cand_y"].tolist(), d1["cand_s"].tolist()))
        b = sorted(zip((W - 1 - d2["cand_x"]).tolist(), d2["cand_y"].tolist(), d2["cand_s"].tolist()))
        assert a == b
        s1 = d1["hyp_score"][d1["hyp_pass"] == 1]
        s2 = d2["hyp_score"][d2["hyp_pass"] == 1]
        assert sorted(s1.tolist()) == sorted(s2.tolist())
        assert r1["valid"] == r2["valid"]
        if r1["valid"]:
            assert abs(r1["cx"] - (W - 1 - r2["cx"])) < 1e-3 and abs(r1["r"] - r2["r"]) < 1e-3


def test_vertical_flip_equivariance(orc):
    p = orc.params(n_strips=16, cands_per_strip=2)
    for i in range(3):
        f, _ = synth.frame(6, i, 480, 640, "centred")
        H = f.shape[0]
        _, d1 = orc.estimate(f, 0, p, debug=True)
        _, d2 = orc.estimate(f[::-1], 0, p, debug=True)
        a = sorted(zip(d1["cand_x"].tolist(), d1["cand_y"].tolist(), d1["cand_s"].tolist()))
        b = sorted(zip(d2["cand_x"].tolist(), (H - 1 - d2["cand_y"]).tolist(), d2["cand_s"].tolist()))
        assert a == b


def test_translation_equivariance(orc):
    """Shifting a full-circle scene by whole pixels shifts the circle."""
    f, gt = synth.frame(8, 0, 480, 640, "full")
    p = orc.params(n_strips=16, cands_per_strip=4, n_hyps=512)
    r0, _ = orc.estimate(f, 0, p)
    tx, ty = 17, -11
    g = np.empty_like(f)
    g[:] = f[2:5, 2:5].mean(axis=(0, 1)).astype(np.uint8)
    g[max(ty, 0):480 + min(ty, 0), max(tx, 0):640 + min(tx, 0)] = \
        f[max(-ty, 0):480 - max(ty, 0), max(-tx, 0):640 - max(tx, 0)]
    r1, _ = orc.estimate(g, 0, p)
    assert r0["valid"] and r1["valid"]
    assert abs(r1["cx"] - r0["cx"] - tx) < 1.5 and abs(r1["cy"] - r0["cy"] - ty) < 1.5
    assert abs(r1["r"] - r0["r"]) < 1.5


def test_mask_is_disc_intersect_rectangle(orc):
    res = dict(cx=301.25, cy=-40.5, r=350.75, score=1.0, valid=1, n_inliers=10)
    m = orc.mask(res, 240, 640).astype(bool)
    ref = metrics.content_mask(240, 640, (res["cx"], res["cy"], res["r"]))
    diff = np.argwhere(m != ref)
    for y, x in diff:   # only where binary32 and binary64 round differently
        assert abs(math.hypot(x - res["cx"], y - res["cy"]) - res["r"]) < 1e-3
    assert len(diff) <= 4


# --------------------------------------------------------- Hausdorff, Eq. 4-6 --


def test_hausdorff_closed_forms():
    H, W = 1080, 1920
    a = metrics.content_mask(H, W, (960, 540, 300))
    b = metrics.content_mask(H, W, (960, 540, 310))
    assert abs(metrics.hausdorff(a, b) - 10) <= 1.5
    assert metrics.hausdorff(a, a) == 0.0
    assert metrics.normalised_hausdorff(a, b) == metrics.hausdorff(a, b)   # d_I = d
    full = metrics.content_mask(H, W, None)
    # circle inside the frame vs the whole rectangle: farthest frame corner
    h = metrics.hausdorff(a, full)
    assert abs(h - (math.hypot(960, 540) - 300)) <= 1.5
    small = np.zeros((540, 960), bool)
    small[:] = metrics.content_mask(540, 960, (480, 270, 150))
    half = metrics.content_mask(540, 960, (480, 270, 155))
    assert abs(metrics.normalised_hausdorff(small, half) - 2 * 5) <= 3.0


def test_synth_deterministic_and_gt():
    f1, g1 = synth.frame(1, 3, 120, 160, "clipped")
    f2, g2 = synth.frame(1, 3, 120, 160, "clipped")
    assert (f1 == f2).all() and g1 == g2
    f3, _ = synth.frame(1, 4, 120, 160, "clipped")
    assert (f1 != f3).any()
    assert synth.gt_valid(80, 60, 50, 120, 160)
    assert not synth.gt_valid(80, 60, 200, 120, 160)
    kinds = [synth.geometry_of("mixed", i) for i in range(10)]
    assert kinds.count("clipped") == 4 and kinds.count("none") == 2
