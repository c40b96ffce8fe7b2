"""The serving admission allocator (host logic, no GPU): first-fit offsets
inside the budget, no overlap, refusal when nothing fits, and adjacent free
blocks merged back into one."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2210_14771_gb300.build import build
    build()
    from paper_2210_14771_gb300 import _native
    return _native


def _pool(L, size, align=256):
    h = C.c_void_p()
    assert L.lib().ca_pool_create(size, align, C.byref(h)) == 0
    return h


def _alloc(L, h, n):
    off = C.c_size_t(0)
    st = L.lib().ca_pool_alloc(h, n, C.byref(off))
    return st, off.value


def test_random_sequence_never_overlaps_and_merges_back(L):
    size = 1 << 20
    h = _pool(L, size)
    rng = np.random.default_rng(0)
    live = {}
    for _ in range(4000):
        if live and (rng.uniform() < 0.45 or len(live) > 60):
            off = int(rng.choice(list(live)))
            assert L.lib().ca_pool_free(h, off) == 0
            del live[off]
        else:
            n = int(rng.integers(1, 40000))
            st, off = _alloc(L, h, n)
            if st == 0:
                need = (n + 255) // 256 * 256
                assert off % 256 == 0 and off + need <= size
                for o, m in live.items():
                    assert off + need <= o or o + m <= off   # disjoint
                live[off] = need
            else:
                assert st == L.CA_ERR_ADMISSION
                largest = C.c_size_t(0)
                L.lib().ca_pool_stats(h, None, C.byref(largest))
                assert largest.value < (n + 255) // 256 * 256   # refused only if nothing fits
    used = C.c_size_t(0)
    L.lib().ca_pool_stats(h, C.byref(used), None)
    assert used.value == sum(live.values())
    for off in list(live):
        assert L.lib().ca_pool_free(h, off) == 0
    largest = C.c_size_t(0)
    L.lib().ca_pool_stats(h, C.byref(used), C.byref(largest))
    assert used.value == 0 and largest.value == size   # one block again
    assert L.lib().ca_pool_free(h, 0) == L.CA_ERR_INVALID_ARG   # not allocated
    L.lib().ca_pool_destroy(h)


def test_budget_refuses_the_frame_that_does_not_fit(L):
    frame_4k = 3840 * 2160 * 3 + 3840 * 2160
    h = _pool(L, 4 << 30)
    n = 0
    while _alloc(L, h, frame_4k)[0] == 0:
        n += 1
    assert n == (4 << 30) // ((frame_4k + 255) // 256 * 256)
    L.lib().ca_pool_destroy(h)


def test_latency_summary_splits_into_feed_queue_and_gpu():
    """serve.summarise on hand-made records: percentiles of arrival-to-result
    latency and of its three parts, which add up per frame."""
    from paper_2210_14771_gb300 import serve
    recs = []
    for i in range(100):
        a = 10.0 + i * 0.01
        s_ = a + 0.001 * (i % 3)               # feeding delay 0-2 ms
        l_ = s_ + 0.0005                       # 0.5 ms queued
        d_ = l_ + 0.002 + (0.050 if i == 99 else 0.0)   # 2 ms of work, one 50 ms stall
        recs.append(dict(t_arrival=a, t_submit=s_, t_launch=l_, t_done=d_, latency=d_ - a))
    st = serve.summarise(recs, 2.0)
    assert st["frames"] == 100 and st["frames_per_s"] == 50.0
    assert st["over_10ms"] == 1 and abs(st["max_ms"] - 52.5) < 1e-6
    assert abs(st["p50_ms"] - 3.5) < 1e-6
    assert abs(st["p99_queue_ms"] - 0.5) < 1e-6
    assert abs(st["p99_feed_ms"] - 2.0) < 1e-6
    for r in recs:
        parts = (r["t_submit"] - r["t_arrival"]) + (r["t_launch"] - r["t_submit"]) + \
            (r["t_done"] - r["t_launch"])
        assert abs(parts - r["latency"]) < 1e-12
