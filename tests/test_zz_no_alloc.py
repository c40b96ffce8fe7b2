"""ca_estimate_static, the entry point for callers that cannot allocate.

Some applications own all device memory and forbid a library from calling
cudaMalloc (a fixed memory budget reserved before a procedure starts, or a host
framework's pool), and some frame loops cannot absorb the device-wide stalls
of cudaMalloc / cudaFree.  For them ca_estimate_static runs the same kernels
with its scratch in one fixed array of library device memory.  These tests
call it through the C ABI and require its results and masks to equal those of
ca_estimate_uniform bit for bit, on two calls in a row with different batches
(the second call reuses the array the first one filled).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2210_14771_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_14771_gb300.build import build
    build()
    from paper_2210_14771_gb300 import _native
    return _native


def _static_call(native, frames, keys, p, res, masks):
    B, H, W, _ = frames.shape
    karr = (C.c_uint64 * B)(*keys)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return native.lib().ca_estimate_static(
        C.c_void_p(frames.data_ptr()), B, H, W, karr, C.byref(p), C.c_void_p(res.data_ptr()),
        C.c_void_p(masks.data_ptr()) if masks is not None else None, stream)


def test_static_entry_matches_handle_entry_on_two_calls(lib):
    from paper_2210_14771_gb300 import api
    ca = api.ContentArea(0)
    cases = [
        (synth.batch(3, 16, 480, 640, "centred"), dict(n_strips=16, cands_per_strip=4, n_hyps=256)),
        (synth.batch(4, 8, 1080, 1920, "mixed"), dict(n_strips=32, cands_per_strip=2, n_hyps=1024)),
    ]
    # inputs, outputs and the reference results are all allocated up front
    prepared = []
    for (frames, _, keys), kw in cases:
        d = torch.from_numpy(frames).cuda()
        p = api.params(**kw)
        ref_res, ref_masks = ca.estimate(d, p, keys=keys, masks=True)
        res = torch.full_like(ref_res, -1.0)
        masks = torch.full_like(ref_masks, 7)
        prepared.append((d, keys, p, ref_res, ref_masks, res, masks))
    # one warm-up call per case: the first use of the library's kernels and of
    # its scratch array loads their code and data, which is not an allocation
    # of the call
    for d, keys, p, _, _, res, masks in prepared:
        assert _static_call(lib, d, keys, p, res, masks) == 0
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    for d, keys, p, _, _, res, masks in prepared:
        res.fill_(-1.0)
        masks.fill_(7)
    torch.cuda.synchronize()
    for d, keys, p, _, _, res, masks in prepared:       # two calls in a row
        assert _static_call(lib, d, keys, p, res, masks) == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before      # nothing taken from torch's pool
    # nor from the device by any other route (cudaMalloc takes whole 2 MiB pages)
    free_after, _ = torch.cuda.mem_get_info()
    assert free_before - free_after < (2 << 20), (free_before, free_after)
    for d, keys, p, ref_res, ref_masks, res, masks in prepared:
        assert res.cpu().numpy().tobytes() == ref_res.cpu().numpy().tobytes()
        assert torch.equal(masks, ref_masks)
    # and once more on the first batch after the second one overwrote the array
    d, keys, p, ref_res, ref_masks, res, masks = prepared[0]
    res.fill_(-1.0)
    masks.fill_(7)
    assert _static_call(lib, d, keys, p, res, None) == 0
    torch.cuda.synchronize()
    assert res.cpu().numpy().tobytes() == ref_res.cpu().numpy().tobytes()
    assert (masks == 7).all()                            # no masks requested, none written
    ca.close()


def test_static_entry_rejects_requests_beyond_its_scratch(lib):
    from paper_2210_14771_gb300 import api
    frames = torch.zeros((257, 16, 16, 3), dtype=torch.uint8, device="cuda")
    res = torch.zeros((257, 6), dtype=torch.float32, device="cuda")
    assert _static_call(lib, frames, list(range(257)), api.params(), res, None) == 1
    few = frames[:4]
    assert _static_call(lib, few, [0, 1, 2, 3], api.params(n_hyps=4097), res[:4], None) == 1
    assert _static_call(lib, few, [0, 1, 2, 3],
                        api.params(n_strips=16, cands_per_strip=4, hyp_mode=1), res[:4], None) == 1
    torch.cuda.synchronize()
    assert (res == 0).all()                              # rejected before any work was queued


def test_static_entry_refuses_stream_capture(lib):
    """A call made while its stream is being captured into a CUDA graph is
    refused (CA_ERR_UNSUPPORTED) before it queues anything: its host-stack
    copies could not be replayed."""
    from paper_2210_14771_gb300 import api
    frames = torch.zeros((2, 64, 96, 3), dtype=torch.uint8, device="cuda")
    res = torch.zeros((2, 6), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        g.capture_begin()
        rc = lib.lib().ca_estimate_static(
            C.c_void_p(frames.data_ptr()), 2, 64, 96, None, C.byref(api.params()),
            C.c_void_p(res.data_ptr()), None, C.c_void_p(side.cuda_stream))
        g.capture_end()
    torch.cuda.synchronize()
    assert rc == 5
    assert (res == 0).all()
