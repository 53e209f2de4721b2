"""cvetl_sort_u64_noalloc: the allocation-free radix sort, for callers that may not allocate
device memory (code inside a framework that owns the device memory pool, latency-critical
loops where cudaMalloc / cudaFree would stall the device).

Called through the C ABI and checked against the ordinary entry points: sorting the packed
(journey id, timestamp) keys of the small-day workload must give exactly the order that
cvetl_extract / cvetl_transform report as the per-point permutation. Two calls in a row
check that the shared scratch array is reset between calls. This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import cvgen

pytestmark = pytest.mark.gpu


def _noalloc_sort(P, keys_dev, n, bits, stream, begin=0):
    import torch

    out_k = torch.empty(n, dtype=torch.int64, device=keys_dev.device)
    out_p = torch.empty(n, dtype=torch.int32, device=keys_dev.device)
    st = P.lib.cvetl_sort_u64_noalloc(keys_dev.data_ptr(), out_k.data_ptr(), out_p.data_ptr(), n, begin,
                                      bits, ctypes.c_void_p(stream.cuda_stream))
    assert st == P.OK, P.lib.cvetl_last_error(None).decode()
    return out_k.cpu().numpy().view(np.uint64), out_p.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_the_pipeline_order_twice():
    import torch

    import paper_2305_07454_b300 as P

    cols = cvgen.generate("small_day", seed=1)
    n = cols["jid"].shape[0]
    assert n <= P.NOALLOC_MAX_PAIRS
    # reference: the per-point permutation of the ordinary entry points
    dev = {k: torch.from_numpy(cols[k]).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
    with P.Pipeline(materialize_points=1) as p:
        ref = p.run(dev)
    assert ref["counters"]["n_valid"] == n  # every row is kept, so positions line up
    want_perm = ref["points"]["perm"]
    # packed (journey id, timestamp) keys: ids < 2^31, timestamps within 2^27 ms of the first
    tmin = int(cols["ts"].min())
    assert cols["jid"].min() >= 0 and cols["jid"].max() < 2 ** 31 and int(cols["ts"].max()) - tmin < 2 ** 27
    keys = (cols["jid"].astype(np.uint64) << np.uint64(27)) | (cols["ts"] - tmin).astype(np.uint64)
    keys_dev = torch.from_numpy(keys.view(np.int64)).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        got_k, got_p = _noalloc_sort(P, keys_dev, n, 58, stream)
        assert np.array_equal(got_p, want_perm)
        assert np.array_equal(got_k, np.sort(keys))


@pytest.mark.parametrize("begin,end,n,dup_bits", [
    (8, 32, 200_003, 0),    # 3 passes (odd: the first pass writes the caller's outputs), begin > 0
    (0, 24, 100_000, 12),   # 3 passes from bit 0, many equal keys
    (0, 58, 150_001, 0),    # the last digit 2 bits wide; keys carry set bits above bit 58
    (5, 12, 70_000, 0),     # one pass narrower than a digit
    (0, 64, None, 0),       # n = CVETL_NOALLOC_MAX_PAIRS exactly, full 64-bit keys
])
def test_noalloc_sort_bit_ranges_against_a_stable_argsort(begin, end, n, dup_bits):
    """Order by bits [begin, end) only, ties in input order: numpy's stable argsort of the keys
    with every other bit cleared. keys_out holds the unmasked keys. Two calls in a row reuse the
    shared scratch array."""
    import torch

    import paper_2305_07454_b300 as P

    n = P.NOALLOC_MAX_PAIRS if n is None else n
    rng = np.random.default_rng(1000 + begin * 64 + end)
    keys = rng.integers(0, 2 ** 63, n, dtype=np.int64).view(np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, n, dtype=np.int64).view(np.uint64)
    if dup_bits:  # only dup_bits bits vary inside the range: long runs of equal keys
        keys &= ~np.uint64(((1 << (end - begin)) - 1) << begin) | np.uint64(((1 << dup_bits) - 1) << begin)
    mask = np.uint64(((1 << end) - 1) if end < 64 else (1 << 64) - 1) & ~np.uint64((1 << begin) - 1)
    want_p = np.argsort(keys & mask, kind="stable").astype(np.uint32)
    keys_dev = torch.from_numpy(keys.view(np.int64)).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        got_k, got_p = _noalloc_sort(P, keys_dev, n, end, stream, begin=begin)
        assert np.array_equal(got_p, want_p)
        assert np.array_equal(got_k, keys[want_p])


def test_noalloc_sort_refuses_a_capturing_stream():
    """The call synchronises its stream, which a capture forbids: it must return CVETL_ESTATE
    and leave the capture intact."""
    import torch

    import paper_2305_07454_b300 as P

    n = 1000
    k = torch.arange(n, 0, -1, dtype=torch.int64, device="cuda")
    o = torch.empty(n, dtype=torch.int64, device="cuda")
    pm = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(g, stream=s):
        codes.append(P.lib.cvetl_sort_u64_noalloc(k.data_ptr(), o.data_ptr(), pm.data_ptr(), n, 0, 64,
                                                  ctypes.c_void_p(s.cuda_stream)))
        o.add_(1)  # the capture still works after the refusal
    assert codes == [P.ESTATE] and b"capturing" in P.lib.cvetl_last_error(None)
    o.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert int(o.sum()) == n


def test_noalloc_sort_rejects_oversize_and_bad_arguments():
    import torch

    import paper_2305_07454_b300 as P

    stream = torch.cuda.current_stream()
    n = P.NOALLOC_MAX_PAIRS + 1
    k = torch.zeros(n, dtype=torch.int64, device="cuda")
    o = torch.empty(n, dtype=torch.int64, device="cuda")
    pm = torch.empty(n, dtype=torch.int32, device="cuda")
    st = P.lib.cvetl_sort_u64_noalloc(k.data_ptr(), o.data_ptr(), pm.data_ptr(), n, 0, 64,
                                      ctypes.c_void_p(stream.cuda_stream))
    assert st == P.EINVAL and b"CVETL_NOALLOC_MAX_PAIRS" in P.lib.cvetl_last_error(None)
    st = P.lib.cvetl_sort_u64_noalloc(k.data_ptr(), k.data_ptr(), pm.data_ptr(), 10, 0, 64,
                                      ctypes.c_void_p(stream.cuda_stream))
    assert st == P.EINVAL
    st = P.lib.cvetl_sort_u64_noalloc(k.data_ptr(), o.data_ptr(), pm.data_ptr(), 10, 0, 65,
                                      ctypes.c_void_p(stream.cuda_stream))
    assert st == P.EINVAL
