"""tl_count_hash_noalloc: the count + hash consumer for callers that cannot
allocate device memory (a consumer runs while the next listing kernel is in
flight; callers that own all device memory through their own pool cannot
let it call cudaMalloc there).

Checked against the allocating consumer tl_count_hash and against the CPU
oracle's hash of the same triples (host copies), through the C ABI, on two
calls in a row (the second with fewer triples, so stale partials left in the
shared scratch would show), and as the consumer of a real listing, whose
count and hash are the oracle's.  This file sorts last so that a run which
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch

    import paper_2203_04774_gb300 as tl
    torch.cuda.set_device(0)
    return tl, torch


def _alloc_consumer(tl, torch, dev_triples, n):
    ch = tl.CountHash(torch.cuda.current_stream().cuda_stream)
    try:
        assert tl.lib().tl_count_hash(dev_triples, n, 0, ch.user) == 0
        return int(ch.state.count), int(ch.state.hash)
    finally:
        ch.release()


def _noalloc_consumer(tl, torch, dev_triples, n, out):
    st = tl.CountHashNoallocState(out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    rc = tl.lib().tl_count_hash_noalloc(dev_triples, n, 0, ctypes.cast(ctypes.pointer(st),
                                                                        ctypes.c_void_p))
    assert rc == 0, tl.lib().tl_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.uint64)


def test_matches_allocating_consumer_two_calls_in_a_row(env):
    tl, torch = env
    g = torch.Generator(device="cuda").manual_seed(7)
    big = torch.randint(0, 1 << 31, (1_000_003, 3), device="cuda", dtype=torch.int64,
                        generator=g).to(torch.int32).contiguous()
    small = torch.randint(0, 1 << 31, (40_000, 3), device="cuda", dtype=torch.int64,
                          generator=g).to(torch.int32).contiguous()
    for buf in (big, small):  # two calls in a row, the second smaller
        n = buf.shape[0]
        want = _alloc_consumer(tl, torch, buf.data_ptr(), n)
        out = torch.zeros(2, dtype=torch.int64, device="cuda")
        got = _noalloc_consumer(tl, torch, buf.data_ptr(), n, out)
        assert (int(got[0]), int(got[1])) == want
        import oracle
        host = buf.cpu().numpy().view(np.uint32)
        assert int(got[1]) == oracle.hash_triples(host) and int(got[0]) == n


def test_rejects_more_than_the_maximum(env):
    tl, torch = env
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = tl.CountHashNoallocState(out.data_ptr(), None)
    rc = tl.lib().tl_count_hash_noalloc(None, tl.TL_NOALLOC_MAX_TRIPLES + 1, 0,
                                        ctypes.cast(ctypes.pointer(st), ctypes.c_void_p))
    assert rc != 0
    assert b"TL_NOALLOC_MAX_TRIPLES" in tl.lib().tl_last_error()
    assert out.cpu().tolist() == [0, 0]


def test_as_the_consumer_of_a_listing(env):
    tl, torch = env
    from paper_2203_04774_gb300 import synth
    n = 300
    e = synth.complete(n)
    gph = tl.Graph(n, torch.from_numpy(e).cuda())
    gph.order_apply(torch.from_numpy(synth.order_random(n, 5)).cuda())
    import oracle
    _, ref_cnt, ref_hash, _ = oracle.Graph(n, e).list(oracle.APP, store=False)
    for alg in (tl.TL_APP, tl.TL_APM):
        nt, cnt, h, _ = gph.list_count_hash(alg, tl.TL_MIN_CHUNK_BYTES)
        out = torch.zeros(2, dtype=torch.int64, device="cuda")
        st = tl.CountHashNoallocState(out.data_ptr(), None)
        fn = ctypes.cast(tl.lib().tl_count_hash_noalloc, ctypes.c_void_p).value
        nt2 = tl.tl_list_triangles(gph.h, alg, tl.TL_MIN_CHUNK_BYTES, fn,
                                   ctypes.cast(ctypes.pointer(st), ctypes.c_void_p))
        got = out.cpu().numpy().astype(np.uint64)
        assert nt2 == nt == cnt == int(got[0]) == n * (n - 1) * (n - 2) // 6
        assert int(got[1]) == h == ref_hash and cnt == ref_cnt
    gph.free()
