"""The allocation-free entry point kh_hdegree_exact_noalloc.

Callers that cannot allocate device memory (a serving process whose device
memory is a pool fixed at start-up, latency-bound code that must not wait on
the allocator) use this variant; it keeps its scratch in a fixed device array
inside the library.  This file is named so that pytest collects it last: a
failure here leaves every other test already run.  It must pass alone in a
fresh process and after the others.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    c = K.kh_ctx_create(0)
    yield c
    c.close()


def reference_degrees(ctx, rp, cl, h):
    """The existing entry point, kh_hdegree_exact, on the same graph."""
    G = K.kh_graph_load_csr(ctx, rp, cl)
    K.kh_set_h(G, h)
    deg = K.kh_hdegree_exact(G)
    G.close()
    return deg


def test_noalloc_matches_hdegree_exact_on_consecutive_calls(ctx):
    import torch
    cases = [(gg.erdos_renyi(2000, 8000, 1001), 2),
             (gg.chung_lu(20000, 20, 2.5, 500, 1102), 3),
             (gg.erdos_renyi(2000, 8000, 1001), 3)]
    for (rp, cl), h in cases:
        want = reference_degrees(ctx, rp, cl, h)
        # the oracle (Sec. 2's definition) agrees with both entry points
        assert (want == O.hdegree_exact(rp, cl, h)).all()
        drp = torch.from_numpy(rp).cuda()
        dcl = torch.from_numpy(cl).cuda()
        for _ in range(2):  # two calls in a row share the scratch array
            out = torch.full((rp.size - 1,), -1, dtype=torch.int32, device="cuda")
            assert K.kh_hdegree_exact_noalloc(drp, dcl, h, out) == K.KH_OK
            torch.cuda.synchronize()
            assert (out.cpu().numpy() == want).all()


def test_noalloc_on_a_caller_stream(ctx):
    import torch
    rp, cl = gg.chung_lu(5000, 12, 2.4, 300, 77)
    want = O.hdegree_exact(rp, cl, 2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        drp = torch.from_numpy(rp).cuda()
        dcl = torch.from_numpy(cl).cuda()
        out = torch.full((rp.size - 1,), -1, dtype=torch.int32, device="cuda")
    s.synchronize()
    assert K.kh_hdegree_exact_noalloc(drp, dcl, 2, out, stream=s) == K.KH_OK
    s.synchronize()
    assert (out.cpu().numpy() == want).all()


def test_noalloc_rejects_sizes_beyond_its_limit(ctx):
    import torch
    lib = K.load()
    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    # n above the stated maximum is refused before any pointer is touched
    assert lib.kh_hdegree_exact_noalloc(819201, dummy.data_ptr(), dummy.data_ptr(), 2,
                                        dummy.data_ptr(), None) == K.KH_EINVAL
    assert lib.kh_hdegree_exact_noalloc(10, dummy.data_ptr(), dummy.data_ptr(), 0,
                                        dummy.data_ptr(), None) == K.KH_EINVAL
    assert lib.kh_hdegree_exact_noalloc(10, dummy.data_ptr(), dummy.data_ptr(), 17,
                                        dummy.data_ptr(), None) == K.KH_EINVAL
    # n = 0 is a no-op
    assert lib.kh_hdegree_exact_noalloc(0, None, None, 2, None, None) == K.KH_OK


def test_noalloc_binding_checks_its_tensors(ctx):
    import torch
    rp, cl = gg.erdos_renyi(200, 600, 3)
    drp = torch.from_numpy(rp).cuda()
    dcl = torch.from_numpy(cl).cuda()
    deg = torch.zeros(200, dtype=torch.int32, device="cuda")
    bad_cases = [
        (drp.to(torch.int32), dcl, deg),                 # rowptr not int64
        (drp, dcl.to(torch.int64), deg),                 # col not int32
        (drp, dcl, deg.to(torch.int64)),                 # deg not int32
        (drp, dcl, torch.zeros(199, dtype=torch.int32, device="cuda")),  # short deg
        (drp.cpu(), dcl, deg),                           # host tensor
        (drp, dcl[::2], deg),                            # not contiguous
        (drp, dcl[:-1], deg),                            # col shorter than rowptr[-1]
    ]
    for args in bad_cases:
        with pytest.raises(K.KhError):
            K.kh_hdegree_exact_noalloc(args[0], args[1], 2, args[2])
    assert K.kh_hdegree_exact_noalloc(drp, dcl, 2, deg) == K.KH_OK
    torch.cuda.synchronize()
    assert (deg.cpu().numpy() == O.hdegree_exact(rp, cl, 2)).all()
