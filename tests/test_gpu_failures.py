"""Failure handling without a GPU fault: device allocations made to fail on
the host (kh_debug_fail_alloc) surface as KH_ENOMEM, and the same context and
graph then finish the decomposition with the oracle's result."""
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
    K.kh_debug_fail_alloc(c, 0)
    c.close()


@pytest.mark.parametrize("exact", [False, True])
def test_injected_allocation_failures(ctx, exact):
    rowptr, col = gg.chung_lu(3000, 10, 2.5, 100, 71)
    n = rowptr.size - 1
    if exact:
        want, _, _ = O.core_exact(rowptr, col, 2)
    else:
        want, _, _ = O.core_sampled(rowptr, col, O.ranks(n, 1), 2, 16)
    failures = 0
    for k in range(1, 48):
        K.kh_debug_fail_alloc(ctx, k)
        try:
            G = K.kh_graph_load_csr(ctx, rowptr, col)
        except K.KhError as e:
            assert e.code == K.KH_ENOMEM and "injected" in K.kh_last_error(ctx)
            failures += 1
            continue
        try:
            K.kh_set_h(G, 2)
            K.kh_set_sampling(G, seed=1, M=16)
            run = K.kh_core_exact if exact else K.kh_core_sampled
            try:
                core = run(G)
            except K.KhError as e:
                assert e.code == K.KH_ENOMEM
                failures += 1
                core = run(G)  # the injection fired once: the retry allocates the rest
            assert np.array_equal(core, want)
        finally:
            G.close()
            K.kh_debug_fail_alloc(ctx, 0)
    assert failures >= 20
