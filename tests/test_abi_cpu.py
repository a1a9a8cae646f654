"""Host-side checks of the C ABI library (no GPU needed): it loads and
exports every entry point that include/khcore.h declares."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2112_06154_gb300 import build as B
from paper_2112_06154_gb300 import khcore as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "khcore.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kh_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ["kh_ctx_create", "kh_graph_load_csr", "kh_set_h", "kh_set_sampling",
                 "kh_ranks", "kh_hdegree_exact", "kh_sampled_counts", "kh_estimate",
                 "kh_core_exact", "kh_core_sampled", "kh_sync", "kh_graph_free",
                 "kh_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    bound = {s[0] for s in K.SIGNATURES}
    assert set(declared_symbols()) <= bound
    for name in declared_symbols():
        assert hasattr(K, name), name


def test_null_arguments_are_rejected_without_a_gpu(lib):
    K.load()
    assert K.load().kh_ctx_create(None, 0, None) == K.KH_EINVAL
    assert K.load().kh_graph_free(None) == K.KH_EINVAL
    assert K.load().kh_set_h(None, 2) == K.KH_EINVAL
    assert K.load().kh_last_error(None) == b"null context"
    assert K.load().kh_peel_stats(None, None, None, None) == K.KH_EINVAL
    assert K.load().kh_prof_trace(None, 0, None, 0, None) == K.KH_EINVAL
    assert K.load().kh_prof_trace_bytes(None, 0, None, 0, None) == K.KH_EINVAL
    assert K.load().kh_debug_fail_alloc(None, 1) == K.KH_EINVAL


def test_binding_rejects_mismatched_csr_before_the_library():
    # the C ABI reads rowptr[n] column ids; the binding checks the arrays agree
    rowptr = np.array([0, 2, 3], np.int64)
    with pytest.raises(K.KhError):
        K.kh_graph_load_csr(None, rowptr, np.array([1], np.int32))
    with pytest.raises(K.KhError):
        K.kh_graph_load_batch(None, np.array([0, 5], np.int64), rowptr, np.array([1, 0, 0], np.int32))
    with pytest.raises(K.KhError):
        K.kh_graph_load_batch(None, np.array([0, 2], np.int64), rowptr, np.array([1, 0, 0], np.int32),
                              h_per_graph=np.array([2, 3], np.int32))
