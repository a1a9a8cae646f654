"""Full-size parity, every node: the library's output vectors on the full-size
graphs against the SHA-256 digests of the CPU oracle's vectors.

tests/golden/fullsize_sha256.txt is written by tests/golden/make_fullsize.py,
which runs only the oracle (exact h-degrees, Sec. 2; fixed-level counts, Alg. 1
with the level forced; estimates through Prop. 3.1 / Alg. 2 levels and Alg. 1).
Both sides hash the raw little-endian bytes of the same dtype and shape, so an
equal digest is an element-by-element equality of the whole vector.  When a
digest differs and the oracle's vector is cached locally (KH_ORACLE_CACHE, else tests/golden/_cache),
the first differing nodes are reported.
"""
import hashlib
import os

import numpy as np
import pytest

from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
DIGESTS = os.path.join(HERE, "golden", "fullsize_sha256.txt")
CACHE = os.environ.get("KH_ORACLE_CACHE") or os.path.join(HERE, "golden", "_cache")


def read_digests():
    rows = {}
    if not os.path.exists(DIGESTS):
        return rows
    with open(DIGESTS) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            case, field, dtype, shape, sha = line.split()[:5]
            rows.setdefault(case, {})[field] = (dtype, shape, sha)
    return rows


ROWS = read_digests()


def digest(a):
    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.astype(a.dtype.newbyteorder("<"), copy=False).tobytes()).hexdigest()


_graphs = {}


def graph(name):
    if name not in _graphs:
        _graphs.clear()  # one full-size graph in host memory at a time
        if name == "c2":
            _graphs[name] = gg.chung_lu(200_000, 20, 2.5, 5000, 1002)
        else:
            _graphs[name] = gg.rmat(22, 16, 0.57, 0.19, 0.19, 1003)
    return _graphs[name]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    c = K.kh_ctx_create(0)
    yield c
    c.close()


def check(case, field, got):
    dtype, shape, sha = ROWS[case][field]
    assert got.dtype.name == dtype and "x".join(map(str, got.shape)) == shape, (case, field)
    if digest(got) == sha:
        return
    msg = f"{case}/{field}: digest differs from the oracle's"
    cached = os.path.join(CACHE, f"{case}_{field}.npy")
    if os.path.exists(cached):
        want = np.load(cached)
        bad = np.nonzero((want != got).reshape(want.shape[0], -1).any(axis=1))[0]
        msg += f"; {bad.size} nodes differ, first {bad[:8].tolist()}"
    pytest.fail(msg)


CASES = sorted(ROWS)


@pytest.mark.parametrize("case", CASES)
def test_full_size_vector_equals_oracle(ctx, case):
    gname, kind, h = case.split("_")[0], case.split("_")[1], int(case.split("_h")[-1])
    rp, cl = graph(gname)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    try:
        K.kh_set_h(G, h)
        K.kh_set_sampling(G, seed=1, M=0, eps=0.5, delta=0.05)
        if kind == "hdeg":
            check(case, "deg", K.kh_hdegree_exact(G))
        elif kind == "counts":
            check(case, "cnt", K.kh_sampled_counts(G, 0, 10))
        elif kind == "est":
            est, level, bsize = K.kh_estimate(G)
            check(case, "est", est)
            check(case, "level", level)
            check(case, "bsize", bsize)
        else:
            pytest.fail(f"unknown case kind {kind}")
    finally:
        G.close()
