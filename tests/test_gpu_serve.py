"""The server on the GPU: requests that overlap on the device (several
slots, each with its own stream) return exactly what each request returns
alone."""
import numpy as np
import pytest

from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K
from paper_2112_06154_gb300 import serve as S

pytestmark = pytest.mark.gpu


def test_results_in_the_mix_equal_results_alone():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    reqs = [(gg.chung_lu(3000, 12, 2.3, 300, 1), 2), (gg.grid(40, 50, 0.01, 2), 3),
            (gg.chung_lu(8000, 8, 2.7, 200, 3), 4), (gg.barabasi_albert(2000, 4, 4), 3),
            (gg.erdos_renyi(2000, 8000, 5), 2), (gg.grid(60, 60, 0.01, 6), 4),
            (gg.chung_lu(5000, 20, 2.1, 400, 7), 3), (gg.rmat(11, 8, .57, .19, .19, 8), 2)]
    srv = S.KhServer(S.gpu_runner(0), slots=3, mem_budget=8 << 30)
    futs = [srv.submit(rp, cl, h) for (rp, cl), h in reqs for _ in range(2)]
    mixed = [f.result(timeout=300)["core"] for f in futs]
    srv.close()
    assert srv.peak_running >= 2  # the requests did overlap
    ctx = K.kh_ctx_create(0)
    for i, ((rp, cl), h) in enumerate(reqs):
        G = K.kh_graph_load_csr(ctx, rp, cl)
        K.kh_set_h(G, h)
        K.kh_set_sampling(G, seed=1, M=0)
        alone = K.kh_core_sampled(G)
        G.close()
        assert (mixed[2 * i] == alone).all() and (mixed[2 * i + 1] == alone).all()
    ctx.close()
