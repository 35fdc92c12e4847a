"""Continuous-batching loop: a request's results are the same alone and inside a mixed
batch of other requests of different sizes (bit for bit: the per-image kernels are
deterministic and independent of what shares a launch), and the loop reports latencies."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2303_00319_gb300 import serve as s
    return s


def _requests(serve, rid0=0):
    sizes = [(256, 256), (384, 512), (256, 256), (512, 384), (320, 320)]
    reqs = []
    for i, (h, w) in enumerate(sizes):
        pr = synth.make_pair(h, w, synth.pair_seed(4, i), angle_deg=None)
        reqs.append(serve.PairRequest(rid0 + i, pr.a, pr.b))
    return reqs


def test_alone_equals_mixed(serve):
    alone = serve.Server(max_keypoints=400, max_batch_pairs=1, hbm_budget=8 << 30, lanes=1)
    mixed = serve.Server(max_keypoints=400, max_batch_pairs=8, hbm_budget=8 << 30, lanes=2)
    ra, rm = _requests(serve), _requests(serve)
    for r in ra:
        alone.submit(r)
        alone.drain()
    for r in rm:
        mixed.submit(r)
    mixed.drain()
    for a, m in zip(ra, rm):
        assert a.result is not None and m.result is not None
        assert len(a.result["kp_a"]) > 0
        for k in ("nn_desc", "d1", "d2", "kp_a", "kp_b", "desc_kp_a"):
            assert np.array_equal(a.result[k], m.result[k]), (a.rid, k)
    alone.close()
    mixed.close()


def test_open_loop_reports_latency(serve):
    srv = serve.Server(max_keypoints=400, max_batch_pairs=4, hbm_budget=8 << 30, lanes=2)
    stats = serve.run_open_loop(srv, _requests(serve) + _requests(serve, 5), rate=200.0, seed=1)
    assert stats["requests"] == 10
    assert 0 < stats["latency_ms_p50"] <= stats["latency_ms_p99"] <= stats["latency_ms_max"]
    assert all(r.done >= r.launched >= r.admitted >= r.arrival for r in srv.finished)
    srv.close()
