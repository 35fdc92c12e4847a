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


def test_resident_state_pools_and_release(serve):
    """keep_resident: each finished request's features, matches, spectrum and MIM stay on
    the device until release; the resident spectrum and MIM equal a standalone context's
    forward DFT and maximum index map of the same image bit for bit; release returns the
    bytes, and a second round of the same sizes creates no new buffers in any pool."""
    import paper_2303_00319_gb300 as pkg
    srv = serve.Server(max_keypoints=400, max_batch_pairs=4, hbm_budget=8 << 30, lanes=2,
                       keep_resident=True)
    reqs = _requests(serve)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert set(srv.resident) == {r.rid for r in reqs} and srv.resident_bytes > 0
    ref = pkg.Context(pkg.default_params(max_keypoints=400), device=0)
    dev = torch.device("cuda:0")
    for r in reqs:
        st = srv.resident[r.rid]
        for img, f in ((r.a, st.fa), (r.b, st.fb)):
            x = torch.from_numpy(img).to(dev)
            spec = ref.fft2(x[None].contiguous())[0]
            assert torch.equal(f.debug["spectrum"], spec)
            g, = ref.extract([x], [ref.alloc_features(tuple(img.shape))])
            ref.sync()
            assert torch.equal(f.debug["mim"], g.debug["mim"])
        # the resident features are the ones the host result was copied from
        assert np.array_equal(st.fa.host()["xy"], r.result["kp_a"])
        assert np.array_equal(st.matches.host()["nn_desc"], r.result["nn_desc"])
    for r in reqs:
        srv.release(r.rid)
    assert srv.resident_bytes == 0 and not srv.resident
    before = srv.pool_stats()
    again = _requests(serve, 100)
    for r in again:
        srv.submit(r)
    srv.drain()
    for r in again:
        srv.release(r.rid)
    assert srv.pool_stats() == before
    for a, b in zip(reqs, again):
        assert np.array_equal(a.result["nn_desc"], b.result["nn_desc"])
    srv.close()


def test_resident_budget_applies_back_pressure(serve):
    """A resident budget that holds about two requests: the loop admits the rest only as
    the caller releases finished state, and refuses to spin when nothing can be admitted."""
    srv = serve.Server(max_keypoints=400, max_batch_pairs=8, hbm_budget=1 << 30, lanes=1,
                       keep_resident=True)
    reqs = _requests(serve)
    need = [srv._resident_need(r) for r in reqs]
    # room for the largest request alone, never for the first two together
    srv.resident_budget = max(need)
    assert need[0] + need[1] > srv.resident_budget
    for r in reqs:
        srv.submit(r)
    with pytest.raises(RuntimeError):
        srv.drain()                       # blocked: nothing released
    assert len(srv.resident) == 1
    done = set()
    while len(done) < len(reqs):
        for rid in list(srv.resident):
            srv.release(rid)
            done.add(rid)
        srv.step(block=True)
        for r in srv.finished:
            done.add(r.rid) if r.rid not in srv.resident else None
    assert all(r.result is not None and "error" not in r.result for r in reqs)
    srv.close()
