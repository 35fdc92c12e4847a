"""Failure paths of the C ABI on a GPU, made on the host or by a bounded device wait that is
told to give up (no fault, no trap, no hang).

* RIFT2_E_NOMEM: a context whose HBM budget is below one image's workspace refuses the
  extraction before enqueuing anything; a budget that holds one image but not two splits
  the launch group and still succeeds.
* RIFT2_E_CAPACITY: feature or match buffers below the context's worst case are refused
  before anything is enqueued (the outputs keep their sentinel values), and
  rift2_required_capacity reports the capacities the call needed.
* RIFT2_E_TIMEOUT: with the descriptor kernel's first-wait limit at 0 every staged copy
  "times out"; the kernel drains its copies, latches the status word and returns, so
  rift2_sync reports RIFT2_E_TIMEOUT, and the next call on the same context (normal limit)
  succeeds and reproduces a fresh context's features bit for bit.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2303_00319_gb300 as p
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return p


@pytest.fixture(scope="module")
def images():
    dev = torch.device("cuda:0")
    pr = synth.make_pair(256, 320, seed=41, angle_deg=25.0, n_blobs=30, n_segments=15)
    return [torch.from_numpy(pr.a).to(dev), torch.from_numpy(pr.b).to(dev)]


def _sentinel(f):
    f.counts.fill_(-7)
    f.kp_xy.fill_(-7)
    return f


def test_nomem_when_budget_below_one_image(pkg, images):
    ctx = pkg.Context(pkg.default_params(max_keypoints=300), device=0, hbm_budget=1 << 20)
    f = _sentinel(ctx.alloc_features())
    with pytest.raises(pkg.Rift2Error) as e:
        ctx.extract([images[0]], [f])
    assert e.value.code == pkg.E_NOMEM
    torch.cuda.synchronize()
    assert f.counts.cpu().tolist() == [-7, -7]          # nothing was enqueued


def test_budget_for_one_image_splits_the_group(pkg, images):
    # one 256 x 320 image needs roughly 300 B/px of workspace: 40 MB holds one, not two
    ref = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    small = pkg.Context(pkg.default_params(max_keypoints=300), device=0, hbm_budget=40 << 20)
    fr = ref.extract(images)
    fs = small.extract(images)
    ref.sync()
    small.sync()
    for a, b in zip(fr, fs):
        ha, hb = a.host(), b.host()
        assert len(ha["xy"]) > 50
        assert np.array_equal(ha["xy"], hb["xy"]) and np.array_equal(ha["desc"], hb["desc"])


def test_capacity_refused_and_required_counts_reported(pkg, images):
    ctx = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    need = ctx.required_capacity()
    assert need == dict(cap_kp=300, cap_desc=600, cap_match=600)
    dev = torch.device("cuda:0")
    short_kp = _sentinel(pkg.Features.alloc(299, dev))
    with pytest.raises(pkg.Rift2Error) as e:
        ctx.extract([images[0]], [short_kp])
    assert e.value.code == pkg.E_CAPACITY
    torch.cuda.synchronize()
    assert short_kp.counts.cpu().tolist() == [-7, -7]
    # enough keypoints, too few descriptor rows (one per keypoint instead of two)
    short_desc = _sentinel(pkg.Features.alloc(300, dev, desc_per_kp=1))
    with pytest.raises(pkg.Rift2Error) as e:
        ctx.extract([images[0]], [short_desc])
    assert e.value.code == pkg.E_CAPACITY
    # the corner flag doubles every requirement
    cc = pkg.Context(pkg.default_params(max_keypoints=300, flags=pkg.FLAG_CORNERS), device=0)
    assert cc.required_capacity() == dict(cap_kp=600, cap_desc=1200, cap_match=1200)
    ring = pkg.Context(pkg.default_params(max_keypoints=300, flags=pkg.FLAG_RIFT_RING), device=0)
    assert ring.required_capacity() == dict(cap_kp=300, cap_desc=1800, cap_match=1800)
    # matches: a buffer one row short of cap_match
    fa, fb = ctx.extract(images)
    m = pkg.Matches.alloc(need["cap_match"] - 1, dev)
    m.count.fill_(-7)
    with pytest.raises(pkg.Rift2Error) as e:
        ctx.match([fa], [fb], [m])
    assert e.value.code == pkg.E_CAPACITY
    ctx.sync()
    assert int(m.count.cpu()[0]) == -7


def test_invalid_arguments_refused_on_the_host(pkg, images):
    ctx = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    with pytest.raises(ValueError):
        ctx.extract([images[0].double()])
    with pytest.raises(pkg.Rift2Error) as e:
        ctx.extract([torch.rand((8, 300), device="cuda:0")])     # side below 16
    assert e.value.code == pkg.E_INVAL
    with pytest.raises(pkg.Rift2Error) as e:
        pkg.Context(pkg.default_params(n_orient=8), device=0)
    assert e.value.code == pkg.E_UNIMPL
    with pytest.raises(pkg.Rift2Error) as e:
        pkg.Context(pkg.default_params(max_keypoints=0), device=0)
    assert e.value.code == pkg.E_INVAL
    with pytest.raises(pkg.Rift2Error) as e:
        ctx.set_wait_limit(-1)
    assert e.value.code == pkg.E_INVAL


def test_descriptor_wait_timeout_is_reported_and_recovers(pkg, images):
    ref = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    fr = ref.extract(images)
    ref.sync()
    ctx = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    ctx.set_wait_limit(0)
    ctx.extract(images)
    with pytest.raises(pkg.Rift2Error) as e:
        ctx.sync()
    assert e.value.code == pkg.E_TIMEOUT
    ctx.sync()                      # the status word was cleared by the failing sync
    ctx.set_wait_limit()
    fs = ctx.extract(images)
    ctx.sync()
    for a, b in zip(fr, fs):
        ha, hb = a.host(), b.host()
        assert len(ha["desc"]) > 50
        assert np.array_equal(ha["xy"], hb["xy"]) and np.array_equal(ha["desc"], hb["desc"])
