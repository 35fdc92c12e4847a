"""RIFT2_FLAG_TWO_LANES: a call's second half of images (or pairs) runs on a second internal
context and stream, forked from and joined back to the caller's stream.  The results are
bit-identical to one lane, the join orders everything before the caller's next work
(including a CUDA-graph capture of the calls), a device timeout on the second lane is
reported by rift2_sync, and the launch count covers both lanes."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(512, 512)] * 6 + [(384, 640), (640, 384), (257, 263), (512, 512)]


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
    return [torch.from_numpy(synth.make_pair(h, w, synth.pair_seed(9, i), angle_deg=None).a).to(dev)
            for i, (h, w) in enumerate(SIZES)]


def _run(pkg, images, flags, stream=None):
    ctx = pkg.Context(pkg.default_params(max_keypoints=400, flags=flags), device=0)
    feats = ctx.extract(images, stream=stream)
    matches = ctx.match(feats[0::2], feats[1::2], stream=stream)
    ctx.sync(stream)
    return [f.host() for f in feats], [m.host() for m in matches], ctx


def _same(a, b):
    for x, y in zip(a, b):
        for k in x:
            assert np.array_equal(np.asarray(x[k]), np.asarray(y[k])), k


def test_two_lanes_bit_identical(pkg, images):
    f1, m1, c1 = _run(pkg, images, 0)
    f2, m2, c2 = _run(pkg, images, pkg.FLAG_TWO_LANES)
    _same(f1, f2)
    _same(m1, m2)
    assert all(len(f["xy"]) > 0 for f in f2) and all(len(m["q_desc"]) > 0 for m in m2)
    # a side stream: the join orders the second lane before the caller's later work
    st = torch.cuda.Stream(device=images[0].device)
    f3, m3, _ = _run(pkg, images, pkg.FLAG_TWO_LANES, stream=st)
    _same(f1, f3)
    _same(m1, m3)
    assert c2.launch_count() >= c1.launch_count()   # both lanes' kernels are counted


def test_two_lanes_graph_capture(pkg, images):
    """extract + match captured on a stream (the fork and join are captured with them) and
    replayed: the outputs equal the direct calls'."""
    ctx = pkg.Context(pkg.default_params(max_keypoints=400, flags=pkg.FLAG_TWO_LANES), device=0)
    feats = [ctx.alloc_features() for _ in images]
    matches = [ctx.alloc_matches() for _ in range(len(images) // 2)]

    def run(st):
        ctx.extract(images, feats, stream=st)
        ctx.match(feats[0::2], feats[1::2], matches, stream=st)

    run(torch.cuda.current_stream())
    ctx.sync()
    ref_f, ref_m = [f.host() for f in feats], [m.host() for m in matches]
    for f in feats:
        f.kp_xy.zero_(); f.desc.zero_(); f.counts.zero_()
    for m in matches:
        m.nn_desc.fill_(-7); m.count.zero_()
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream(device=images[0].device)
    gs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(gs):
        with torch.cuda.graph(g, stream=gs):
            run(gs)
    g.replay()
    torch.cuda.synchronize()
    _same(ref_f, [f.host() for f in feats])
    _same(ref_m, [m.host() for m in matches])


def test_two_lanes_timeout_reported_and_recovers(pkg, images):
    ref, _, _ = _run(pkg, images, 0)
    ctx = pkg.Context(pkg.default_params(max_keypoints=400, flags=pkg.FLAG_TWO_LANES), device=0)
    ctx.extract(images)          # makes the second lane
    ctx.sync()
    ctx.set_wait_limit(0)        # both lanes
    ctx.extract(images)
    with pytest.raises(pkg.Rift2Error) as e:
        ctx.sync()
    assert e.value.code == pkg.E_TIMEOUT
    ctx.sync()
    ctx.set_wait_limit()
    fs = ctx.extract(images)
    ctx.sync()
    _same([{k: r[k] for k in ("xy", "desc")} for r in ref],
          [{k: f.host()[k] for k in ("xy", "desc")} for f in fs])


def test_two_lanes_workspace_figure(pkg, images):
    """With two lanes the figure is the sum of the halves' one-lane figures (the first half
    of the images and pairs on the context, the rest on the second lane)."""
    sizes = [tuple(im.shape) for im in images]
    one = pkg.Context(pkg.default_params(max_keypoints=400), device=0)
    two = pkg.Context(pkg.default_params(max_keypoints=400, flags=pkg.FLAG_TWO_LANES), device=0)
    h = len(sizes) // 2
    assert two.workspace_bytes(sizes, 5) == (one.workspace_bytes(sizes[:h], 2) +
                                             one.workspace_bytes(sizes[h:], 3))
