"""Allocation-free keypoint detection (rift2_detect_static) against rift2_detect.

rift2_detect_static serves callers that must not allocate device memory: it keeps its
scratch in one fixed device array instead of a context workspace.  Through the C ABI,
two calls in a row (the second on a different map, so a stale candidate list or min/max
from the first call would show) must return exactly what the context-based entry point
returns for the same maps.  This file is collected last on purpose.
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


def _map(h, w, seed):
    # any non-negative structured map will do: a synthetic scene plus a floor
    img = synth.scene(h, w, np.random.Generator(np.random.PCG64(seed)))
    return (img + 1e-3).astype(np.float32)


def test_static_detect_matches_context_detect_twice(pkg):
    dev = torch.device("cuda:0")
    params = pkg.default_params(max_keypoints=3000)
    ctx = pkg.Context(params, device=0)
    for h, w, seed in ((1024, 1024, 5), (480, 640, 9)):
        m = torch.from_numpy(_map(h, w, seed)).to(dev)
        ref, = ctx.detect(m[None].contiguous())
        got = pkg.detect_static(m, ctx.alloc_features(), params)
        torch.cuda.synchronize()
        r, g = ref.host(), got.host()
        assert len(r["xy"]) > 100
        assert int(got.counts.cpu()[0]) == int(ref.counts.cpu()[0])
        assert np.array_equal(g["xy"], r["xy"])
        assert np.array_equal(g["score"], r["score"])


def test_static_detect_refuses_maps_beyond_its_scratch(pkg):
    dev = torch.device("cuda:0")
    m = torch.zeros((1026, 1026), device=dev)
    with pytest.raises(pkg.Rift2Error) as e:
        pkg.detect_static(m, pkg.Features.alloc(5000, dev))
    assert e.value.code == pkg.E_CAPACITY
