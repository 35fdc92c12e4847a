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


def test_static_detect_allocates_no_device_memory(pkg):
    """After a warm-up call (which loads the kernels), repeated calls on preallocated
    outputs leave the device's free memory unchanged: nothing is allocated per call."""
    dev = torch.device("cuda:0")
    params = pkg.default_params(max_keypoints=2000)
    m = torch.from_numpy(_map(768, 1024, 21)).to(dev)
    feats = pkg.Features.alloc(2000, dev)
    pkg.detect_static(m, feats, params)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(5):
        pkg.detect_static(m, feats, params)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert int(feats.counts.cpu()[0]) > 100


def test_static_detect_refuses_host_buffers(pkg):
    """Through the C ABI directly (the Python wrapper refuses earlier): a host map or host
    outputs are refused on the host with RIFT2_E_INVAL before anything is enqueued."""
    import ctypes as C
    dev = torch.device("cuda:0")
    m_host = torch.from_numpy(_map(256, 256, 3))
    m_dev = m_host.to(dev)
    feats = pkg.Features.alloc(5000, dev)
    fc, _ = feats.to_c()
    L = pkg.lib()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.rift2_detect_static(None, C.c_void_p(m_host.data_ptr()), 256, 256, C.byref(fc), st)
    assert rc == pkg.E_INVAL
    host_xy = torch.zeros((5000, 2), dtype=torch.int32)
    fc.kp_xy = host_xy.data_ptr()
    rc = L.rift2_detect_static(None, C.c_void_p(m_dev.data_ptr()), 256, 256, C.byref(fc), st)
    assert rc == pkg.E_INVAL
    with pytest.raises(ValueError):
        pkg.detect_static(m_host, feats)
    with pytest.raises(ValueError):   # a strided view is refused, not read as a dense map
        pkg.detect_static(m_dev.t(), feats)
