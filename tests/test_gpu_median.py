"""The noise threshold's median against the exact median of the GPU's own |EO_0,o| planes.

T_o is a fixed multiple of the median smallest-scale amplitude of orientation o (§II-A,
reading R2: the noise model of the phase-congruency measure RIFT builds on).  The library
selects that median exactly, by a radix select on the float bit patterns, so T_o must
equal noise_c x (the mean of the plane's two middle values) to the last bit of the FP32
sum and product, where the plane is the |EO_0,o| map the filter bank itself wrote (the
debug output `an0`) and noise_c is the oracle's constant T / median rounded to FP32.

The sizes cover an even and an odd pixel count, slices of 16-byte and of scalar loads
(P % 4 != 0), planes spread over several CTAs, one mixed-size call (packed planes), and
planes of one repeated value (a constant image: every amplitude is +0; a grating: one
amplitude nearly everywhere), whose selection takes the warp-aggregated counting path."""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(256, 256), (512, 512), (257, 263), (258, 259), (301, 303), (384, 640)]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2303_00319_gb300 as p
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return p


def _noise_c32():
    # T is linear in the median: T(plane of one value 1.0) is the constant itself
    return np.float32(O.noise_threshold(np.ones((1, 1))))


def _expected(an0_plane, c32):
    v = np.sort(an0_plane.astype(np.float32).ravel())
    n = v.size
    lo, hi = v[(n - 1) // 2], v[n // 2]
    return np.float32(np.float32(0.5) * np.float32(lo + hi)) * c32


def _check(feats, c32, what):
    for i, f in enumerate(feats):
        an0 = f.debug["an0"].cpu().numpy()
        got = f.debug["noise_t"].cpu().numpy()
        assert an0.shape[0] == len(got)
        for o in range(len(got)):
            exp = _expected(an0[o], c32)
            # bit-exact up to one ulp of the final product (the library rounds the same
            # double-precision constant to FP32 as the oracle's)
            assert abs(float(got[o]) - float(exp)) <= float(np.spacing(np.float32(exp))), \
                f"{what}: image {i} orientation {o}: {got[o]!r} vs {exp!r}"


def test_median_exact_on_own_planes(pkg):
    dev = torch.device("cuda:0")
    imgs = [torch.from_numpy(synth.make_pair(h, w, synth.pair_seed(11, i), angle_deg=None).a).to(dev)
            for i, (h, w) in enumerate(SIZES)]
    ctx = pkg.Context(pkg.default_params(max_keypoints=200), device=0)
    c32 = _noise_c32()
    # one mixed-size call (one launch group of packed planes) and each size alone
    feats = ctx.extract(imgs, debug=True)
    ctx.sync()
    _check(feats, c32, "mixed call")
    for h_w, im in zip(SIZES[:3], imgs[:3]):
        f, = ctx.extract([im], debug=True)
        ctx.sync()
        _check([f], c32, f"alone {h_w}")
    # a second call on the same context: the histograms start from zero again
    feats2 = ctx.extract(imgs, debug=True)
    ctx.sync()
    for a, b in zip(feats, feats2):
        assert np.array_equal(a.debug["noise_t"].cpu().numpy(), b.debug["noise_t"].cpu().numpy())


def test_median_repeated_values(pkg):
    dev = torch.device("cuda:0")
    h, w = 256, 320
    y, x = np.mgrid[0:h, 0:w]
    grating = (0.5 + 0.4 * np.cos(2 * np.pi * (96 * x / w + 13 * y / h))).astype(np.float32)
    flat = np.full((h, w), 0.37, dtype=np.float32)
    ctx = pkg.Context(pkg.default_params(max_keypoints=100), device=0)
    feats = ctx.extract([torch.from_numpy(grating).to(dev), torch.from_numpy(flat).to(dev)],
                        debug=True)
    ctx.sync()
    c32 = _noise_c32()
    _check(feats, c32, "repeated values")
    assert np.all(feats[1].debug["noise_t"].cpu().numpy() == 0)
    assert float(feats[0].debug["noise_t"].max()) > 0
