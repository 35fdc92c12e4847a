"""GPU parity: every stage of the CUDA path through the C ABI against the FP64 oracle.

Stage tests feed the oracle's upstream outputs to the GPU stage, so a near tie upstream
cannot cascade.  End-to-end tests compare the whole path on the seeded pairs.

Tolerances (float maps): the CUDA path computes the filter bank in FP32; its FFT leaves an
absolute error of a few ulp of a map's maximum, so element-wise errors are measured
against max(|oracle|, floor * max|oracle|).  Integer outputs (MIM, keypoints, dominant indices,
descriptor counts, NN indices) must be identical except at oracle-certified near ties
(relative top-two margin below 1e-5).
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from parity_util import (assert_map, assert_nn_matches, common_keypoint_descriptors,
                         compare_keypoints, rel_err)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIE = 1e-5
# An FP32 transform of 2^20 points leaves an absolute error of a few ulp of a map's
# maximum; 1e-4 relative is asserted down to 2.5e-3 of the maximum (4 ulp / 1e-4).
AMP_FLOOR = 2.5e-3


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2303_00319_gb300 as p
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return p


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def small(pkg, dev):
    """256^2 pair (30 degrees), <= 500 keypoints: oracle with all maps + GPU with debug maps."""
    pr = synth.config_pair(0)
    p = O.Params(max_keypoints=500)
    ctx = pkg.Context(pkg.default_params(max_keypoints=500), device=0)
    oa = O.extract(pr.a.astype(np.float64), p, keep_maps=True)
    ob = O.extract(pr.b.astype(np.float64), p, keep_maps=True)
    fa, fb = ctx.extract([torch.from_numpy(pr.a).to(dev), torch.from_numpy(pr.b).to(dev)],
                         debug=True)
    m = ctx.match([fa], [fb])[0]
    ctx.sync()
    return dict(pr=pr, p=p, ctx=ctx, oa=oa, ob=ob, fa=fa, fb=fb, m=m)


# --------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("h,w", [(16, 16), (256, 256), (1024, 1024), (48, 80), (105, 63),
                                 (384, 640), (224, 448), (1408, 176), (1664, 208), (2048, 1920),
                                 # Bluestein lengths (a prime factor above 13): primes, 17,
                                 # the largest side, and wide smooth rows beyond the register path
                                 (257, 263), (17, 34), (1021, 97), (4093, 24), (40, 4091),
                                 (64, 6144),
                                 # radix-9 and radix-16 passes (1296 = 16 9 9, 162 = 2 9 9)
                                 (1296, 96), (288, 162)])
def test_fft2_matches_numpy(pkg, dev, h, w):
    ctx = pkg.Context(pkg.default_params(), device=0)
    x = np.random.default_rng(h * 7 + w).random((2, h, w)).astype(np.float32)
    got = ctx.fft2(torch.from_numpy(x).to(dev)).cpu().numpy()
    exp = np.fft.fft2(x.astype(np.float64))
    err = np.max(np.abs(got - exp)) / np.max(np.abs(exp))
    assert err < 2e-6, err


# ------------------------------------------------------------------------- maps
def test_amplitude_sums(small):
    d = small["fa"].debug
    assert rel_err(d["amp"].cpu().numpy(), small["oa"].maps["A"], AMP_FLOOR) < 1e-4


def test_mim_exact_except_near_ties(small):
    for f, o in ((small["fa"], small["oa"]), (small["fb"], small["ob"])):
        mim = f.debug["mim"].cpu().numpy()
        mis = mim != o.maps["mim"]
        assert np.all(o.maps["mim_margin"][mis] < TIE), int(mis.sum())


def test_noise_threshold(small):
    t = small["fa"].debug["noise_t"].cpu().numpy()
    np.testing.assert_allclose(t, small["oa"].maps["T"], rtol=1e-5)


def test_noise_threshold_concentrated_amplitudes(pkg, dev):
    """A grating's filter responses have one amplitude everywhere (|EO| = |G(k)| / 2 for a
    one-sided filter), so nearly every |EO_0,o| falls in one bucket of both rounds of the
    median's selection (the second round's counting then aggregates equal buckets per
    warp).  T_o against the oracle (absolute tolerance: orientations whose window misses
    the grating have amplitudes at FP32 round-off)."""
    h, w = 256, 320
    y, x = np.mgrid[0:h, 0:w]
    img = (0.5 + 0.4 * np.cos(2 * np.pi * (96 * x / w + 13 * y / h))).astype(np.float32)
    ctx = pkg.Context(pkg.default_params(max_keypoints=100), device=0)
    f, = ctx.extract([torch.from_numpy(img).to(dev)], debug=True)
    ctx.sync()
    t = f.debug["noise_t"].cpu().numpy()
    o = O.extract(img.astype(np.float64), O.Params(max_keypoints=100), keep_maps=True)
    np.testing.assert_allclose(t, o.maps["T"], rtol=1e-5, atol=1e-5 * float(np.max(o.maps["T"])))
    assert np.max(o.maps["T"]) > 0


def test_pc_terms_and_moment(small):
    # both images: PC in [0, 1] against its scale; M also in FAST's normalised units, well
    # inside the 1e-5 certification margin
    _check_all_maps(small["fa"].debug, small["oa"], "256 A")
    _check_all_maps(small["fb"].debug, small["ob"], "256 B")


# --------------------------------------------------------------------- stages
def test_detect_stage_on_oracle_moment(pkg, dev, small):
    p = small["p"]
    for o in (small["oa"], small["ob"]):
        m32 = o.maps["M"].astype(np.float32)
        f, = small["ctx"].detect(torch.from_numpy(m32[None].copy()).to(dev))
        g = f.host()
        xy, v, unc, btie = O.detect(m32.astype(np.float64), p)
        r = compare_keypoints(g["xy"], g["score"], xy, v, unc, btie)
        assert not r["bad"] and r["inversions"] == 0, r
        common = min(len(v), len(g["score"]))
        np.testing.assert_allclose(g["score"][:common], v[:common], rtol=1e-5)


def test_detect_stage_edge_cases(pkg, dev):
    ctx = pkg.Context(pkg.default_params(max_keypoints=50), device=0)
    # constant map: no keypoints
    f, = ctx.detect(torch.full((1, 128, 160), 0.3, device=dev))
    assert f.counts.cpu().tolist() == [0, 0]
    # map too small for a patch: no keypoints
    f, = ctx.detect(torch.rand((1, 90, 90), device=dev))
    assert f.counts.cpu()[0] == 0
    # more survivors than max_keypoints, with many exact ties (checkerboard + plateaus)
    rng = np.random.default_rng(3)
    m = (np.round(rng.random((200, 232)) * 8) / 8).astype(np.float32)
    f, = ctx.detect(torch.from_numpy(m[None].copy()).to(dev))
    g = f.host()
    xy, v, unc, btie = O.detect(m.astype(np.float64), O.Params(max_keypoints=50))
    assert len(g["xy"]) == len(xy) == 50
    r = compare_keypoints(g["xy"], g["score"], xy, v, unc, btie)
    assert not r["bad"], r


@pytest.mark.parametrize("k", [20000, 30000])
def test_detect_stage_large_top_k(pkg, dev, k):
    """More than 16384 keypoints per image: the any-size shared-memory sort (k <= 26624)
    and the global-memory sort beyond it, against the oracle's detection on a noise map
    with more NMS survivors than k."""
    rng = np.random.default_rng(11)
    m = rng.random((640, 800)).astype(np.float32)
    ctx = pkg.Context(pkg.default_params(max_keypoints=k), device=0)
    f, = ctx.detect(torch.from_numpy(m[None].copy()).to(dev))
    g = f.host()
    xy, v, unc, btie = O.detect(m.astype(np.float64), O.Params(max_keypoints=k))
    assert len(g["xy"]) == len(xy) == k
    r = compare_keypoints(g["xy"], g["score"], xy, v, unc, btie)
    assert not r["bad"] and r["inversions"] == 0, r


@pytest.mark.parametrize("k,pattern", [(5000, "noise"), (20000, "noise"), (300, "dots")])
def test_detect_stage_multi_cta_selection(pkg, dev, k, pattern):
    """Maps above 4 MPix select the top K from a histogram of the candidates' leading key
    bits with many CTAs: against the oracle on a 2048 x 2112 noise map (the boundary
    bucket fits the sort), and on a grid of isolated bright pixels, ~250000 corners with
    one and the same score, whose bucket overflows the sort and sends it back to refining
    on the full list (ties ordered by raster index)."""
    if pattern == "noise":
        m = np.random.default_rng(12).random((2048, 2112)).astype(np.float32)
    else:
        m = np.zeros((2048, 2112), np.float32)
        m[2::4, 3::4] = 1.0
    ctx = pkg.Context(pkg.default_params(max_keypoints=k), device=0)
    f, = ctx.detect(torch.from_numpy(m[None].copy()).to(dev))
    g = f.host()
    xy, v, unc, btie = O.detect(m.astype(np.float64), O.Params(max_keypoints=k))
    assert len(g["xy"]) == len(xy) == k
    r = compare_keypoints(g["xy"], g["score"], xy, v, unc, btie)
    assert not r["bad"] and r["inversions"] == 0, r
    if pattern == "dots":   # equal FP32 scores: raster order
        ridx = g["xy"][:, 1].astype(np.int64) * m.shape[1] + g["xy"][:, 0]
        assert np.all(np.diff(ridx) > 0) and np.all(g["score"] == g["score"][0])


def test_describe_stage_bit_exact(pkg, dev, small):
    ctx = small["ctx"]
    for o in (small["oa"], small["ob"]):
        f = ctx.alloc_features()
        n = len(o.xy)
        f.kp_xy[:n] = torch.from_numpy(o.xy.astype(np.int32)).to(dev)
        f.counts[0] = n
        ctx.describe(torch.from_numpy(o.maps["mim"][None].copy()).to(dev), [f])
        g = f.host()
        assert np.array_equal(g["desc"].astype(np.int64), o.desc)
        assert np.array_equal(g["desc_kp"], o.desc_kp)
        assert np.array_equal(g["desc_dom"], o.desc_dom)
        np.testing.assert_allclose(g["desc_norm"], np.sqrt((o.desc ** 2).sum(axis=1)), rtol=1e-7)


def test_describe_stage_patch_edges_and_ragged(pkg, dev):
    # keypoints at the extreme corners of the admissible region, odd width (x start not
    # 16-aligned), random MIM
    ctx = pkg.Context(pkg.default_params(max_keypoints=64), device=0)
    h, w = 150, 203
    mim = np.random.default_rng(8).integers(0, 6, size=(h, w)).astype(np.uint8)
    pts = [(48, 48), (w - 49, 48), (48, h - 49), (w - 49, h - 49), (100, 75), (61, 99), (63, 50)]
    xy = np.array(pts, dtype=np.int64)
    f = ctx.alloc_features()
    f.kp_xy[:len(xy)] = torch.from_numpy(xy.astype(np.int32)).to(dev)
    f.counts[0] = len(xy)
    ctx.describe(torch.from_numpy(mim[None].copy()).to(dev), [f])
    g = f.host()
    desc, dkp, ddom, _ = O.describe(mim, xy, O.Params(max_keypoints=64))
    assert np.array_equal(g["desc"].astype(np.int64), desc)
    assert np.array_equal(g["desc_kp"], dkp) and np.array_equal(g["desc_dom"], ddom)


def _features_from(ctx, dev, desc, dkp):
    f = ctx.alloc_features()
    f.desc[:len(desc)] = torch.from_numpy(desc.astype(np.int16)).to(dev)
    f.desc_kp[:len(desc)] = torch.from_numpy(dkp.astype(np.int32)).to(dev)
    f.counts[1] = len(desc)
    return f


def test_match_stage_exact(pkg, dev, small):
    ctx = small["ctx"]
    oa, ob = small["oa"], small["ob"]
    fa = _features_from(ctx, dev, oa.desc, oa.desc_kp)
    fb = _features_from(ctx, dev, ob.desc, ob.desc_kp)
    m = ctx.match([fa], [fb])[0].host()
    nn, d1, d2, near = O.match(oa.desc, ob.desc)
    assert len(m["nn_desc"]) == len(nn)
    assert np.all((m["nn_desc"] == nn) | near)
    assert np.array_equal(m["kp_b"][~near], ob.desc_kp[nn][~near])
    np.testing.assert_allclose(m["d1"], d1, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(m["d2"], d2, rtol=1e-5, atol=1e-9)
    assert np.array_equal(m["near_tie"].astype(bool), near)


def test_match_stage_duplicates_and_single(pkg, dev):
    ctx = pkg.Context(pkg.default_params(max_keypoints=100), device=0)
    rng = np.random.default_rng(4)
    a = rng.integers(0, 40, size=(70, 216))
    b = rng.integers(0, 40, size=(130, 216))
    b[5] = a[0]
    b[77] = a[0]          # exact duplicate: the lower index must win
    fa = _features_from(ctx, dev, a, np.arange(70))
    fb = _features_from(ctx, dev, b, np.arange(130))
    m = ctx.match([fa], [fb])[0].host()
    nn, d1, d2, near = O.match(a, b)
    assert m["nn_desc"][0] == 5 and nn[0] == 5
    assert np.all((m["nn_desc"] == nn) | near)
    # one descriptor in B: d2 = inf
    fb1 = _features_from(ctx, dev, b[:1], np.arange(1))
    m1 = ctx.match([fa], [fb1])[0].host()
    assert np.all(m1["nn_desc"] == 0) and np.all(np.isinf(m1["d2"]))
    # empty A
    fa0 = _features_from(ctx, dev, a[:0], np.arange(0))
    m0 = ctx.match([fa0], [fb])[0]
    assert int(m0.count.cpu()[0]) == 0


def test_match_stage_screen_fallback(pkg, dev):
    """Ten exact copies of a query's descriptor spread over B's tiles and column halves
    fill every candidate list with equal scores: the screen cannot certify the top two and
    the exhaustive pass must return the lowest copy, as the oracle does."""
    ctx = pkg.Context(pkg.default_params(max_keypoints=700), device=0)
    rng = np.random.default_rng(11)
    a = rng.integers(0, 40, size=(300, 216))
    b = rng.integers(0, 40, size=(1300, 216))
    copies = [37, 130, 131, 300, 555, 700, 901, 1024, 1100, 1299]
    for j in copies:
        b[j] = a[0]
    for j in (12, 400, 800, 1250, 1251, 1252):   # a second query with six copies
        b[j] = a[7]
    fa = _features_from(ctx, dev, a, np.arange(300))
    fb = _features_from(ctx, dev, b, np.arange(1300))
    m = ctx.match([fa], [fb])[0].host()
    nn, d1, d2, near = O.match(a, b)
    assert nn[0] == 37 and m["nn_desc"][0] == 37 and m["d1"][0] == 0 and m["d2"][0] == 0
    assert nn[7] == 12 and m["nn_desc"][7] == 12
    assert np.all((m["nn_desc"] == nn) | near)
    np.testing.assert_allclose(m["d1"], d1, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(m["d2"], d2, rtol=1e-5, atol=1e-9)
    assert np.array_equal(m["near_tie"].astype(bool), near)


# -------------------------------------------------------------------- end to end
def _e2e_check(f, o, ctx_p):
    g = f.host()
    r = compare_keypoints(g["xy"], g["score"], o.xy, o.score, o.maps["kp_uncertain"],
                          o.maps["kp_boundary_tie"])
    assert not r["bad"] and r["inversions"] == 0, r
    return g, r


def _check_descriptors_and_nn(ga, gb, fa_dbg, fb_dbg, oa, ob, m, min_checked, label):
    """Descriptors of keypoints both lists share, whose patch has no MIM pixel that differs
    from the oracle's, are identical; the GPU matches equal the oracle's exhaustive search
    run on the GPU's own descriptors except at certified near ties."""
    checked = 0
    for g, dbg, o in ((ga, fa_dbg, oa), (gb, fb_dbg, ob)):
        mis = dbg["mim"].cpu().numpy() != o.maps["mim"]
        pairs = common_keypoint_descriptors(g, o, mis)
        for jg, jo in pairs:
            assert np.array_equal(g["desc"][jg].astype(np.int64), o.desc[jo]), label
            assert np.array_equal(g["desc_dom"][jg], o.desc_dom[jo]), label
        checked += len(pairs)
    assert checked >= min_checked, (label, checked)
    nn, d1, d2, near = O.match(ga["desc"].astype(np.int64), gb["desc"].astype(np.int64))
    assert_nn_matches(m, nn, d1, d2, near, label)
    assert np.array_equal(m["kp_a"], ga["desc_kp"][m["q_desc"]])
    assert np.array_equal(m["kp_b"], gb["desc_kp"][m["nn_desc"]])
    return checked


def test_end_to_end_small_pair(small):
    ga, ra = _e2e_check(small["fa"], small["oa"], small["p"])
    gb, rb = _e2e_check(small["fb"], small["ob"], small["p"])
    _check_descriptors_and_nn(ga, gb, small["fa"].debug, small["fb"].debug, small["oa"],
                              small["ob"], small["m"].host(), 100, "256x256")


def _check_all_maps(dbg, o, label):
    """Every debug map of one image against the oracle (floors as in the module header);
    all maps are compared before the first failure is raised, and each reports its worst
    element."""
    d = {k: v.cpu().numpy() for k, v in dbg.items()}
    m = o.maps
    mis = d["mim"] != m["mim"]
    errs = []

    def check(fn):
        try:
            fn()
        except AssertionError as e:
            errs.append(" ".join(ln.strip() for ln in str(e).splitlines() if ln.strip())[:400])

    def mim_check():
        assert np.all(m["mim_margin"][mis] < TIE), f"{label}: MIM {int(mis.sum())} mismatches"
    check(mim_check)
    amax = float(np.max(m["A"]))
    check(lambda: assert_map(f"{label} A_o", d["amp"], m["A"], AMP_FLOOR))
    check(lambda: assert_map(f"{label} |EO0|", d["an0"], m["An0"], 1e-2))
    # q = w / A_o inherits the amplitude's absolute error floor (AMP_FLOOR of its maximum):
    # its relative error grows like that floor over A_o where the amplitude is small
    with np.errstate(divide="ignore", invalid="ignore"):
        cond_q = np.where(m["A"] > 0, m["q"] * AMP_FLOOR * amax / m["A"], 0.0)
    check(lambda: assert_map(f"{label} q", d["q"], m["q"], 1e-3, extra_den=cond_q))
    # Er projects every scale onto the mean-phase direction sum EO / X: an FP32 rounding
    # delta of the responses turns that direction by delta / X, so Er's absolute error
    # grows like A_o / X where the summed vector is short.  Its denominator carries that
    # conditioning (A_o / (Ns X) relative to 1e-2 of the amplitude map's maximum).
    cond_er = m["A"] / (4.0 * m["X"]) * 1e-2 * amax
    check(lambda: assert_map(f"{label} Er", d["er"], m["Er"], 5e-2, extra_den=cond_er))
    check(lambda: assert_map(f"{label} PC", d["pc"], m["pc"], 1.0))
    # T_o is the median smallest-scale amplitude times a constant: the amplitude bar (1e-4
    # relative) applies; the 256^2 direct-size tests hold it to 1e-5
    check(lambda: np.testing.assert_allclose(d["noise_t"], m["T"], rtol=1e-4,
                                             err_msg=f"{label} T_o"))
    mo = m["M"]
    dn = np.max(np.abs(d["moment"] - mo)) / (mo.max() - mo.min())

    def m_norm():
        assert dn < 5e-6, f"{label}: M in normalised units {dn:.3e}"
    check(m_norm)
    # M is quadratic in PC: its relative error is twice PC's at leading order, so both its
    # bar (2e-4) and its floor (2e-2) are twice PC's; what the detector thresholds is M in
    # normalised units, checked above against the certification margin
    check(lambda: assert_map(f"{label} M", d["moment"], mo, 2e-2, bar=2e-4))
    assert not errs, "; ".join(errs)
    return int(mis.sum())


@pytest.mark.slow
def test_end_to_end_1024(pkg, dev):
    """Full-size workload (1024^2, <= 5000 keypoints) in the benchmark's launch grouping:
    both images of a pair in one extract call, every map of both images against the
    oracle, keypoints, descriptors of the shared keypoints, and the matches against the
    oracle's exhaustive search on the GPU's descriptors."""
    pr = synth.config_pair(1)
    ctx = pkg.Context(pkg.default_params(), device=0)
    fa, fb = ctx.extract([torch.from_numpy(pr.a).to(dev), torch.from_numpy(pr.b).to(dev)],
                         debug=True)
    m = ctx.match([fa], [fb])[0]
    ctx.sync()
    oa = O.extract(pr.a.astype(np.float64), O.Params(), keep_maps=True)
    ob = O.extract(pr.b.astype(np.float64), O.Params(), keep_maps=True)
    _check_all_maps(fa.debug, oa, "1024 A")
    _check_all_maps(fb.debug, ob, "1024 B")
    ga, _ = _e2e_check(fa, oa, None)
    gb, _ = _e2e_check(fb, ob, None)
    assert len(ga["xy"]) == 5000 and len(gb["xy"]) == 5000
    _check_descriptors_and_nn(ga, gb, fa.debug, fb.debug, oa, ob, m.host(), 1000, "1024")


@pytest.mark.slow
@pytest.mark.parametrize("h,w", [(384, 640), (1408, 256),
                                 # Bluestein sides: both prime; and rows too wide for four
                                 # scales at once: 6144 = 2^11 3 (split pass), prime 2053
                                 # (two-halves pass)
                                 (257, 263), (150, 6144), (160, 2053),
                                 # a Bluestein width whose length the row kernels' occupancy
                                 # decides (1289 -> 2704), radix-9 heights
                                 (162, 1289), (1296, 200)])
def test_mixed_radix_maps_and_descriptors(pkg, dev, h, w):
    """Sizes whose transforms run the shared-memory kernels (lg_cols_inverse, lg_rows_reduce;
    384 = 2^7 3, 640 = 2^7 5, 1408 = 2^7 11), Bluestein's chirp-z form for sides with a
    prime factor above 13, and the split row pass for rows too wide for four scales in
    shared memory: every map, keypoints, descriptors and matches of a pair against the
    oracle, as for the register path."""
    pr = synth.make_pair(h, w, synth.pair_seed(2, h + w), angle_deg=None)
    ctx = pkg.Context(pkg.default_params(max_keypoints=600), device=0)
    fa, fb = ctx.extract([torch.from_numpy(pr.a).to(dev), torch.from_numpy(pr.b).to(dev)],
                         debug=True)
    m = ctx.match([fa], [fb])[0]
    ctx.sync()
    p = O.Params(max_keypoints=600)
    oa = O.extract(pr.a.astype(np.float64), p, keep_maps=True)
    ob = O.extract(pr.b.astype(np.float64), p, keep_maps=True)
    _check_all_maps(fa.debug, oa, f"{h}x{w} A")
    _check_all_maps(fb.debug, ob, f"{h}x{w} B")
    ga, _ = _e2e_check(fa, oa, None)
    gb, _ = _e2e_check(fb, ob, None)
    _check_descriptors_and_nn(ga, gb, fa.debug, fb.debug, oa, ob, m.host(), 100, f"{h}x{w}")


def test_edge_images(pkg, dev):
    ctx = pkg.Context(pkg.default_params(max_keypoints=100), device=0)
    # constant image: every amplitude is zero, no keypoints, no descriptors
    z = torch.full((128, 128), 0.5, device=dev)
    # smaller than a patch: no keypoints; ragged mixed-radix sizes
    s = torch.rand((64, 80), device=dev)
    r = torch.from_numpy(synth.make_pair(120, 210, 5, 10.0, 8, 4).a).to(dev)
    f = ctx.extract([z, s, r])
    ctx.sync()
    assert f[0].counts.cpu().tolist() == [0, 0]
    assert f[1].counts.cpu().tolist() == [0, 0]
    o = O.extract(r.cpu().numpy().astype(np.float64), O.Params(max_keypoints=100), keep_maps=True)
    g, _ = _e2e_check(f[2], o, None)
    # sides the transforms do not take are refused, not computed wrongly: a length with a
    # prime factor above 13 beyond 4096, and any side beyond 8192
    for shape in ((4099, 128), (128, 8200)):
        with pytest.raises(pkg.Rift2Error) as e:
            ctx.extract([torch.rand(shape, device=dev)])
        assert e.value.code == pkg.E_UNIMPL


@pytest.mark.parametrize("na,nb", [(3000, 4500), (129, 127), (1, 300), (640, 1)])
def test_tensor_core_matcher_matches_oracle_and_cuda_core_form(pkg, dev, na, nb):
    """tcgen05 path (default) against the oracle and the CUDA-core form, several tiles and
    ragged edges; descriptors are random count vectors with cells summing to 256."""
    rng = np.random.default_rng(na + 7 * nb)

    def rand_desc(n):
        d = np.zeros((n, 216), dtype=np.int64)
        for c in range(36):
            w = rng.dirichlet(np.full(6, 0.7), size=n)
            d[:, c * 6:(c + 1) * 6] = rng.multinomial(256, [1 / 6] * 6, size=n) if False else \
                np.array([rng.multinomial(256, wi) for wi in w])
        return d
    a, b = rand_desc(na), rand_desc(nb)
    b[nb // 2] = a[0]
    ctx_tc = pkg.Context(pkg.default_params(max_keypoints=2500), device=0)
    ctx_pl = pkg.Context(pkg.default_params(max_keypoints=2500, flags=pkg.FLAG_PLAIN_MATCH),
                         device=0)
    out = []
    for ctx in (ctx_tc, ctx_pl):
        fa = _features_from(ctx, dev, a, np.arange(na))
        fb = _features_from(ctx, dev, b, np.arange(nb))
        m = ctx.match([fa], [fb])[0]
        ctx.sync()
        out.append(m.host())
    nn, d1, d2, near = O.match(a, b)
    for m in out:
        assert len(m["nn_desc"]) == na
        assert np.all((m["nn_desc"] == nn) | near)
        np.testing.assert_allclose(m["d1"], d1, rtol=1e-5, atol=1e-9)
        if nb > 1:
            np.testing.assert_allclose(m["d2"], d2, rtol=1e-5, atol=1e-9)
    assert np.array_equal(out[0]["nn_desc"], out[1]["nn_desc"])


def test_tensor_core_matcher_batch_of_pairs(pkg, dev):
    """Several pairs of different sizes in one call share the launches."""
    rng = np.random.default_rng(11)
    ctx = pkg.Context(pkg.default_params(max_keypoints=800), device=0)
    sizes = [(900, 1500), (1, 1), (1600, 200), (0, 50)]
    fas, fbs, exp = [], [], []
    for na, nb in sizes:
        a = rng.integers(0, 60, size=(na, 216))
        b = rng.integers(0, 60, size=(nb, 216))
        fas.append(_features_from(ctx, dev, a, np.arange(na)))
        fbs.append(_features_from(ctx, dev, b, np.arange(nb)))
        exp.append(O.match(a, b) if na else None)
    ms = ctx.match(fas, fbs)
    ctx.sync()
    for m, e, (na, nb) in zip(ms, exp, sizes):
        h = m.host()
        assert len(h["nn_desc"]) == na
        if na:
            nn, d1, d2, near = e
            assert np.all((h["nn_desc"] == nn) | near)


@pytest.mark.slow
def test_uneven_batch_in_one_call(pkg, dev):
    """Images of different sizes (mixed radices 3, 5, 7, 11, 13 among them) in one extract
    call: each matches the oracle image by image."""
    ctx = pkg.Context(pkg.default_params(max_keypoints=400), device=0)
    sizes = [(384, 640), (1408, 256), (256, 1664), (640, 384), (896, 1152)]
    imgs = []
    for i, (h, w) in enumerate(sizes):
        imgs.append(synth.make_pair(h, w, synth.pair_seed(2, i), angle_deg=None).a)
    feats = ctx.extract([torch.from_numpy(a).to(dev) for a in imgs])
    ctx.sync()
    for a, f in zip(imgs, feats):
        o = O.extract(a.astype(np.float64), O.Params(max_keypoints=400), keep_maps=True)
        g, _ = _e2e_check(f, o, None)
        assert len(g["xy"]) == len(o.xy)


def test_graph_capture_replays_the_calls(pkg, dev):
    """extract + match of a mixed-size batch captured into a CUDA graph (after the calls
    that create plans and workspace) and replayed: the outputs equal the direct calls'."""
    ctx = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    sizes = [(256, 256), (256, 256), (384, 320), (384, 320)]
    imgs = [torch.from_numpy(synth.make_pair(h, w, synth.pair_seed(5, i), angle_deg=None).a).to(dev)
            for i, (h, w) in enumerate(sizes)]
    feats = [ctx.alloc_features() for _ in imgs]
    matches = [ctx.alloc_matches() for _ in range(2)]

    def run(st):
        ctx.extract(imgs, feats, stream=st)
        ctx.match(feats[0::2], feats[1::2], matches, stream=st)

    run(torch.cuda.current_stream())
    ctx.sync()
    ref_f = [f.host() for f in feats]
    ref_m = [m.host() for m in matches]
    for f in feats:   # clear the outputs so the replay has to write them again
        f.kp_xy.zero_(); f.desc.zero_(); f.counts.zero_()
    for m in matches:
        m.nn_desc.fill_(-7); m.count.zero_()
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream(device=dev)
    gs.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=gs):
        run(torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    ctx.sync()
    for f, r in zip(feats, ref_f):
        h = f.host()
        assert np.array_equal(h["xy"], r["xy"]) and np.array_equal(h["desc"], r["desc"])
    for m, r in zip(matches, ref_m):
        h = m.host()
        assert np.array_equal(h["nn_desc"], r["nn_desc"]) and np.array_equal(h["d1"], r["d1"])


def test_corner_keypoints_merge(pkg, dev):
    """With corner keypoints (FAST on the minimum moment, reading R13) the keypoint list is
    the edge list followed by the corners not already in it: each part matches the
    oracle's (up to certified near ties), and the descriptors cover the merged list."""
    pr = synth.config_pair(0)
    p = O.Params(max_keypoints=300, corners=True)
    o = O.extract(pr.a.astype(np.float64), p, keep_maps=True)
    ctx = pkg.Context(pkg.default_params(max_keypoints=300, flags=pkg.FLAG_CORNERS), device=0)
    f = ctx.extract([torch.from_numpy(pr.a).to(dev)])[0]
    ctx.sync()
    g = f.host()
    ne = o.maps["n_edge"]
    r = compare_keypoints(g["xy"][:ne], g["score"][:ne], o.xy[:ne], o.score[:ne],
                          o.maps["kp_uncertain"], o.maps["kp_boundary_tie"])
    assert not r["bad"] and r["inversions"] == 0, r
    if r["flips"] == 0:
        edge = {tuple(map(int, q)) for q in o.xy[:ne]}
        keep = np.array([tuple(map(int, q)) not in edge for q in o.maps["corner_xy"]], dtype=bool)
        unc = o.maps["corner_uncertain"]
        rc = compare_keypoints(g["xy"][ne:], g["score"][ne:], o.xy[ne:], o.score[ne:], unc,
                               o.maps["corner_boundary_tie"])
        assert not rc["bad"] and rc["inversions"] == 0, rc
        assert keep.sum() == len(o.xy) - ne
    assert len(g["xy"]) > ne   # the synthetic scene has corner keypoints beyond the edge ones
    # every keypoint got 1 or 2 descriptors
    assert set(np.unique(g["desc_kp"])) == set(range(len(g["xy"])))


def test_autotuned_column_tile_gives_identical_features(pkg, dev):
    """With AUTOTUNE the first call of a size whose columns run in shared memory times the
    candidate tiles and keeps one; the features equal those of the default tile bit for bit."""
    sizes = [(640, 384), (640, 384)]
    imgs = [torch.from_numpy(synth.make_pair(h, w, synth.pair_seed(6, i), angle_deg=None).a).to(dev)
            for i, (h, w) in enumerate(sizes)]
    ref = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    tuned = pkg.Context(pkg.default_params(max_keypoints=300, flags=pkg.FLAG_AUTOTUNE), device=0)
    fr = ref.extract(imgs)
    ft = tuned.extract(imgs)
    ft2 = tuned.extract(imgs)   # the kept tile
    ref.sync(); tuned.sync()
    tile = tuned.tuned_tile(640, 384)
    assert tile >= 1 and ref.tuned_tile(640, 384) == 0
    for a, b, c in zip(fr, ft, ft2):
        ha, hb, hc = a.host(), b.host(), c.host()
        for k in ("xy", "desc"):
            assert np.array_equal(ha[k], hb[k]) and np.array_equal(ha[k], hc[k])
    assert tuned.tuned_tile(1024, 1024) == 0   # never seen


def test_autotuned_match_split_bit_identical(pkg, dev, small):
    """The matcher's split of B's columns, timed over 1..4 on the first call of a batch
    shape: every split gives the same matches (exact re-rank and certification), and the
    kept split reproduces them on the next call."""
    fa, fb = small["fa"], small["fb"]
    ref = pkg.Context(pkg.default_params(max_keypoints=500), device=0)
    tuned = pkg.Context(pkg.default_params(max_keypoints=500, flags=pkg.FLAG_AUTOTUNE), device=0)
    mr = ref.match([fa], [fb])
    m1 = tuned.match([fa], [fb])   # tunes: the last timed run's results
    m2 = tuned.match([fa], [fb])   # the kept split
    ref.sync(); tuned.sync()
    assert 1 <= tuned.tuned_match_split(1) <= 4 and ref.tuned_match_split(1) == 0
    r, a, b = mr[0].host(), m1[0].host(), m2[0].host()
    assert len(r["q_desc"]) > 100
    for k in ("q_desc", "nn_desc", "d1", "d2", "near_tie"):
        assert np.array_equal(r[k], a[k]) and np.array_equal(r[k], b[k]), k


# ------------------------------------------------------ RIFT ring baseline (§II-C)
def test_rift_ring_and_template_descriptors_bit_exact(pkg, dev, small):
    o = small["oa"]
    n = len(o.xy)
    for flag, mode, per in ((pkg.FLAG_RIFT_RING, "rift_ring", 6),
                            (pkg.FLAG_RIFT_TEMPLATE, "rift_template", 1)):
        ctx = pkg.Context(pkg.default_params(max_keypoints=500, flags=flag), device=0)
        f = ctx.alloc_features()
        assert f.desc.shape[0] >= per * 500
        f.kp_xy[:n] = torch.from_numpy(o.xy.astype(np.int32)).to(dev)
        f.counts[0] = n
        ctx.describe(torch.from_numpy(o.maps["mim"][None].copy()).to(dev), [f])
        g = f.host()
        desc, dkp, ddom, _ = O.describe(o.maps["mim"], o.xy, O.Params(max_keypoints=500), mode)
        assert len(g["desc"]) == per * n
        assert np.array_equal(g["desc"].astype(np.int64), desc)
        assert np.array_equal(g["desc_kp"], dkp) and np.array_equal(g["desc_dom"], ddom)


def test_rift_baseline_matching_and_ground_truth(pkg, dev, small):
    """RIFT baseline end to end (template A against the ring of B), and the library's
    ground-truth evaluation (rift2_evaluate) of both methods' matches against the oracle's
    evaluation of the SAME correspondences; the GPU path's correct-match count also stays
    within 2 of the count the oracle's own features reach."""
    pr, p = small["pr"], small["p"]
    ring = pkg.Context(pkg.default_params(max_keypoints=500, flags=pkg.FLAG_RIFT_RING), device=0)
    tmpl = pkg.Context(pkg.default_params(max_keypoints=500, flags=pkg.FLAG_RIFT_TEMPLATE), device=0)
    fa = tmpl.extract([torch.from_numpy(pr.a).to(dev)])[0]
    fb = ring.extract([torch.from_numpy(pr.b).to(dev)])[0]
    m = ring.match([fa], [fb])[0]
    ring.sync()
    ga, gb, gm = fa.host(), fb.host(), m.host()
    assert len(gb["desc"]) == 6 * len(gb["xy"]) and len(ga["desc"]) == len(ga["xy"])
    oa = O.extract(pr.a.astype(np.float64), p, mode="rift_template")
    ob = O.extract(pr.b.astype(np.float64), p, mode="rift_ring")
    nn, d1, d2, near = O.match(ga["desc"].astype(np.int64), gb["desc"].astype(np.int64))
    assert_nn_matches(gm, nn, d1, d2, near, "RIFT ring")
    tf = synth.ground_truth_affine(pr.angle_deg, pr.a.shape)
    cases = (((fa, fb, m), (ga, gb, gm), (oa, ob)),
             ((small["fa"], small["fb"], small["m"]),
              (small["fa"].host(), small["fb"].host(), small["m"].host()),
              (small["oa"], small["ob"])))
    for (dfa, dfb, dm), (g_a, g_b, g_m), (o_a, o_b) in cases:
        ev = small["ctx"].evaluate([dfa], [dfb], [dm], [tf])
        mg = pkg.Context.evaluation_host(ev)[0]
        same = O.evaluate(g_a["xy"], g_b["xy"], g_m["nn_desc"], g_a["desc_kp"], g_b["desc_kp"],
                          pr.angle_deg, pr.a.shape)
        assert mg["correct"] == same["correct"] and mg["matches"] == same["matches"], (mg, same)
        assert mg["success"] == same["success"]
        assert abs(mg["rmse"] - same["rmse"]) <= 1e-9 * max(1.0, same["rmse"])
        o_nn, _, _, _ = O.match(o_a.desc, o_b.desc)
        mo = O.evaluate(o_a.xy, o_b.xy, o_nn, o_a.desc_kp, o_b.desc_kp, pr.angle_deg, pr.a.shape)
        assert abs(mg["correct"] - mo["correct"]) <= 2, (mg, mo)
        assert mg["matches"] == mo["matches"]


def test_evaluate_hand_placed_correspondences(pkg, dev):
    """rift2_evaluate on hand-placed keypoints with known residuals (0, 2, 4, 5 px under a
    90-degree turn), a row without a correspondence, and two pairs in one call."""
    ctx = pkg.Context(pkg.default_params(max_keypoints=8), device=0)
    h = w = 101
    tf = synth.ground_truth_affine(90.0, (h, w))
    xa = np.array([[10, 20], [30, 40], [50, 50], [70, 15], [5, 5]], dtype=np.int32)
    # where A's points land under the turn, then displaced by the wanted residuals
    land = np.array([[tf[0] * x + tf[1] * y + tf[2], tf[3] * x + tf[4] * y + tf[5]] for x, y in xa])
    xb = np.round(land).astype(np.int32)
    xb[1, 0] += 2
    xb[2, 1] += 4
    xb[3, 0] += 5
    fa = ctx.alloc_features()
    fb = ctx.alloc_features()
    fa.kp_xy[:5] = torch.from_numpy(xa).to(dev)
    fb.kp_xy[:5] = torch.from_numpy(xb).to(dev)
    m = ctx.alloc_matches()
    m.kp_a[:5] = torch.arange(5, dtype=torch.int32, device=dev)
    m.kp_b[:5] = torch.tensor([0, 1, 2, 3, -1], dtype=torch.int32, device=dev)
    m.count[0] = 5
    res = pkg.Context.evaluation_host(ctx.evaluate([fa, fa], [fb, fb], [m, m], [tf, tf],
                                                   min_correct=2))
    for r in res:
        assert r["matches"] == 4 and r["correct"] == 2 and r["success"]
        assert abs(r["rmse"] - math.sqrt(2.0)) < 1e-12
    with pytest.raises(pkg.Rift2Error):
        ctx.evaluate([fa], [fb], [m], [tf], tol=0.0)


@pytest.mark.slow
def test_large_scene_4096(pkg, dev):
    """Large scene (4096^2, up to 20000 keypoints, 20000 x 20000-class matching).  The
    oracle computes orientation 0 of the filter bank in full (amplitude sum and noise
    threshold); keypoints, descriptors and matches are checked by properties that hold at
    any size, and sampled queries by exhaustive search over the returned descriptors."""
    pr = synth.config_pair(3)
    ctx = pkg.Context(pkg.default_params(max_keypoints=20000), device=0, hbm_budget=48 << 30)
    fa, fb = ctx.extract([torch.from_numpy(pr.a).to(dev), torch.from_numpy(pr.b).to(dev)],
                         debug=True)
    m = ctx.match([fa], [fb])[0]
    ctx.sync()
    # orientation 0 against the oracle's definition
    img = pr.a.astype(np.float64)
    F = np.fft.fft2(img)
    r, th = O.frequency_grid(*img.shape)
    ang = O.angular(th, 0)
    amp0 = np.zeros(img.shape)
    an0 = None
    for s in range(4):
        e = np.abs(np.fft.ifft2(F * (O.radial(r, s) * ang)))
        amp0 += e
        if s == 0:
            an0 = e
    got = fa.debug["amp"][0].cpu().numpy()
    assert rel_err(got, amp0, AMP_FLOOR) < 1e-4
    t0 = O.noise_threshold(an0)
    assert abs(float(fa.debug["noise_t"][0].cpu()) - t0) <= 1e-5 * t0
    # keypoints / descriptors / matches: properties
    g, gb, mh = fa.host(), fb.host(), m.host()
    h, w = img.shape
    assert len(g["xy"]) == 20000
    assert np.all(np.diff(g["score"]) <= 0)
    x, y = g["xy"][:, 0], g["xy"][:, 1]
    assert np.all((x >= 48) & (y >= 48) & (x < w - 48) & (y < h - 48))
    d = g["desc"].astype(np.int64).reshape(len(g["desc"]), 36, 6)
    assert np.all(d.sum(axis=2) == 256)
    assert np.all(np.diff(g["desc_kp"]) >= 0) and np.all(g["desc_dom"] < 6)
    assert len(mh["nn_desc"]) == len(g["desc"])
    assert np.all((mh["nn_desc"] >= 0) & (mh["nn_desc"] < len(gb["desc"])))
    assert np.all(mh["d1"] <= mh["d2"])
    A = g["desc"].astype(np.float64)
    B = gb["desc"].astype(np.float64)
    nb = np.sqrt((B * B).sum(axis=1))
    for q in np.random.default_rng(3).choice(len(A), size=64, replace=False):
        dist = 2.0 - 2.0 * (B @ A[q]) / (nb * np.sqrt(A[q] @ A[q]))
        j = int(np.argmin(dist))
        srt = np.sort(dist)
        if srt[1] - srt[0] >= 1e-5 * max(srt[0], 1e-12):
            assert mh["nn_desc"][q] == j
        assert abs(mh["d1"][q] - srt[0]) <= 1e-5 * max(srt[0], 1e-6) + 1e-9


# --------------------------- spatial orientation normalisation (variant, reading R14)
def test_spatial_descriptors_bit_exact_on_oracle_inputs(pkg, dev, small):
    """desc_spatial on the oracle's keypoints and MIM: disc histogram, frame choice, rotated
    grid sampling and recoding identical to the oracle's integer arithmetic."""
    ctx = pkg.Context(pkg.default_params(max_keypoints=500, flags=pkg.FLAG_SPATIAL_NORM),
                      device=0)
    for o in (small["oa"], small["ob"]):
        f = ctx.alloc_features()
        n = len(o.xy)
        f.kp_xy[:n] = torch.from_numpy(o.xy.astype(np.int32)).to(dev)
        f.counts[0] = n
        ctx.describe(torch.from_numpy(o.maps["mim"][None].copy()).to(dev), [f])
        g = f.host()
        desc, dkp, ddom, _ = O.describe(o.maps["mim"], o.xy, O.Params(max_keypoints=500),
                                        "rift2_spatial")
        assert np.array_equal(g["desc"].astype(np.int64), desc)
        assert np.array_equal(g["desc_kp"], dkp) and np.array_equal(g["desc_dom"], ddom)
        np.testing.assert_allclose(g["desc_norm"], np.sqrt((desc ** 2).sum(axis=1)), rtol=1e-7)


def test_spatial_descriptors_at_the_border_and_ragged(pkg, dev):
    """Keypoints whose rotated grid and disc leave the image (samples not counted), odd
    width, structured MIM with every dominant index and both frame sides."""
    ctx = pkg.Context(pkg.default_params(max_keypoints=200, flags=pkg.FLAG_SPATIAL_NORM),
                      device=0)
    h, w = 171, 203
    rng = np.random.default_rng(12)
    f0 = rng.standard_normal((h, w)) + 1j * rng.standard_normal((h, w))
    lp = np.exp(-(np.fft.fftfreq(h)[:, None] ** 2 + np.fft.fftfreq(w)[None, :] ** 2) / 8e-4)
    ang = np.angle(np.fft.ifft2(np.fft.fft2(f0) * lp)) + np.pi
    mim = (np.floor(ang / (2 * np.pi) * 6).astype(np.int64) % 6).astype(np.uint8)
    pts = [(48, 48), (w - 49, 48), (48, h - 49), (w - 49, h - 49), (100, 85), (61, 99),
           (63, 50), (150, 120), (49, 130), (130, 49)]
    pts += [tuple(v) for v in rng.integers(48, [w - 48, h - 48], size=(80, 2)).tolist()]
    xy = np.array(pts, dtype=np.int64)
    f = ctx.alloc_features()
    f.kp_xy[:len(xy)] = torch.from_numpy(xy.astype(np.int32)).to(dev)
    f.counts[0] = len(xy)
    ctx.describe(torch.from_numpy(mim[None].copy()).to(dev), [f])
    g = f.host()
    desc, dkp, ddom, info = O.describe(mim, xy, O.Params(max_keypoints=200), "rift2_spatial")
    assert len({i[0] for i in info}) >= 4           # several dominant indices exercised
    assert np.array_equal(g["desc"].astype(np.int64), desc)
    assert np.array_equal(g["desc_kp"], dkp) and np.array_equal(g["desc_dom"], ddom)


def test_spatial_descriptors_end_to_end(pkg, dev, small):
    """The whole pipeline with the variant flag: keypoints as RIFT2's, descriptors of the
    shared keypoints whose 133 x 133 window has no MIM pixel differing from the oracle's
    are identical, matches as the oracle's exhaustive search on the GPU's descriptors."""
    pr = small["pr"]
    ctx = pkg.Context(pkg.default_params(max_keypoints=500, flags=pkg.FLAG_SPATIAL_NORM),
                      device=0)
    fa, fb = ctx.extract([torch.from_numpy(pr.a).to(dev), torch.from_numpy(pr.b).to(dev)],
                         debug=True)
    m = ctx.match([fa], [fb])[0]
    ctx.sync()
    checked = 0
    hosts = []
    for f, o in ((fa, small["oa"]), (fb, small["ob"])):
        g, _ = _e2e_check(f, o, None)
        hosts.append(g)
        mim_g = f.debug["mim"].cpu().numpy()
        mis = mim_g != o.maps["mim"]
        xy_o = o.xy
        desc, dkp, _, _ = O.describe(o.maps["mim"], xy_o, small["p"], "rift2_spatial")
        gi = {tuple(map(int, q)): i for i, q in enumerate(g["xy"])}
        for k, (x, y) in enumerate(xy_o.tolist()):
            if (x, y) not in gi or mis[max(0, y - 66):y + 67, max(0, x - 66):x + 67].any():
                continue
            jg = np.flatnonzero(g["desc_kp"] == gi[(x, y)])
            assert np.array_equal(g["desc"][jg].astype(np.int64), desc[dkp == k])
            checked += 1
    assert checked >= 100
    nn, d1, d2, near = O.match(hosts[0]["desc"].astype(np.int64), hosts[1]["desc"].astype(np.int64))
    assert_nn_matches(m.host(), nn, d1, d2, near, "spatial")
