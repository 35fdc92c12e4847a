"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a direct DFT, properties
of the log-Gabor transfer function, a closed form for gratings, the 90-degree rotation
invariant of the MIM, the paper's worked histogram example, hand-built FAST patterns and
brute-force search.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------- FFT
def direct_dft2(x):
    h, w = x.shape
    out = np.zeros((h, w), dtype=np.complex128)
    for v in range(h):
        for u in range(w):
            acc = 0j
            for y in range(h):
                for xx in range(w):
                    acc += x[y, xx] * np.exp(-2j * math.pi * (u * xx / w + v * y / h))
            out[v, u] = acc
    return out


@pytest.mark.parametrize("n", [16, 15])
def test_fft_matches_direct_dft(n):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((n, n))
    ref = direct_dft2(x)
    got = np.fft.fft2(x)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_responses_use_fft_convolution_definition():
    # EO = ifft2(fft2(I) G) is the circular convolution of I with the filter's kernel;
    # check one response against a direct circular convolution on a 12x10 image.
    rng = np.random.default_rng(2)
    img = rng.random((12, 10))
    eo = O.responses(img)
    g = O.log_gabor_bank(12, 10)[1, 2]
    kern = np.fft.ifft2(g)                       # spatial kernel of the filter
    conv = np.zeros((12, 10), dtype=np.complex128)
    for y in range(12):
        for x in range(10):
            for yy in range(12):
                for xx in range(10):
                    conv[y, x] += img[yy, xx] * kern[(y - yy) % 12, (x - xx) % 10]
    assert np.max(np.abs(eo[1, 2] - conv)) < 1e-12


# --------------------------------------------------------------------- filters
def test_frequency_grid_convention():
    r, th = O.frequency_grid(8, 10)
    assert r[0, 0] == 1.0
    assert math.isclose(r[0, 1], 0.1) and math.isclose(r[1, 0], 0.125)
    assert math.isclose(r[0, 5], 0.5)            # Nyquist column of an even width
    assert th[0, 1] == 0.0                       # +u axis is theta = 0
    assert math.isclose(th[7, 0], math.pi / 2)   # negative row frequency is theta = +90 deg
    assert math.isclose(th[1, 0], -math.pi / 2)


def test_radial_peak_bandwidth_and_lowpass():
    p = O.DEFAULT
    for s in range(p.n_scales):
        f = O.center_frequency(s, p)
        assert math.isclose(f, 1.0 / (3.0 * 1.6 ** s))
        lp = O.lowpass(np.array(f), p)
        # unit peak (before the low-pass) exactly at the centre frequency
        assert math.isclose(float(O.radial(np.array(f), s, p)), float(lp), rel_tol=1e-14)
        # the Gaussian on a log axis falls to exp(-1/2) one log-sigma away on both sides
        for fac in (p.sigma_onf, 1.0 / p.sigma_onf):
            rr = np.array(f * fac)
            val = float(O.radial(rr, s, p)) / float(O.lowpass(rr, p))
            assert math.isclose(val, math.exp(-0.5), rel_tol=1e-12)
        # and is symmetric on the log axis
        a = float(O.radial(np.array(f * 1.3), s, p) / O.lowpass(np.array(f * 1.3), p))
        b = float(O.radial(np.array(f / 1.3), s, p) / O.lowpass(np.array(f / 1.3), p))
        assert math.isclose(a, b, rel_tol=1e-12)
    # Butterworth: 1/2 at the cutoff, 1/3 where (r/c)^(2n) = 2
    assert math.isclose(float(O.lowpass(np.array(0.45))), 0.5)
    assert math.isclose(float(O.lowpass(np.array(0.45 * 2 ** (1 / 30)))), 1 / 3, rel_tol=1e-12)
    # DC is removed
    r, _ = O.frequency_grid(6, 6)
    assert O.radial(r, 0)[0, 0] == 0.0


def test_angular_window_values_partition_and_one_sidedness():
    no = 6
    d = math.pi / no
    for o in range(no):
        t0 = o * d
        vals = O.angular(np.array([t0, t0 + d / 2, t0 - d, t0 + d, t0 + 2 * d, t0 - 2 * d,
                                   t0 + math.pi, t0 + 2.5 * d]), o)
        np.testing.assert_allclose(vals, [1.0, (1 + math.cos(math.pi / 4)) / 2, 0.5, 0.5,
                                          0.0, 0.0, 0.0, 0.0], atol=1e-15)
    th = np.linspace(-math.pi, math.pi, 2001)
    total = sum(O.angular(th, o) for o in range(no))
    inner = (th >= math.pi / 6) & (th <= 2 * math.pi / 3)
    np.testing.assert_allclose(total[inner], 2.0, atol=1e-12)
    for o in range(no):
        prod = O.angular(th, o) * O.angular(th + math.pi, o)
        assert np.max(prod) == 0.0


# -------------------------------------------------------- grating closed form
@pytest.mark.parametrize("k1,k2", [(5, 0), (3, 4), (-6, 7), (0, 9), (11, -2)])
def test_grating_amplitude_and_mim_closed_form(k1, k2):
    h, w = 64, 48
    y, x = np.mgrid[0:h, 0:w]
    img = np.cos(2 * math.pi * (k1 * x / w + k2 * y / h))
    eo = O.responses(img)
    u, v = k1 / w, k2 / h
    r = math.hypot(u, v)
    th_pos = math.atan2(-v, u)
    th_neg = math.atan2(v, -u)
    expect = np.zeros((4, 6))
    for s in range(4):
        for o in range(6):
            gp = float(O.radial(np.array(r), s)) * float(O.angular(np.array(th_pos), o))
            gn = float(O.radial(np.array(r), s)) * float(O.angular(np.array(th_neg), o))
            assert gp * gn == 0.0  # one-sided: at most one of the two deltas passes
            expect[s, o] = (gp + gn) / 2.0
    np.testing.assert_allclose(np.abs(eo), np.broadcast_to(expect[:, :, None, None], eo.shape),
                               atol=1e-12)
    a = O.amplitude_sums(eo)
    mim, _ = O.max_index_map(a)
    tot = expect.sum(axis=0)
    best = np.flatnonzero(tot >= tot.max() * (1 - 1e-9))   # exact ties: any of the tied set
    assert np.all(np.isin(mim, best))
    if len(best) == 1:
        assert np.all(mim == best[0])


def test_grating_phase_congruency_closed_form():
    # A pure grating gives every scale the same phase: E_s = a_s cos(phi), O_s = a_s sin(phi),
    # so Er = A^2/(A+eps), the median of |EO_0| is a_0 itself, width = (A/a_max - 1)/3.
    h, w = 40, 40
    y, x = np.mgrid[0:h, 0:w]
    img = np.cos(2 * math.pi * (4 * x / w + 3 * y / h))
    p = O.DEFAULT
    eo = O.responses(img, p)
    pc, t = O.phase_congruency(eo, p)
    amp = np.abs(eo)[:, :, 0, 0]                 # a_s per (s, o), constant over pixels
    for o in range(6):
        a_s = amp[:, o]
        big_a = a_s.sum()
        tau = a_s[0] / math.sqrt(math.log(4))
        tot = tau * (1 - 1.6 ** -4) / (1 - 1 / 1.6)
        t_exp = tot * (math.sqrt(math.pi / 2) + math.sqrt((4 - math.pi) / 2))
        assert math.isclose(t[o], t_exp, rel_tol=1e-9, abs_tol=1e-15)
        if big_a < 1e-9:
            assert np.all(pc[o] == 0)
            continue
        width = (big_a / (a_s.max() + p.eps) - 1) / 3
        wgt = 1 / (1 + math.exp((0.5 - width) * 3))
        energy = big_a * big_a / (big_a + p.eps)
        expect = wgt * max(energy - t_exp, 0.0) / big_a
        np.testing.assert_allclose(pc[o], expect, rtol=1e-7, atol=1e-12)


# -------------------------------------------------- rotation invariant (§III, Fig. 3)
def test_mim_shifts_by_half_the_orientations_under_rot90():
    # Odd size: the DFT grid is symmetric under a quarter turn, so the invariant is exact.
    rng = np.random.default_rng(3)
    from synth import scene
    img = scene(63, 63, np.random.Generator(np.random.PCG64(7)), n_blobs=12, n_segments=6)
    img = img + 0.02 * rng.standard_normal(img.shape)
    a = O.amplitude_sums(O.responses(img))
    ar = O.amplitude_sums(O.responses(np.rot90(img)))
    mim, margin = O.max_index_map(a)
    mim_r, _ = O.max_index_map(ar)
    ok = np.rot90(margin) >= 1e-5
    assert ok.mean() > 0.99
    expect = (np.rot90(mim).astype(int) + 3) % 6
    assert np.array_equal(mim_r[ok], expect[ok])
    # amplitudes themselves rotate with the orientation shift
    for o in range(6):
        np.testing.assert_allclose(ar[(o + 3) % 6], np.rot90(a[o]), atol=1e-10)


def test_recoded_histogram_invariant_under_rot90():
    from synth import scene
    img = scene(105, 105, np.random.Generator(np.random.PCG64(11)), n_blobs=25, n_segments=12)
    mim, _ = O.max_index_map(O.amplitude_sums(O.responses(img)))
    mim_r, margin_r = O.max_index_map(O.amplitude_sums(O.responses(np.rot90(img))))
    # patch around the centre; in the rotated frame take the rotated window explicitly
    c = 52
    # the same pixels seen from both frames: rotate the whole map, then cut the window
    win = np.rot90(mim)[c - 20:c + 20, c - 20:c + 20]
    win_r = mim_r[c - 20:c + 20, c - 20:c + 20]
    hist = np.bincount(win.ravel(), minlength=6)
    hist_r = np.bincount(win_r.ravel(), minlength=6)
    s, _, _ = O.dominant_indices(hist)
    s_r, _, _ = O.dominant_indices(hist_r)
    assert (s_r - s) % 6 == 3
    # recoded patches agree pixel by pixel after the spatial quarter turn (Fig. 3(h))
    rec = O.recode(win, s)
    rec_r = O.recode(win_r, s_r)
    ok = margin_r[c - 20:c + 20, c - 20:c + 20] >= 1e-5
    assert np.array_equal(rec[ok], rec_r[ok])
    hn = np.bincount(rec.ravel(), minlength=6)
    hn_r = np.bincount(rec_r.ravel(), minlength=6)
    assert np.array_equal(hn, hn_r)


# ------------------------------------------------- dominant index (§III, Eq. 1-2)
def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [int(v) for v in vals]
    return out


def test_worked_example_histogram_shift_and_recode():
    g = _golden("worked_example_histogram.txt")
    h1 = np.array(g["hist_mim1"])
    # moving the initial layer by one shifts every bin down by one (MIM 2 -> 1)
    mim1 = np.repeat(np.arange(6), h1)
    mim2 = O.recode(mim1, 1)
    assert np.array_equal(np.bincount(mim2, minlength=6), g["hist_mim2"])
    s, s2, has2 = O.dominant_indices(h1)
    assert s + 1 == g["dominant_1based"][0]
    assert has2 == bool(g["has_secondary"][0])
    rec = np.bincount(O.recode(mim1, s), minlength=6)
    assert np.array_equal(rec, g["recoded"])
    # the recoded histogram does not depend on the initial layer
    for shift in range(6):
        m = O.recode(mim1, shift)
        sm, _, _ = O.dominant_indices(np.bincount(m, minlength=6))
        assert np.array_equal(np.bincount(O.recode(m, sm), minlength=6), g["recoded"])


def test_recode_is_eq2_one_based():
    # Eq. 2 in the paper's 1-based indices, evaluated literally for every (MIM, s)
    for s1 in range(1, 7):
        for m1 in range(1, 7):
            lit = m1 - s1 + 1 if m1 >= s1 else m1 + 6 - s1 + 1
            assert int(O.recode(m1 - 1, s1 - 1)) + 1 == lit


def test_secondary_ratio_boundary():
    assert O.dominant_indices([100, 80, 0, 0, 0, 0])[2]           # exactly 80 %
    assert not O.dominant_indices([100, 79, 0, 0, 0, 0])[2]
    assert O.dominant_indices([5, 4, 0, 0, 0, 0])[2]
    s, s2, has2 = O.dominant_indices([7, 9, 9, 1, 0, 0])          # tie: lowest index wins
    assert (s, s2, has2) == (1, 2, True)


def test_descriptor_counts_and_permutation():
    rng = np.random.default_rng(5)
    mim = rng.integers(0, 6, size=(200, 200)).astype(np.uint8)
    xy = np.array([[60, 70], [100, 120], [48, 48], [151, 151]])
    desc, dkp, ddom, info = O.describe(mim, xy)
    for i in range(len(desc)):
        x, y = xy[dkp[i]]
        patch = mim[y - 48:y + 48, x - 48:x + 48].astype(int)
        rec = O.recode(patch, ddom[i])
        for ci in range(6):
            for cj in range(6):
                cell = rec[ci * 16:(ci + 1) * 16, cj * 16:(cj + 1) * 16]
                np.testing.assert_array_equal(desc[i, (ci * 6 + cj) * 6:(ci * 6 + cj + 1) * 6],
                                              np.bincount(cell.ravel(), minlength=6))
        assert desc[i].sum() == 96 * 96
        assert desc[i].reshape(36, 6).sum(axis=1).tolist() == [256] * 36


# ------------------------------------------------------------------------- FAST
def brute_fast(mn, t, arc=9):
    h, w = mn.shape
    corner = np.zeros((h, w), bool)
    score = np.zeros((h, w))
    for y in range(3, h - 3):
        for x in range(3, w - 3):
            p = mn[y, x]
            vals = [mn[y + dy, x + dx] for dx, dy in O.CIRCLE]
            for sign in (1, -1):
                ok = [sign * (q - p) > t for q in vals]
                if any(all(ok[(st + j) % 16] for j in range(arc)) for st in range(16)):
                    corner[y, x] = True
            if corner[y, x]:
                vb = sum(q - p - t for q in vals if q > p + t)
                vd = sum(p - q - t for q in vals if q < p - t)
                score[y, x] = max(vb, vd)
    return corner, score


def test_fast_hand_built_patterns():
    p = O.Params(patch=6, cells=6)        # 3-pixel border: the whole interior is a candidate
    img = np.zeros((15, 15))
    img[7, 7] = 1.0                        # isolated bright pixel: all 16 circle pixels darker
    c, v, _ = O.fast_corners(img, p)
    assert c[7, 7] and math.isclose(v[7, 7], 16 * (1.0 - 0.001))
    img = np.zeros((15, 15))
    img[:, 7] = 1.0                        # thin line: at most 2 contiguous darker pixels
    c, _, _ = O.fast_corners(img, p)
    assert not c[7, 7]
    img = np.zeros((15, 15))
    img[7:, 7:] = 1.0                      # block corner: dark pixel just outside it is a corner
    c, _, _ = O.fast_corners(img, p)
    assert c[7, 7] or c[6, 6]


def test_fast_matches_brute_force():
    rng = np.random.default_rng(9)
    mn = rng.random((20, 22)) * 0.02
    p = O.Params(patch=6, cells=6, fast_threshold=0.002)
    c, v, _ = O.fast_corners(mn, p)
    cb, vb = brute_fast(mn, 0.002)
    assert np.array_equal(c, cb)
    np.testing.assert_allclose(v, vb, atol=1e-15)


def test_nms_and_topk_brute_force():
    rng = np.random.default_rng(10)
    corner = rng.random((12, 13)) < 0.5
    score = np.round(rng.random((12, 13)) * 4) / 4 * corner      # many exact ties
    keep, _ = O.nms3x3(corner, score)
    h, w = corner.shape
    for y in range(h):
        for x in range(w):
            exp = corner[y, x]
            for dy, dx in itertools.product((-1, 0, 1), repeat=2):
                yy, xx = y + dy, x + dx
                if (dy or dx) and 0 <= yy < h and 0 <= xx < w and corner[yy, xx]:
                    if not ((score[y, x], -(y * w + x)) > (score[yy, xx], -(yy * w + xx))):
                        exp = False
            assert keep[y, x] == exp
    xy, v, _ = O.top_k(keep, score, 5)
    allk = sorted([(-score[y, x], y * w + x) for y, x in zip(*np.nonzero(keep))])[:5]
    assert [(-vv, yy * w + xx) for (xx, yy), vv in zip(xy, v)] == allk


# -------------------------------------------------------------------------- NN
def test_match_brute_force():
    rng = np.random.default_rng(12)
    a = rng.integers(0, 20, size=(30, 216))
    b = rng.integers(0, 20, size=(40, 216))
    b[7] = a[3]                     # an exact match
    b[9] = b[7]                     # and its duplicate: lowest index must win
    nn, d1, d2, near = O.match(a, b)
    for i in range(30):
        ds = []
        for j in range(40):
            ai, bj = a[i].astype(float), b[j].astype(float)
            ds.append(np.sum((ai / np.linalg.norm(ai) - bj / np.linalg.norm(bj)) ** 2))
        j = int(np.argmin(ds))
        srt = sorted(ds)
        if srt[1] - srt[0] > 1e-9:
            assert nn[i] == j
        assert math.isclose(d1[i], srt[0], abs_tol=1e-12)
        assert math.isclose(d2[i], srt[1], abs_tol=1e-12)
    assert nn[3] == 7 and near[3]


def test_median_even_count():
    assert O.median_even_mean([4.0, 1.0, 3.0, 2.0]) == 2.5
    x = np.random.default_rng(4).random(1001)
    assert O.median_even_mean(x) == sorted(x)[500]


@pytest.mark.parametrize("k", [1.0, 2.0])
def test_noise_threshold_against_rayleigh_statistics(k):
    """Noise model of reading R2 (§II-A names phase congruency with noise compensation):
    the smallest-scale amplitude of pure noise is the modulus of a complex Gaussian, i.e.
    Rayleigh(sigma).  With one scale the scale-sum factor is 1, so the threshold must equal
    the noise energy's mean + k std, taken here from the SAMPLE moments of 1.2e6 moduli:
    an estimate independent of the median route the oracle takes (median / sqrt(ln 4)
    recovers sigma; mean sigma sqrt(pi/2), std sigma sqrt((4 - pi)/2)).  A wrong Rayleigh
    constant, a dropped or mis-scaled k, or a median of the wrong quantity moves T by
    several percent; the Monte-Carlo error here is about 0.1 %.  The scale-sum factor is
    pinned on its own against the explicit series sum_{s < Ns} mult^-s."""
    rng = np.random.default_rng(20230301)
    sigma = 0.37
    z = sigma * (rng.standard_normal(1_200_000) + 1j * rng.standard_normal(1_200_000))
    mod = np.abs(z)
    p1 = O.Params(n_scales=1, k=k)
    # sigma from the median (the oracle's route) against the known sigma of the draw
    assert abs(O.median_even_mean(mod) / math.sqrt(math.log(4.0)) - sigma) < 3e-3 * sigma
    t1 = O.noise_threshold(mod, p1)
    mc = mod.mean() + k * mod.std()
    assert abs(t1 - mc) < 3e-3 * mc, (t1, mc)
    # the scale-sum factor: T grows by the geometric series of the scale amplitudes
    for ns, mult in ((4, 1.6), (3, 2.1), (6, 1.3)):
        series = sum(mult ** -s for s in range(ns))
        tn = O.noise_threshold(mod, O.Params(n_scales=ns, mult=mult, k=k))
        t1m = O.noise_threshold(mod, O.Params(n_scales=1, mult=mult, k=k))
        assert abs(tn / t1m - series) < 1e-12 * series


def test_energy_polar_form_and_frequency_spread():
    """The phase-congruency energy in its polar form: for scale components A_s e^(i phi_s)
    with mean phase phibar = arg(sum_s A_s e^(i phi_s)), Er = sum_s A_s (cos(phi_s - phibar)
    - |sin(phi_s - phibar)|) (eps -> 0).  Two equal components in quadrature give zero
    energy, components in phase give sum A.  The frequency-spread width is 1 for equal
    amplitudes on all scales and 0 for one scale alone, fixing the weight."""
    p = O.Params(eps=1e-15)
    rng = np.random.default_rng(5)
    amp = rng.uniform(0.1, 2.0, (4, 64))
    phi = rng.uniform(-math.pi, math.pi, (4, 64))
    eo = (amp * np.exp(1j * phi))[:, None, None, :]          # [Ns][No=1][1][64]
    er, q, an0, a_sum = O.pc_terms(eo, p)
    phibar = np.angle((amp * np.exp(1j * phi)).sum(axis=0))
    d = phi - phibar
    polar = (amp * (np.cos(d) - np.abs(np.sin(d)))).sum(axis=0)
    np.testing.assert_allclose(er[0, 0], polar, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(a_sum[0, 0], amp.sum(axis=0), rtol=1e-12)
    np.testing.assert_allclose(an0[0, 0], amp[0], rtol=1e-12)
    # quadrature pair (the other scales silent) and an in-phase set
    quad = np.array([1.0, 1j, 0.0, 0.0])[:, None, None, None] * np.exp(0.7j)
    assert abs(O.pc_terms(quad, p)[0][0, 0, 0]) < 1e-12
    inph = np.array([0.3, 1.1, 0.6, 2.0])[:, None, None, None] * np.exp(-2.1j)
    assert abs(O.pc_terms(inph, p)[0][0, 0, 0] - 4.0) < 1e-12
    # spread weight: width 1 (equal amplitudes) and 0 (one scale), q = w / sum A
    w = lambda width: 1.0 / (1.0 + math.exp((p.cutoff - width) * p.g))
    eq = np.full((4, 1, 1, 1), 0.5 + 0.5j)
    assert abs(O.pc_terms(eq, p)[1][0, 0, 0] - w(1.0) / (4 * abs(0.5 + 0.5j))) < 1e-12
    one = np.array([0.0, 0.8, 0.0, 0.0])[:, None, None, None] + 0j
    assert abs(O.pc_terms(one, p)[1][0, 0, 0] - w(0.0) / 0.8) < 1e-12


def test_step_edge_phase_congruency_invariants():
    """A bright vertical stripe on an odd-width circle (edges between columns 39 | 40 and
    120 | 121, no Nyquist column): phase congruency lies in [0, 1], is the same on every
    row, is zero for the orientations whose angular window misses the horizontal
    frequency axis (60, 90, 120 degrees), mirrors under x -> 160 - x with orientation o
    going to -o (the stripe maps to itself; global sign and conjugation leave PC
    unchanged), sits on the edges only, and puts the maximum moment there."""
    img = np.full((128, 161), 0.2)
    img[:, 40:121] = 0.8
    p = O.Params()
    pc, _ = O.phase_congruency(O.responses(img, p), p)
    M, m = O.moments(pc, p)
    assert pc.min() >= 0.0 and pc.max() <= 1.0
    assert np.array_equal(pc, np.broadcast_to(pc[:, :1, :], pc.shape))
    for o in (2, 3, 4):
        assert pc[o].max() < 1e-12
    mir = pc[:, :, ::-1]
    for o in range(6):
        np.testing.assert_allclose(pc[o], mir[(6 - o) % 6], atol=1e-12)
    # PC only next to the edges; the stripe's centre and the background far from it see none
    assert pc[0, 64, 80] == 0.0 and pc[0, 64, 0] == 0.0
    assert pc[0, 64, 39] > 0.3 and pc[0, 64, 40] > 0.3
    assert set(np.argsort(M[64])[-4:].tolist()) == {39, 40, 120, 121}
    assert np.all(M >= m)


def test_moments_of_single_orientation():
    # PC only in orientation o: M = PC^2 (edge), m ~ 0 (no corner)
    pc = np.zeros((6, 1, 1))
    for o in range(6):
        pc[:] = 0
        pc[o] = 0.7
        mx, mn = O.moments(pc)
        # (Sxx + Syy) = PC^2 / 3, den = PC^2/3 + eps  ->  M = PC^2/3 + eps/2, m = -eps/2
        assert math.isclose(mx.item(), 0.49 / 3 + 0.5e-4, rel_tol=1e-12)
        assert math.isclose(mn.item(), -0.5e-4, rel_tol=1e-9)
    # isotropic PC: equal in all orientations gives den = eps (Sxy = 0, Sxx = Syy)
    pc[:] = 0.5
    mx, mn = O.moments(pc)
    assert math.isclose(mx.item(), mn.item() + 1e-4, rel_tol=1e-9)


# ------------------------------------------------------------ RIFT ring baseline (§II-C)
def test_ring_members_are_the_cyclic_shifts_and_contain_rift2():
    rng = np.random.default_rng(21)
    mim = rng.integers(0, 6, size=(160, 170)).astype(np.uint8)
    xy = np.array([[60, 70], [100, 100], [121, 111]])
    ring, rkp, rdom, info = O.describe(mim, xy, mode="rift_ring")
    tmpl, tkp, tdom, _ = O.describe(mim, xy, mode="rift_template")
    r2, r2kp, r2dom, _ = O.describe(mim, xy, mode="rift2")
    assert len(ring) == 6 * len(xy) and len(tmpl) == len(xy)
    for k in range(len(xy)):
        members = ring[rkp == k]
        assert list(rdom[rkp == k]) == list(range(6))
        # member w: every cell's bins rotated by w relative to the unshifted template
        for w in range(6):
            np.testing.assert_array_equal(
                members[w].reshape(36, 6), np.roll(tmpl[k].reshape(36, 6), -w, axis=1))
        # RIFT2's descriptor is the ring member whose initial layer is the dominant index
        for d, s in zip(r2[r2kp == k], r2dom[r2kp == k]):
            np.testing.assert_array_equal(d, members[s])


def test_ground_truth_evaluation_on_exact_correspondences():
    # identity transform: a keypoint matched to itself has residual 0
    xy = np.array([[10, 20], [30, 40], [55, 65]])
    ev = O.evaluate(xy, xy, np.array([0, 1, 2]), np.arange(3), np.arange(3), 0.0, (100, 100))
    assert ev["correct"] == 3 and ev["rmse"] == 0.0 and not ev["success"]
    # quarter turn: the point p maps to R^-1 (p - c) + c
    h = w = 101
    c = 50.0
    pa = np.array([[60.0, 50.0]])                      # dx = 10, dy = 0
    pb = np.array([[50.0, 40.0]])                      # 90 deg sampling rotation sends it here
    ev = O.evaluate(pa, pb, np.array([0]), np.array([0]), np.array([0]), 90.0, (h, w))
    assert ev["correct"] == 1 and ev["rmse"] < 1e-9
    ev = O.evaluate(pa, pb + 5, np.array([0]), np.array([0]), np.array([0]), 90.0, (h, w))
    assert ev["correct"] == 0 and ev["rmse"] == 20.0


# ----------------------------------------------- corner keypoints (§II-A, reading R13)
def test_corner_keypoints_on_the_minimum_moment():
    """A bright square: the minimum moment (cornerness) peaks at its four corners and stays
    small along its sides, where the maximum moment (edgeness) is large; FAST on the
    normalised minimum moment ranks exactly the four corners first, far ahead of the rest."""
    img = np.zeros((160, 160))
    img[56:104, 56:104] = 1.0
    p = O.Params(max_keypoints=50, corners=True)
    pc, _ = O.phase_congruency(O.responses(img, p), p)
    m_max, m_min = O.moments(pc, p)
    corners = ((56, 56), (56, 103), (103, 56), (103, 103))
    mids = ((56, 80), (80, 56), (103, 80), (80, 103))
    assert min(m_min[y, x] for y, x in corners) > 3 * max(m_min[y, x] for y, x in mids)
    assert min(m_max[y, x] for y, x in mids) > 3 * max(m_min[y, x] for y, x in mids)
    xy, v, _, _ = O.detect(m_min, p)
    assert {tuple(map(int, q)) for q in xy[:4]} == {(x, y) for y, x in corners}
    assert v[3] > 3 * v[4]


def test_merge_keypoints_brute_force():
    """Edge keypoints unchanged and first; then the corner keypoints in their order, minus
    the pixels already present; no pixel twice."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        pts = rng.integers(0, 12, size=(40, 2))
        _, first = np.unique(pts, axis=0, return_index=True)
        pts = pts[np.sort(first)]
        ne = int(rng.integers(0, len(pts)))
        nc = int(rng.integers(0, len(pts)))
        edge = pts[:ne]
        corner = rng.permutation(pts)[:nc]
        ve, vc = rng.random(ne), rng.random(nc)
        xy, v = O.merge_keypoints(edge, ve, corner, vc)
        assert np.array_equal(xy[:ne], edge) and np.array_equal(v[:ne], ve)
        seen = {tuple(q) for q in edge}
        exp = [(tuple(q), w) for q, w in zip(corner, vc) if tuple(q) not in seen]
        assert [tuple(q) for q in xy[ne:]] == [q for q, _ in exp]
        assert np.array_equal(v[ne:], np.array([w for _, w in exp]))
        assert len({tuple(q) for q in xy}) == len(xy)


# ------------------------------------------- spatial orientation normalisation (R14)
def _structured_mim(n, seed):
    """A MIM with spatial structure (smoothed random orientation field, quantised) so that
    dominant indices and centroids vary between keypoints; int values 0..5."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    k = np.fft.fftfreq(n)
    lp = np.exp(-(k[:, None] ** 2 + k[None, :] ** 2) / (2 * 0.02 ** 2))
    z = np.fft.ifft2(np.fft.fft2(f) * lp)
    ang = np.angle(z) + math.pi                           # [0, 2 pi)
    return (np.floor(ang / (2 * math.pi) * 6).astype(np.int64) % 6).astype(np.uint8)


def _unambiguous(mim, x, y, p):
    """Keypoints whose dominant / secondary choice and frame sides have no exact tie (ties
    break by the lowest index, which a rotation of the values does not preserve)."""
    off = O.disc_offsets(p)
    vals, inside = O.mim_at(mim, x, y, off)
    hist = np.bincount(vals[inside], minlength=6)[:6]
    srt = np.sort(hist)[::-1]
    if srt[0] == srt[1] or srt[1] == srt[2]:
        return False
    s, s2, has2 = O.dominant_indices(hist, p)
    if 1000 * hist[s2] == 800 * hist[s]:
        return False
    for w in ([s, s2] if has2 else [s]):
        c, sn = O.rotation_q14(w, p)
        sel = vals == w
        if int(off[sel, 0].sum()) * c - int(off[sel, 1].sum()) * sn == 0:
            return False
    return True


def test_spatial_frame_zero_is_the_axis_aligned_descriptor():
    """In frame 0 (dominant index 0, centroid on the +x side) with the whole patch inside
    the image, the rotated grid is the R7 window itself: the R14 descriptor equals RIFT2's
    descriptor recoded by 0, built here from explicit cell slices."""
    p = O.Params()
    rng = np.random.default_rng(17)
    mim = rng.integers(1, 6, size=(200, 220)).astype(np.uint8)
    mim[:, 110:] = np.where(rng.random((200, 110)) < 0.6, 0, mim[:, 110:])
    x, y = 110, 100
    d, dkp, ddom, info = O.describe_spatial(mim, np.array([[x, y]]), p)
    assert info[0][0] == 0 and ddom[0] == 0
    assert O.spatial_frame(mim, x, y, 0, p) == (1 << 14, 0)
    patch = mim[y - 48:y + 48, x - 48:x + 48].astype(np.int64)
    exp = np.concatenate([np.bincount(patch[16 * i:16 * i + 16, 16 * j:16 * j + 16].ravel(),
                                      minlength=6) for i in range(6) for j in range(6)])
    assert np.array_equal(d[0], exp)
    # Q14 table: exact values at 0 and 90 degrees, symmetric rounding elsewhere
    assert O.rotation_q14(0) == (16384, 0) and O.rotation_q14(3) == (0, 16384)
    assert O.rotation_q14(1) == (round(16384 * math.sqrt(3) / 2), 8192)


@pytest.mark.parametrize("turns", [1, 2, 3])
def test_spatial_descriptor_invariant_under_quarter_turns(turns):
    """R14 makes the descriptor itself rotation invariant, not only up to a permutation of
    its cells (as RIFT2's index recoding alone is, §III): on an odd-size MIM turned by
    turns x 90 degrees (the values shifting by 3 turns mod 6, as the filter bank's
    orientations do) every keypoint without an exact tie has identical descriptors,
    including keypoints whose rotated grid leaves the image."""
    p = O.Params()
    n = 151
    mim = _structured_mim(n, 5)
    mim_r = ((np.rot90(mim, turns).astype(np.int64) + 3 * turns) % 6).astype(np.uint8)
    rng = np.random.default_rng(9)
    pts = rng.integers(48, n - 48, size=(60, 2))
    checked = 0
    for x, y in pts.tolist():
        # np.rot90 (k=1): pixel (x, y) moves to (y, n-1-x)
        xr, yr = x, y
        for _ in range(turns):
            xr, yr = yr, n - 1 - xr
        if not (_unambiguous(mim, x, y, p) and 48 <= xr < n - 48 and 48 <= yr < n - 48):
            continue
        d, _, dom, _ = O.describe_spatial(mim, np.array([[x, y]]), p)
        dr, _, dom_r, _ = O.describe_spatial(mim_r, np.array([[xr, yr]]), p)
        assert np.array_equal((dom + 3 * turns) % 6, dom_r)
        assert np.array_equal(d, dr), (x, y)
        checked += 1
    assert checked >= 30
    # RIFT2's recoding alone leaves the cells permuted: its descriptors differ here
    x, y = 75, 75
    a = O.describe(mim, np.array([[x, y]]), p)[0]
    b = O.describe(mim_r, np.array([[x if turns == 2 else y, n - 1 - x if turns == 1 else
                                     (n - 1 - x if turns == 2 else x)]]), p)[0]
    assert not np.array_equal(a[:1], b[:1])


def test_spatial_normalisation_follows_the_rotation_direction():
    """The grid turns the way the filter bank's orientation index does (counter-clockwise
    as displayed, pinned by the grating tests): for a scene and its copy turned by 30
    degrees (bilinear, so only approximately equal), R14 descriptors of corresponding
    keypoints are far closer than with the grid turned the other way."""
    from synth import rotate_bilinear, scene
    p = O.Params()
    n = 161
    img = scene(n, n, np.random.Generator(np.random.PCG64(31)), n_blobs=25, n_segments=12)
    rot = rotate_bilinear(img, 30.0)
    mim = O.max_index_map(O.amplitude_sums(O.responses(img)))[0]
    mim_r = O.max_index_map(O.amplitude_sums(O.responses(rot)))[0]
    c = (n - 1) / 2
    th = math.radians(30.0)
    dists = {"ccw": [], "cw": []}
    rng = np.random.default_rng(4)
    for x, y in rng.integers(60, n - 60, size=(40, 2)).tolist():
        # where (x, y) of img lands in rot: rotate_bilinear samples img at R^-1 (q - c) + c
        dx, dy = x - c, y - c
        xr = int(round(math.cos(th) * dx + math.sin(th) * dy + c))
        yr = int(round(-math.sin(th) * dx + math.cos(th) * dy + c))
        if not (48 <= xr < n - 48 and 48 <= yr < n - 48):
            continue
        d0 = O.describe_spatial(mim, np.array([[x, y]]), p)[0][0].astype(float)
        d1 = O.describe_spatial(mim_r, np.array([[xr, yr]]), p)[0][0].astype(float)
        dists["ccw"].append(np.linalg.norm(d0 - d1))
        # the other turning sense: the same construction on the mirrored scene
        m0 = O.describe_spatial(mim[:, ::-1], np.array([[n - 1 - x, y]]), p)[0][0].astype(float)
        dists["cw"].append(np.linalg.norm(m0 - d1))
    assert len(dists["ccw"]) >= 15
    assert np.median(dists["ccw"]) < 0.6 * np.median(dists["cw"]), dists
