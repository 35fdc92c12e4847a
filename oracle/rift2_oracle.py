"""RIFT2 feature pipeline: FP64 CPU oracle.  TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct numpy restatement of what the RIFT2 hot path computes:
log-Gabor bank -> phase congruency -> maximum moment -> FAST keypoints; amplitude sums ->
maximum index map (MIM); dominant index (Eq. 1) -> index recoding (Eq. 2) -> 6x6-cell
MIM-histogram descriptor; brute-force nearest-neighbour matching.

Only the tests, the smoke check and the benchmark's CPU-baseline / reference arm import
this module.  The CUDA library never does and shares no code with it.

Every floating-point step runs in float64 (numpy.fft in complex128).  Integer steps
(MIM indices, histograms, descriptors, dot products) are exact.

Where the paper is silent the module takes a reading, tagged [R1]..[R9]:
  R1 log-Gabor parameters: sigma_f=0.75, low-pass 0.45 / order 15, cycles-per-pixel grid
     theta = atan2(-v, u), circular (unpadded) filtering, ifft2 with 1/(HW).
  R2 phase congruency: Kovesi-model noise compensation from the median of the
     smallest-scale amplitude, k=1, g=3, cutoff 0.5, eps=1e-4.
  R3 moments: covariance of PC_o (cos, sin) over orientations (maximum / minimum moment).
  R4 FAST-9 with Rosten's sum-of-differences score, lexicographic 3x3 NMS on
     (score, -raster index), top-K by (score desc, raster index asc).
  R5 MIM ties go to the lowest orientation.
  R6 plain integer cell counts (no weighting), descriptor value = counts / L2 norm.
  R7 patch rows y-48..y+47 and columns x-48..x+47; keypoints only where it fits.
  R8 secondary descriptor iff 1000*H[s2] >= round(1000*ratio)*H[s] (ratio 0.8).
  R9 matching A -> B, lowest index on ties, duplicates kept.
  R13 RIFT's corner keypoints (§II-A): FAST on the min-max normalised minimum moment with
     the edge detector's threshold, NMS and ordering, capped at max_keypoints; merged after
     the edge keypoints, pixels already in the edge list dropped.
  R14 (a variant the paper does not have) spatial orientation normalisation of the patch:
     dominant index from the disc |d| <= 48, a frame of angle w pi / No or that + 180 deg
     chosen by the side of the centroid of the w-pixels, the 96x96 grid rotated into it in
     Q14 fixed point with rounding half away from zero, out-of-image samples not counted.

Pins (tests/test_oracle_*.py): FFT vs a direct DFT; filter properties (peak, bandwidth,
low-pass half point, raised-cosine window values, partition of unity, one-sidedness);
grating closed form for |EO| and MIM; 90-degree rotation invariant of MIM and of the
recoded histograms; the paper's worked histogram example (§III); FAST on hand-built
patterns and brute force; NN brute force; the phase-congruency energy against its polar
form with quadrature / in-phase special cases and the spread weight at widths 0 and 1;
step-edge and single-orientation invariants of PC and the moments.  The paper prints no
phase-congruency formula, so those pins hold PC and the moment map to the reading R2/R3,
not to the paper ("parity partially unpinned").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------- params
@dataclass(frozen=True)
class Params:
    """Pipeline parameters.  Table 1 gives 5000 keypoints, patch 96, FAST threshold 0.001
    and dominant ratio 0.8; §II-B gives the 6x6 grid and No bins; Ns, No, minimum
    wavelength and multiplier follow the log-Gabor bank of §II; the rest are readings."""
    n_scales: int = 4
    n_orient: int = 6
    min_wavelength: float = 3.0
    mult: float = 1.6
    sigma_onf: float = 0.75
    k: float = 1.0
    g: float = 3.0
    cutoff: float = 0.5
    eps: float = 1e-4
    lp_cutoff: float = 0.45
    lp_order: int = 15
    fast_threshold: float = 0.001
    fast_arc: int = 9
    max_keypoints: int = 5000
    patch: int = 96
    cells: int = 6
    second_ratio: float = 0.8
    corners: bool = False          # RIFT's corner keypoints on the minimum moment too [R13]

    @property
    def half_patch(self) -> int:
        return self.patch // 2

    @property
    def cell_size(self) -> int:
        return self.patch // self.cells

    @property
    def desc_dim(self) -> int:
        return self.cells * self.cells * self.n_orient


DEFAULT = Params()


# ------------------------------------------------------------------ log-Gabor bank [R1]
def frequency_grid(h: int, w: int):
    """Radius r (cycles/px) and angle theta = atan2(-v, u) of every DFT bin (§II, [R1]).
    r[0,0] is set to 1 as a placeholder so that log(r) is finite there."""
    u = np.fft.fftfreq(w)[None, :]
    v = np.fft.fftfreq(h)[:, None]
    uu = np.broadcast_to(u, (h, w))
    vv = np.broadcast_to(v, (h, w))
    r = np.sqrt(uu * uu + vv * vv)
    theta = np.arctan2(-vv, uu)
    r = r.copy()
    r[0, 0] = 1.0
    return r, theta


def lowpass(r, p: Params = DEFAULT):
    """Butterworth low-pass 1 / (1 + (r/cutoff)^(2n)) that tames the corner frequencies."""
    return 1.0 / (1.0 + (r / p.lp_cutoff) ** (2 * p.lp_order))


def center_frequency(s: int, p: Params = DEFAULT) -> float:
    """f_s = 1 / (min_wavelength * mult^s)."""
    return 1.0 / (p.min_wavelength * p.mult ** s)


def radial(r, s: int, p: Params = DEFAULT):
    """Radial log-Gabor component of scale s: exp(-ln^2(r/f_s) / (2 ln^2 sigma_f)) * LP(r),
    zero at DC."""
    f = center_frequency(s, p)
    out = np.exp(-(np.log(r / f) ** 2) / (2.0 * math.log(p.sigma_onf) ** 2)) * lowpass(r, p)
    out = np.array(out, dtype=np.float64)
    if out.ndim == 2:
        out[0, 0] = 0.0
    return out


def angular(theta, o: int, p: Params = DEFAULT):
    """Raised-cosine angular window of orientation o centred on theta_o = o*pi/No.
    It spans theta_o +- 2pi/No and is one-sided (zero at theta_o + pi), so every
    filtered response is analytic: its real part is the even and its imaginary part the
    odd response."""
    th_o = o * math.pi / p.n_orient
    d = np.abs(np.arctan2(np.sin(theta - th_o), np.cos(theta - th_o)))
    d = np.minimum(d * p.n_orient / 2.0, math.pi)
    return (1.0 + np.cos(d)) / 2.0


def log_gabor_bank(h: int, w: int, p: Params = DEFAULT):
    """G[s][o] = radial_s * angular_o on the (h, w) DFT grid, float64 [Ns][No][h][w]."""
    r, theta = frequency_grid(h, w)
    g = np.empty((p.n_scales, p.n_orient, h, w), dtype=np.float64)
    for s in range(p.n_scales):
        rs = radial(r, s, p)
        for o in range(p.n_orient):
            g[s, o] = rs * angular(theta, o, p)
    return g


def responses(img, p: Params = DEFAULT):
    """EO[s][o] = ifft2(fft2(img) * G[s][o]) — the complex log-Gabor responses of §II-B.
    Circular convolution, no padding [R1]."""
    img = np.asarray(img, dtype=np.float64)
    f = np.fft.fft2(img)
    g = log_gabor_bank(img.shape[0], img.shape[1], p)
    eo = np.empty(g.shape, dtype=np.complex128)
    for s in range(p.n_scales):
        for o in range(p.n_orient):
            eo[s, o] = np.fft.ifft2(f * g[s, o])
    return eo


# ------------------------------------------------------------------------ MIM (§II-B)
def amplitude_sums(eo):
    """A_o(x) = sum_s |EO_{s,o}(x)|, float64 [No][H][W]."""
    return np.abs(eo).sum(axis=0)


def max_index_map(a):
    """MIM(x) = argmax_o A_o(x), 0-based, lowest o on ties [R5] (np.argmax keeps the first).
    Also returns the relative top-two margin (A_(1) - A_(2)) / A_(1) per pixel, used to
    certify near-ties."""
    mim = np.argmax(a, axis=0).astype(np.uint8)
    srt = np.sort(a, axis=0)
    top, second = srt[-1], srt[-2]
    with np.errstate(invalid="ignore", divide="ignore"):
        margin = np.where(top > 0, (top - second) / top, 0.0)
    return mim, margin


# ------------------------------------------------------------ phase congruency [R2, R3]
def median_even_mean(x):
    """Median of all values; for an even count the mean of the two middle values."""
    return float(np.median(np.asarray(x, dtype=np.float64).ravel()))


def noise_threshold(an0, p: Params = DEFAULT) -> float:
    """Noise energy threshold T_o from the median amplitude of the smallest scale [R2]:
    tau = median/sqrt(ln 4) (Rayleigh mode), tau_total = tau (1 - mult^-Ns)/(1 - mult^-1),
    T = tau_total sqrt(pi/2) + k tau_total sqrt((4 - pi)/2)."""
    tau = median_even_mean(an0) / math.sqrt(math.log(4.0))
    tot = tau * (1.0 - (1.0 / p.mult) ** p.n_scales) / (1.0 - 1.0 / p.mult)
    return tot * math.sqrt(math.pi / 2.0) + p.k * tot * math.sqrt((4.0 - math.pi) / 2.0)


def mean_phase_energy(eo, p: Params = DEFAULT):
    """X_o = |sum_s EO_{s,o}| + eps, the length of the summed response vector whose
    direction is the mean phase [R2]."""
    sum_e = eo.real.sum(axis=0)
    sum_o = eo.imag.sum(axis=0)
    return np.sqrt(sum_e ** 2 + sum_o ** 2) + p.eps


def pc_terms(eo, p: Params = DEFAULT):
    """Per orientation, the terms of phase congruency before the noise threshold [R2]:
    Er_o = sum_s (E mE + O mO - |E mO - O mE|) with (mE, mO) the unit mean phase vector,
    q_o = w_o / A_o (0 where A_o = 0) with the frequency-spread weight w_o, An0_o = |EO_0,o|.
    Returns (Er, q, An0, A) each float64 [No][H][W]."""
    e = eo.real
    od = eo.imag
    an = np.abs(eo)
    sum_e = e.sum(axis=0)
    sum_o = od.sum(axis=0)
    sum_an = an.sum(axis=0)
    max_an = an.max(axis=0)
    x_energy = mean_phase_energy(eo, p)
    me = sum_e / x_energy
    mo = sum_o / x_energy
    er = (e * me + od * mo - np.abs(e * mo - od * me)).sum(axis=0)
    width = (sum_an / (max_an + p.eps) - 1.0) / (p.n_scales - 1)
    weight = 1.0 / (1.0 + np.exp((p.cutoff - width) * p.g))
    with np.errstate(invalid="ignore", divide="ignore"):
        q = np.where(sum_an > 0, weight / sum_an, 0.0)
    return er, q, an[0], sum_an


def phase_congruency(eo, p: Params = DEFAULT):
    """PC_o = w_o max(Er_o - T_o, 0) / A_o for each orientation (§II-A names the model).
    Returns (PC [No][H][W], T [No])."""
    er, q, an0, _ = pc_terms(eo, p)
    t = np.array([noise_threshold(an0[o], p) for o in range(p.n_orient)])
    pc = q * np.maximum(er - t[:, None, None], 0.0)
    return pc, t


def moments(pc, p: Params = DEFAULT):
    """Maximum and minimum moments of PC over orientations [R3]:
    a = PC_o cos(theta_o), b = PC_o sin(theta_o); Sxx = sum a^2/(No/2), Syy = sum b^2/(No/2),
    Sxy = 4 sum ab / No; M = (Sxx+Syy+den)/2, m = (Sxx+Syy-den)/2, den = sqrt(Sxy^2+(Sxx-Syy)^2)+eps.
    M is the edge map §II-A detects on; m the corner map."""
    no = p.n_orient
    sxx = np.zeros(pc.shape[1:])
    syy = np.zeros(pc.shape[1:])
    sxy = np.zeros(pc.shape[1:])
    for o in range(no):
        ang = o * math.pi / no
        a = pc[o] * math.cos(ang)
        b = pc[o] * math.sin(ang)
        sxx += a * a
        syy += b * b
        sxy += a * b
    sxx /= no / 2.0
    syy /= no / 2.0
    sxy *= 4.0 / no
    den = np.sqrt(sxy ** 2 + (sxx - syy) ** 2) + p.eps
    return (sxx + syy + den) / 2.0, (sxx + syy - den) / 2.0


def normalise(m):
    """Min-max normalisation to [0, 1]; None when the map is constant (no keypoints)."""
    lo, hi = float(m.min()), float(m.max())
    if not hi > lo:
        return None
    return (m - lo) / (hi - lo)


# ------------------------------------------------------------------------ FAST [R4]
# The 16-pixel Bresenham circle of radius 3, in cyclic order.
CIRCLE = ((0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
          (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3))


def candidate_region(h: int, w: int, p: Params = DEFAULT):
    """Pixels whose 96x96 patch [y-48, y+47] x [x-48, x+47] lies inside the image [R7]."""
    hp = p.half_patch
    return hp, max(hp, h - hp), hp, max(hp, w - hp)   # y0, y1, x0, x1 (half-open)


def fast_corners(mn, p: Params = DEFAULT, tie_eps: float = 1e-5):
    """FAST segment test with arc >= fast_arc and threshold t on the normalised map mn
    (§II-A, Table 1).  Returns (corner mask, score V, uncertain mask) over the full image;
    only the candidate region can be set.  V = max(sum over brighter circle pixels of
    (I_q - p - t), sum over darker ones of (p - I_q - t)).  A pixel is uncertain when any
    circle comparison is within tie_eps of its threshold."""
    h, w = mn.shape
    t = p.fast_threshold
    y0, y1, x0, x1 = candidate_region(h, w, p)
    corner = np.zeros((h, w), dtype=bool)
    score = np.zeros((h, w), dtype=np.float64)
    unc = np.zeros((h, w), dtype=bool)
    if y1 <= y0 or x1 <= x0:
        return corner, score, unc
    c = mn[y0:y1, x0:x1]
    ring = np.stack([mn[y0 + dy:y1 + dy, x0 + dx:x1 + dx] for dx, dy in CIRCLE])
    bright = ring > c + t
    dark = ring < c - t
    margin = np.minimum(np.abs(ring - (c + t)), np.abs(ring - (c - t))).min(axis=0)
    n = len(CIRCLE)
    arc = p.fast_arc

    def has_arc(b):
        ok = np.zeros(b.shape[1:], dtype=bool)
        for start in range(n):
            run = np.ones(b.shape[1:], dtype=bool)
            for j in range(arc):
                run &= b[(start + j) % n]
            ok |= run
        return ok

    is_corner = has_arc(bright) | has_arc(dark)
    vb = np.where(bright, ring - c - t, 0.0).sum(axis=0)
    vd = np.where(dark, c - ring - t, 0.0).sum(axis=0)
    corner[y0:y1, x0:x1] = is_corner
    score[y0:y1, x0:x1] = np.where(is_corner, np.maximum(vb, vd), 0.0)
    unc[y0:y1, x0:x1] = margin < tie_eps
    return corner, score, unc


def nms3x3(corner, score, tie_rel: float = 1e-5):
    """Keep a corner p iff for every corner q in its 8-neighbourhood (V_p, -idx_p) >
    (V_q, -idx_q) lexicographically, idx = y*W + x [R4].  Also flags pixels whose decision
    rests on a score gap below tie_rel * V_p (uncertain)."""
    h, w = corner.shape
    keep = corner.copy()
    unc = np.zeros_like(corner)
    pad_c = np.zeros((h + 2, w + 2), dtype=bool)
    pad_v = np.zeros((h + 2, w + 2))
    pad_c[1:-1, 1:-1] = corner
    pad_v[1:-1, 1:-1] = score
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            qc = pad_c[1 + dy:1 + dy + h, 1 + dx:1 + dx + w]
            qv = pad_v[1 + dy:1 + dy + h, 1 + dx:1 + dx + w]
            q_before = (dy < 0) or (dy == 0 and dx < 0)   # idx_q < idx_p
            if q_before:
                wins = score > qv
            else:
                wins = score >= qv
            keep &= ~qc | wins
            unc |= corner & qc & (np.abs(score - qv) < tie_rel * np.maximum(score, 1e-300))
    return keep, unc


def top_k(keep, score, k: int, tie_rel: float = 1e-5):
    """Strongest k survivors by (V desc, raster index asc).  Returns int64 [n][2] (x, y),
    float64 scores, and whether the k-th / (k+1)-th boundary is a near tie."""
    h, w = keep.shape
    ys, xs = np.nonzero(keep)
    v = score[ys, xs]
    idx = ys.astype(np.int64) * w + xs
    order = np.lexsort((idx, -v))
    order = order[:k] if k < len(order) else order
    boundary_tie = False
    if len(v) > k > 0:
        srt = np.sort(v)[::-1]
        boundary_tie = bool(srt[k - 1] - srt[k] < tie_rel * srt[k - 1])
    xy = np.stack([xs[order], ys[order]], axis=1).astype(np.int64)
    return xy, v[order], boundary_tie


# ------------------------------------------------------- descriptor (§II-B, §III, Eq. 1-2)
def cell_histograms(mim, xy, p: Params = DEFAULT):
    """Per keypoint, No-bin histograms of the MIM over the cells x cells grid of the patch
    rows y-48..y+47, columns x-48..x+47 [R6, R7].  int64 [K][cells*cells][No], cells in
    row-major (i, j) order."""
    hp, cs, nc, no = p.half_patch, p.cell_size, p.cells, p.n_orient
    out = np.zeros((len(xy), nc * nc, no), dtype=np.int64)
    for kidx, (x, y) in enumerate(xy):
        patch = mim[y - hp:y + hp, x - hp:x + hp].astype(np.int64)
        for i in range(nc):
            for j in range(nc):
                cell = patch[i * cs:(i + 1) * cs, j * cs:(j + 1) * cs]
                out[kidx, i * nc + j] = np.bincount(cell.ravel(), minlength=no)[:no]
    return out


def dominant_indices(hist, p: Params = DEFAULT):
    """Eq. 1: s = argmax of the whole-patch histogram (lowest bin on ties).  The secondary
    index s2 = argmax over the other bins; it yields a second descriptor iff its count is
    within the dominant ratio of the peak (§III), compared exactly in integers [R8]."""
    hist = np.asarray(hist, dtype=np.int64)
    s = int(np.argmax(hist))
    rest = hist.copy()
    rest[s] = -1
    s2 = int(np.argmax(rest))
    r_pm = int(round(p.second_ratio * 1000))
    has2 = 1000 * int(hist[s2]) >= r_pm * int(hist[s])
    return s, s2, bool(has2)


def recode(mim_values, s: int, p: Params = DEFAULT):
    """Eq. 2 in 0-based form: MIM_n = MIM - s if MIM >= s else MIM + No - s."""
    m = np.asarray(mim_values, dtype=np.int64)
    return np.where(m >= s, m - s, m + p.n_orient - s)


def descriptor_from_cells(cells, s: int, p: Params = DEFAULT):
    """216-D count vector of the recoded MIM patch: entry (c, b') counts the pixels of
    cell c whose recoded index is b', i.e. desc[c*No + recode(b, s)] = cells[c][b]."""
    no = p.n_orient
    d = np.zeros(cells.shape[0] * no, dtype=np.int64)
    for c in range(cells.shape[0]):
        for b in range(no):
            d[c * no + int(recode(b, s, p))] = cells[c, b]
    return d


def describe(mim, xy, p: Params = DEFAULT, mode: str = "rift2"):
    """Descriptors of the keypoints xy on the MIM.

    mode "rift2" (§III): one descriptor per keypoint recoded by its dominant index, plus a
    second one where the secondary index qualifies (both images).
    mode "rift_template" (§II-C, RIFT's baseline): one descriptor from the unshifted MIM.
    mode "rift_ring" (§II-C): the No descriptors of the convolution-sequence ring, the MIM
    with each layer w = 0..No-1 as the initial one, i.e. recoded by w.
    mode "rift2_spatial" (a variant, reading R14): describe_spatial.
    Returns (desc int64 [n][216], desc_kp, desc_dom, per-keypoint (s, s2, has2, whole))."""
    if mode == "rift2_spatial":
        return describe_spatial(mim, xy, p)
    cells = cell_histograms(mim, xy, p)
    descs, dkp, ddom, info = [], [], [], []
    for kidx in range(len(xy)):
        whole = cells[kidx].sum(axis=0)
        s, s2, has2 = dominant_indices(whole, p)
        info.append((s, s2, has2, whole))
        if mode == "rift2":
            shifts = [s, s2] if has2 else [s]
        elif mode == "rift_template":
            shifts = [0]
        elif mode == "rift_ring":
            shifts = list(range(p.n_orient))
        else:
            raise ValueError(mode)
        for w in shifts:
            descs.append(descriptor_from_cells(cells[kidx], w, p))
            dkp.append(kidx)
            ddom.append(w)
    d = np.array(descs, dtype=np.int64).reshape(-1, p.desc_dim)
    return d, np.array(dkp, dtype=np.int64), np.array(ddom, dtype=np.int64), info


# ------------------------- spatial orientation normalisation (a variant, reading R14)
# The paper normalises rotation through the dominant index alone (§III): the MIM values
# are recoded, but the 6x6 cell layout stays axis-aligned, so the descriptor of a rotated
# patch is the original one with its cells permuted (exactly so only for quarter turns).
# Reading R14 adds the missing spatial step:
#  * dominant index from the histogram over the disc |d| <= 48 around the keypoint (a
#    rotation-symmetric region), pixels inside the image only; s, s2 and the secondary
#    test as in Eq. 1 / R8;
#  * an orientation index fixes an axis only up to 180 degrees: the frame for index w
#    points along +a_w or -a_w, a_w = (cos th_w, -sin th_w) in array coordinates
#    (th_w = w pi / No, y down), whichever side holds the centroid of the disc pixels
#    whose MIM is w (exact integer sums; +a_w on a tie);
#  * the patch grid d = (dx, dy), dx, dy in [-48, 47], is rotated by that frame's angle
#    counter-clockwise (as displayed) with cos / sin in Q14 fixed point (rounded half away
#    from zero) and each sample rounded half away from zero: sample = p + rnd(R d), so a
#    quarter turn of the image maps every sample exactly;
#  * samples outside the image are not counted; the counts are recoded by w (Eq. 2).
ROT_Q = 14


def _rnd_q(v):
    """round(v / 2^ROT_Q) to the nearest integer, ties away from zero, on exact integers."""
    v = np.asarray(v, dtype=np.int64)
    return np.sign(v) * ((np.abs(v) + (1 << (ROT_Q - 1))) >> ROT_Q)


def rotation_q14(w: int, p: Params = DEFAULT):
    """(cos, sin) of th_w = w pi / No in Q14 fixed point, rounded half away from zero."""
    th = w * math.pi / p.n_orient
    def q(v):
        a = abs(v) * (1 << ROT_Q)
        return int(math.copysign(math.floor(a + 0.5), v)) if a > 0 else 0
    return q(math.cos(th)), q(math.sin(th))


def disc_offsets(p: Params = DEFAULT):
    """Integer offsets d with |d|^2 <= half_patch^2, int64 [n][2] (dx, dy)."""
    r = p.half_patch
    dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
    keep = dx * dx + dy * dy <= r * r
    return np.stack([dx[keep], dy[keep]], axis=1).astype(np.int64)


def mim_at(mim, x, y, off):
    """MIM values at (x, y) + off and whether each sample lies inside the image."""
    h, w = mim.shape
    qx, qy = x + off[:, 0], y + off[:, 1]
    inside = (qx >= 0) & (qx < w) & (qy >= 0) & (qy < h)
    vals = np.full(len(off), -1, dtype=np.int64)
    vals[inside] = mim[qy[inside], qx[inside]]
    return vals, inside


def spatial_frame(mim, x, y, w: int, p: Params = DEFAULT):
    """(cos, sin) in Q14 of the frame for index w at (x, y): th_w, or th_w + 180 degrees
    when the centroid of the disc pixels with MIM == w lies on the -a_w side."""
    c, sn = rotation_q14(w, p)
    off = disc_offsets(p)
    vals, _ = mim_at(mim, x, y, off)
    sel = vals == w
    sx, sy = int(off[sel, 0].sum()), int(off[sel, 1].sum())
    proj = sx * c - sy * sn          # centroid . a_w, a_w = (c, -sn) in array coordinates
    return (-c, -sn) if proj < 0 else (c, sn)


def rotated_samples(x, y, c, sn, p: Params = DEFAULT):
    """Sample pixels of the grid d in [-hp, hp)^2 rotated by the frame (c, sn):
    (x + rnd(c dx + sn dy), y + rnd(-sn dx + c dy)), ordered cell by cell (cells row-major,
    pixels row-major within a cell).  int64 [cells^2][cell^2][2]."""
    hp, cs, nc = p.half_patch, p.cell_size, p.cells
    out = np.zeros((nc * nc, cs * cs, 2), dtype=np.int64)
    for i in range(nc):
        for j in range(nc):
            dy, dx = np.mgrid[-hp + i * cs:-hp + (i + 1) * cs, -hp + j * cs:-hp + (j + 1) * cs]
            dx, dy = dx.ravel(), dy.ravel()
            out[i * nc + j, :, 0] = x + _rnd_q(c * dx + sn * dy)
            out[i * nc + j, :, 1] = y + _rnd_q(-sn * dx + c * dy)
    return out


def describe_spatial(mim, xy, p: Params = DEFAULT):
    """Descriptors with the spatial orientation normalisation of reading R14: one per
    keypoint from its dominant index (disc histogram) and a second one where the secondary
    index qualifies (R8), each from the patch grid rotated into its index's frame and
    recoded by that index (Eq. 2).  Returns (desc int64 [n][216], desc_kp, desc_dom,
    per-keypoint (s, s2, has2, disc histogram))."""
    h, w = mim.shape
    no = p.n_orient
    off = disc_offsets(p)
    descs, dkp, ddom, info = [], [], [], []
    for kidx, (x, y) in enumerate(np.asarray(xy).tolist()):
        vals, inside = mim_at(mim, x, y, off)
        whole = np.bincount(vals[inside], minlength=no)[:no]
        s, s2, has2 = dominant_indices(whole, p)
        info.append((s, s2, has2, whole))
        for wi in ([s, s2] if has2 else [s]):
            c, sn = spatial_frame(mim, x, y, wi, p)
            smp = rotated_samples(x, y, c, sn, p)
            d = np.zeros(p.desc_dim, dtype=np.int64)
            for cell in range(p.cells * p.cells):
                qx, qy = smp[cell, :, 0], smp[cell, :, 1]
                ok = (qx >= 0) & (qx < w) & (qy >= 0) & (qy < h)
                cnt = np.bincount(mim[qy[ok], qx[ok]].astype(np.int64), minlength=no)[:no]
                for b in range(no):
                    d[cell * no + int(recode(b, wi, p))] = cnt[b]
            descs.append(d)
            dkp.append(kidx)
            ddom.append(wi)
    d = np.array(descs, dtype=np.int64).reshape(-1, p.desc_dim)
    return d, np.array(dkp, dtype=np.int64), np.array(ddom, dtype=np.int64), info


# ------------------------------------------------------------------- matching [R9]
def match(desc_a, desc_b, chunk: int = 1024, tie_rel: float = 1e-5):
    """Brute-force nearest neighbour (§IV): for every descriptor of A, the descriptor of B
    at the smallest distance ||a/|a| - b/|b|||^2 = 2 - 2 a.b/(|a||b|), lowest index on
    ties.  The dot products are exact integers (float64 holds them exactly).  Returns
    (nn, d1, d2, near_tie) with d2 the second-smallest distance (inf if B has one row)."""
    a = np.asarray(desc_a, dtype=np.float64)
    b = np.asarray(desc_b, dtype=np.float64)
    na, nb = len(a), len(b)
    nn = np.full(na, -1, dtype=np.int64)
    d1 = np.full(na, np.inf)
    d2 = np.full(na, np.inf)
    if na == 0 or nb == 0:
        return nn, d1, d2, np.zeros(na, dtype=bool)
    norm_a = np.sqrt((a * a).sum(axis=1))
    norm_b = np.sqrt((b * b).sum(axis=1))
    for i0 in range(0, na, chunk):
        dots = a[i0:i0 + chunk] @ b.T
        den = norm_a[i0:i0 + chunk, None] * norm_b[None, :]
        with np.errstate(invalid="ignore", divide="ignore"):
            d = 2.0 - 2.0 * np.where(den > 0, dots / den, 0.0)
        j = np.argmin(d, axis=1)
        rows = np.arange(len(j))
        nn[i0:i0 + chunk] = j
        d1[i0:i0 + chunk] = d[rows, j]
        if nb > 1:
            d[rows, j] = np.inf
            d2[i0:i0 + chunk] = d.min(axis=1)
    with np.errstate(invalid="ignore"):
        near = (d2 - d1) < tie_rel * np.maximum(d1, 1e-12)
    return nn, d1, d2, near


# ---------------------------------------------------------------------- pipeline
@dataclass
class Features:
    xy: np.ndarray                 # int64 [n_kp][2] (x, y)
    score: np.ndarray              # float64 [n_kp]
    desc: np.ndarray               # int64 [n_desc][216] counts
    desc_kp: np.ndarray            # int64 [n_desc]
    desc_dom: np.ndarray           # int64 [n_desc]
    maps: dict = field(default_factory=dict)


def detect(m_map, p: Params = DEFAULT, tie_eps: float = 1e-5):
    """FAST on the normalised maximum-moment map, 3x3 NMS, top-K (§II-A, Table 1, [R4]).
    Returns (xy, score, uncertain-pixel mask, boundary_tie)."""
    mn = normalise(m_map)
    h, w = m_map.shape
    if mn is None:
        return np.zeros((0, 2), np.int64), np.zeros(0), np.zeros((h, w), bool), False
    corner, score, unc_fast = fast_corners(mn, p, tie_eps)
    keep, unc_nms = nms3x3(corner, score, tie_eps)
    xy, v, btie = top_k(keep, score, p.max_keypoints, tie_eps)
    # A flipped corner decision also changes its neighbours' NMS outcome.
    unc = unc_fast | unc_nms
    pad = np.zeros((h + 2, w + 2), dtype=bool)
    pad[1:-1, 1:-1] = unc_fast
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            unc |= pad[1 + dy:1 + dy + h, 1 + dx:1 + dx + w] & corner
    return xy, v, unc, btie


def merge_keypoints(xy_edge, v_edge, xy_corner, v_corner):
    """Edge keypoints (maximum moment) followed by the corner keypoints (minimum moment)
    that are not already edge keypoints, each list in its own (score desc, index asc)
    order [R13]: RIFT takes both kinds, corners for repeatability and edges for number
    (§II-A)."""
    have = {(int(x), int(y)) for x, y in xy_edge}
    keep = np.array([(int(x), int(y)) not in have for x, y in xy_corner], dtype=bool)
    xy = np.concatenate([np.asarray(xy_edge).reshape(-1, 2), np.asarray(xy_corner).reshape(-1, 2)[keep]])
    v = np.concatenate([np.asarray(v_edge, dtype=np.float64), np.asarray(v_corner, dtype=np.float64)[keep]])
    return xy.astype(np.int64), v


def extract(img, p: Params = DEFAULT, keep_maps: bool = False, mode: str = "rift2") -> Features:
    """Whole single-image path: responses -> (MIM, PC -> M -> keypoints) -> descriptors
    (`mode` as in describe).  With p.corners the keypoints are merge_keypoints of FAST on
    the maximum moment and FAST on the minimum moment, each capped at max_keypoints."""
    eo = responses(img, p)
    a = amplitude_sums(eo)
    mim, mim_margin = max_index_map(a)
    pc, t = phase_congruency(eo, p)
    m_max, m_min = moments(pc, p)
    xy, v, unc, btie = detect(m_max, p)
    n_edge = len(xy)
    if p.corners:
        xy_c, v_c, unc_c, btie_c = detect(m_min, p)
        xy, v = merge_keypoints(xy, v, xy_c, v_c)
    desc, dkp, ddom, _ = describe(mim, xy, p, mode)
    maps = {}
    if keep_maps:
        er, q, an0, _ = pc_terms(eo, p)
        maps = dict(A=a, mim=mim, mim_margin=mim_margin, pc=pc, T=t, M=m_max, m=m_min,
                    Er=er, q=q, An0=an0, X=mean_phase_energy(eo, p), kp_uncertain=unc,
                    kp_boundary_tie=btie, n_edge=n_edge)
        if p.corners:
            maps.update(corner_xy=xy_c, corner_score=v_c, corner_uncertain=unc_c,
                        corner_boundary_tie=btie_c)
    return Features(xy, v, desc, dkp, ddom, maps)


# ------------------------------------------------------ ground-truth evaluation (§IV)
def evaluate(xy_a, xy_b, nn, desc_kp_a, desc_kp_b, angle_deg, shape, tol: float = 3.0,
             rmse_cap: float = 20.0, min_correct: int = 10):
    """Correct matches, RMSE and success of one pair against the known rotation (§IV:
    a match is correct if its residual is below 3 px; RMSE over the correct matches,
    capped at 20 px; a pair succeeds with at least 10 correct matches).  Image B is image A
    rotated by angle_deg about ((W-1)/2, (H-1)/2), so a point p of A appears in B at
    R^-1 (p - c) + c with R the sampling rotation [[cos, -sin], [sin, cos]]."""
    h, w = shape
    cy, cx = (h - 1) / 2.0, (w - 1) / 2.0
    a = math.radians(angle_deg)
    ca, sa = math.cos(a), math.sin(a)
    ok = nn >= 0
    pa = np.asarray(xy_a, dtype=np.float64)[np.asarray(desc_kp_a)[ok]]
    pb = np.asarray(xy_b, dtype=np.float64)[np.asarray(desc_kp_b)[nn[ok]]]
    dx, dy = pa[:, 0] - cx, pa[:, 1] - cy
    ex = ca * dx + sa * dy + cx
    ey = -sa * dx + ca * dy + cy
    res = np.hypot(ex - pb[:, 0], ey - pb[:, 1])
    good = res < tol
    n = int(good.sum())
    rmse = float(np.sqrt(np.mean(res[good] ** 2))) if n else rmse_cap
    return {"correct": n, "rmse": min(rmse, rmse_cap), "success": n >= min_correct,
            "matches": int(ok.sum())}
