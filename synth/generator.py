"""Seeded synthetic multimodal image pairs.

This module only draws inputs. It holds none of the feature pipeline's arithmetic and
is shared by the oracle tests, the GPU tests and the benchmark so that every side sees
the same pixels.

The pairs stand in for the paper's SAR-optical and infrared-optical datasets (§IV),
which are not available: image A is an "optical-like" scene of Gaussian blobs and
anti-aliased line segments; image B is A rotated about its centre, passed through a
nonlinear intensity remap and multiplied by gamma speckle (SAR-like multiplicative
noise). The rotation is returned so that ground-truth residuals can be computed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 20230301


def pair_seed(config: int, pair_index: int) -> int:
    """Seed of pair `pair_index` of workload `config`: 20230301 + 1000*config + index."""
    return SEED_BASE + 1000 * config + pair_index


def default_counts(h: int, w: int) -> tuple[int, int]:
    """Blob / segment counts: 40/20 at 256^2 and 400/200 at 1024^2, power law between."""
    n_blobs = int(round(40.0 * (h * w / 65536.0) ** 0.83))
    n_blobs = max(n_blobs, 4)
    return n_blobs, n_blobs // 2


@dataclass
class Pair:
    a: np.ndarray          # float32 [H][W] in [0, 1]
    b: np.ndarray          # float32 [H][W] in [0, 1]
    angle_deg: float       # rotation applied to A to make B (counter-clockwise on screen)
    seed: int


def _add_blob(img, rng):
    h, w = img.shape
    cy = rng.uniform(0, h)
    cx = rng.uniform(0, w)
    sigma = rng.uniform(3.0, 20.0)
    amp = rng.uniform(0.2, 1.0)
    r = int(math.ceil(4.0 * sigma))
    y0, y1 = max(0, int(cy) - r), min(h, int(cy) + r + 1)
    x0, x1 = max(0, int(cx) - r), min(w, int(cx) + r + 1)
    if y0 >= y1 or x0 >= x1:
        return
    yy = np.arange(y0, y1, dtype=np.float64)[:, None]
    xx = np.arange(x0, x1, dtype=np.float64)[None, :]
    img[y0:y1, x0:x1] += amp * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sigma * sigma))


def _add_segment(img, rng):
    h, w = img.shape
    n = min(h, w)
    py = rng.uniform(0, h)
    px = rng.uniform(0, w)
    length = rng.uniform(n / 16.0, n / 4.0)
    ang = rng.uniform(0.0, 2.0 * math.pi)
    amp = rng.uniform(0.2, 1.0)
    qx = px + length * math.cos(ang)
    qy = py + length * math.sin(ang)
    half = 1.5
    y0 = max(0, int(math.floor(min(py, qy) - half - 1)))
    y1 = min(h, int(math.ceil(max(py, qy) + half + 2)))
    x0 = max(0, int(math.floor(min(px, qx) - half - 1)))
    x1 = min(w, int(math.ceil(max(px, qx) + half + 2)))
    if y0 >= y1 or x0 >= x1:
        return
    dx, dy = qx - px, qy - py
    l2 = dx * dx + dy * dy
    # tiles of the bounding box whose centre lies farther than half + the tile's half
    # diagonal from the segment hold no pixel within `half` of it: they would add 0
    tile = 64
    for ty in range(y0, y1, tile):
        for tx in range(x0, x1, tile):
            ty1, tx1 = min(y1, ty + tile), min(x1, tx + tile)
            mx, my = 0.5 * (tx + tx1 - 1), 0.5 * (ty + ty1 - 1)
            tc = min(1.0, max(0.0, ((mx - px) * dx + (my - py) * dy) / l2))
            if math.hypot(mx - (px + tc * dx), my - (py + tc * dy)) > half + 0.75 * tile:
                continue
            yy = np.arange(ty, ty1, dtype=np.float64)[:, None]
            xx = np.arange(tx, tx1, dtype=np.float64)[None, :]
            t = np.clip(((xx - px) * dx + (yy - py) * dy) / l2, 0.0, 1.0)
            dist = np.hypot(xx - (px + t * dx), yy - (py + t * dy))
            img[ty:ty1, tx:tx1] += amp * np.clip(1.0 - dist / half, 0.0, 1.0)


def scene(h: int, w: int, rng: np.random.Generator, n_blobs: int | None = None,
          n_segments: int | None = None, noise_std: float = 0.01) -> np.ndarray:
    """Optical-like image A: blobs + anti-aliased segments + Gaussian noise, clipped to [0,1]."""
    nb, ns = default_counts(h, w)
    if n_blobs is None:
        n_blobs = nb
    if n_segments is None:
        n_segments = ns
    img = np.zeros((h, w), dtype=np.float64)
    for _ in range(n_blobs):
        _add_blob(img, rng)
    for _ in range(n_segments):
        _add_segment(img, rng)
    img += rng.normal(0.0, noise_std, size=(h, w))
    return np.clip(img, 0.0, 1.0)


def rotate_bilinear(img: np.ndarray, angle_deg: float) -> np.ndarray:
    """Rotate about ((W-1)/2, (H-1)/2), bilinear sampling, zero outside the source."""
    h, w = img.shape
    cy, cx = (h - 1) / 2.0, (w - 1) / 2.0
    a = math.radians(angle_deg)
    ca, sa = math.cos(a), math.sin(a)
    # destination (x, y) samples the source at R^-1 (x - c) + c; screen y points down,
    # so a counter-clockwise on-screen rotation uses +sin in the y row.
    dx = np.arange(w, dtype=np.float64)[None, :] - cx
    flat = img.ravel()
    out = np.zeros_like(img)
    band = 128   # destination rows per band: the band's source samples stay cache-local
    for r0 in range(0, h, band):
        dy = np.arange(r0, min(h, r0 + band), dtype=np.float64)[:, None] - cy
        sx = ca * dx - sa * dy + cx
        sy = sa * dx + ca * dy + cy
        x0 = np.floor(sx).astype(np.int64)
        y0 = np.floor(sy).astype(np.int64)
        fx = sx - x0
        fy = sy - y0
        acc = out[r0:r0 + band]
        # the four taps in a fixed order; a tap outside the source adds exactly 0
        for oy in (0, 1):
            for ox in (0, 1):
                xi = x0 + ox
                yi = y0 + oy
                wgt = (fx if ox else 1 - fx) * (fy if oy else 1 - fy)
                ok = (xi >= 0) & (xi < w) & (yi >= 0) & (yi < h)
                val = flat[np.where(ok, yi * w + xi, 0)]
                acc += np.where(ok, wgt * val, 0.0)
    return out


def ground_truth_affine(angle_deg: float, shape) -> tuple:
    """The known transform of a pair as (t0..t5), (x', y') = (t0 x + t1 y + t2,
    t3 x + t4 y + t5): image B is image A sampled through the rotation by angle_deg about
    ((W-1)/2, (H-1)/2) (rotate_bilinear), so a point p of A appears in B at
    [[cos, sin], [-sin, cos]] (p - c) + c."""
    h, w = shape
    cy, cx = (h - 1) / 2.0, (w - 1) / 2.0
    t = math.radians(angle_deg)
    c, s = math.cos(t), math.sin(t)
    return (c, s, cx - c * cx - s * cy, -s, c, cy + s * cx - c * cy)


def make_pair(h: int, w: int, seed: int, angle_deg: float | None = None,
              n_blobs: int | None = None, n_segments: int | None = None) -> Pair:
    """One seeded pair. angle_deg=None draws the rotation uniformly from [0, 360)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = scene(h, w, rng, n_blobs, n_segments)
    if angle_deg is None:
        angle_deg = float(rng.uniform(0.0, 360.0))
    b = rotate_bilinear(a, angle_deg)
    b = 1.0 - np.power(np.clip(b, 0.0, 1.0), 0.6)
    b = b * rng.gamma(4.0, 0.25, size=b.shape)
    b = np.clip(b, 0.0, 1.0)
    return Pair(a.astype(np.float32), b.astype(np.float32), float(angle_deg), seed)


def config_pair(config: int, pair_index: int = 0) -> Pair:
    """The pair shapes of the two single-pair workloads: 256^2 at 30 deg, 1024^2 random."""
    seed = pair_seed(config, pair_index)
    if config == 0:
        return make_pair(256, 256, seed, angle_deg=30.0, n_blobs=40, n_segments=20)
    if config == 1:
        return make_pair(1024, 1024, seed, angle_deg=None, n_blobs=400, n_segments=200)
    if config == 3:
        return make_pair(4096, 4096, seed, angle_deg=None)
    raise ValueError(f"no single-pair shape for workload {config}")


def batch_sizes(n: int, seed: int, lo: int = 384, hi: int = 2048, step: int = 128):
    """Uneven batch shapes: sides uniform on {lo..hi step}, aspect <= 2 (redrawn otherwise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = np.arange(lo, hi + 1, step)
    out = []
    while len(out) < n:
        h, w = int(rng.choice(sides)), int(rng.choice(sides))
        if max(h, w) <= 2 * min(h, w):
            out.append((h, w))
    return out


def smooth_sizes(lo: int = 16, hi: int = 8192, primes=(2, 3, 5, 7, 11, 13)):
    """Integers in [lo, hi] whose prime factors all lie in `primes` (sizes the FFT takes)."""
    out = []
    for n in range(lo, hi + 1):
        m = n
        for p in primes:
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return np.array(out)


def serving_sizes(n: int, seed: int, lo: int = 256, hi: int = 4096, smooth: bool = False,
                  max_width: int = 3584):
    """Pair sizes of the serving workload: each side an integer log-uniform in [lo, hi]
    (rounded to the nearest integer).  With smooth=True each side is instead snapped to the
    nearest 13-smooth size (width at most max_width)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ok = smooth_sizes(lo, hi) if smooth else None
    out = []
    for _ in range(n):
        side = []
        for lim in (hi, max_width):
            x = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
            if smooth:
                cand = ok[ok <= lim]
                side.append(int(cand[np.argmin(np.abs(cand - x))]))
            else:
                side.append(int(min(hi, max(lo, round(x)))))
        out.append((side[0], side[1]))
    return out
