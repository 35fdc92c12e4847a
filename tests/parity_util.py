"""Comparison helpers for the GPU-vs-oracle parity tests (no pipeline arithmetic here)."""
from __future__ import annotations

import numpy as np


def rel_err(got, exp, floor_frac):
    """max |got - exp| / max(|exp|, floor_frac * max|exp|)."""
    got = np.asarray(got, dtype=np.float64)
    exp = np.asarray(exp, dtype=np.float64)
    scale = np.max(np.abs(exp))
    if scale == 0:
        return float(np.max(np.abs(got)))
    den = np.maximum(np.abs(exp), floor_frac * scale)
    return float(np.max(np.abs(got - exp) / den))


def compare_keypoints(gpu_xy, gpu_score, ora_xy, ora_score, uncertain, boundary_tie,
                      tie_rel=1e-5):
    """Keypoint lists must agree except where the oracle certifies a near tie.

    Returns a dict with the unexplained differences (must be empty), the number of
    certified flips, and the number of order inversions not explained by a near tie."""
    g = [tuple(map(int, p)) for p in gpu_xy]
    o = [tuple(map(int, p)) for p in ora_xy]
    gs, osset = set(g), set(o)
    only_g = [p for p in g if p not in osset]
    only_o = [p for p in o if p not in gs]
    # certified: an uncertain corner / NMS decision, or a score within tie_rel of the
    # oracle's top-K cut (an exact or near tie at the cut may resolve either way)
    cut = float(ora_score[-1]) if len(ora_score) else 0.0
    score_g = {p: float(v) for p, v in zip(g, gpu_score)}
    score_o0 = {p: float(v) for p, v in zip(o, ora_score)}

    def certified(p):
        if uncertain[p[1], p[0]]:
            return True
        v = score_o0.get(p, score_g.get(p, 0.0))
        return cut > 0 and abs(v - cut) < tie_rel * cut

    flips = [p for p in only_g + only_o if certified(p)]
    un_g = [p for p in only_g if not certified(p)]
    un_o = [p for p in only_o if not certified(p)]
    # a flipped keypoint above the top-K cut displaces one at the cut in the other list
    slack = len(flips) + (1 if boundary_tie else 0)
    rank_g = {p: i for i, p in enumerate(g)}
    rank_o = {p: i for i, p in enumerate(o)}
    bad = [p for p in un_g if rank_g[p] < len(g) - slack]
    bad += [p for p in un_o if rank_o[p] < len(o) - slack]
    # order of the common keypoints: adjacent inversions need a near tie of the scores
    score_o = {p: float(v) for p, v in zip(o, ora_score)}
    common = [p for p in g if p in osset]
    inv = 0
    for a, b in zip(common, common[1:]):
        if rank_o[a] > rank_o[b]:
            va, vb = score_o[a], score_o[b]
            if abs(va - vb) >= tie_rel * max(va, vb):
                inv += 1
    return {"bad": bad, "flips": len(flips), "inversions": inv, "n_gpu": len(g), "n_oracle": len(o)}
