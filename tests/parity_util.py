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


def worst_above_floor(got, exp, floor_frac):
    """(worst relative error, its flat index, how many elements exceed 1e-4): the figures a
    failing map assertion reports."""
    got = np.asarray(got, dtype=np.float64)
    exp = np.asarray(exp, dtype=np.float64)
    scale = np.max(np.abs(exp))
    den = np.maximum(np.abs(exp), floor_frac * scale) if scale > 0 else np.ones_like(exp)
    r = np.abs(got - exp) / den
    i = int(np.argmax(r))
    return float(r.flat[i]), i, int((r > 1e-4).sum())


def assert_map(name, got, exp, floor_frac, bar=1e-4, extra_den=None):
    """Element-wise |got - exp| / max(|exp|, floor * max|exp|[, extra_den]) < bar, reporting
    the worst element."""
    if extra_den is not None:
        got = np.asarray(got, dtype=np.float64)
        exp = np.asarray(exp, dtype=np.float64)
        scale = np.max(np.abs(exp))
        den = np.maximum(np.maximum(np.abs(exp), floor_frac * scale), extra_den)
        r = np.abs(got - exp) / den
        i = int(np.argmax(r))
        w, n = float(r.flat[i]), int((r > bar).sum())
        assert w < bar, f"{name}: worst rel err {w:.3e} at flat index {i} ({n} elements above {bar})"
        return w
    w, i, n = worst_above_floor(got, exp, floor_frac)
    assert w < bar, f"{name}: worst rel err {w:.3e} at flat index {i} ({n} elements above {bar})"
    return w


def common_keypoint_descriptors(g, o, mim_mismatch, hp=48):
    """Pairs (gpu rows, oracle rows) of descriptors of keypoints present in both lists whose
    patch holds no MIM pixel that differs between the two maps (there the counts must be
    identical).  g: host dict of the GPU features; o: oracle Features."""
    gi = {tuple(map(int, p)): i for i, p in enumerate(g["xy"])}
    out = []
    for k, (x, y) in enumerate(np.asarray(o.xy).tolist()):
        if (x, y) not in gi:
            continue
        if mim_mismatch[y - hp:y + hp, x - hp:x + hp].any():
            continue
        jo = np.flatnonzero(np.asarray(o.desc_kp) == k)
        jg = np.flatnonzero(g["desc_kp"] == gi[(x, y)])
        out.append((jg, jo))
    return out


def assert_nn_matches(m, nn, d1, d2, near, label=""):
    """GPU matches against the oracle's exhaustive search on the same descriptors: indices
    identical except at certified near ties, distances within 1e-5 relative."""
    assert len(m["nn_desc"]) == len(nn), label
    bad = ~((m["nn_desc"] == nn) | near)
    assert not bad.any(), f"{label}: {int(bad.sum())} NN mismatches away from near ties"
    np.testing.assert_allclose(m["d1"], d1, rtol=1e-5, atol=1e-9, err_msg=label)
    fin = np.isfinite(d2)
    np.testing.assert_allclose(m["d2"][fin], d2[fin], rtol=1e-5, atol=1e-9, err_msg=label)
    return int(near.sum())
