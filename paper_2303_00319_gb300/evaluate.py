"""Ground-truth evaluation of putative correspondences on synthetic pairs (§IV metrics).

A match is correct when the matched keypoint of B lies within 3 px of where the A keypoint
lands under the known transform; RMSE is taken over the correct matches and capped at
20 px; a pair succeeds with at least 10 correct matches.  The synthetic image B is image A
rotated about ((W-1)/2, (H-1)/2) with the sampling rotation [[cos, -sin], [sin, cos]], so
a point p of A appears in B at [[cos, sin], [-sin, cos]] (p - c) + c.  Host-side analysis of
results already copied back; not part of the device path.
"""
from __future__ import annotations

import math

import numpy as np


def rotation_residuals(kp_a, kp_b, nn, desc_kp_a, desc_kp_b, angle_deg: float, shape):
    h, w = shape
    cy, cx = (h - 1) / 2.0, (w - 1) / 2.0
    t = math.radians(angle_deg)
    c, s = math.cos(t), math.sin(t)
    nn = np.asarray(nn)
    keep = nn >= 0
    pa = np.asarray(kp_a, dtype=np.float64)[np.asarray(desc_kp_a)[keep]]
    pb = np.asarray(kp_b, dtype=np.float64)[np.asarray(desc_kp_b)[nn[keep]]]
    dx, dy = pa[:, 0] - cx, pa[:, 1] - cy
    return np.hypot(c * dx + s * dy + cx - pb[:, 0], -s * dx + c * dy + cy - pb[:, 1])


def pair_metrics(residuals, tol: float = 3.0, rmse_cap: float = 20.0, min_correct: int = 10):
    good = residuals < tol
    n = int(good.sum())
    rmse = float(np.sqrt(np.mean(residuals[good] ** 2))) if n else rmse_cap
    return {"correct": n, "rmse": min(rmse, rmse_cap), "success": n >= min_correct,
            "matches": int(len(residuals))}
