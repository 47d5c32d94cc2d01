"""Reconstruction accuracy metrics (host-side evaluation; not part of the per-frame path).

Accuracy, completeness, Chamfer-L1 and F-score as the paper evaluates maps (Sec. 4.1.2): accuracy is the mean distance
from each reconstructed point to its nearest ground-truth point, completeness the mean distance from each ground-truth
point to its nearest reconstructed point, Chamfer-L1 their mean. F-score at threshold d: the harmonic mean of the
fractions of reconstructed and ground-truth points within d of the other set.
"""
from __future__ import annotations

import numpy as np


def backproject(depth: np.ndarray, fx: float, fy: float, cx: float, cy: float, T_wc: np.ndarray,
                stride: int = 1) -> np.ndarray:
    """World points (n, 3) of the valid (> 0, finite) pixels of a z-depth image, every ``stride``-th pixel."""
    d = np.asarray(depth, dtype=np.float64)[::stride, ::stride]
    v, u = np.mgrid[0:depth.shape[0]:stride, 0:depth.shape[1]:stride]
    ok = np.isfinite(d) & (d > 0)
    z = d[ok]
    pc = np.stack([(u[ok] - cx) / fx * z, (v[ok] - cy) / fy * z, z], axis=1)
    T = np.asarray(T_wc, dtype=np.float64).reshape(4, 4)
    return pc @ T[:3, :3].T + T[:3, 3]


def chamfer(recon: np.ndarray, truth: np.ndarray, f_threshold: float = 0.1) -> dict:
    """Accuracy, completeness, Chamfer-L1 and F-score of point sets recon and truth (metres)."""
    from scipy.spatial import cKDTree
    if len(recon) == 0 or len(truth) == 0:
        return dict(acc=float("inf"), comp=float("inf"), chamfer=float("inf"), fscore=0.0)
    d_rt = cKDTree(truth).query(recon, workers=-1)[0]
    d_tr = cKDTree(recon).query(truth, workers=-1)[0]
    p = float(np.mean(d_rt < f_threshold))
    r = float(np.mean(d_tr < f_threshold))
    acc, comp = float(d_rt.mean()), float(d_tr.mean())
    return dict(acc=acc, comp=comp, chamfer=0.5 * (acc + comp), fscore=0.0 if p + r == 0 else 2 * p * r / (p + r))
