"""Map quality as the paper measures it (Sec. IV): the area under the ROC curve
(AUC) and the negative log-likelihood (NLL) of labelled points under the
occupancy probabilities of their cells.  Host-side evaluation (NumPy)."""
from __future__ import annotations

import numpy as np


def auc(scores: np.ndarray, labels: np.ndarray) -> float:
    """ROC AUC by the rank statistic (Mann-Whitney U), ties counted half."""
    s = np.asarray(scores, np.float64).ravel()
    y = np.asarray(labels).ravel().astype(bool)
    n_pos, n_neg = int(y.sum()), int((~y).sum())
    if n_pos == 0 or n_neg == 0:
        return float("nan")
    order = np.argsort(s, kind="mergesort")
    ranks = np.empty(len(s), np.float64)
    ss = s[order]
    # average ranks over runs of equal scores
    edges = np.flatnonzero(np.diff(ss)) + 1
    starts = np.concatenate([[0], edges])
    ends = np.concatenate([edges, [len(ss)]])
    avg = (starts + ends + 1) / 2.0  # 1-based average rank of each run
    ranks[order] = np.repeat(avg, ends - starts)
    return float((ranks[y].sum() - n_pos * (n_pos + 1) / 2.0) / (n_pos * n_neg))


def nll(prob: np.ndarray, labels: np.ndarray, eps: float = 1e-7) -> float:
    """Mean negative log-likelihood of binary labels under probabilities prob."""
    p = np.clip(np.asarray(prob, np.float64).ravel(), eps, 1.0 - eps)
    y = np.asarray(labels).ravel().astype(np.float64)
    return float(-np.mean(y * np.log(p) + (1.0 - y) * np.log(1.0 - p)))


def point_cells(xy: np.ndarray, W: int, H: int, res: float, x_min: float, y_min: float):
    """Cell (i, j) of each point and a mask of the points inside the map."""
    xy = np.asarray(xy, np.float64)
    i = np.floor((xy[:, 0] - x_min) / res).astype(np.int64)
    j = np.floor((xy[:, 1] - y_min) / res).astype(np.int64)
    inside = (i >= 0) & (i < W) & (j >= 0) & (j < H)
    return i, j, inside


def evaluate(occ: np.ndarray, xy: np.ndarray, labels: np.ndarray, res: float, x_min: float,
             y_min: float) -> dict:
    """AUC and NLL of labelled points (1 = occupied) under the occupancy map occ [H][W]."""
    H, W = occ.shape
    i, j, inside = point_cells(xy, W, H, res, x_min, y_min)
    p = occ[j[inside], i[inside]]
    y = np.asarray(labels)[inside]
    return {"auc": auc(p, y), "nll": nll(p, y), "points": int(inside.sum())}
