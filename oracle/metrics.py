"""Evaluation metrics -- oracle side (TEST INFRASTRUCTURE ONLY).

``lagged_pcc`` is the lagged Pearson correlation of Supplementary Sec. 6
("Correlation coefficients"): pcc(x_model(t + lag), x_exp(t)); the paper
uses lag = 2 TR.  ``isi_cv`` and ``rates`` summarise rasters for the
long-run statistical comparisons.
"""
from __future__ import annotations

import numpy as np


def pcc(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    da = a - a.mean()
    db = b - b.mean()
    return float((da * db).sum() / np.sqrt((da * da).sum() * (db * db).sum()))


def lagged_pcc(x_model: np.ndarray, x_exp: np.ndarray, lag: int = 2) -> float:
    T = len(x_exp)
    assert len(x_model) == T and 0 <= lag < T - 1
    return pcc(x_model[lag:], x_exp[:T - lag])


def rates_hz(steps: np.ndarray, ids: np.ndarray, n_neurons: int, n_steps: int, dt_ms: float):
    counts = np.bincount(ids, minlength=n_neurons)
    return counts / (n_steps * dt_ms * 1e-3)


def isi_cv(steps: np.ndarray, ids: np.ndarray, min_spikes: int = 3) -> float:
    """Mean coefficient of variation of the inter-spike intervals over neurons
    with at least `min_spikes` spikes."""
    order = np.lexsort((steps, ids))
    s = steps[order].astype(np.int64)
    i = ids[order]
    cvs = []
    bounds = np.flatnonzero(np.diff(i)) + 1
    for seg in np.split(np.arange(len(i)), bounds):
        if len(seg) >= min_spikes:
            isi = np.diff(s[seg]).astype(np.float64)
            if isi.mean() > 0:
                cvs.append(isi.std() / isi.mean())
    return float(np.mean(cvs)) if cvs else float("nan")
