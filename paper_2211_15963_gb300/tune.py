"""Drive tuning for a target firing rate.

The paper initialises its conductances iteratively until the network fires
at the wanted rate (Supplementary Algorithm 1: run the model, compare the
obtained synaptic current with the wanted one, rescale, repeat).  Here the
knob is the background drive (``w_ext`` by default) and the comparison is the
steady-state population rate; the search is a bisection on the logarithm of
the knob, each evaluation a short simulation on the GPU through the C ABI.
"""
from __future__ import annotations

import math

from . import dbnet


def measure_rate(graph, params, *, sim_ms: float = 300.0, measure_ms: float = 200.0,
                 dt_ms: float = 0.1, seed: int = 1, stream=None) -> float:
    """Mean rate (Hz) over the last measure_ms of a sim_ms run."""
    n_total = int(round(sim_ms / dt_ms))
    n_meas = int(round(measure_ms / dt_ms))
    net = dbnet.Network(graph, params, dict(dt_ms=dt_ms, seed=seed), stream)
    try:
        net.step(n_total - n_meas)
        s0 = net.stats()["spikes"]
        net.step(n_meas)
        s1 = net.stats()["spikes"]
    finally:
        net.close()
    return (s1 - s0) / graph.n_neurons / (measure_ms * 1e-3)


def tune_drive(graph, params: dict, target_hz: float, *, knob: str = "w_ext", lo: float = 0.05,
               hi: float = 50.0, iters: int = 12, rel_tol: float = 0.03, **kw):
    """Bisection on log(knob) until the rate is within rel_tol of target_hz.
    Returns (knob value, rate reached, history)."""
    hist = []

    def rate_at(v):
        p = dict(params)
        p[knob] = v
        r = measure_rate(graph, p, **kw)
        hist.append((v, r))
        return r

    a, b = math.log(lo), math.log(hi)
    best = None
    for _ in range(iters):
        m = 0.5 * (a + b)
        r = rate_at(math.exp(m))
        if best is None or abs(r - target_hz) < abs(best[1] - target_hz):
            best = (math.exp(m), r)
        if abs(r - target_hz) <= rel_tol * target_hz:
            break
        if r < target_hz:
            a = m
        else:
            b = m
    return best[0], best[1], hist
