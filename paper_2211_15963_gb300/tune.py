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


# ------------------------------------------------------------------------
# Conductance initialisation (Supplementary Algorithm 1).
#
# Step 1 computes the target synaptic current of each channel from two
# rates.  The leak is linearised at the middle of the voltage range,
# I_leak = -gL ((V_th + V_reset) / 2 - V_L), so a neuron that climbs from
# V_reset to V_th under a constant total current I fires at
# r(I) = 1 / (T_ref + C (V_th - V_reset) / (I + I_leak)).  The excitatory
# current is the one that gives r_max with no inhibition, the inhibitory
# current the one that brings the rate down to r_normal, both net of the
# constant injected current (and the mean OU current, where on).  The
# excitatory current is split 0.3 / 0.7 over AMPA / NMDA (less of the fast
# channel, against collective oscillation), the inhibitory current 0.5 / 0.5
# over GABA_A / GABA_B.  Steps 2-8 run the model, measure the mean current
# of each channel, I_u = g_u J_u (V_u - V) averaged over neurons and time,
# and rescale g_u by target / measured until they agree.
EXC_SPLIT = (0.3, 0.7)
INH_SPLIT = (0.5, 0.5)


def channel_targets(p: dict, r_max_hz: float, r_normal_hz: float):
    """Step 1: target mean synaptic current (nA) of AMPA, NMDA, GABA_A, GABA_B."""
    C, gL, VL = p["C"], p["gL"], p["VL"]
    Vth, Vr, Tref = p["Vth"], p["Vreset"], p["Tref"]
    i_leak = -gL * ((Vth + Vr) / 2.0 - VL)
    i_other = p["I_ext"] + (p.get("ou_mu", 0.0) if p.get("ou_sigma", 0.0) or p.get("ou_mu", 0.0) else 0.0)

    def total_for(r_hz):
        climb = 1000.0 / r_hz - Tref  # ms from reset to threshold
        if climb <= 0:
            raise ValueError("rate above 1 / T_ref")
        return C * (Vth - Vr) / climb - i_leak

    i_exc = total_for(r_max_hz) - i_other
    i_inh = total_for(r_normal_hz) - i_other - i_exc
    return (EXC_SPLIT[0] * i_exc, EXC_SPLIT[1] * i_exc, INH_SPLIT[0] * i_inh, INH_SPLIT[1] * i_inh)


def measure_channel_currents(sim, p: dict, warm_steps: int, steps: int, every: int):
    """Mean I_u = g_u J_u (V_u - V) over neurons, sampled every `every` steps
    after `warm_steps`.  `sim` has step(n) and state() -> (V, J[4][N], ref)."""
    import numpy as np
    sim.step(warm_steps)
    acc = np.zeros(4)
    n = 0
    for _ in range(max(steps // every, 1)):
        sim.step(every)
        V, J, _ = sim.state()
        V = np.asarray(V, dtype=np.float64)
        J = np.asarray(J, dtype=np.float64)
        for u in range(4):
            acc[u] += np.mean(p["g_u"][u] * J[u] * (p["Vu"][u] - V))
        n += 1
    return acc / n


def init_conductances(make_sim, p: dict, r_max_hz: float, r_normal_hz: float, *, iters: int = 8,
                      tol: float = 0.05, warm_steps: int = 1000, steps: int = 1000,
                      every: int = 10, step_exp: float = 0.5, max_factor: float = 2.0):
    """Supplementary Algorithm 1.  make_sim(params) builds a simulator
    (a dbnet.Network or an oracle.Sim) of one network whose regions all use
    `params`.  Each iteration multiplies g_u by (target / measured) ** step_exp,
    clipped to [1 / max_factor, max_factor]: the paper's step is step_exp = 1,
    which in a recurrent network near its transition swings between a silent
    and a runaway state, so the default takes half the logarithmic step.
    Returns (g_u, history of (g_u, measured currents), targets)."""
    target = channel_targets(p, r_max_hz, r_normal_hz)
    q = dict(p)
    hist = []
    for _ in range(iters):
        sim = make_sim(q)
        try:
            cur = measure_channel_currents(sim, q, warm_steps, steps, every)
        finally:
            if hasattr(sim, "close"):
                sim.close()
        hist.append((tuple(q["g_u"]), tuple(float(c) for c in cur)))
        ratio = [t / c if c * t > 0 else max_factor for t, c in zip(target, cur)]
        if all(abs(c / t - 1.0) < tol for t, c in zip(target, cur)):
            break
        g = [gu * min(max(r ** step_exp, 1.0 / max_factor), max_factor)
             for gu, r in zip(q["g_u"], ratio)]
        q["g_u"] = tuple(g)
    return tuple(q["g_u"]), hist, target
