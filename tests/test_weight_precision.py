"""What storing weights in BF16 costs (the device keeps one BF16 weight per
edge; the paper's connection table, Supplementary Table 5, holds float32).

The same network is run by the FP64 oracle twice: once with the BF16-rounded
weights every other test uses, once with the unrounded FP64 weights they
were rounded from (still accumulated as rint(w 2^16), an absolute error of
at most 2^-17 per edge, a hundred times below the BF16 step).  The network
is chaotic, so single trajectories part; the statistics must not.
"""
import dataclasses

import numpy as np

import oracle
import synth
from oracle import metrics

STEPS = 5000  # 0.5 s at dt = 0.1 ms


def test_bf16_weight_rounding_changes_statistics_little(small_graph):
    rng = np.random.default_rng(2026)
    w64 = rng.lognormal(-1.0, 0.5, small_graph.n_edges)
    g = dataclasses.replace(small_graph, w_bf16=synth.f64_to_bf16(w64))
    rel = np.abs(g.weights_f64() - w64) / w64
    assert rel.max() <= 2.0 ** -8 and rel.mean() > 2.0 ** -12   # BF16: 8 significant bits
    p = synth.default_region_params()
    a = oracle.Sim(g, p, seed=21, precision=64)
    b = oracle.Sim(g, p, seed=21, precision=64, weights_f64=w64)
    a.step(STEPS)
    b.step(STEPS)
    (sa, ia), (sb, ib) = a.raster(), b.raster()
    N = g.n_neurons
    ra = metrics.rates_hz(sa, ia, N, STEPS, 0.1).mean()
    rb = metrics.rates_hz(sb, ib, N, STEPS, 0.1).mean()
    assert len(ia) > 10_000
    assert abs(ra - rb) / rb < 0.02
    cva, cvb = metrics.isi_cv(sa, ia), metrics.isi_cv(sb, ib)
    assert abs(cva - cvb) / cvb < 0.05
    # population rate in 1 ms bins
    pa = np.bincount(sa // 10, minlength=STEPS // 10)[:STEPS // 10]
    pb = np.bincount(sb // 10, minlength=STEPS // 10)[:STEPS // 10]
    assert np.corrcoef(pa, pb)[0, 1] > 0.9
