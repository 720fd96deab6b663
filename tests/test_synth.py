"""The seeded input generator draws the network shapes the paper describes
(Extended Data Table 2): fixed in-degree, uniform sources without autapses
or multapses, 4:1 E/I, cross-region sources excitatory, rows sorted by
(delay, target)."""
import numpy as np

import synth


def _check(g, k_in, k_within, d_within, d_cross):
    N = g.n_neurons
    rp = np.asarray(g.row_ptr)
    col = np.asarray(g.col)
    d = np.asarray(g.delay)
    src = np.repeat(np.arange(N), np.diff(rp))
    assert rp[0] == 0 and rp[-1] == N * k_in and np.all(np.diff(rp) >= 0)
    assert np.all(src != col)
    assert np.all(np.bincount(col, minlength=N) == k_in)
    key = src.astype(np.int64) * N + col
    assert len(np.unique(key)) == len(key)
    # rows sorted by (delay, target)
    rk = d.astype(np.int64) * N + col
    same = src[1:] == src[:-1]
    assert np.all(rk[1:][same] > rk[:-1][same])
    region = np.searchsorted(g.region_offsets, np.arange(N), side="right") - 1
    within = region[src] == region[col]
    per_tgt_within = np.bincount(col[within], minlength=N)
    assert np.all(per_tgt_within == k_within)
    assert np.all((d[within] >= d_within[0]) & (d[within] <= d_within[1]))
    if (~within).any():
        assert np.all((d[~within] >= d_cross[0]) & (d[~within] <= d_cross[1]))
        exc_end = g.region_offsets[:-1] + g.n_exc
        assert np.all(src[~within] < exc_end[region[src[~within]]])


def test_single_region_network(small_graph):
    g = small_graph
    assert g.n_neurons == 10_000 and list(g.n_exc) == [8000]
    _check(g, 100, 100, (1, 20), None)
    w = g.weights_f64()
    assert abs(np.log(w).mean() + 1.0) < 0.01 and abs(np.log(w).std() - 0.5) < 0.01


def test_multi_region_network_is_deterministic_and_thread_independent():
    a = synth.make_graph([300] * 5, 50, 11, k_within=40, d_within=(1, 50), d_cross=(50, 200),
                         threads=1)
    b = synth.make_graph([300] * 5, 50, 11, k_within=40, d_within=(1, 50), d_cross=(50, 200),
                         threads=4)
    for f in ("row_ptr", "col", "w_bf16", "delay"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    _check(a, 50, 40, (1, 50), (50, 200))


def test_region_matrix_density_and_rows():
    M = synth.region_matrix(100, 0.3, 5)
    assert np.allclose(M.sum(1), 1.0)
    assert np.all(np.diag(M) == 0)
    dens = (M > 0).sum() / (100 * 99)
    assert 0.27 < dens < 0.33


def test_bf16_round_trip():
    x = np.exp(np.random.default_rng(0).normal(-1, 0.5, 1000))
    b = synth.f64_to_bf16(x)
    y = synth.bf16_to_f64(b)
    assert np.all(np.abs(y - x) <= np.abs(x) * 2.0**-8)
    assert np.array_equal(synth.f64_to_bf16(y), b)
