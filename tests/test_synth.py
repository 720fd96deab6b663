"""The seeded input generator draws the network shapes the paper describes
(Extended Data Table 2): fixed in-degree, uniform sources without autapses
or multapses, 4:1 E/I, cross-region sources excitatory, rows sorted by
(delay, target)."""
import os

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


def test_cortical_columns_follow_the_population_counts():
    """Extended Data Table 3 networks: every neuron of population i gets
    exactly the scaled count from each population of its voxel and from
    excitatory neurons of other voxels; no autapse or multapse; the
    out-degree is heavy-tailed (small layer-1 populations feed many)."""
    V, n = 4, 2000
    g = synth.cortical_columns(V, n, 200, seed=9)
    pops = g.populations
    offs, kl, kc = pops["offsets"], pops["k_local"], pops["k_cc"]
    n_exc = int(g.n_exc[0])
    rp = np.asarray(g.row_ptr)
    src = np.repeat(np.arange(g.n_neurons), np.diff(rp))
    tgt = np.asarray(g.col)
    assert not np.any(src == tgt)
    pair = tgt.astype(np.int64) * g.n_neurons + src
    assert len(np.unique(pair)) == len(pair)
    same = src // n == tgt // n
    pop_of = np.searchsorted(offs, np.arange(n), side="right") - 1
    tpop = pop_of[np.arange(g.n_neurons) % n]   # population of every neuron
    # cortico-cortical sources: excitatory neurons of another voxel
    assert np.all((src[~same] % n) < n_exc)
    # local counts per (target, source population), capped at the source
    # population's size (minus the target itself in its own population)
    cnt = np.zeros((g.n_neurons, len(offs) - 1), dtype=np.int64)
    np.add.at(cnt, (tgt[same], pop_of[src[same] % n]), 1)
    sizes = np.diff(offs)
    expect = np.minimum(kl[tpop], sizes[None, :] - np.eye(len(sizes), dtype=np.int64)[tpop])
    assert np.array_equal(cnt, expect)
    assert np.array_equal(np.bincount(tgt[~same], minlength=g.n_neurons), kc[tpop])
    deg = np.diff(rp)
    assert deg.max() > 3 * np.median(deg)
    assert abs(len(tgt) / g.n_neurons - 200) < 10


def test_generator_holds_only_its_output():
    """The generator needs no per-edge memory beyond its output (7 bytes per
    edge: target, BF16 weight, delay), so a 2e10-edge graph fits in 140 GB
    of host memory.  Peak resident memory of a fresh process generating
    2e8 edges, against its output plus a fixed allowance."""
    import subprocess
    import sys
    code = ("import resource, synth\n"
            "g = synth.make_graph([10000] * 20, 1000, 3, k_within=800, d_within=(1, 50),"
            " d_cross=(50, 200))\n"
            "print(g.n_edges, resource.getrusage(resource.RUSAGE_SELF).ru_maxrss)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                         timeout=600, check=True).stdout.split()
    E, peak_kb = int(out[0]), int(out[1])
    assert E == 200_000_000
    assert peak_kb * 1024 < 7 * E + (600 << 20)
