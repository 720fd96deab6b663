"""The benchmark's own workload, in the benchmark's launch configuration,
against the oracle element by element.

The mid-size network (2,000,000 neurons in 100 regions of 20,000, in-degree
1,000, delays 1-50 steps within and 50-200 across regions, ~15 Hz drive) is
built by the same generator and seed, with the same parameters and options,
and stepped the way the benchmark steps it: on its own stream, replayed from
the captured 64-step graph, with the delivery grid autotuned part-way.  Over
the first 200 steps (every delay the graph has comes due at least once) the
raster, the membrane potentials, traces and refractory counters must equal
the matched-FP32 oracle bit for bit, the synaptic events (spikes times
out-degree) must equal the oracle's, and the FP64 Balloon-Windkessel state
must agree to 1e-12.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEPS = 200


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_mid_network_first_200_steps_bit_exact():
    import bench
    from paper_2211_15963_gb300 import dbnet
    seed = synth.seed_for(1)
    g = synth.make_graph([20000] * 100, 1000, seed, k_within=800, d_within=(1, 50),
                         d_cross=(50, 200))
    params = bench.params_for(15, 1000)
    stream = torch.cuda.Stream(torch.device("cuda", 0))
    net = dbnet.Network(g, params, dict(seed=seed + 1, net_id=0, autotune_at=64,
                                        raster_capacity=1 << 24), stream)
    # 64 plain steps, then the launch-shape tuner's chunks (each candidate
    # grid and schedule in turn, captured graphs) and a tail of direct steps
    net.step(STEPS)
    assert net.stats()["emit_delay"] == 0
    o = oracle.Sim(g, params, seed=seed + 1, net_id=0, precision=32)
    o.step(STEPS)

    st, ids = net.spikes()
    rs, rids = o.raster()
    assert len(ids) > 100_000
    assert np.array_equal(st, rs) and np.array_equal(ids, rids)
    V, J, ref = net.state()
    Vo, Jo, refo = o.state()
    assert np.array_equal(V.astype(np.float64), Vo)
    assert np.array_equal(J.astype(np.float64), Jo)
    assert np.array_equal(ref, refo)
    s, so = net.stats(), o.info()
    assert s["spikes"] == so["spikes"] == len(rids)
    # the device counts an event when it comes due, the oracle when its spike
    # is emitted: compare with the edges due by the last step
    assert s["events"] == so["events"]   # spikes x out-degree, counted at emission
    assert s["events"] > 100_000_000
    assert np.allclose(net.bw(), o.bw_state(), rtol=1e-12, atol=1e-15)
    net.close()


def test_graph_beyond_2_31_edges_bit_exact():
    """The paths only the largest networks take: 2,200,000 neurons (110
    regions of 20,000) at in-degree 1,000 give 2.2e9 edges, so rows start
    beyond edge 2^31 and record byte offsets beyond 2^32 (int64 row
    pointers, 64-bit record addressing in ingest and delivery).  The graph is
    ingested from pageable host memory as the largest benchmark does.
    Raster, state and synaptic events equal the matched-FP32 oracle over 120
    steps."""
    import bench
    from paper_2211_15963_gb300 import dbnet
    seed = synth.seed_for(4) + 7
    g = synth.make_graph([20000] * 110, 1000, seed, k_within=800, d_within=(1, 50),
                         d_cross=(50, 200))
    assert g.n_edges > 2**31
    params = bench.params_for(15, 1000)
    stream = torch.cuda.Stream(torch.device("cuda", 0))
    steps = 120
    net = dbnet.Network(g, params, dict(seed=seed + 1, raster_capacity=1 << 24), stream)
    net.step(steps)
    o = oracle.Sim(g, params, seed=seed + 1, precision=32)
    o.step(steps)
    st, ids = net.spikes()
    rs, rids = o.raster()
    assert len(ids) > 50_000 and int(rids.max()) > 2_100_000
    assert np.array_equal(st, rs) and np.array_equal(ids, rids)
    V, J, ref = net.state()
    Vo, Jo, refo = o.state()
    assert np.array_equal(V.astype(np.float64), Vo)
    assert np.array_equal(J.astype(np.float64), Jo)
    assert np.array_equal(ref, refo)
    assert net.stats()["events"] == o.info()["events"]
    net.close()
