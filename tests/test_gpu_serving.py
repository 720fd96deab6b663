"""Request server on the GPU: continuous batching must not change results.

Every request is an independent network; served in a mix -- admitted while
others run, on tiles another request used before, sharing a device graph --
it must give the same raster, BOLD samples and spike count, bit for bit, as
the same network created alone with dbnet_create (integer accumulation makes
delivery order-independent, and each request's Philox counter is its own
step index).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RUN = dict(tr_ms=20.0)


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _request(i, n, R, k, d_cross=(20, 60)):
    sizes = [n // R] * R
    sizes[-1] += n - sum(sizes)
    g = synth.make_graph(sizes, k, 900 + i, d_within=(1, 20), d_cross=d_cross)
    p = [synth.default_region_params(I_ext=0.85 + 0.02 * r) for r in range(R)]
    return g, p


def _alone(g, p, n_steps, seed, net_id):
    from paper_2211_15963_gb300 import dbnet
    net = dbnet.Network(g, p, dict(RUN, seed=seed, net_id=net_id, raster_capacity=1 << 20,
                                   bold_capacity=4096))
    net.step(n_steps)
    out = net.spikes(), net.bold(), net.stats()["spikes"]
    net.close()
    return out


def _check(srv, rid, ref):
    (st, ids), bold, nsp = ref
    s = srv.poll(rid)
    assert s["state"] == 2, s
    a_st, a_id = srv.spikes(rid)
    assert np.array_equal(a_st, st) and np.array_equal(a_id, ids)
    assert np.array_equal(srv.bold(rid), bold)
    assert s["spikes"] == nsp and len(st) == nsp
    assert s["latency_s"] >= s["run_s"] > 0.0


def test_requests_in_a_mix_equal_alone_runs():
    from paper_2211_15963_gb300 import dbnet
    reqs = [(_request(0, 3000, 2, 80), 1234, 11, 1),
            (_request(1, 5200, 3, 120), 777, 12, 2),
            (_request(2, 1500, 1, 60), 2000, 13, 3),
            (_request(3, 4100, 4, 100), 3001, 14, 4)]
    srv = dbnet.Server(max_neurons=1 << 15, max_requests=4, max_regions=32, max_delay=60,
                       chunk_steps=128, arena_bytes=1 << 30, run=RUN)
    ids = []
    for (g, p), n, seed, nid in reqs[:2]:
        ids.append(srv.submit(g, p, n, seed=seed, net_id=nid, raster_capacity=1 << 20))
    for _ in range(3):      # the first two are running when the others arrive
        srv.pump()
    assert srv.poll(ids[0])["state"] == 1
    for (g, p), n, seed, nid in reqs[2:]:
        ids.append(srv.submit(g, p, n, seed=seed, net_id=nid, raster_capacity=1 << 20))
    srv.drain()
    for rid, ((g, p), n, seed, nid) in zip(ids, reqs):
        _check(srv, rid, _alone(g, p, n, seed, nid))
    st = srv.stats()
    assert st["done"] == 4 and st["running"] == 0 and st["queued"] == 0
    assert st["events"] > 0
    srv.close()


def test_admission_waits_for_room_and_reuses_tiles():
    """Two tiles of room: the second request waits in the queue, then runs on
    the tiles the first one left after cooling down."""
    from paper_2211_15963_gb300 import dbnet
    (g, p) = _request(5, 1800, 2, 70)
    (h, q) = _request(6, 2000, 2, 90)
    srv = dbnet.Server(max_neurons=2048, max_requests=2, max_regions=8, max_delay=60,
                       chunk_steps=64, arena_bytes=256 << 20, run=RUN)
    a = srv.submit(g, p, 900, seed=3, net_id=7, raster_capacity=1 << 20)
    b = srv.submit(h, q, 700, seed=4, net_id=8, raster_capacity=1 << 20)
    srv.pump()
    assert srv.poll(a)["state"] == 1 and srv.poll(b)["state"] == 0
    srv.drain()
    assert srv.poll(b)["queued_s"] > 0
    _check(srv, a, _alone(g, p, 900, 3, 7))
    _check(srv, b, _alone(h, q, 700, 4, 8))
    srv.close()


def test_shared_graph_key_and_failed_neighbour():
    """Requests with one graph_key share a device copy; a request whose
    delays exceed the pool's ring fails alone."""
    from paper_2211_15963_gb300 import dbnet
    (g, p) = _request(7, 2500, 2, 100)
    (bad, pb) = _request(8, 1200, 2, 50, d_cross=(70, 90))   # delays above max_delay
    srv = dbnet.Server(max_neurons=1 << 14, max_requests=4, max_regions=16, max_delay=60,
                       chunk_steps=128, arena_bytes=512 << 20, run=RUN)
    a = srv.submit(g, p, 1500, seed=5, net_id=1, graph_key=42, raster_capacity=1 << 20)
    srv.pump()
    used_one = srv.stats()["arena_used"]
    b = srv.submit(g, p, 1100, seed=6, net_id=2, graph_key=42, raster_capacity=1 << 20)
    c = srv.submit(bad, pb, 500, seed=7, net_id=3)
    srv.pump()
    used_two = srv.stats()["arena_used"]
    # the second request adds its own buffers, not another copy of the edges
    assert used_two - used_one <= used_one - 6 * g.n_edges
    srv.drain()
    sc = srv.poll(c)
    assert sc["state"] == 3 and sc["error"] == dbnet.DBNET_EINVAL
    _check(srv, a, _alone(g, p, 1500, 5, 1))
    _check(srv, b, _alone(g, p, 1100, 6, 2))
    srv.release(a)
    with pytest.raises(dbnet.DbnetError):
        srv.poll(a)
    srv.close()


def test_random_stream_through_a_tight_pool():
    """Twelve random requests (sizes, regions, in-degrees, durations) arrive
    at random rounds into a pool too small for all of them: they queue,
    reuse tiles and region slots, and each still equals its run alone."""
    from paper_2211_15963_gb300 import dbnet
    rng = np.random.default_rng(123)
    reqs = []
    for i in range(12):
        n = int(rng.integers(800, 4000))
        R = int(rng.integers(1, 4))
        k = int(rng.integers(30, 90))
        g, p = _request(20 + i, n, R, k)
        reqs.append((g, p, int(rng.integers(200, 1500)), 100 + i, 50 + i, int(rng.integers(0, 12))))
    srv = dbnet.Server(max_neurons=8192, max_requests=3, max_regions=8, max_delay=60,
                       chunk_steps=64, arena_bytes=256 << 20, run=RUN)
    ids = {}
    for rnd in range(400):
        for i, r in enumerate(reqs):
            if r[5] == rnd:
                ids[i] = srv.submit(r[0], r[1], r[2], seed=r[3], net_id=r[4],
                                    raster_capacity=1 << 20)
        srv.pump()
        if len(ids) == len(reqs) and all(srv.poll(v)["state"] == 2 for v in ids.values()):
            break
    srv.drain()
    for i, (g, p, n, seed, nid, _) in enumerate(reqs):
        _check(srv, ids[i], _alone(g, p, n, seed, nid))
    srv.close()


def test_two_weight_requests_share_a_four_channel_pool():
    """A server created with four accumulator channels serves one-weight and
    two-weight requests together, each equal to its run alone; a server
    without them refuses a two-weight request at submission."""
    from paper_2211_15963_gb300 import dbnet
    (g, p) = _request(40, 2600, 2, 90)
    (h, q) = _request(41, 3100, 3, 110)
    h = synth.with_second_weight(h, 42)
    srv = dbnet.Server(max_neurons=1 << 14, max_requests=4, max_regions=16, max_delay=60,
                       chunk_steps=128, arena_bytes=512 << 20, run=RUN, two_weights=1)
    a = srv.submit(g, p, 1200, seed=9, net_id=1, raster_capacity=1 << 20)
    srv.pump()
    b = srv.submit(h, q, 900, seed=10, net_id=2, raster_capacity=1 << 20)
    srv.drain()
    _check(srv, a, _alone(g, p, 1200, 9, 1))
    _check(srv, b, _alone(h, q, 900, 10, 2))
    srv.close()
    plain = dbnet.Server(max_neurons=1 << 13, max_requests=2, max_regions=8, max_delay=60,
                         chunk_steps=64, arena_bytes=256 << 20, run=RUN)
    with pytest.raises(dbnet.DbnetError) as ei:
        plain.submit(h, q, 100, seed=1)
    assert ei.value.code == dbnet.DBNET_EUNSUPPORTED
    plain.close()
