"""The allocation-free entry point gives what the ordinary one gives.

dbnet_run_noalloc serves callers that cannot allocate device memory while
they run (an arena that owns the whole GPU, a loop that cannot pay for
cudaMalloc's synchronisation): its scratch is one static device array shared
by every call.  Two calls in a row, on different networks and seeds, must
each match dbnet_create + dbnet_step bit for bit (the same kernels run in the
same order, so the parity tolerance of the other GPU tests -- exact -- holds),
which also shows that each call starts from cleared scratch.  This file is
named to be collected last.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _run_noalloc(g, p, opts, n_steps, raster_cap=1 << 18):
    from paper_2211_15963_gb300 import dbnet
    dev = torch.device("cuda", 0)
    n_pad = (g.n_neurons + 1023) // 1024 * 1024
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)  # noqa: E731
    row_ptr = t(g.row_ptr, np.int64)
    col = t(g.col, np.int32)
    w = t(np.asarray(g.w_bf16).view(np.int16), np.int16)
    d = t(g.delay, np.uint8)
    V = torch.empty(n_pad, dtype=torch.float32, device=dev)
    J = torch.empty(4, n_pad, dtype=torch.float32, device=dev)
    ref = torch.empty(n_pad, dtype=torch.uint8, device=dev)
    rs = torch.empty(raster_cap, dtype=torch.int32, device=dev)
    ri = torch.empty(raster_cap, dtype=torch.int32, device=dev)
    n_sp, n_ev = dbnet.dbnet_run_noalloc(g.n_neurons, g.region_offsets, g.n_exc, row_ptr, col, w,
                                         d, p, opts, n_steps, V, J, ref, rs, ri)
    torch.cuda.synchronize()
    N = g.n_neurons
    k = min(n_sp, raster_cap)
    st, ids = rs[:k].cpu().numpy(), ri[:k].cpu().numpy()
    order = np.lexsort((ids, st))
    return (V[:N].cpu().numpy(), J[:, :N].cpu().numpy(), ref[:N].cpu().numpy().astype(np.int32),
            st[order], ids[order], n_sp, n_ev)


def _run_handle(g, p, opts, n_steps):
    from paper_2211_15963_gb300 import dbnet
    net = dbnet.Network(g, p, dict(opts, raster_capacity=1 << 18))
    net.step(n_steps)
    V, J, ref = net.state()
    st, ids = net.spikes()
    s = net.stats()
    net.close()
    return V, J, ref, st, ids, s["spikes"], s["events"]


def test_noalloc_matches_ordinary_entry_point_twice_in_a_row():
    g1 = synth.make_graph([1500, 700, 333, 2049], 80, 21, k_within=64, d_within=(1, 30),
                          d_cross=(30, 120))
    g2 = synth.small_network()
    cases = [(g1, [synth.default_region_params(I_ext=0.8 + 0.05 * r) for r in range(4)],
              dict(seed=4, net_id=1), 700),
             (g2, synth.default_region_params(), dict(seed=15964), 900)]
    for g, p, opts, n in cases:
        a = _run_noalloc(g, p, opts, n)
        b = _run_handle(g, p, opts, n)
        names = ("V", "J", "ref", "raster steps", "raster ids", "spikes", "events")
        assert a[5] > 100
        for name, x, y in zip(names, a, b):
            assert np.array_equal(np.asarray(x), np.asarray(y)), name


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2211_15963_gb300 import dbnet
    N = 70_000
    n_pad = (N + 1023) // 1024 * 1024
    dev = torch.device("cuda", 0)
    z64 = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    z32 = torch.zeros(1, dtype=torch.int32, device=dev)
    zw = torch.zeros(1, dtype=torch.int16, device=dev)
    zd = torch.zeros(1, dtype=torch.uint8, device=dev)
    V = torch.empty(n_pad, dtype=torch.float32, device=dev)
    J = torch.empty(4 * n_pad, dtype=torch.float32, device=dev)
    ref = torch.empty(n_pad, dtype=torch.uint8, device=dev)
    with pytest.raises(dbnet.DbnetError) as ei:
        dbnet.dbnet_run_noalloc(N, [0, N], [N], z64, z32, zw, zd, synth.default_region_params(),
                                {}, 10, V, J, ref)
    assert ei.value.code == dbnet.DBNET_ERANGE and "limit" in str(ei.value)


def _device_graph(g):
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)  # noqa: E731
    return dict(row_ptr=t(g.row_ptr, np.int64), col=t(g.col, np.int32),
                w=t(np.asarray(g.w_bf16).view(np.int16), np.int16), d=t(g.delay, np.uint8))


def _state(n):
    dev = torch.device("cuda", 0)
    n_pad = (n + 1023) // 1024 * 1024
    return (torch.empty(n_pad, dtype=torch.float32, device=dev),
            torch.empty(4 * n_pad, dtype=torch.float32, device=dev),
            torch.empty(n_pad, dtype=torch.uint8, device=dev))


@pytest.mark.parametrize("fault", ["target", "zero_delay", "delay_order", "negative_weight",
                                   "infinite_weight"])
def test_noalloc_validates_the_device_graph_then_runs_cleanly(fault):
    """The device-side checks of the allocation-free entry point (its own
    validation kernel, separate from dbnet_create's ingest): a graph that
    breaks one rule is rejected with DBNET_EINVAL, and a valid call right
    after still equals the ordinary entry point, so the shared scratch is
    cleared after an error."""
    from paper_2211_15963_gb300 import dbnet
    g = synth.make_graph([300, 212], 30, 5, k_within=24, d_within=(1, 9), d_cross=(9, 25))
    dg = _device_graph(g)
    row = 17
    a, b = int(g.row_ptr[row]), int(g.row_ptr[row + 1])
    assert b - a >= 2
    if fault == "target":
        dg["col"][a] = g.n_neurons
    elif fault == "zero_delay":
        dg["d"][a] = 0
    elif fault == "delay_order":
        dg["d"][a] = int(g.delay[b - 1]) + 1
    elif fault == "negative_weight":
        dg["w"][a] = -16512   # 0xBF80: -1.0 in BF16
    else:
        dg["w"][a] = 32640    # 0x7F80: +inf in BF16
    V, J, ref = _state(g.n_neurons)
    p = synth.default_region_params()
    with pytest.raises(dbnet.DbnetError) as ei:
        dbnet.dbnet_run_noalloc(g.n_neurons, g.region_offsets, g.n_exc, dg["row_ptr"], dg["col"],
                                dg["w"], dg["d"], p, dict(seed=2), 50, V, J, ref)
    assert ei.value.code == dbnet.DBNET_EINVAL
    a1 = _run_noalloc(g, p, dict(seed=2), 300)
    b1 = _run_handle(g, p, dict(seed=2), 300)
    assert a1[5] > 0
    for x, y in zip(a1, b1):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_noalloc_rejects_a_ring_beyond_its_limit_and_unaligned_state():
    from paper_2211_15963_gb300 import dbnet
    # 65,536 neurons with a delay of 64 steps need 65,536 x 65 ring entries > 2^22
    N = 65_536
    g = synth.make_graph([N], 2, 9, d_within=(64, 64))
    dg = _device_graph(g)
    V, J, ref = _state(N)
    p = synth.default_region_params()
    with pytest.raises(dbnet.DbnetError) as ei:
        dbnet.dbnet_run_noalloc(N, g.region_offsets, g.n_exc, dg["row_ptr"], dg["col"], dg["w"],
                                dg["d"], p, {}, 5, V, J, ref)
    assert ei.value.code == dbnet.DBNET_ERANGE and "ring" in str(ei.value)
    # V that does not start on a 16-byte boundary
    g2 = synth.make_graph([500], 10, 3, d_within=(1, 5))
    dg2 = _device_graph(g2)
    V2, J2, ref2 = _state(500)
    Vbig = torch.empty(1024 + 4, dtype=torch.float32, device=V2.device)
    with pytest.raises(dbnet.DbnetError) as ei:
        dbnet.dbnet_run_noalloc(500, g2.region_offsets, g2.n_exc, dg2["row_ptr"], dg2["col"],
                                dg2["w"], dg2["d"], p, {}, 5, Vbig[1:], J2, ref2)
    assert ei.value.code == dbnet.DBNET_EINVAL and "aligned" in str(ei.value)
