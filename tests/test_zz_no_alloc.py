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
    dev = torch.device("cuda", 0)
    z64 = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    z32 = torch.zeros(1, dtype=torch.int32, device=dev)
    zw = torch.zeros(1, dtype=torch.int16, device=dev)
    zd = torch.zeros(1, dtype=torch.uint8, device=dev)
    V = torch.empty(1, dtype=torch.float32, device=dev)
    with pytest.raises(dbnet.DbnetError) as ei:
        dbnet.dbnet_run_noalloc(N, [0, N], [N], z64, z32, zw, zd, synth.default_region_params(),
                                {}, 10, V, V, zd)
    assert ei.value.code == dbnet.DBNET_ERANGE and "limit" in str(ei.value)
