"""The C-ABI library loads and exports every entry point include/dbnet.h
declares, and rejects malformed inputs on the host before any device work
(these tests make no compute calls and run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from paper_2211_15963_gb300 import dbnet

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b((?:dbnet|ens|dbsrv)_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return dbnet.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 18
    raw = ctypes.CDLL(dbnet.library_path())
    for n in names:
        assert hasattr(raw, n), n
    assert set(names) <= set(dbnet._SIGS), "binding misses a declared function"


def test_strerror_and_defaults(lib):
    for code in range(0, -9, -1):
        assert lib.dbnet_strerror(code)
    o = dbnet.dbnet_options_default()
    assert o.dt_ms == 0.1 and o.bin_ms == 1.0 and o.tr_ms == 800.0 and o.precision == 32
    assert abs(o.bw_rho - 0.34) < 1e-15 and o.bold_capacity == 4096
    assert o.autotune_at == 2000


def _tiny_graph():
    W = np.zeros((6, 6))
    W[1, 0] = 0.5
    W[2, 1] = 0.25
    return synth.graph_from_dense(W, np.full((6, 6), 2), [4, 2])


def _expect(code, graph, params=None, **opts):
    params = params or synth.default_region_params()
    with pytest.raises(dbnet.DbnetError) as ei:
        dbnet.dbnet_create(graph, params, opts)
    assert ei.value.code == code, str(ei.value)


def test_host_validation_rejects_malformed_inputs(lib):
    g = _tiny_graph()
    bad = _tiny_graph()
    bad.region_offsets = np.array([0, 4, 7], dtype=np.int32)
    _expect(dbnet.DBNET_EINVAL, bad)
    bad = _tiny_graph()
    bad.region_offsets = np.array([0, 6, 6], dtype=np.int32)
    _expect(dbnet.DBNET_EINVAL, bad)
    bad = _tiny_graph()
    bad.n_exc = np.array([5, 1], dtype=np.int32)
    _expect(dbnet.DBNET_EINVAL, bad)
    bad = _tiny_graph()
    bad.row_ptr = bad.row_ptr.copy()
    bad.row_ptr[3] = bad.row_ptr[4] + 1
    _expect(dbnet.DBNET_EINVAL, bad)
    _expect(dbnet.DBNET_EINVAL, g, synth.default_region_params(C=0.0))
    _expect(dbnet.DBNET_EINVAL, g, synth.default_region_params(tau_u=(2.0, -1.0, 10.0, 100.0)))
    _expect(dbnet.DBNET_EINVAL, g, synth.default_region_params(Tref=30.0))  # 300 steps > 255
    _expect(dbnet.DBNET_EINVAL, g, synth.default_region_params(w_ext=-1.0))
    _expect(dbnet.DBNET_EINVAL, g, bin_ms=0.25)
    _expect(dbnet.DBNET_EINVAL, g, tr_ms=800.5)
    _expect(dbnet.DBNET_EUNSUPPORTED, g, precision=64)
    _expect(dbnet.DBNET_EINVAL, g, fixed_shift=31)
    _expect(dbnet.DBNET_EINVAL, g, autotune_at=-2)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(dbnet, "_lib", None)
    monkeypatch.setattr(dbnet, "_SO", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        dbnet.lib()


def test_ensemble_host_validation(lib):
    g = _tiny_graph()
    p = synth.default_region_params()
    th = np.zeros((3, 2, 2))

    def expect(code, M=3, theta=th, **k):
        with pytest.raises(dbnet.DbnetError) as ei:
            dbnet.ens_create(g, p, M, theta if theta.shape[0] == M else np.zeros((M, 2, 2)), {},
                             dbnet.enkf_options(**k))
        assert ei.value.code == code, str(ei.value)

    expect(dbnet.DBNET_EINVAL, M=1)
    expect(dbnet.DBNET_EINVAL, obs_var=0.0)
    expect(dbnet.DBNET_EINVAL, gamma=1.5)
    expect(dbnet.DBNET_EINVAL, rw_sigma=-1.0)
    expect(dbnet.DBNET_EINVAL, theta_lo=1.0, theta_hi=0.0)
    expect(dbnet.DBNET_EINVAL, mode=7)
    expect(dbnet.DBNET_EINVAL, theta=np.full((3, 2, 2), np.nan))


def test_server_host_validation(lib):
    """dbsrv_create checks its options on the host before touching a device."""
    for bad in (dict(max_requests=0), dict(max_delay=0), dict(max_delay=256),
                dict(chunk_steps=0), dict(arena_bytes=1024), dict(max_neurons=0),
                dict(two_weights=2)):
        with pytest.raises(dbnet.DbnetError) as ei:
            dbnet.Server(**bad)
        assert ei.value.code == dbnet.DBNET_EINVAL, bad
    o = dbnet.dbsrv_options_default()
    assert o.max_requests == 64 and o.max_delay == 255 and o.chunk_steps == 256
    assert o.run.dt_ms == 0.1 and o.run.autotune_at == 2000


def test_ou_parameters_are_validated(lib):
    g = _tiny_graph()
    _expect(dbnet.DBNET_EINVAL, g, synth.default_region_params(ou_mu=0.5, ou_tau=0.0))
    _expect(dbnet.DBNET_EINVAL, g, synth.default_region_params(ou_sigma=-0.1, ou_tau=5.0))
    _expect(dbnet.DBNET_EINVAL, g, synth.default_region_params(ou_mu=float("nan"), ou_tau=5.0))


def test_enkf_targets_are_validated(lib):
    g = _tiny_graph()
    p = synth.default_region_params()
    th = np.zeros((3, 2, 2))
    for tgt in [(7, 0), (-2, 0), (dbnet.DBENS_T_IEXT, dbnet.DBENS_T_IEXT),
                (dbnet.DBENS_T_GABA_A, dbnet.DBENS_T_DEFAULT)]:
        with pytest.raises(dbnet.DbnetError) as ei:
            dbnet.ens_create(g, p, 3, th, {}, dbnet.enkf_options(target=tgt))
        assert ei.value.code == dbnet.DBNET_EINVAL, tgt
    _expect(dbnet.DBNET_EINVAL, g, synth.default_region_params(iext_shape=-1.0))


def test_struct_layouts_match_the_library(lib):
    """Every ctypes mirror has the size the C compiler gave the struct (a
    field added on one side only shifts everything after it)."""
    import ctypes
    sizes = dbnet.abi_sizes()
    assert set(sizes) == set(dbnet.ABI_STRUCTS)
    for name, size in sizes.items():
        assert ctypes.sizeof(getattr(dbnet, name)) == size, name


class _FakeCudaTensor:
    """Stands in for a CUDA tensor in the wrapper's argument checks (no GPU
    here, and the checks read only metadata)."""

    def __init__(self, dtype, n, device=0, contiguous=True, cuda=True):
        self.dtype, self._n, self._contig, self.is_cuda = dtype, n, contiguous, cuda

        class _D:
            index = device
        self.device = _D()

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._contig


def _noalloc_args(N=3000, E=9000):
    import torch
    n_pad = (N + 1023) // 1024 * 1024
    F = _FakeCudaTensor
    return dict(n_neurons=N, region_offsets=[0, 1000, N], n_exc=[800, 1600],
                row_ptr=F(torch.int64, N + 1), col=F(torch.int32, E), weight_bf16=F(torch.int16, E),
                delay=F(torch.uint8, E), V=F(torch.float32, n_pad), J=F(torch.float32, 4 * n_pad),
                ref=F(torch.uint8, n_pad), raster_step=F(torch.int32, 100),
                raster_id=F(torch.int32, 100), n_edges=E)


def test_noalloc_wrapper_rejects_mismatched_tensors_without_touching_a_gpu(monkeypatch):
    """dbnet_run_noalloc receives bare device pointers, so its binding checks
    dtype, length, contiguity and device of every tensor first; none of
    these cases reaches the library."""
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(dbnet, "_current_device", lambda: 0)
    F = _FakeCudaTensor
    dbnet.noalloc_check(**_noalloc_args())  # the well-formed case passes
    n_pad = 3072
    bad = {
        "row_ptr": F(torch.int32, 3001),             # int32 row pointers
        "col": F(torch.int32, 8999),                 # one edge short
        "weight_bf16": F(torch.float32, 9000),       # float weights
        "delay": F(torch.int32, 9000),               # wide delays
        "V": F(torch.float32, 3000),                 # not padded to whole tiles
        "J": F(torch.float32, 3 * n_pad),            # three channels
        "ref": F(torch.int32, n_pad),                # wide refractory counters
        "raster_id": F(torch.int32, 99),             # shorter than raster_step
    }
    for name, t in bad.items():
        a = _noalloc_args()
        a[name] = t
        with pytest.raises(ValueError):
            dbnet.noalloc_check(**a)
    for t in (F(torch.float32, n_pad, device=1), F(torch.float32, n_pad, contiguous=False),
              F(torch.float32, n_pad, cuda=False)):
        a = _noalloc_args()
        a["V"] = t
        with pytest.raises(ValueError):
            dbnet.noalloc_check(**a)
    a = _noalloc_args()
    a["region_offsets"] = [0, 3000]                 # one entry short for two regions
    with pytest.raises(ValueError):
        dbnet.noalloc_check(**a)
    a = _noalloc_args()
    a["raster_id"] = None
    with pytest.raises(ValueError):
        dbnet.noalloc_check(**a)
