"""ctypes binding of include/dbnet.h.

Argument marshalling only: every step of the simulation runs in the CUDA
library (libdbnet.so, built in place by ``_build.build``).  The functions
carry the C names; ``Network`` and ``Ensemble`` are small owners of a handle.
Host arrays may be numpy arrays or CPU torch tensors (pinned ones included);
a CUDA stream may be given as a ``torch.cuda.Stream``, an integer handle or
None (the library then uses a stream of its own).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdbnet.so")
_lock = threading.Lock()
_lib = None

DBNET_OK = 0
DBNET_EINVAL = -1
DBNET_ENOMEM = -2
DBNET_ECUDA = -3
DBNET_ETIMEOUT = -4
DBNET_EOVERFLOW = -5
DBNET_ESTATE = -6
DBNET_ERANGE = -7
DBNET_EUNSUPPORTED = -8
DBNET_WEIGHT_F32 = 0
DBNET_WEIGHT_BF16 = 1
DBNET_SCHEDULE_AUTO, DBNET_SCHEDULE_SEQUENTIAL, DBNET_SCHEDULE_PIPELINED, DBNET_SCHEDULE_PERSISTENT = \
    0, 1, 2, 3
DBENS_DIFFUSION = 0
DBENS_GLOBAL = 1

_d, _i32, _i64, _u64, _vp = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p


dbnet_alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
dbnet_free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                 ctypes.c_void_p)


class dbnet_allocator_t(ctypes.Structure):
    _fields_ = [("alloc", dbnet_alloc_fn), ("free", dbnet_free_fn), ("ctx", ctypes.c_void_p)]


class dbnet_graph_t(ctypes.Structure):
    _fields_ = [("n_neurons", _i32), ("n_regions", _i32), ("region_offsets", _vp),
                ("n_exc", _vp), ("row_ptr", _vp), ("col", _vp), ("weight", _vp),
                ("weight_dtype", _i32), ("delay", _vp), ("weight2", _vp)]


class dbnet_region_params_t(ctypes.Structure):
    _fields_ = [("C", _d), ("gL", _d), ("VL", _d), ("Vth", _d), ("Vreset", _d), ("Tref", _d),
                ("Vu", _d * 4), ("tau_u", _d * 4), ("g_u", _d * 4), ("I_ext", _d),
                ("drive_rate_hz", _d), ("drive_K", _d), ("w_ext", _d),
                ("ou_mu", _d), ("ou_sigma", _d), ("ou_tau", _d), ("iext_shape", _d)]


class dbnet_options_t(ctypes.Structure):
    _fields_ = [("dt_ms", _d), ("bin_ms", _d), ("tr_ms", _d), ("z_scale", _d),
                ("bw_kappa", _d), ("bw_gamma", _d), ("bw_tau", _d), ("bw_alpha", _d),
                ("bw_rho", _d), ("bw_V0", _d), ("seed", _u64), ("net_id", _u64),
                ("fixed_shift", _i32), ("precision", _i32), ("raster_capacity", _i64),
                ("bold_capacity", _i64), ("autotune_at", _i64), ("bin_spikes", _i32),
                ("emit_delay", _i32), ("schedule", _i32), ("deliver_blocks", _i32)]


class dbnet_stats_t(ctypes.Structure):
    _fields_ = [("step", _i64), ("spikes", _i64), ("events", _i64), ("raster_len", _i64),
                ("raster_dropped", _i64), ("bold_samples", _i64), ("fixed_shift", _i32),
                ("max_delay", _i32), ("packed_edges", _i32), ("weights_rounded", _i32),
                ("deliver_blocks", _i32), ("autotuned", _i32), ("two_weights", _i32),
                ("seg_ring", _i32), ("emit_delay", _i32), ("schedule", _i32)]


class dbnet_device_graph_t(ctypes.Structure):
    _fields_ = [("n_neurons", _i32), ("n_regions", _i32), ("region_offsets", _vp),
                ("n_exc", _vp), ("row_ptr", _vp), ("col", _vp), ("weight_bf16", _vp),
                ("delay", _vp)]


class dbsrv_options_t(ctypes.Structure):
    _fields_ = [("max_neurons", _i64), ("max_requests", _i32), ("max_regions", _i32),
                ("max_delay", _i32), ("chunk_steps", _i32), ("arena_bytes", _i64),
                ("max_inflight", _i32), ("two_weights", _i32), ("run", dbnet_options_t)]


class dbsrv_request_t(ctypes.Structure):
    _fields_ = [("n_steps", _i64), ("seed", _u64), ("net_id", _u64), ("graph_key", _u64),
                ("bold_capacity", _i64), ("raster_capacity", _i64)]


class dbsrv_status_t(ctypes.Structure):
    _fields_ = [("state", _i32), ("error", _i32), ("steps", _i64), ("spikes", _i64),
                ("bold_samples", _i64), ("raster_len", _i64), ("queued_s", _d), ("run_s", _d),
                ("latency_s", _d)]


class dbsrv_stats_t(ctypes.Structure):
    _fields_ = [("iterations", _i64), ("events", _i64), ("running", _i32), ("queued", _i32),
                ("cooling", _i32), ("done", _i32), ("arena_used", _i64), ("arena_bytes", _i64),
                ("tiles_in_use", _i32), ("tile_extent", _i32)]


DBSRV_QUEUED, DBSRV_RUNNING, DBSRV_DONE, DBSRV_FAILED = 0, 1, 2, 3


class dbens_enkf_t(ctypes.Structure):
    _fields_ = [("obs_var", _d), ("gamma", _d), ("rw_sigma", _d), ("theta_lo", _d),
                ("theta_hi", _d), ("floor", _d), ("mode", _i32), ("target", _i32 * 2)]


# what each of a region's two log scales multiplies
DBENS_T_DEFAULT, DBENS_T_AMPA, DBENS_T_NMDA, DBENS_T_GABA_A, DBENS_T_GABA_B, DBENS_T_IEXT = range(6)
DBENS_T_NONE = -1


_SIGS = {
    "dbnet_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "dbnet_last_error": (ctypes.c_char_p, []),
    "dbnet_set_allocator": (ctypes.c_int, [ctypes.POINTER(dbnet_allocator_t)]),
    "dbnet_barrier_probe": (ctypes.c_int, [_i32, _i32, _i32, _i64]),
    "dbnet_abi_sizes": (ctypes.c_int, [_vp, ctypes.c_int]),
    "dbnet_options_default": (ctypes.c_int, [ctypes.POINTER(dbnet_options_t)]),
    "dbnet_create": (ctypes.c_int, [ctypes.POINTER(dbnet_graph_t), _vp,
                                    ctypes.POINTER(dbnet_options_t), _vp, ctypes.POINTER(_vp)]),
    "dbnet_step": (ctypes.c_int, [_vp, _i64]),
    "dbnet_sync": (ctypes.c_int, [_vp]),
    "dbnet_step_timed": (ctypes.c_int, [_vp, _i64, _vp]),
    "dbnet_read_spikes": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "dbnet_read_bold": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "dbnet_read_bw": (ctypes.c_int, [_vp, _vp]),
    "dbnet_read_state": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "dbnet_set_state": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "dbnet_stats": (ctypes.c_int, [_vp, ctypes.POINTER(dbnet_stats_t)]),
    "dbnet_read_ibg": (ctypes.c_int, [_vp, _vp]),
    "dbnet_set_ibg": (ctypes.c_int, [_vp, _vp]),
    "dbnet_destroy": (None, [_vp]),
    "ens_create": (ctypes.c_int, [ctypes.POINTER(dbnet_graph_t), _vp, _i32, _vp,
                                  ctypes.POINTER(dbnet_options_t), ctypes.POINTER(dbens_enkf_t),
                                  _vp, ctypes.POINTER(_vp)]),
    "ens_step": (ctypes.c_int, [_vp, _i64]),
    "ens_assimilate": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ens_read": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "ens_member": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_vp)]),
    "ens_destroy": (None, [_vp]),
    "dbsrv_options_default": (ctypes.c_int, [ctypes.POINTER(dbsrv_options_t)]),
    "dbsrv_create": (ctypes.c_int, [ctypes.POINTER(dbsrv_options_t), _vp, ctypes.POINTER(_vp)]),
    "dbsrv_submit": (ctypes.c_int, [_vp, ctypes.POINTER(dbnet_graph_t), _vp,
                                    ctypes.POINTER(dbsrv_request_t), ctypes.POINTER(_i64)]),
    "dbsrv_pump": (ctypes.c_int, [_vp, _vp]),
    "dbsrv_drain": (ctypes.c_int, [_vp]),
    "dbsrv_poll": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(dbsrv_status_t)]),
    "dbsrv_read_bold": (ctypes.c_int, [_vp, _i64, _vp, _i64, ctypes.POINTER(_i64)]),
    "dbsrv_read_spikes": (ctypes.c_int, [_vp, _i64, _vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "dbsrv_release": (ctypes.c_int, [_vp, _i64]),
    "dbsrv_stats": (ctypes.c_int, [_vp, ctypes.POINTER(dbsrv_stats_t)]),
    "dbsrv_destroy": (None, [_vp]),
    "dbnet_run_noalloc": (ctypes.c_int, [ctypes.POINTER(dbnet_device_graph_t), _vp,
                                         ctypes.POINTER(dbnet_options_t), _i64, _vp, _vp, _vp,
                                         _vp, _vp, _i64, ctypes.POINTER(_i64),
                                         ctypes.POINTER(_i64), _vp]),
}


def library_path() -> str:
    return _SO


def lib():
    """Load the in-tree CUDA library; fail loudly when it was not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_SO):
                raise RuntimeError("libdbnet.so is not built: run __graft_entry__.build() "
                                   "(nvcc for sm_103a); there is no CPU fallback")
            L = ctypes.CDLL(_SO)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


ABI_STRUCTS = ("dbnet_graph_t", "dbnet_region_params_t", "dbnet_options_t", "dbnet_stats_t",
               "dbens_enkf_t", "dbnet_device_graph_t", "dbsrv_options_t", "dbsrv_request_t",
               "dbsrv_status_t", "dbsrv_stats_t")


def abi_sizes() -> dict:
    """sizeof of each public struct as the library was compiled, by name."""
    out = np.zeros(11, dtype=np.int64)
    n = lib().dbnet_abi_sizes(out.ctypes.data, len(out))
    return dict(zip(ABI_STRUCTS[:n], (int(x) for x in out[:n])))


class DbnetError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = lib()
        self.code = code
        msg = "%s: %s (%s)" % (where, L.dbnet_strerror(code).decode(),
                               L.dbnet_last_error().decode())
        super().__init__(msg)


def _check(rc: int, where: str) -> None:
    if rc != DBNET_OK:
        raise DbnetError(rc, where)


def _addr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if hasattr(a, "is_cuda") and a.is_cuda:
            raise ValueError("graph arrays are host memory")
        return int(a.data_ptr())
    raise TypeError("expected a numpy array or a CPU tensor")


def _stream(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def dbnet_barrier_probe(blocks: int, missing: int = 0, rounds: int = 1,
                        limit_us: int = 1_000_000) -> int:
    """One cooperative launch of the persistent stepper's grid barrier on
    the current device: `rounds` barriers over `blocks` blocks, each
    expecting `missing` arrivals more than the grid makes.  Returns the
    status code: DBNET_OK, or DBNET_ETIMEOUT when a wait gave up at
    limit_us (always, for missing > 0); raises DbnetError for others."""
    rc = lib().dbnet_barrier_probe(int(blocks), int(missing), int(rounds), int(limit_us))
    if rc not in (DBNET_OK, DBNET_ETIMEOUT):
        raise DbnetError(rc, "dbnet_barrier_probe")
    return rc


# ------------------------------------------------------------- allocator ----
_allocators = []   # installed callbacks stay alive for the handles that used them


def dbnet_set_allocator(alloc=None, free=None) -> None:
    """Install Python callables as the library's device allocator:
    alloc(nbytes, stream) -> device address (int) or 0, free(ptr, nbytes,
    stream).  With no arguments, cudaMalloc is restored.  Affects handles
    created afterwards."""
    if alloc is None:
        _check(lib().dbnet_set_allocator(None), "dbnet_set_allocator")
        return

    def _a(nbytes, stream, ctx):
        try:
            return int(alloc(int(nbytes), int(stream or 0))) or None
        except Exception:  # noqa: BLE001  -- reported as DBNET_ENOMEM by the library
            return None

    def _f(ptr, nbytes, stream, ctx):
        try:
            free(int(ptr), int(nbytes), int(stream or 0))
        except Exception:  # noqa: BLE001
            pass
    a = dbnet_allocator_t(dbnet_alloc_fn(_a), dbnet_free_fn(_f), None)
    _allocators.append(a)
    _check(lib().dbnet_set_allocator(ctypes.byref(a)), "dbnet_set_allocator")


def use_torch_allocator(device=None) -> None:
    """Back every device allocation of later handles with PyTorch's caching
    allocator (torch.cuda.caching_allocator_alloc / _delete) on `device`
    (default: the current device), each on the stream of its handle."""
    import torch
    dev = torch.cuda.current_device() if device is None else device

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, device=dev, stream=stream)

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)
    dbnet_set_allocator(alloc, free)


# ------------------------------------------------------------ structures ----
def dbnet_options_default(**over) -> dbnet_options_t:
    o = dbnet_options_t()
    _check(lib().dbnet_options_default(ctypes.byref(o)), "dbnet_options_default")
    for k, v in over.items():
        if k.startswith("bw") and isinstance(v, dict):
            continue
        setattr(o, k, v)
    return o


def options_from(opts) -> dbnet_options_t:
    if isinstance(opts, dbnet_options_t):
        return opts
    opts = dict(opts or {})
    bw = opts.pop("bw", None)
    o = dbnet_options_default(**opts)
    if bw:
        for k, v in bw.items():
            setattr(o, "bw_" + k, float(v))
    return o


def region_params(p: dict) -> dbnet_region_params_t:
    r = dbnet_region_params_t()
    for k in ("C", "gL", "VL", "Vth", "Vreset", "Tref", "I_ext", "drive_rate_hz", "drive_K", "w_ext"):
        setattr(r, k, float(p[k]))
    r.ou_mu = float(p.get("ou_mu", 0.0))
    r.ou_sigma = float(p.get("ou_sigma", 0.0))
    r.ou_tau = float(p.get("ou_tau", 10.0))
    r.iext_shape = float(p.get("iext_shape", 0.0))
    for k in ("Vu", "tau_u", "g_u"):
        arr = getattr(r, k)
        for u in range(4):
            arr[u] = float(p[k][u])
    return r


def params_array(params, n_regions: int):
    if isinstance(params, dict):
        params = [params] * n_regions
    if len(params) != n_regions:
        raise ValueError("one parameter set per region is needed")
    return (dbnet_region_params_t * n_regions)(*[region_params(p) for p in params])


def graph_struct(graph):
    """dbnet_graph_t over the arrays of a graph object with fields n_neurons,
    n_regions, region_offsets, n_exc, row_ptr, col, w_bf16 (or weight) and
    delay, and optionally w2_bf16 (or weight2): a second weight per edge.
    Returns (struct, keepalive)."""
    ro = np.ascontiguousarray(graph.region_offsets, dtype=np.int32)
    ne = np.ascontiguousarray(graph.n_exc, dtype=np.int32)
    rp = graph.row_ptr
    if isinstance(rp, np.ndarray):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
    w = getattr(graph, "w_bf16", None)
    w2 = getattr(graph, "w2_bf16", None)
    dtype = DBNET_WEIGHT_BF16
    if w is None:
        w = graph.weight
        w2 = getattr(graph, "weight2", None)
        dtype = DBNET_WEIGHT_F32
    g = dbnet_graph_t(int(graph.n_neurons), int(graph.n_regions), _addr(ro), _addr(ne), _addr(rp),
                      _addr(graph.col), _addr(w), dtype, _addr(graph.delay),
                      _addr(w2) if w2 is not None else None)
    return g, (ro, ne, rp, graph)


# --------------------------------------------------------------- network ----
def dbnet_create(graph, params, options=None, stream=None) -> ctypes.c_void_p:
    g, keep = graph_struct(graph)
    P = params_array(params, int(graph.n_regions))
    o = options_from(options)
    h = _vp()
    _check(lib().dbnet_create(ctypes.byref(g), ctypes.cast(P, _vp), ctypes.byref(o),
                              _stream(stream), ctypes.byref(h)), "dbnet_create")
    return h


def dbnet_step(h, n_steps: int) -> None:
    _check(lib().dbnet_step(h, int(n_steps)), "dbnet_step")


def dbnet_step_timed(h, n_steps: int):
    """Returns (delivery ms, update ms) summed over the n_steps launches."""
    ms = np.zeros(2)
    _check(lib().dbnet_step_timed(h, int(n_steps), ms.ctypes.data), "dbnet_step_timed")
    return float(ms[0]), float(ms[1])


def dbnet_sync(h) -> None:
    _check(lib().dbnet_sync(h), "dbnet_sync")


def dbnet_stats(h) -> dict:
    s = dbnet_stats_t()
    _check(lib().dbnet_stats(h, ctypes.byref(s)), "dbnet_stats")
    return {k: getattr(s, k) for k, _ in dbnet_stats_t._fields_}


def dbnet_read_spikes(h, t0: int = 0, t1: int = 2**62, cap: int | None = None):
    if cap is None:
        cap = max(dbnet_stats(h)["raster_len"], 0)
    st = np.zeros(max(cap, 1), dtype=np.int32)
    ids = np.zeros(max(cap, 1), dtype=np.int32)
    n = _i64(0)
    _check(lib().dbnet_read_spikes(h, int(t0), int(t1), st.ctypes.data, ids.ctypes.data, int(cap),
                                   ctypes.byref(n)), "dbnet_read_spikes")
    return st[:n.value].copy(), ids[:n.value].copy()


def dbnet_read_bold(h, n_regions: int, cap: int = 4096) -> np.ndarray:
    y = np.zeros((max(cap, 1), n_regions))
    n = _i64(0)
    _check(lib().dbnet_read_bold(h, y.ctypes.data, int(cap), ctypes.byref(n)), "dbnet_read_bold")
    return y[:n.value].copy()


def dbnet_read_bw(h, n_regions: int) -> np.ndarray:
    x = np.zeros((n_regions, 4))
    _check(lib().dbnet_read_bw(h, x.ctypes.data), "dbnet_read_bw")
    return x


def dbnet_read_state(h, n_neurons: int):
    V = np.zeros(n_neurons, dtype=np.float32)
    J = np.zeros((4, n_neurons), dtype=np.float32)
    ref = np.zeros(n_neurons, dtype=np.int32)
    _check(lib().dbnet_read_state(h, V.ctypes.data, J.ctypes.data, ref.ctypes.data),
           "dbnet_read_state")
    return V, J, ref


def dbnet_set_state(h, V=None, J=None, ref=None) -> None:
    Va = None if V is None else np.ascontiguousarray(V, dtype=np.float32)
    Ja = None if J is None else np.ascontiguousarray(J, dtype=np.float32)
    ra = None if ref is None else np.ascontiguousarray(ref, dtype=np.int32)
    _check(lib().dbnet_set_state(h, _addr(Va), _addr(Ja), _addr(ra)), "dbnet_set_state")


def dbnet_read_ibg(h, n_neurons: int) -> np.ndarray:
    I = np.zeros(n_neurons, dtype=np.float32)
    _check(lib().dbnet_read_ibg(h, I.ctypes.data), "dbnet_read_ibg")
    return I


def dbnet_set_ibg(h, I) -> None:
    a = np.ascontiguousarray(I, dtype=np.float32)
    _check(lib().dbnet_set_ibg(h, a.ctypes.data), "dbnet_set_ibg")


def dbnet_destroy(h) -> None:
    if h:
        lib().dbnet_destroy(h)


class Network:
    """Owner of one dbnet handle."""

    def __init__(self, graph, params, options=None, stream=None):
        self.N = int(graph.n_neurons)
        self.R = int(graph.n_regions)
        self.h = dbnet_create(graph, params, options, stream)

    def step(self, n: int) -> None:
        dbnet_step(self.h, n)

    def sync(self) -> None:
        dbnet_sync(self.h)

    def step_timed(self, n: int):
        return dbnet_step_timed(self.h, n)

    def stats(self) -> dict:
        return dbnet_stats(self.h)

    def spikes(self, t0: int = 0, t1: int = 2**62):
        return dbnet_read_spikes(self.h, t0, t1)

    def bold(self, cap: int = 4096) -> np.ndarray:
        return dbnet_read_bold(self.h, self.R, cap)

    def bw(self) -> np.ndarray:
        return dbnet_read_bw(self.h, self.R)

    def state(self):
        return dbnet_read_state(self.h, self.N)

    def set_state(self, V=None, J=None, ref=None) -> None:
        dbnet_set_state(self.h, V, J, ref)

    def ibg(self) -> np.ndarray:
        return dbnet_read_ibg(self.h, self.N)

    def set_ibg(self, I) -> None:
        dbnet_set_ibg(self.h, I)

    def close(self) -> None:
        if getattr(self, "h", None):
            dbnet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------- allocation-free ----
def noalloc_check(n_neurons, region_offsets, n_exc, row_ptr, col, weight_bf16, delay, V, J, ref,
                  raster_step=None, raster_id=None, n_edges=None):
    """Argument checks of dbnet_run_noalloc that the C side cannot make (it
    sees bare device pointers): every tensor is contiguous CUDA memory on the
    current device with the dtype and at least the element count the
    kernels index -- row_ptr int64 [N+1]; col int32, weight_bf16 int16 or
    uint16 and delay uint8 with n_edges elements each; V float32 [n_pad];
    J float32 [4 n_pad]; ref uint8 [n_pad]; raster_step and raster_id int32
    of equal length -- where n_pad = ceil(N / 1024) x 1024, and
    region_offsets has one entry more than n_exc.  Raises ValueError on the
    first mismatch.  `n_edges` is row_ptr[N] (read from the device by the
    caller).  Touches no GPU."""
    N = int(n_neurons)
    if N < 1:
        raise ValueError("n_neurons must be >= 1")
    if len(region_offsets) != len(n_exc) + 1:
        raise ValueError("region_offsets needs len(n_exc) + 1 entries")
    n_pad = (N + 1023) // 1024 * 1024
    cur = _current_device()

    def need(name, t, dtypes, count):
        if t is None:
            raise ValueError("%s is required" % name)
        if not (getattr(t, "is_cuda", False) and t.is_contiguous()):
            raise ValueError("%s must be a contiguous CUDA tensor" % name)
        if cur is not None and t.device.index != cur:
            raise ValueError("%s is on cuda:%s, not the current device cuda:%d" % (name, t.device.index, cur))
        if str(t.dtype) not in dtypes:
            raise ValueError("%s must be %s, not %s" % (name, " or ".join(dtypes), t.dtype))
        if t.numel() < count:
            raise ValueError("%s has %d elements, needs %d" % (name, t.numel(), count))

    need("row_ptr", row_ptr, ("torch.int64",), N + 1)
    E = 0 if n_edges is None else int(n_edges)
    need("col", col, ("torch.int32",), E)
    need("weight_bf16", weight_bf16, ("torch.int16", "torch.uint16", "torch.bfloat16"), E)
    need("delay", delay, ("torch.uint8",), E)
    need("V", V, ("torch.float32",), n_pad)
    need("J", J, ("torch.float32",), 4 * n_pad)
    need("ref", ref, ("torch.uint8",), n_pad)
    if (raster_step is None) != (raster_id is None):
        raise ValueError("raster_step and raster_id go together")
    if raster_step is not None:
        need("raster_step", raster_step, ("torch.int32",), 0)
        need("raster_id", raster_id, ("torch.int32",), raster_step.numel())
        if raster_id.numel() != raster_step.numel():
            raise ValueError("raster_step and raster_id must have the same length")


def _current_device():
    try:
        import torch
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except Exception:  # noqa: BLE001
        return None


def dbnet_run_noalloc(n_neurons, region_offsets, n_exc, row_ptr, col, weight_bf16, delay, params,
                      options, n_steps, V, J, ref, raster_step=None, raster_id=None, stream=None):
    """Run through the allocation-free entry point.  row_ptr, col,
    weight_bf16, delay, V [n_pad], J [4, n_pad], ref [n_pad] (uint8) and the
    optional raster buffers are CUDA tensors the caller allocated;
    region_offsets and n_exc are host arrays.  Every tensor is checked
    (noalloc_check) before the call.  Returns (n_spikes, n_events)."""
    ro = np.ascontiguousarray(region_offsets, dtype=np.int32)
    ne = np.ascontiguousarray(n_exc, dtype=np.int32)
    n_edges = None
    if getattr(row_ptr, "is_cuda", False) and row_ptr.numel() >= int(n_neurons) + 1:
        n_edges = int(row_ptr[int(n_neurons)].item())   # one 8-byte read of the caller's row_ptr
    noalloc_check(n_neurons, ro, ne, row_ptr, col, weight_bf16, delay, V, J, ref, raster_step,
                  raster_id, n_edges)
    R = len(ne)
    g = dbnet_device_graph_t(int(n_neurons), R, ro.ctypes.data, ne.ctypes.data,
                             int(row_ptr.data_ptr()), int(col.data_ptr()),
                             int(weight_bf16.data_ptr()), int(delay.data_ptr()))
    P = params_array(params, R)
    o = options_from(options)
    cap = 0 if raster_step is None else int(raster_step.numel())
    rs = 0 if raster_step is None else int(raster_step.data_ptr())
    ri = 0 if raster_id is None else int(raster_id.data_ptr())
    ns, ne_ = _i64(0), _i64(0)
    _check(lib().dbnet_run_noalloc(ctypes.byref(g), ctypes.cast(P, _vp), ctypes.byref(o),
                                   int(n_steps), int(V.data_ptr()), int(J.data_ptr()),
                                   int(ref.data_ptr()), rs, ri, cap, ctypes.byref(ns),
                                   ctypes.byref(ne_), _stream(stream)), "dbnet_run_noalloc")
    return ns.value, ne_.value


# -------------------------------------------------------------- ensemble ----
def enkf_options(obs_var=1e-6, gamma=0.5, rw_sigma=0.02, theta_lo=-0.6931471805599453,
                 theta_hi=0.6931471805599453, floor=1e-2, mode=DBENS_DIFFUSION,
                 target=(DBENS_T_DEFAULT, DBENS_T_DEFAULT)) -> dbens_enkf_t:
    k = dbens_enkf_t(obs_var, gamma, rw_sigma, theta_lo, theta_hi, floor, mode)
    k.target[0], k.target[1] = int(target[0]), int(target[1])
    return k


def ens_create(graph, base_params, n_members: int, log_scale_init, options=None, enkf=None,
               stream=None):
    g, keep = graph_struct(graph)
    P = params_array(base_params, int(graph.n_regions))
    o = options_from(options)
    th = np.ascontiguousarray(log_scale_init, dtype=np.float64)
    assert th.shape == (n_members, int(graph.n_regions), 2)
    k = enkf if isinstance(enkf, dbens_enkf_t) else enkf_options(**(enkf or {}))
    h = _vp()
    _check(lib().ens_create(ctypes.byref(g), ctypes.cast(P, _vp), int(n_members), th.ctypes.data,
                            ctypes.byref(o), ctypes.byref(k), _stream(stream), ctypes.byref(h)),
           "ens_create")
    return h


def ens_step(h, n_steps: int) -> None:
    _check(lib().ens_step(h, int(n_steps)), "ens_step")


def ens_assimilate(h, y_obs, n_members: int, eps_obs=None, xi_rw=None) -> np.ndarray:
    y = np.ascontiguousarray(y_obs, dtype=np.float64)
    R = len(y)
    e = None if eps_obs is None else np.ascontiguousarray(eps_obs, dtype=np.float64)
    x = None if xi_rw is None else np.ascontiguousarray(xi_rw, dtype=np.float64)
    if e is not None:
        assert e.shape == (n_members, R)
    if x is not None:
        assert x.shape == (n_members, R, 2)
    out = np.zeros(R)
    _check(lib().ens_assimilate(h, y.ctypes.data, _addr(e), _addr(x), out.ctypes.data),
           "ens_assimilate")
    return out


def ens_read(h, n_members: int, n_regions: int):
    th = np.zeros((n_members, n_regions, 2))
    bw = np.zeros((n_members, n_regions, 4))
    y = np.zeros((n_members, n_regions))
    _check(lib().ens_read(h, th.ctypes.data, bw.ctypes.data, y.ctypes.data), "ens_read")
    return th, bw, y


def ens_member(h, member: int):
    v = _vp()
    _check(lib().ens_member(h, int(member), ctypes.byref(v)), "ens_member")
    return v


def ens_destroy(h) -> None:
    if h:
        lib().ens_destroy(h)


class Ensemble:
    """Owner of one dbens handle (M networks sharing a graph)."""

    def __init__(self, graph, base_params, n_members, log_scale_init, options=None, enkf=None,
                 stream=None):
        self.M = int(n_members)
        self.R = int(graph.n_regions)
        self.N = int(graph.n_neurons)
        self.h = ens_create(graph, base_params, n_members, log_scale_init, options, enkf, stream)

    def step(self, n: int) -> None:
        ens_step(self.h, n)

    def assimilate(self, y_obs, eps_obs=None, xi_rw=None) -> np.ndarray:
        return ens_assimilate(self.h, y_obs, self.M, eps_obs, xi_rw)

    def read(self):
        return ens_read(self.h, self.M, self.R)

    def member_state(self, m: int):
        return dbnet_read_state(ens_member(self.h, m), self.N)

    def member_bold(self, m: int, cap: int = 4096):
        return dbnet_read_bold(ens_member(self.h, m), self.R, cap)

    def member_spikes(self, m: int):
        v = ens_member(self.h, m)
        return dbnet_read_spikes(v)

    def member_stats(self, m: int) -> dict:
        return dbnet_stats(ens_member(self.h, m))

    def stats(self) -> dict:
        """Ensemble totals: events (engine-wide) and spikes summed over members."""
        s = [self.member_stats(m) for m in range(self.M)]
        out = dict(s[0])
        out["spikes"] = sum(x["spikes"] for x in s)
        return out

    def close(self) -> None:
        if getattr(self, "h", None):
            ens_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- serving ----
def dbsrv_options_default(**over) -> dbsrv_options_t:
    o = dbsrv_options_t()
    _check(lib().dbsrv_options_default(ctypes.byref(o)), "dbsrv_options_default")
    run = over.pop("run", None)
    for k, v in over.items():
        setattr(o, k, v)
    if run:
        r = options_from(run)
        o.run = r
    return o


def _fields(st) -> dict:
    return {k: getattr(st, k) for k, _ in type(st)._fields_}


class Server:
    """Owner of one dbsrv handle: a request server that batches independent
    simulations on one GPU (continuous batching, admission by pool room)."""

    def __init__(self, stream=None, **options):
        self.opt = dbsrv_options_default(**options)
        self.h = _vp()
        _check(lib().dbsrv_create(ctypes.byref(self.opt), _stream(stream), ctypes.byref(self.h)),
               "dbsrv_create")
        self._keep = {}   # request id -> host arrays the server may still read
        self._R = {}

    def submit(self, graph, params, n_steps: int, *, seed: int = 1, net_id: int = 0,
               graph_key: int = 0, bold_capacity: int = 0, raster_capacity: int = 0) -> int:
        g, keep = graph_struct(graph)
        P = params_array(params, int(graph.n_regions))
        rq = dbsrv_request_t(int(n_steps), int(seed), int(net_id), int(graph_key),
                             int(bold_capacity), int(raster_capacity))
        rid = _i64()
        _check(lib().dbsrv_submit(self.h, ctypes.byref(g), ctypes.cast(P, _vp), ctypes.byref(rq),
                                  ctypes.byref(rid)), "dbsrv_submit")
        self._keep[rid.value] = (g, keep, graph)
        self._R[rid.value] = int(graph.n_regions)
        return rid.value

    def pump(self) -> dict:
        st = dbsrv_stats_t()
        _check(lib().dbsrv_pump(self.h, ctypes.byref(st)), "dbsrv_pump")
        return _fields(st)

    def drain(self) -> None:
        _check(lib().dbsrv_drain(self.h), "dbsrv_drain")

    def poll(self, rid: int) -> dict:
        st = dbsrv_status_t()
        _check(lib().dbsrv_poll(self.h, int(rid), ctypes.byref(st)), "dbsrv_poll")
        d = _fields(st)
        if d["state"] != DBSRV_QUEUED:
            self._keep.pop(rid, None)   # admitted or failed: the arrays are no longer read
        return d

    def bold(self, rid: int) -> np.ndarray:
        R = self._R[rid]
        n = self.poll(rid)["bold_samples"]
        y = np.zeros((max(n, 1), R))
        got = _i64()
        _check(lib().dbsrv_read_bold(self.h, int(rid), y.ctypes.data, int(n), ctypes.byref(got)),
               "dbsrv_read_bold")
        return y[:got.value]

    def spikes(self, rid: int):
        n = self.poll(rid)["raster_len"]
        st = np.zeros(max(n, 1), dtype=np.int32)
        ids = np.zeros(max(n, 1), dtype=np.int32)
        got = _i64()
        _check(lib().dbsrv_read_spikes(self.h, int(rid), st.ctypes.data, ids.ctypes.data, int(n),
                                       ctypes.byref(got)), "dbsrv_read_spikes")
        return st[:got.value], ids[:got.value]

    def release(self, rid: int) -> None:
        _check(lib().dbsrv_release(self.h, int(rid)), "dbsrv_release")
        self._keep.pop(rid, None)
        self._R.pop(rid, None)

    def stats(self) -> dict:
        st = dbsrv_stats_t()
        _check(lib().dbsrv_stats(self.h, ctypes.byref(st)), "dbsrv_stats")
        return _fields(st)

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().dbsrv_destroy(self.h)
            self.h = None
        self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
