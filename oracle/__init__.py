"""CPU oracle for the Digital Brain hot path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The CUDA library never calls it and the
two share no code: the oracle's C++ (`oracle.cc`) and numpy (`enkf.py`,
`metrics.py`) restate the paper's equations on their own, and only the seeded
input generator (`synth`) feeds both sides.

Functions and the passages they follow:

* ``Sim``: conductance LIF update (Methods, capacitance-voltage equation and
  Eq. 2; Supplementary Sec. 3, Eqs. 3 and 5), push delivery into a per-delay
  ring (Supplementary Algorithm 2), Poisson background (Extended Data
  Table 2), Balloon-Windkessel readout (Extended Data Table 4), optional
  spike binning (Supplementary Sec. 3, "Numerical method").  FP64 and
  op-order-matched FP32 modes; an all-core timing variant (``threads``)
  with identical results.
* ``bw_step``: one forward-Euler step of Extended Data Table 4.
* ``philox4x64``: Philox4x64-10 (Salmon et al., SC'11), the counter-based
  generator the drive draws from.
* ``enkf.diffusion_enkf``: Supplementary Algorithm 3 (diffusion EnKF) with the
  random walk of the hyperparameters (Supplementary Sec. 6).
* ``metrics.lagged_pcc``: lagged Pearson correlation (Supplementary Sec. 6).

Every function has pins in ``tests/test_oracle_pins.py`` that do not come from
the oracle itself: closed forms, library routines, brute force and
Monte-Carlo bounds.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.cc")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


class OgGraph(ctypes.Structure):
    _fields_ = [("n_neurons", ctypes.c_int32), ("n_regions", ctypes.c_int32),
                ("region_offsets", ctypes.c_void_p), ("n_exc", ctypes.c_void_p),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("w_bf16", ctypes.c_void_p), ("delay", ctypes.c_void_p),
                ("w2_bf16", ctypes.c_void_p), ("w_f64", ctypes.c_void_p)]


class OgRegion(ctypes.Structure):
    _fields_ = [("C", ctypes.c_double), ("gL", ctypes.c_double), ("VL", ctypes.c_double),
                ("Vth", ctypes.c_double), ("Vreset", ctypes.c_double), ("Tref", ctypes.c_double),
                ("Vu", ctypes.c_double * 4), ("tau_u", ctypes.c_double * 4),
                ("g_u", ctypes.c_double * 4), ("I_ext", ctypes.c_double),
                ("drive_rate_hz", ctypes.c_double), ("drive_K", ctypes.c_double),
                ("w_ext", ctypes.c_double), ("ou_mu", ctypes.c_double),
                ("ou_sigma", ctypes.c_double), ("ou_tau", ctypes.c_double),
                ("iext_shape", ctypes.c_double)]


class OgOptions(ctypes.Structure):
    _fields_ = [("dt_ms", ctypes.c_double), ("bin_ms", ctypes.c_double),
                ("tr_ms", ctypes.c_double), ("z_scale", ctypes.c_double),
                ("bw_kappa", ctypes.c_double), ("bw_gamma", ctypes.c_double),
                ("bw_tau", ctypes.c_double), ("bw_alpha", ctypes.c_double),
                ("bw_rho", ctypes.c_double), ("bw_V0", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("net_id", ctypes.c_uint64),
                ("fixed_shift", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("bin_spikes", ctypes.c_int32), ("pad", ctypes.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            L.og_create.restype = vp
            L.og_create.argtypes = [ctypes.POINTER(OgGraph), vp, ctypes.POINTER(OgOptions),
                                    ctypes.POINTER(ctypes.c_int)]
            L.og_destroy.argtypes = [vp]
            L.og_set_threads.argtypes = [vp, i32]
            L.og_step.argtypes = [vp, i64]
            L.og_deliver_only.argtypes = [vp, vp, i64, i64]
            L.og_read_state.argtypes = [vp, vp, vp, vp]
            L.og_set_state.argtypes = [vp, vp, vp, vp]
            L.og_read_ibg.argtypes = [vp, vp]
            L.og_set_ibg.argtypes = [vp, vp]
            L.og_box_muller.restype = d
            L.og_box_muller.argtypes = [ctypes.c_uint64]
            L.og_gamma_draw.restype = d
            L.og_gamma_draw.argtypes = [d, ctypes.c_uint64, ctypes.c_uint64, i64]
            L.og_info.argtypes = [vp, vp]
            for f in (L.og_read_raster,):
                f.argtypes = [vp, vp, vp]
            for f in (L.og_read_bold, L.og_read_bw, L.og_read_ring, L.og_read_counts):
                f.argtypes = [vp, vp]
            L.og_philox4x64_10.argtypes = [vp, vp, vp]
            L.og_poisson_thresholds.restype = i32
            L.og_poisson_thresholds.argtypes = [d, vp]
            L.og_bw_step.restype = d
            L.og_bw_step.argtypes = [vp, d, d, d, d, d, d, d, d]
            _lib = L
    return _lib


def _addr(a) -> int:
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    return int(a.data_ptr())


def philox4x64(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().og_philox4x64_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def poisson_thresholds(lam: float) -> np.ndarray:
    thr = np.zeros(16, dtype=np.uint32)
    n = lib().og_poisson_thresholds(lam, thr.ctypes.data)
    assert n >= 0
    return thr[:n].copy()


def bw_step(x: np.ndarray, z: float, h: float, bw: dict) -> float:
    """Advance x = [s, f, v, q] (float64, in place) by one Euler step; return y."""
    assert x.dtype == np.float64 and x.shape == (4,)
    return lib().og_bw_step(x.ctypes.data, z, h, bw["kappa"], bw["gamma"], bw["tau"],
                            bw["alpha"], bw["rho"], bw["V0"])


def region_struct(p: dict) -> OgRegion:
    r = OgRegion()
    for k in ("C", "gL", "VL", "Vth", "Vreset", "Tref", "I_ext", "drive_rate_hz", "drive_K",
              "w_ext"):
        setattr(r, k, float(p[k]))
    for k in ("Vu", "tau_u", "g_u"):
        arr = getattr(r, k)
        for u in range(4):
            arr[u] = float(p[k][u])
    r.ou_mu = float(p.get("ou_mu", 0.0))
    r.ou_sigma = float(p.get("ou_sigma", 0.0))
    r.ou_tau = float(p.get("ou_tau", 10.0))
    r.iext_shape = float(p.get("iext_shape", 0.0))
    return r


def gamma_draw(k: float, seed: int, net_id: int, i: int) -> float:
    """The oracle's Gamma(k, 1) draw for neuron i's injected-current factor."""
    return lib().og_gamma_draw(float(k), int(seed), int(net_id), int(i))


def box_muller(word: int) -> float:
    """The oracle's standard normal from one 64-bit Philox word."""
    return lib().og_box_muller(int(word))


class Sim:
    """One network simulated by the oracle."""

    def __init__(self, graph, region_params, *, dt_ms=0.1, bin_ms=1.0, tr_ms=800.0,
                 z_scale=1.0, bw=None, seed=1, net_id=0, fixed_shift=0, precision=32,
                 weights_f64=None, bin_spikes=False, threads=1):
        from synth import BW_DEFAULT
        bw = dict(BW_DEFAULT if bw is None else bw)
        if isinstance(region_params, dict):
            region_params = [region_params] * graph.n_regions
        assert len(region_params) == graph.n_regions
        self.graph = graph  # keep the arrays alive
        self._regs = (OgRegion * graph.n_regions)(*[region_struct(p) for p in region_params])
        w2 = getattr(graph, "w2_bf16", None)
        w2 = _addr(w2) if w2 is not None else None
        wf = None
        if weights_f64 is not None:   # unrounded first weights, [E]
            self._wf = np.ascontiguousarray(weights_f64, dtype=np.float64)
            assert len(self._wf) == graph.n_edges
            wf = _addr(self._wf)
        g = OgGraph(graph.n_neurons, graph.n_regions, _addr(graph.region_offsets),
                    _addr(graph.n_exc), _addr(graph.row_ptr), _addr(graph.col),
                    _addr(graph.w_bf16), _addr(graph.delay), w2, wf)
        o = OgOptions(dt_ms, bin_ms, tr_ms, z_scale, bw["kappa"], bw["gamma"], bw["tau"],
                      bw["alpha"], bw["rho"], bw["V0"], seed, net_id, fixed_shift, precision,
                      1 if bin_spikes else 0, 0)
        err = ctypes.c_int(0)
        self._h = lib().og_create(ctypes.byref(g), ctypes.cast(self._regs, ctypes.c_void_p),
                                  ctypes.byref(o), ctypes.byref(err))
        if not self._h:
            raise ValueError("oracle rejected the network (code %d)" % err.value)
        self.N = graph.n_neurons
        self.R = graph.n_regions
        if threads != 1:
            self.set_threads(threads)

    def set_threads(self, n: int) -> None:
        """Threads of the timing variant (OpenMP; 0 = every core).  The
        results do not depend on it: neuron ranges are joined in order and
        the accumulators are exact integers."""
        if n <= 0:
            n = os.cpu_count() or 1
        self.threads = int(n)
        lib().og_set_threads(self._h, self.threads)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().og_destroy(h)
            self._h = None

    def info(self) -> dict:
        a = np.zeros(10, dtype=np.int64)
        lib().og_info(self._h, a.ctypes.data)
        keys = ("N", "R", "D", "S", "step", "events", "spikes", "raster_len", "bold_samples",
                "bins_done")
        return {k: int(v) for k, v in zip(keys, a)}

    def step(self, n: int) -> None:
        lib().og_step(self._h, int(n))

    def deliver_only(self, ids, n: int) -> None:
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        lib().og_deliver_only(self._h, ids.ctypes.data, len(ids), int(n))

    def state(self):
        V = np.zeros(self.N)
        J = np.zeros((4, self.N))
        ref = np.zeros(self.N, dtype=np.int32)
        lib().og_read_state(self._h, V.ctypes.data, J.ctypes.data, ref.ctypes.data)
        return V, J, ref

    def ibg(self) -> np.ndarray:
        """The background OU current of every neuron."""
        I = np.zeros(self.N)
        lib().og_read_ibg(self._h, I.ctypes.data)
        return I

    def set_ibg(self, I) -> None:
        a = np.ascontiguousarray(I, dtype=np.float64)
        lib().og_set_ibg(self._h, a.ctypes.data)

    def set_state(self, V=None, J=None, ref=None) -> None:
        def p(a, dt):
            if a is None:
                return None, None
            a = np.ascontiguousarray(a, dtype=dt)
            return a, a.ctypes.data
        Va, Vp = p(V, np.float64)
        Ja, Jp = p(J, np.float64)
        ra, rp = p(ref, np.int32)
        lib().og_set_state(self._h, Vp, Jp, rp)

    def raster(self):
        n = self.info()["raster_len"]
        st = np.zeros(n, dtype=np.int32)
        ids = np.zeros(n, dtype=np.int32)
        lib().og_read_raster(self._h, st.ctypes.data, ids.ctypes.data)
        return st, ids

    def bold(self) -> np.ndarray:
        n = self.info()["bold_samples"]
        y = np.zeros((n, self.R))
        lib().og_read_bold(self._h, y.ctypes.data)
        return y

    def bw_state(self) -> np.ndarray:
        x = np.zeros((self.R, 4))
        lib().og_read_bw(self._h, x.ctypes.data)
        return x

    def ring(self) -> np.ndarray:
        """[D][N][channels]: the 2 classes (E, I), or with two weights per
        edge the 4 channels (AMPA, NMDA, GABA_A, GABA_B)."""
        D = self.info()["D"]
        nch = 4 if getattr(self.graph, "w2_bf16", None) is not None else 2
        r = np.zeros((D, self.N, nch), dtype=np.int64)
        lib().og_read_ring(self._h, r.ctypes.data)
        return r

    def counts(self) -> np.ndarray:
        c = np.zeros(self.R, dtype=np.int32)
        lib().og_read_counts(self._h, c.ctypes.data)
        return c
