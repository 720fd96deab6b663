"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no simulation arithmetic.  It draws

* networks shaped like the paper's (Extended Data Table 2: 4:1 E/I split,
  fixed in-degree, uniform sources without autapses or multapses; Methods
  "Constructing the Digital Brain model"; Supplementary Section 2 for the
  within-/cross-region structure), returned as a CSR by source whose rows are
  sorted by (delay, target), with BF16 weights and integer delays in steps;
* per-region neuron and synapse constants (the paper lists the fields of its
  property table, Supplementary Table 5, but prints no values; the defaults
  here are textbook conductance-LIF values and are stated as such);
* the workload recipes (sizes, seeds, delay ranges) used by the tests and the
  benchmark.

Everything is a deterministic function of the seed.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator (plain C++ with OpenMP) in place."""
    src = os.path.join(_HERE, "synth.cc")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


class _Spec(ctypes.Structure):
    _fields_ = [
        ("n_neurons", ctypes.c_int32),
        ("n_regions", ctypes.c_int32),
        ("region_offsets", ctypes.c_void_p),
        ("n_exc", ctypes.c_void_p),
        ("k_in", ctypes.c_int32),
        ("k_within", ctypes.c_int32),
        ("cross_exc_only", ctypes.c_int32),
        ("d_within_min", ctypes.c_int32),
        ("d_within_max", ctypes.c_int32),
        ("d_cross_min", ctypes.c_int32),
        ("d_cross_max", ctypes.c_int32),
        ("w_mu", ctypes.c_double),
        ("w_sigma", ctypes.c_double),
        ("region_prob", ctypes.c_void_p),
        ("seed", ctypes.c_uint64),
    ]


class _ColumnSpec(ctypes.Structure):
    _fields_ = [("n_voxels", ctypes.c_int32), ("n_pops", ctypes.c_int32),
                ("pop_offset", ctypes.c_void_p), ("voxel_size", ctypes.c_int32),
                ("n_exc", ctypes.c_int32), ("k_local", ctypes.c_void_p),
                ("k_cc", ctypes.c_void_p), ("region_prob", ctypes.c_void_p),
                ("d_within_min", ctypes.c_int32), ("d_within_max", ctypes.c_int32),
                ("d_cross_min", ctypes.c_int32), ("d_cross_max", ctypes.c_int32),
                ("w_mu", ctypes.c_double), ("w_sigma", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.synth_graph.restype = ctypes.c_int
            L.synth_graph.argtypes = [ctypes.POINTER(_Spec), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
            L.synth_columns.restype = ctypes.c_int
            L.synth_columns.argtypes = [ctypes.POINTER(_ColumnSpec), ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32]
            L.synth_region_matrix.restype = ctypes.c_int
            L.synth_region_matrix.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p]
            _lib = L
    return _lib


def _ptr(a) -> int:
    """Address of a contiguous numpy array or CPU torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    return int(a.data_ptr())


@dataclasses.dataclass
class Graph:
    """CSR by source.  Neurons are sorted by region and, inside each region,
    excitatory before inhibitory.  Rows are sorted by (delay, target)."""
    n_neurons: int
    n_regions: int
    region_offsets: np.ndarray  # int32 [R+1]
    n_exc: np.ndarray           # int32 [R]
    row_ptr: object             # int64 [N+1]
    col: object                 # int32 [E]
    w_bf16: object              # uint16 [E] (BF16 bit patterns)
    delay: object               # uint8 [E], steps, >= 1
    max_delay: int
    w2_bf16: object = None      # uint16 [E] second channel's weight, or None

    @property
    def n_edges(self) -> int:
        return int(self.row_ptr[-1])

    def weights_f64(self) -> np.ndarray:
        return bf16_to_f64(np.asarray(self.w_bf16))


def bf16_to_f64(w_bf16: np.ndarray) -> np.ndarray:
    return (np.asarray(w_bf16, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def f64_to_bf16(w: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 (ties to even) via float32."""
    b = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return b.astype(np.uint16)


def region_layout(sizes, exc_frac: float = 0.8):
    sizes = np.asarray(sizes, dtype=np.int64)
    ro = np.zeros(len(sizes) + 1, dtype=np.int32)
    ro[1:] = np.cumsum(sizes)
    n_exc = np.rint(sizes * exc_frac).astype(np.int32)
    return ro, n_exc


def region_matrix(R: int, density: float, seed: int, mu: float = 0.0, sigma: float = 1.0):
    out = np.zeros((R, R), dtype=np.float64)
    rc = lib().synth_region_matrix(R, density, mu, sigma, seed, out.ctypes.data)
    assert rc == 0
    return out


def make_graph(sizes, k_in: int, seed: int, *, k_within: int | None = None,
               exc_frac: float = 0.8, d_within=(1, 20), d_cross=(50, 200),
               w_mu: float = -1.0, w_sigma: float = 0.5, region_density: float = 0.3,
               cross_exc_only: bool = True, threads: int = 0, alloc=None) -> Graph:
    """Draw a network.  `sizes` lists the region sizes.  `alloc(n, dtype)` may
    supply the edge arrays (for instance pinned host memory)."""
    sizes = list(sizes)
    R = len(sizes)
    ro, n_exc = region_layout(sizes, exc_frac)
    N = int(ro[-1])
    if k_within is None:
        k_within = k_in if R == 1 else int(round(0.8 * k_in))
    prob = region_matrix(R, region_density, seed + 7) if R > 1 else None
    E = N * k_in
    if alloc is None:
        alloc = lambda n, dt: np.empty(n, dtype=dt)  # noqa: E731
    row_ptr = np.empty(N + 1, dtype=np.int64)
    col = alloc(E, np.int32)
    w = alloc(E, np.uint16)
    d = alloc(E, np.uint8)
    sp = _Spec(N, R, ro.ctypes.data, n_exc.ctypes.data, k_in, k_within, int(cross_exc_only),
               d_within[0], d_within[1], d_cross[0], d_cross[1], w_mu, w_sigma,
               prob.ctypes.data if prob is not None else None, seed)
    rc = lib().synth_graph(ctypes.byref(sp), row_ptr.ctypes.data, _ptr(col), _ptr(w), _ptr(d),
                           threads)
    if rc != 0:
        raise ValueError("synth_graph rejected the spec (code %d)" % rc)
    dmax = max(d_within[1], d_cross[1] if R > 1 else 0)
    return Graph(N, R, ro, n_exc, row_ptr, col, w, d, dmax)


# ---------------------------------------------------------------------------
# Cortical micro-columns.  Extended Data Table 3: the average number of
# synapses a neuron of each postsynaptic population receives from each
# presynaptic population of its column, and from other columns (CC).  Rows
# and columns follow the populations below; the table has no e1 source
# column (0 here) and blank cells are 0.
COLUMN_POPS = ("e1", "i1", "e2/3", "i2/3", "e4", "i4", "e5", "i5", "e6", "i6")
COLUMN_SOURCES = ("i1", "e2/3", "i2/3", "e4", "i4", "e5", "i5", "e6", "i6", "CC")
COLUMN_TABLE = (  # rows: COLUMN_POPS; columns: COLUMN_SOURCES
    (1323, 823, 200, 15, 1, 9, 0, 0, 0, 10133),
    (901, 560, 149, 10, 1, 6, 0, 0, 0, 6899),
    (133, 3554, 804, 881, 45, 431, 0, 136, 0, 1020),
    (52, 1778, 532, 456, 29, 217, 0, 69, 0, 396),
    (27, 417, 84, 1070, 782, 79, 8, 1686, 0, 1489),
    (0, 168, 41, 628, 538, 36, 0, 1028, 0, 790),
    (147, 2550, 176, 765, 99, 621, 596, 363, 0, 1591),
    (0, 1357, 76, 380, 32, 375, 403, 129, 0, 214),
    (2, 643, 46, 549, 196, 327, 126, 925, 597, 2609),
    (0, 80, 8, 92, 3, 159, 11, 76, 499, 1794),
)
# Share of a column's neurons in layers 1, 2/3, 4, 5, 6.  The paper weights
# layers by thickness but prints no values; these are generic proportions
# (a thin, sparse layer 1), not the paper's.
LAYER_FRACTION = (0.015, 0.30, 0.25, 0.20, 0.235)


def cortical_columns(n_voxels: int, voxel_size: int, d_in: int = 1000, seed: int = 1, *,
                     exc_frac: float = 0.8, d_within=(1, 20), d_cross=(20, 100),
                     w_mu: float = -1.0, w_sigma: float = 0.5, density: float = 0.3,
                     threads: int = 0) -> Graph:
    """Micro-column network (Extended Data Table 3; Supplementary Sec. 2,
    Eqs. 5-6): each voxel is a region of ten populations (E and I of layers
    1, 2/3, 4, 5, 6; E populations first).  A neuron of population i gets
    k_i * M[i][j] / sum_k M[i][k] synapses from population j of its voxel and
    k_i * M[i][CC] / sum_k M[i][k] from excitatory neurons of other voxels
    (source voxel by a seeded region matrix), where k_i is proportional to
    the row sum of M and scaled so the mean in-degree is d_in (the table's
    counts exceed the paper's in-degree cap of 1000).  Counts above a local
    population's size are capped at it."""
    layer_of = (0, 0, 1, 1, 2, 2, 3, 3, 4, 4)
    exc = (1, 0) * 5
    size = []
    for p in range(10):
        f = LAYER_FRACTION[layer_of[p]] * (exc_frac if exc[p] else 1.0 - exc_frac)
        size.append(max(2, int(round(f * voxel_size))))
    size[2] += voxel_size - sum(size)  # e2/3 absorbs the rounding
    order = [p for p in range(10) if exc[p]] + [p for p in range(10) if not exc[p]]
    M = np.array(COLUMN_TABLE, dtype=np.float64)
    src_col = {name: c for c, name in enumerate(COLUMN_SOURCES)}
    rows = M.sum(axis=1)
    mean_row = sum(rows[p] * size[p] for p in range(10)) / voxel_size
    K = rows * (d_in / mean_row)
    P = 10
    k_local = np.zeros((P, P), dtype=np.int32)
    k_cc = np.zeros(P, dtype=np.int32)
    pos = {p: i for i, p in enumerate(order)}
    for ti, p in enumerate(order):
        for si, q in enumerate(order):
            name = COLUMN_POPS[q]
            if name in src_col:
                k_local[ti, si] = int(round(K[p] * M[p, src_col[name]] / rows[p]))
        k_cc[ti] = int(round(K[p] * M[p, src_col["CC"]] / rows[p]))
    offs = np.zeros(P + 1, dtype=np.int32)
    offs[1:] = np.cumsum([size[p] for p in order])
    n_exc_v = int(sum(size[p] for p in order if exc[p]))
    V = int(n_voxels)
    prob = region_matrix(V, density, seed + 7) if V > 1 else None
    sp = _ColumnSpec(V, P, offs.ctypes.data, int(voxel_size), n_exc_v, k_local.ctypes.data,
                     k_cc.ctypes.data, prob.ctypes.data if prob is not None else None,
                     d_within[0], d_within[1], d_cross[0], d_cross[1], w_mu, w_sigma, seed)
    N = V * int(voxel_size)
    row_ptr = np.empty(N + 1, dtype=np.int64)
    rc = lib().synth_columns(ctypes.byref(sp), row_ptr.ctypes.data, None, None, None, threads)
    if rc != 0:
        raise ValueError("synth_columns rejected the spec (code %d)" % rc)
    E = int(row_ptr[-1])
    col = np.empty(E, dtype=np.int32)
    w = np.empty(E, dtype=np.uint16)
    d = np.empty(E, dtype=np.uint8)
    rc = lib().synth_columns(ctypes.byref(sp), row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                             d.ctypes.data, threads)
    if rc != 0:
        raise ValueError("synth_columns rejected the spec (code %d)" % rc)
    ro = np.arange(V + 1, dtype=np.int32) * int(voxel_size)
    n_exc = np.full(V, n_exc_v, dtype=np.int32)
    g = Graph(N, V, ro, n_exc, row_ptr, col, w, d, max(d_within[1], d_cross[1] if V > 1 else 0))
    g.populations = dict(order=[COLUMN_POPS[p] for p in order], offsets=offs, k_local=k_local,
                         k_cc=k_cc)
    return g


def graph_from_dense(W: np.ndarray, Dl: np.ndarray, sizes, exc_frac: float = 0.8,
                     W2: np.ndarray | None = None) -> Graph:
    """Build a Graph from dense matrices W[target, source] (0 = no edge, values
    already representable in BF16) and Dl[target, source] (delays in steps).
    With W2, every edge also carries a second weight (an edge exists where W
    or W2 is non-zero).  Used for brute-force checks on tiny networks."""
    N = W.shape[0]
    ro, n_exc = region_layout(sizes, exc_frac)
    assert int(ro[-1]) == N
    cols, ws, w2s, ds = [], [], [], []
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    mask = W != 0 if W2 is None else (W != 0) | (W2 != 0)
    for j in range(N):
        tg = np.nonzero(mask[:, j])[0]
        order = np.lexsort((tg, Dl[tg, j]))
        tg = tg[order]
        cols.append(tg.astype(np.int32))
        ws.append(f64_to_bf16(W[tg, j]))
        if W2 is not None:
            w2s.append(f64_to_bf16(W2[tg, j]))
        ds.append(Dl[tg, j].astype(np.uint8))
        row_ptr[j + 1] = row_ptr[j] + len(tg)
    col = np.concatenate(cols) if cols else np.zeros(0, np.int32)
    w = np.concatenate(ws) if ws else np.zeros(0, np.uint16)
    d = np.concatenate(ds) if ds else np.zeros(0, np.uint8)
    w2 = None
    if W2 is not None:
        w2 = np.concatenate(w2s) if w2s else np.zeros(0, np.uint16)
    dmax = int(d.max()) if len(d) else 1
    return Graph(N, len(sizes), ro, n_exc, row_ptr, col, w, d, dmax, w2)


def with_second_weight(g: Graph, seed: int, w_mu: float = -1.0, w_sigma: float = 0.5,
                       alloc=None) -> Graph:
    """The same graph with a second weight on every edge, drawn independently
    from the lognormal(w_mu, w_sigma) of the first and rounded to BF16 (the
    connection table of Supplementary Table 5 stores one weight per channel,
    the channels' weights sharing a distribution).  Drawn in chunks;
    `alloc(n, dtype)` may supply the output array."""
    rng = np.random.default_rng(seed)
    E = g.n_edges
    w2 = np.empty(E, dtype=np.uint16) if alloc is None else alloc(E, np.uint16)
    out = w2 if isinstance(w2, np.ndarray) else w2.numpy().view(np.uint16)
    CH = 1 << 24
    for e0 in range(0, E, CH):
        e1 = min(E, e0 + CH)
        out[e0:e1] = f64_to_bf16(rng.lognormal(w_mu, w_sigma, e1 - e0))
    return dataclasses.replace(g, w2_bf16=w2)


# ---------------------------------------------------------------------------
# Neuron and synapse constants.  Channel order: AMPA, NMDA, GABA_A, GABA_B.
# Units: mV, ms, nF, microsiemens, nA.  The paper (Supplementary Table 5)
# names these fields but gives no values; these are textbook conductance-LIF
# values (membrane time constant 20 ms, reversal potentials 0/0/-70/-100 mV,
# decay times 2/100/10/100 ms), not the paper's.  The conductances and the
# constant current put the in-degree-100 network in an inhibition-dominated
# asynchronous irregular state near 9-10 Hz; `scale_for_degree` applies the in-degree rescaling of the
# conductances for other in-degrees.
# ---------------------------------------------------------------------------
PARAM_FIELDS = ("C", "gL", "VL", "Vth", "Vreset", "Tref", "Vu", "tau_u", "g_u",
                "I_ext", "drive_rate_hz", "drive_K", "w_ext")


def default_region_params(**over) -> dict:
    p = dict(C=0.5, gL=0.025, VL=-70.0, Vth=-50.0, Vreset=-55.0, Tref=2.0,
             Vu=(0.0, 0.0, -70.0, -100.0), tau_u=(2.0, 100.0, 10.0, 100.0),
             g_u=(0.006, 0.00002, 0.6, 0.002),
             I_ext=0.9, drive_rate_hz=10.0, drive_K=1.0, w_ext=2.0)
    p.update(over)
    return p


def scale_for_degree(p: dict, k_in: int, k_ref: int = 100) -> dict:
    """Rescale the synaptic conductances of a parameter set tuned at in-degree
    k_ref for in-degree k_in by k_ref/k_in, which keeps the mean synaptic
    input per neuron fixed.  (Methods Eq. 3 prints the factor as D/d; read
    dimensionally, conserving the input needs d/D.)"""
    q = dict(p)
    q["g_u"] = tuple(float(g) * k_ref / k_in for g in p["g_u"])
    return q


# Hemodynamic constants (Friston et al. 2000 standard values; the paper's
# Extended Data Table 4 gives the equations but no values).  Seconds.
BW_DEFAULT = dict(kappa=0.65, gamma=0.41, tau=0.98, alpha=0.32, rho=0.34, V0=0.02)


# ---------------------------------------------------------------------------
# Workload recipes.  Graph seed = 15963 + 10 * index, drive seed = +1,
# ensemble prior seed = +2.
# ---------------------------------------------------------------------------
def seed_for(index: int) -> int:
    return 15963 + 10 * index


def small_network(seed: int | None = None, threads: int = 0) -> Graph:
    """10,000 neurons (8,000 E / 2,000 I), one region, in-degree 100 from
    uniform sources, delays 1..20 steps at dt = 0.1 ms."""
    return make_graph([10_000], 100, seed_for(0) if seed is None else seed,
                      d_within=(1, 20), threads=threads)


def mid_network(threads: int = 0, alloc=None, n_regions: int = 100, region_size: int = 20_000,
                seed: int | None = None) -> Graph:
    """2,000,000 neurons in 100 regions of 20,000, in-degree 1,000 (800
    within, 200 across from excitatory sources); within delays 0.1-5 ms,
    across 5-20 ms at dt = 0.1 ms."""
    return make_graph([region_size] * n_regions, 1000, seed_for(1) if seed is None else seed,
                      k_within=800, d_within=(1, 50), d_cross=(50, 200), threads=threads,
                      alloc=alloc)


def ensemble_network(threads: int = 0, seed: int | None = None) -> Graph:
    """100,000 neurons in 20 regions of 5,000, in-degree 500 (400 within)."""
    return make_graph([5_000] * 20, 500, seed_for(2) if seed is None else seed,
                      k_within=400, d_within=(1, 50), d_cross=(50, 200), threads=threads)


def serving_request(rng: np.random.Generator) -> dict:
    """One request of the serving trace: size log-uniform in [1e4, 1e6],
    in-degree uniform in [100, 1000], 1-50 regions, 0.5-5 s of biological time."""
    n = int(round(math.exp(rng.uniform(math.log(1e4), math.log(1e6)))))
    R = int(rng.integers(1, 51))
    k = int(rng.integers(100, 1001))
    base = n // R
    sizes = [base] * R
    sizes[-1] += n - base * R
    bio_s = float(rng.uniform(0.5, 5.0))
    seed = int(rng.integers(1, 2**31))
    return dict(sizes=sizes, k_in=k, bio_s=bio_s, seed=seed)
