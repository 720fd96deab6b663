"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test names the passage of the paper it checks and the external fact it
checks against (a library routine, a closed form, a hand-derived linearisation,
brute force, or a Monte-Carlo bound on an exact Kalman posterior).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import enkf, metrics
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- Philox ----
def _numpy_philox(ctr, key):
    """numpy's Philox (4x64-10) increments its 256-bit counter before each
    block, so block(ctr) is what numpy returns from counter ctr - 1."""
    c = [int(x) for x in ctr]
    for i in range(4):
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = 2**64 - 1
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return np.array(bg.random_raw(4), dtype=np.uint64)


def test_philox_matches_numpy_library():
    rng = np.random.default_rng(1)
    cases = [((0, 0, 0, 0), (0, 0)), ((1, 0, 0, 0), (0, 0)),
             ((2**64 - 1,) * 4, (2**64 - 1,) * 2), ((12345, 678, 1, 0), (15964, 3))]
    for _ in range(20):
        cases.append((tuple(int(x) for x in rng.integers(0, 2**63, 4, dtype=np.uint64)),
                      tuple(int(x) for x in rng.integers(0, 2**63, 2, dtype=np.uint64))))
    for ctr, key in cases:
        assert np.array_equal(oracle.philox4x64(ctr, key), _numpy_philox(ctr, key)), (ctr, key)


# ------------------------------------------------------ Poisson drive -------
@pytest.mark.parametrize("lam", [0.0, 1e-3, 0.05, 0.5, 2.0])
def test_poisson_thresholds_match_scipy_cdf(lam):
    from scipy.stats import poisson
    thr = oracle.poisson_thresholds(lam)
    ref = []
    for k in range(16):
        t = math.floor(poisson.cdf(k, lam) * 2**32)
        if t >= 2**32:
            break
        ref.append(t)
    assert len(thr) == len(ref)
    assert np.all(np.abs(thr.astype(np.int64) - np.array(ref, dtype=np.int64)) <= 1)


def test_poisson_inversion_counts_follow_pmf():
    from scipy.stats import poisson
    lam = 0.7
    thr = oracle.poisson_thresholds(lam).astype(np.uint64)
    u = np.random.default_rng(2).integers(0, 2**32, 2_000_000, dtype=np.uint64)
    c = (u[:, None] >= thr[None, :]).sum(axis=1)
    n = len(u)
    obs = np.bincount(c, minlength=8)[:6]
    exp = poisson.pmf(np.arange(6), lam) * n
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 30.0  # 5 dof; p < 1e-5 above this
    assert abs(c.mean() - lam) < 5 * math.sqrt(lam / n)


# ---------------------------------------------------------------- LIF -------
def _iso_graph(n=4, exc_frac=0.8):
    W = np.zeros((n, n))
    return synth.graph_from_dense(W, np.ones((n, n), dtype=np.int64), [n], exc_frac)


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("case", [
    dict(dt=0.1, C=0.5, gL=0.025, I=0.6, Tref=2.0),
    dict(dt=0.05, C=0.25, gL=0.03, I=0.7, Tref=1.5),
])
def test_lif_interspike_interval_closed_form(precision, case):
    """Methods capacitance-voltage equation + Supp. Eq. 5 reset: under a
    constant current the discrete scheme is a linear recursion
    V' - Vinf = a (V - Vinf), a = 1 - dt gL / C, Vinf = VL + I/gL, so from
    V_reset the k-th free step crosses V_th for the first k >= k*,
    k* = ln((Vinf - Vth)/(Vinf - Vreset)) / ln a, and the period is n_ref + k."""
    p = synth.default_region_params(C=case["C"], gL=case["gL"], I_ext=case["I"], drive_rate_hz=0.0,
                                    Tref=case["Tref"], g_u=(0.0, 0.0, 0.0, 0.0))
    dt = case["dt"]
    a = 1.0 - dt * p["gL"] / p["C"]
    Vinf = p["VL"] + p["I_ext"] / p["gL"]
    kstar = math.log((Vinf - p["Vth"]) / (Vinf - p["Vreset"])) / math.log(a)
    assert 0.05 < kstar - math.floor(kstar) < 0.95  # away from a rounding tie
    k = math.ceil(kstar)
    n_ref = round(p["Tref"] / dt)
    g = _iso_graph()
    s = oracle.Sim(g, p, dt_ms=dt, bin_ms=1.0, precision=precision)
    s.set_state(V=np.full(4, p["Vreset"]), J=np.zeros((4, 4)), ref=np.zeros(4, np.int32))
    T = 5 * (n_ref + k) + 3
    s.step(T)
    st, ids = s.raster()
    first = st[ids == 0]
    expect = np.arange(k - 1, T, n_ref + k)
    assert np.array_equal(first, expect)


def test_lif_continuous_limit():
    """As dt -> 0 the discrete period approaches T_ref + tau_m ln((Vinf - Vreset)/(Vinf - Vth))."""
    p = synth.default_region_params(I_ext=0.6, drive_rate_hz=0.0, g_u=(0.0, 0.0, 0.0, 0.0))
    tau_m = p["C"] / p["gL"]
    Vinf = p["VL"] + p["I_ext"] / p["gL"]
    T_cont = p["Tref"] + tau_m * math.log((Vinf - p["Vreset"]) / (Vinf - p["Vth"]))
    dt = 0.002
    g = _iso_graph()
    s = oracle.Sim(g, p, dt_ms=dt, bin_ms=1.0, precision=64)
    s.set_state(V=np.full(4, p["Vreset"]), J=np.zeros((4, 4)), ref=np.zeros(4, np.int32))
    s.step(int(3 * T_cont / dt))
    st, ids = s.raster()
    period = np.diff(st[ids == 0]).mean() * dt
    assert abs(period - T_cont) < 2 * dt + 1e-3 * T_cont


# -------------------------------------------------- synaptic traces ---------
@pytest.mark.parametrize("exc_frac,channels", [(1.0, (0, 1)), (0.0, (2, 3))])
def test_trace_arrival_and_exponential_decay(exc_frac, channels):
    """Supp. Eq. 3: J(t+dt) = exp(-dt/tau) J(t) + w A(t).  A spike of neuron 0
    at step 0 over an edge of delay 3 reaches neuron 1's traces of the
    source's class at step 3; afterwards J_n = w exp(-dt/tau)^n."""
    W = np.zeros((2, 2))
    W[1, 0] = 0.75
    Dl = np.full((2, 2), 3)
    g = synth.graph_from_dense(W, Dl, [2], exc_frac)
    p = synth.default_region_params(I_ext=0.0, drive_rate_hz=0.0)
    s = oracle.Sim(g, p, precision=64)
    s.set_state(V=np.array([-49.0, -70.0]), J=np.zeros((4, 2)), ref=np.zeros(2, np.int32))
    traj = []
    for _ in range(200):
        s.step(1)
        traj.append(s.state()[1][:, 1].copy())
    traj = np.array(traj)  # [step, channel]
    st, ids = s.raster()
    assert list(zip(st, ids)) == [(0, 0)]
    assert np.all(traj[:3] == 0.0)
    other = [u for u in range(4) if u not in channels]
    assert np.all(traj[:, other] == 0.0)
    for u in channels:
        dec = math.exp(-0.1 / p["tau_u"][u])
        m = np.arange(197)
        expect = 0.75 * dec ** m
        assert np.allclose(traj[3:, u], expect, rtol=1e-13, atol=0)


def test_conductance_steady_state():
    """Methods, I_u = g_u (V_u - V) J_u with frozen traces: V converges to
    (gL VL + sum g J V_u + I) / (gL + sum g J)."""
    p = synth.default_region_params(I_ext=0.05, drive_rate_hz=0.0, Vth=100.0,
                                    tau_u=(1e300,) * 4, g_u=(0.01, 0.002, 0.03, 0.004))
    g = _iso_graph()
    s = oracle.Sim(g, p, precision=64)
    J = np.array([[0.8] * 4, [5.0] * 4, [0.6] * 4, [2.0] * 4])
    s.set_state(V=np.full(4, -60.0), J=J, ref=np.zeros(4, np.int32))
    s.step(40000)
    V = s.state()[0]
    gJ = np.array(p["g_u"]) * J[:, 0]
    Vss = (p["gL"] * p["VL"] + (gJ * np.array(p["Vu"])).sum() + p["I_ext"]) / (p["gL"] + gJ.sum())
    assert np.allclose(V, Vss, rtol=1e-9)


# ------------------------------------------------------------ delivery ------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_delivery_matches_brute_force_all_pairs(seed):
    """Supp. Algorithm 2 (push delivery) against a dense all-pairs sum:
    ring[(n + d_ij) mod D][i][class j] = sum over spiking j of q(W_ij)."""
    rng = np.random.default_rng(seed)
    sizes = [60, 36]
    N = sum(sizes)
    W = np.where(rng.random((N, N)) < 0.3, np.exp(rng.normal(-1, 0.5, (N, N))), 0.0)
    np.fill_diagonal(W, 0.0)
    W = synth.bf16_to_f64(synth.f64_to_bf16(W))
    Dl = rng.integers(1, 8, (N, N))
    g = synth.graph_from_dense(W, Dl, sizes)
    p = synth.default_region_params(drive_rate_hz=0.0)
    s = oracle.Sim(g, p, precision=32)
    info = s.info()
    D, S = info["D"], info["S"]
    exc = np.zeros(N, dtype=bool)
    for r in range(len(sizes)):
        exc[g.region_offsets[r]:g.region_offsets[r] + g.n_exc[r]] = True
    expect = np.zeros((D, N, 2), dtype=np.int64)
    total = 0
    for call in range(4):
        n = int(rng.integers(0, 50))
        ids = np.sort(rng.choice(N, size=int(rng.integers(1, 20)), replace=False)).astype(np.int32)
        s.deliver_only(ids, n)
        for i in range(N):
            for j in ids:
                if W[i, j] != 0.0:
                    expect[(n + Dl[i, j]) % D, i, 0 if exc[j] else 1] += int(np.rint(W[i, j] * 2.0**S))
                    total += 1
    assert np.array_equal(s.ring(), expect)
    assert s.info()["events"] == total


@pytest.mark.parametrize("seed", [3, 4])
def test_two_weight_delivery_matches_brute_force_all_pairs(seed):
    """Supp. Algorithm 2 with the two weights per edge of Supp. Table 5,
    against dense all-pairs sums: channel 2c + 0 of target i gets
    sum over spiking j of class c of q(W_ij), channel 2c + 1 sum of q(W2_ij).
    Some edges carry only one of the two weights."""
    rng = np.random.default_rng(seed)
    sizes = [50, 30]
    N = sum(sizes)
    E = rng.random((N, N)) < 0.3
    W = np.where(E & (rng.random((N, N)) < 0.9), np.exp(rng.normal(-1, 0.5, (N, N))), 0.0)
    W2 = np.where(E & (rng.random((N, N)) < 0.9), np.exp(rng.normal(-1, 0.5, (N, N))), 0.0)
    np.fill_diagonal(W, 0.0)
    np.fill_diagonal(W2, 0.0)
    W = synth.bf16_to_f64(synth.f64_to_bf16(W))
    W2 = synth.bf16_to_f64(synth.f64_to_bf16(W2))
    Dl = rng.integers(1, 8, (N, N))
    g = synth.graph_from_dense(W, Dl, sizes, W2=W2)
    s = oracle.Sim(g, synth.default_region_params(drive_rate_hz=0.0), precision=32)
    D, S = s.info()["D"], s.info()["S"]
    exc = np.zeros(N, dtype=bool)
    for r in range(len(sizes)):
        exc[g.region_offsets[r]:g.region_offsets[r] + g.n_exc[r]] = True
    expect = np.zeros((D, N, 4), dtype=np.int64)
    total = 0
    for call in range(4):
        n = int(rng.integers(0, 50))
        ids = np.sort(rng.choice(N, size=int(rng.integers(1, 20)), replace=False)).astype(np.int32)
        s.deliver_only(ids, n)
        for i in range(N):
            for j in ids:
                if W[i, j] != 0.0 or W2[i, j] != 0.0:
                    c = 0 if exc[j] else 2
                    slot = (n + Dl[i, j]) % D
                    expect[slot, i, c] += int(np.rint(W[i, j] * 2.0**S))
                    expect[slot, i, c + 1] += int(np.rint(W2[i, j] * 2.0**S))
                    total += 1
    assert np.array_equal(s.ring(), expect)
    assert s.info()["events"] == total


@pytest.mark.parametrize("exc_frac,channels", [(1.0, (0, 1)), (0.0, (2, 3))])
def test_two_weight_traces_take_their_own_weight(exc_frac, channels):
    """Supp. Eq. 3 per channel with two weights per edge: a spike of neuron 0
    at step 0 over an edge of delay 3 with weights (0.75, 0.3125) reaches
    neuron 1's first channel of the source's class with 0.75 and its second
    with 0.3125; afterwards each decays with its own exp(-dt/tau_u)."""
    W = np.zeros((2, 2))
    W2 = np.zeros((2, 2))
    W[1, 0], W2[1, 0] = 0.75, 0.3125
    g = synth.graph_from_dense(W, np.full((2, 2), 3), [2], exc_frac, W2=W2)
    p = synth.default_region_params(I_ext=0.0, drive_rate_hz=0.0)
    s = oracle.Sim(g, p, precision=64)
    s.set_state(V=np.array([-49.0, -70.0]), J=np.zeros((4, 2)), ref=np.zeros(2, np.int32))
    traj = []
    for _ in range(100):
        s.step(1)
        traj.append(s.state()[1][:, 1].copy())
    traj = np.array(traj)
    assert np.all(traj[:3] == 0.0)
    other = [u for u in range(4) if u not in channels]
    assert np.all(traj[:, other] == 0.0)
    for u, w in zip(channels, (0.75, 0.3125)):
        dec = math.exp(-0.1 / p["tau_u"][u])
        assert np.allclose(traj[3:, u], w * dec ** np.arange(97), rtol=1e-13, atol=0)


@pytest.mark.parametrize("precision", [32, 64])
def test_two_equal_weights_reduce_to_the_one_weight_form(small_graph, precision):
    """With the second weight equal to the first on every edge, the four
    channels receive what the two classes do in the one-weight form (the
    background drive included): raster and state are identical."""
    import dataclasses
    g2 = dataclasses.replace(small_graph, w2_bf16=np.array(small_graph.w_bf16).copy())
    p = synth.default_region_params()
    a = oracle.Sim(small_graph, p, seed=9, precision=precision)
    b = oracle.Sim(g2, p, seed=9, precision=precision)
    a.step(400)
    b.step(400)
    assert a.info()["spikes"] > 50
    for x, y in zip(a.raster(), b.raster()):
        assert np.array_equal(x, y)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    assert a.info()["S"] == b.info()["S"]


def test_two_weights_drive_feeds_both_excitatory_channels():
    """The Poisson background (Ext. Data Table 2) with two weights per edge
    and no recurrent edges: AMPA and NMDA traces follow the same arrivals,
    each decaying with its own constant; GABA traces stay 0."""
    W = np.zeros((4, 4))
    g = synth.graph_from_dense(W, np.ones((4, 4), int), [4], 1.0, W2=W)
    p = synth.default_region_params(I_ext=0.0, drive_rate_hz=2000.0, drive_K=1.0, w_ext=0.5)
    s = oracle.Sim(g, p, seed=5, precision=64)
    deA, deN = (math.exp(-0.1 / p["tau_u"][u]) for u in (0, 1))
    prev = np.zeros((4, 4))
    arrivals = 0
    for _ in range(300):
        s.step(1)
        J = s.state()[1]
        xA = J[0] - deA * prev[0]
        xN = J[1] - deN * prev[1]
        assert np.allclose(xA, xN, atol=1e-12)
        arrivals += int(np.count_nonzero(xA > 0.25))
        assert np.all(J[2:] == 0.0)
        prev = J.copy()
    assert arrivals > 120


def test_events_equal_spikes_times_out_degree(small_graph):
    """Every spike delivers exactly its out-degree (Supp. Algorithm 2)."""
    s = oracle.Sim(small_graph, synth.default_region_params(), seed=15964, precision=32)
    s.step(300)
    st, ids = s.raster()
    outdeg = np.diff(small_graph.row_ptr)
    info = s.info()
    assert info["spikes"] == len(ids) > 0
    assert info["events"] == int(outdeg[ids].sum())


# ---------------------------------------------------- Balloon-Windkessel ----
def test_bw_rest_is_exact_fixed_point():
    """Extended Data Table 4 with z = 0 from s=0, f=v=q=1: every derivative is
    zero exactly (E(1, rho) = rho) and y = 0."""
    x = np.array([0.0, 1.0, 1.0, 1.0])
    for _ in range(1000):
        y = oracle.bw_step(x, 0.0, 1e-3, synth.BW_DEFAULT)
        assert y == 0.0
    assert np.array_equal(x, [0.0, 1.0, 1.0, 1.0])


@pytest.mark.parametrize("z", [0.005, 0.02, 0.1])
def test_bw_constant_input_fixed_point(z):
    """Closed-form fixed point for constant z: s* = 0, f* = 1 + z/gamma,
    v* = f*^alpha, q* = v* E(f*, rho)/rho, y* from the BOLD equation."""
    bw = synth.BW_DEFAULT
    x = np.array([0.0, 1.0, 1.0, 1.0])
    for _ in range(300_000):
        y = oracle.bw_step(x, z, 1e-3, bw)
    f = 1 + z / bw["gamma"]
    v = f ** bw["alpha"]
    q = v * (1 - (1 - bw["rho"]) ** (1 / f)) / bw["rho"]
    k1, k2, k3 = 7 * bw["rho"], 2.0, 2 * bw["rho"] - 0.2
    ystar = bw["V0"] * (k1 * (1 - q) + k2 * (1 - q / v) + k3 * (1 - v))
    assert np.allclose(x, [0.0, f, v, q], rtol=1e-7, atol=1e-9)
    assert abs(y - ystar) <= 1e-7 * abs(ystar)


def test_bw_linear_response_matches_hand_jacobian():
    """Small-signal response against the Jacobian of Extended Data Table 4 at
    rest, derived by hand: E'(1) = (1 - rho) ln(1 - rho)."""
    bw = synth.BW_DEFAULT
    ka, ga, ta, al, rho, V0 = (bw[k] for k in ("kappa", "gamma", "tau", "alpha", "rho", "V0"))
    A = np.zeros((4, 4))
    A[0, 0], A[0, 1] = -ka, -ga
    A[1, 0] = 1.0
    A[2, 1], A[2, 2] = 1 / ta, -1 / (al * ta)
    A[3, 1] = (rho + (1 - rho) * math.log(1 - rho)) / rho / ta
    A[3, 2] = -(1 / al - 1) / ta
    A[3, 3] = -1 / ta
    B = np.array([1.0, 0, 0, 0])
    c = V0 * np.array([0.0, 0.0, (2.0 - (2 * rho - 0.2)), -(7 * rho + 2.0)])
    h, eps = 1e-3, 1e-6
    x = np.array([0.0, 1.0, 1.0, 1.0])
    dx = np.zeros(4)
    y_or, y_lin = [], []
    for k in range(20000):
        z = eps if k < 200 else 0.0
        y_or.append(oracle.bw_step(x, z, h, bw))
        dx = dx + h * (A @ dx + B * z)
        y_lin.append(c @ dx)
    y_or, y_lin = np.array(y_or), np.array(y_lin)
    assert np.max(np.abs(y_or - y_lin)) < 1e-4 * np.max(np.abs(y_lin))


# ---------------------------------------------------------------- EnKF ------
def _prior(R, rng, block_diag=False):
    n = enkf.BLOCK * R
    G = rng.normal(size=(n, n)) * 0.3
    if block_diag:
        mask = np.kron(np.eye(R), np.ones((enkf.BLOCK, enkf.BLOCK)))
        G = G * mask
    P = G @ G.T + 0.2 * np.eye(n)
    mu = rng.normal(size=n)
    return mu, P


def test_enkf_global_mode_matches_exact_kalman_posterior():
    """Textbook stochastic EnKF (one observer, all regions): as M grows the
    analysis mean and covariance approach the exact linear-Gaussian
    posterior mu + P H^T (H P H^T + G)^-1 (y - H mu), (I - K H) P."""
    rng = np.random.default_rng(5)
    R, M, obs_var = 2, 40000, 0.5
    mu, P = _prior(R, rng)
    n = len(mu)
    X = rng.multivariate_normal(mu, P, size=M)
    y = rng.normal(size=R) * 2
    eps = rng.normal(size=(M, R))
    Xa = enkf.diffusion_enkf(X, y, obs_var, 1.0, eps, mode="global")
    H = np.zeros((R, n))
    for r in range(R):
        H[r, enkf.BLOCK * r + enkf.Y_INDEX] = 1
    K = P @ H.T @ np.linalg.inv(H @ P @ H.T + obs_var * np.eye(R))
    mu_a = mu + K @ (y - H @ mu)
    P_a = (np.eye(n) - K @ H) @ P
    sd = np.sqrt(np.diag(P))
    assert np.all(np.abs(Xa.mean(0) - mu_a) < 8 * sd / np.sqrt(M) * (1 + np.abs(y - H @ mu).max()))
    Pa_hat = np.cov(Xa.T)
    assert np.allclose(np.diag(Pa_hat), np.diag(P_a), rtol=0.06, atol=0.01)


def test_enkf_diffusion_fusion_weights_own_observer_by_gamma():
    """Supp. Algorithm 3 step 7 with independent regions: the other observers'
    gains on block b vanish, so block b moves by gamma times its own exact
    single-observer correction."""
    rng = np.random.default_rng(6)
    R, M, obs_var, gamma = 3, 40000, 0.3, 0.7
    mu, P = _prior(R, rng, block_diag=True)
    X = rng.multivariate_normal(mu, P, size=M)
    y = mu[[enkf.BLOCK * r + enkf.Y_INDEX for r in range(R)]] + rng.normal(size=R)
    eps = rng.normal(size=(M, R))
    Xa = enkf.diffusion_enkf(X, y, obs_var, gamma, eps)
    for b in range(R):
        h = enkf.BLOCK * b + enkf.Y_INDEX
        blk = slice(enkf.BLOCK * b, enkf.BLOCK * (b + 1))
        K = P[blk, h] / (P[h, h] + obs_var)
        expect = mu[blk] + gamma * K * (y[b] - mu[h])
        sd = np.sqrt(np.diag(P)[blk])
        assert np.all(np.abs(Xa.mean(0)[blk] - expect) < 10 * sd / np.sqrt(M) * (1 + abs(y[b] - mu[h])))


def test_enkf_perfect_observation_and_no_information_limits():
    rng = np.random.default_rng(7)
    R, M = 4, 64
    mu, P = _prior(R, rng)
    X = rng.multivariate_normal(mu, P, size=M)
    y = rng.normal(size=R)
    zero = np.zeros((M, R))
    # Gamma -> 0, gamma = 1: every observed BOLD value lands on the observation
    Xa = enkf.diffusion_enkf(X, y, 1e-14, 1.0, zero)
    for r in range(R):
        assert np.allclose(Xa[:, enkf.BLOCK * r + enkf.Y_INDEX], y[r], atol=1e-9)
    # Gamma -> infinity: nothing moves
    Xb = enkf.diffusion_enkf(X, y, 1e14, 0.6, rng.normal(size=(M, R)))
    assert np.allclose(Xb, X, atol=1e-5)


def test_enkf_single_observer_is_textbook_enkf():
    """With one region the diffusion filter has one observer and is the
    textbook stochastic EnKF (the global mode)."""
    rng = np.random.default_rng(8)
    mu, P = _prior(1, rng)
    X = rng.multivariate_normal(mu, P, size=50)
    y = rng.normal(size=1)
    eps = rng.normal(size=(50, 1))
    assert np.allclose(enkf.diffusion_enkf(X, y, 0.4, 0.3, eps),
                       enkf.diffusion_enkf(X, y, 0.4, 0.3, eps, mode="global"), atol=1e-12)


def test_lagged_pcc_matches_numpy_corrcoef():
    rng = np.random.default_rng(9)
    a = rng.normal(size=100)
    b = np.roll(a, 2) + 0.1 * rng.normal(size=100)
    for lag in (0, 1, 2, 5):
        ref = np.corrcoef(b[lag:], a[:100 - lag])[0, 1]
        assert abs(metrics.lagged_pcc(b, a, lag) - ref) < 1e-12


# ------------------------------------------------ FP32 against FP64 ---------
@pytest.mark.slow
def test_matched_fp32_statistics_agree_with_fp64(small_graph):
    """The op-order-matched FP32 oracle and the FP64 oracle describe the same
    dynamics: over 2 s the rate and ISI CV agree to within what two
    trajectories of this chaotic network differ by (the rasters themselves
    diverge after the first near-threshold crossing)."""
    res = {}
    for prec in (32, 64):
        s = oracle.Sim(small_graph, synth.default_region_params(), seed=15964, precision=prec)
        s.step(20000)
        st, ids = s.raster()
        res[prec] = (len(ids), metrics.isi_cv(st, ids))
    r32, r64 = res[32][0], res[64][0]
    assert abs(r32 - r64) / r64 < 0.03
    assert abs(res[32][1] - res[64][1]) < 0.05


# ---------------------------------------------------- background OU current --
def _empty_graph(N):
    """N unconnected neurons in one region (all excitatory)."""
    return synth.Graph(N, 1, np.array([0, N], np.int32), np.array([N], np.int32),
                       np.zeros(N + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint16),
                       np.zeros(0, np.uint8), 1)


def test_box_muller_draws_are_standard_normal():
    """The OU noise xi: Box-Muller of Philox words is N(0, 1) (KS test and
    the first two moments)."""
    stats = pytest.importorskip("scipy.stats")
    words = np.concatenate([oracle.philox4x64([n, 7, 4, 0], [3, 9]) for n in range(12000)])
    z = np.array([oracle.box_muller(int(w)) for w in words])
    assert abs(z.mean()) < 5.0 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_ou_current_stationary_moments():
    """Eq. 1 discretised (Euler-Maruyama) is the AR(1) process
    I' = a I + (1 - a) mu + s xi with a = 1 - dt/tau, s = sigma sqrt(2 dt/tau):
    stationary mean mu, variance s^2 / (1 - a^2) = sigma^2 / (1 - dt / (2 tau)),
    lag-1 autocorrelation a (Extended Data Table 2 values)."""
    N, dt, mu, sigma, tau = 20000, 0.1, 0.66, 0.12, 10.0
    p = synth.default_region_params(ou_mu=mu, ou_sigma=sigma, ou_tau=tau, drive_rate_hz=0.0)
    s = oracle.Sim(_empty_graph(N), p, precision=64)
    s.step(1500)  # 15 time constants from I = mu
    a_prev = s.ibg()
    s.step(1)
    a_now = s.ibg()
    var_st = sigma ** 2 / (1.0 - dt / (2.0 * tau))
    assert abs(a_now.mean() - mu) < 5.0 * math.sqrt(var_st / N)
    assert abs(a_now.var() / var_st - 1.0) < 5.0 * math.sqrt(2.0 / N)
    a = 1.0 - dt / tau
    r = np.corrcoef(a_prev, a_now)[0, 1]
    assert abs(r - a) < 5.0 * (1.0 - a * a) / math.sqrt(N)


def test_ou_relaxation_without_noise_is_exact():
    """sigma = 0: I_n = mu + (I_0 - mu) (1 - dt/tau)^n."""
    N, mu, tau = 64, 0.5, 7.0
    p = synth.default_region_params(ou_mu=mu, ou_sigma=0.0, ou_tau=tau, drive_rate_hz=0.0)
    s = oracle.Sim(_empty_graph(N), p, precision=64)
    I0 = np.linspace(-1.0, 2.0, N)
    s.set_ibg(I0)
    s.step(137)
    expect = mu + (I0 - mu) * (1.0 - 0.1 / tau) ** 137
    assert np.allclose(s.ibg(), expect, rtol=1e-12, atol=1e-14)


def test_ou_current_enters_the_membrane_bracket_with_its_old_value():
    """Eq. 5 (bracket times dt/C): one step from a chosen state with no
    synaptic input gives V' = V + (dt/C)(-gL (V - VL) + I_ext + I_bg(t))."""
    N = 8
    p = synth.default_region_params(ou_mu=0.3, ou_sigma=0.0, ou_tau=5.0, drive_rate_hz=0.0,
                                    Vth=100.0)
    s = oracle.Sim(_empty_graph(N), p, precision=64)
    V0 = np.linspace(-70.0, -52.0, N)
    I0 = np.linspace(-0.4, 0.9, N)
    s.set_state(V=V0, J=np.zeros((4, N)), ref=np.zeros(N, np.int32))
    s.set_ibg(I0)
    s.step(1)
    expect = V0 + (0.1 / p["C"]) * (-p["gL"] * (V0 - p["VL"]) + p["I_ext"] + I0)
    assert np.allclose(s.state()[0], expect, rtol=1e-13, atol=1e-12)


# -------------------------------------------- heterogeneous injected current --
@pytest.mark.parametrize("k", [0.5, 2.5, 9.0])
def test_gamma_draws_follow_the_gamma_law(k):
    """Per-neuron I_ext factors (Methods: I_ext,i Gamma distributed):
    Marsaglia-Tsang draws against scipy's Gamma(k) (KS), mean and variance k
    (k < 1 goes through G(k + 1) U^(1/k))."""
    stats = pytest.importorskip("scipy.stats")
    n = 20000
    g = np.array([oracle.gamma_draw(k, 11, 3, i) for i in range(n)])
    assert abs(g.mean() - k) < 5.0 * math.sqrt(k / n)
    assert abs(g.var() / k - 1.0) < 5.0 * math.sqrt((2.0 + 6.0 / k) / n)
    assert stats.kstest(g, stats.gamma(k).cdf).pvalue > 1e-3


def test_heterogeneous_current_enters_the_membrane_bracket():
    """With iext_shape k, neuron i's injected current is I_ext * G_i / k
    inside the dt/C bracket."""
    N, k = 16, 3.0
    p = synth.default_region_params(I_ext=0.4, iext_shape=k, drive_rate_hz=0.0, Vth=100.0)
    s = oracle.Sim(_empty_graph(N), p, seed=21, net_id=2, precision=64)
    V0 = np.linspace(-70.0, -52.0, N)
    s.set_state(V=V0, J=np.zeros((4, N)), ref=np.zeros(N, np.int32))
    s.step(1)
    f = np.array([oracle.gamma_draw(k, 21, 2, i) / k for i in range(N)])
    expect = V0 + (0.1 / p["C"]) * (-p["gL"] * (V0 - p["VL"]) + p["I_ext"] * f)
    assert np.allclose(s.state()[0], expect, rtol=1e-13, atol=1e-12)
    assert f.std() > 0.1  # the factors differ between neurons


# ------------------------------------------- bins, z and the BOLD samples ----
def _isolated_spike_steps(k, n_ref, m0, T):
    """Spike steps of an isolated neuron under constant current that starts at
    V_reset with m0 refractory steps left: it is clamped for m0 steps, then
    needs k free steps to cross (the closed form of the ISI pin above), so it
    fires at m0 + k - 1 and every n_ref + k steps after."""
    return list(range(m0 + k - 1, T, n_ref + k))


@pytest.mark.parametrize("precision", [32, 64])
def test_bin_counts_z_and_bold_samples_follow_the_spike_schedule(precision):
    """Fig. 2a and Extended Data Table 4: at the end of every bin of spb
    steps, z_r = z_scale x (spikes of region r in that bin) / N_r drives one
    Euler step of the hemodynamic model, the count restarts from zero, and
    the BOLD value after every bins_per_tr-th bin is sampled.  Regions of
    different sizes and currents, a bin of 5 steps and a TR of 7 bins (not
    a multiple of any spike period): the spike schedule comes from the
    closed-form ISI, the hemodynamic steps from the pinned bw_step, so a
    count divided by N instead of N_r, a count that is not reset, or a bin
    or TR index off by one fails."""
    sizes = [3, 5, 2, 6]
    currents = [0.6, 0.75, 0.9, 0.68]
    dt, bin_ms, tr_ms, z_scale = 0.1, 0.5, 3.5, 3.0
    spb, bins_per_tr = 5, 7
    N, R = sum(sizes), len(sizes)
    g = synth.graph_from_dense(np.zeros((N, N)), np.ones((N, N), dtype=np.int64), sizes, 0.5)
    params = [synth.default_region_params(I_ext=I, drive_rate_hz=0.0, g_u=(0.0, 0.0, 0.0, 0.0))
              for I in currents]
    rng = np.random.default_rng(11)
    m0 = rng.integers(0, 40, N).astype(np.int32)
    T = 2 * spb * bins_per_tr * 13 + 17  # ends inside a bin
    s = oracle.Sim(g, params, dt_ms=dt, bin_ms=bin_ms, tr_ms=tr_ms, z_scale=z_scale,
                   precision=precision)
    s.set_state(V=np.full(N, params[0]["Vreset"]), J=np.zeros((4, N)), ref=m0)
    s.step(T)
    ro = np.asarray(g.region_offsets)
    counts = np.zeros((T // spb + 1, R), dtype=np.int64)
    spikes = []
    for r in range(R):
        p = params[r]
        a = 1.0 - dt * p["gL"] / p["C"]
        Vinf = p["VL"] + p["I_ext"] / p["gL"]
        kstar = math.log((Vinf - p["Vth"]) / (Vinf - p["Vreset"])) / math.log(a)
        assert 0.05 < kstar - math.floor(kstar) < 0.95  # away from a rounding tie
        k, n_ref = math.ceil(kstar), round(p["Tref"] / dt)
        for i in range(ro[r], ro[r + 1]):
            for n in _isolated_spike_steps(k, n_ref, int(m0[i]), T):
                counts[n // spb, r] += 1
                spikes.append((n, i))
    st, ids = s.raster()
    assert sorted(spikes) == sorted(zip(st.tolist(), ids.tolist()))
    x = np.tile(np.array([0.0, 1.0, 1.0, 1.0]), (R, 1))
    bold = []
    n_bins = T // spb
    for b in range(n_bins):
        y = np.zeros(R)
        for r in range(R):
            z = z_scale * float(counts[b, r]) / float(sizes[r])
            xr = x[r].copy()
            y[r] = oracle.bw_step(xr, z, bin_ms * 1e-3, synth.BW_DEFAULT)
            x[r] = xr
        if (b + 1) % bins_per_tr == 0:
            bold.append(y)
    got = s.bold()
    assert got.shape == (n_bins // bins_per_tr, R) and len(bold) == got.shape[0] > 10
    assert np.array_equal(got, np.array(bold))
    assert np.array_equal(s.bw_state(), x)
    # the partial last bin is still counting
    assert np.array_equal(s.counts(), counts[n_bins])
    assert s.info()["bins_done"] == n_bins


# ------------------------------------------- EnKF state helpers (Sec. 6) ----
def test_pack_and_unpack_state_follow_the_region_block_layout():
    """Supplementary Sec. 6: the state of a member holds, per region, the
    hyperparameters and the hemodynamic state with its BOLD value.  The
    block of region r is [theta_AMPA, theta_GABA_A, s, f, v, q, y], written
    out by hand here for two members and two regions."""
    theta = np.array([[[0.1, 0.2], [0.3, 0.4]], [[-0.1, -0.2], [-0.3, -0.4]]])
    bw = np.array([[[1.0, 1.1, 1.2, 1.3], [2.0, 2.1, 2.2, 2.3]],
                   [[3.0, 3.1, 3.2, 3.3], [4.0, 4.1, 4.2, 4.3]]])
    y = np.array([[0.01, 0.02], [0.03, 0.04]])
    X = enkf.pack_state(theta, bw, y)
    expect = np.array([
        [0.1, 0.2, 1.0, 1.1, 1.2, 1.3, 0.01, 0.3, 0.4, 2.0, 2.1, 2.2, 2.3, 0.02],
        [-0.1, -0.2, 3.0, 3.1, 3.2, 3.3, 0.03, -0.3, -0.4, 4.0, 4.1, 4.2, 4.3, 0.04],
    ])
    assert np.array_equal(X, expect)
    th2, bw2, y2 = enkf.unpack_state(expect)
    assert np.array_equal(th2, theta) and np.array_equal(bw2, bw) and np.array_equal(y2, y)
    # the named positions agree with the layout
    assert enkf.BLOCK == 7 and enkf.Y_INDEX == 6 and enkf.THETA == (0, 1)


def test_constrain_clips_hyperparameters_and_floors_flow_volume_q():
    """After an analysis the log scales go back into the prior support
    [theta_lo, theta_hi] and f, v, q are kept at or above the floor; s and y
    are left as they are.  Expected values written out by hand."""
    lo, hi, floor = -0.5, 0.5, 0.01
    X = np.array([
        [0.7, -0.9, -0.3, 0.005, -1.0, 0.02, -0.04, 0.2, -0.5, 0.1, 1.5, 0.01, -2.0, 0.3],
        [-0.5, 0.5, 0.4, 2.0, 0.0, 0.009, 0.05, 1e3, -1e3, -0.2, 0.011, 0.5, 0.0099, -0.1],
    ])
    expect = np.array([
        [0.5, -0.5, -0.3, 0.01, 0.01, 0.02, -0.04, 0.2, -0.5, 0.1, 1.5, 0.01, 0.01, 0.3],
        [-0.5, 0.5, 0.4, 2.0, 0.01, 0.01, 0.05, 0.5, -0.5, -0.2, 0.011, 0.5, 0.01, -0.1],
    ])
    got = enkf.constrain(X, lo, hi, floor)
    assert np.array_equal(got, expect)
    assert np.array_equal(X[0, :2], [0.7, -0.9])  # the input is not modified


def test_random_walk_moves_only_the_hyperparameters_and_clips():
    """Supplementary Sec. 6: theta(t) = theta(t - 1) + eps_theta with eps_theta
    = rw_sigma x xi, clipped to the prior support; nothing else moves.
    Expected values written out by hand (rw_sigma = 0.5)."""
    lo, hi = -1.0, 1.0
    X = np.array([[0.2, -0.8, 9.0, 9.1, 9.2, 9.3, 9.4, 0.9, 0.0, 8.0, 8.1, 8.2, 8.3, 8.4]])
    xi = np.array([[[1.0, -1.0], [0.4, 0.6]]])   # [M=1, R=2, 2]
    expect = np.array([[0.7, -1.0, 9.0, 9.1, 9.2, 9.3, 9.4, 1.0, 0.3, 8.0, 8.1, 8.2, 8.3, 8.4]])
    got = enkf.random_walk(X, 0.5, xi, lo, hi)
    assert np.allclose(got, expect, rtol=0, atol=1e-15)
    assert np.array_equal(got[:, 2:7], X[:, 2:7]) and np.array_equal(got[:, 9:], X[:, 9:])


# ------------------------------------------------ spike binning (b_t) -------
@pytest.mark.parametrize("spb,dt", [(5, 0.1), (10, 0.1), (1, 0.1), (2, 0.5)])
def test_binned_delivery_matches_brute_force(spb, dt):
    """Supplementary Sec. 3, "Numerical method": with a spike bin b_t the
    accumulated spike A_j(t) is non-zero only at bin edges t = k b_t, where it
    marks a spike of j in (t - b_t, t]; Eq. 3 then adds w A_j(t).  So a spike
    emitted in any step of bin [k spb, (k + 1) spb) acts as if emitted in the
    bin's last step and reaches, over an edge of delay d, the accumulator
    consumed at step (k + 1) spb - 1 + d; a neuron that fires twice in one bin
    counts once.  Isolated sources (one of them fast enough to fire twice in
    a bin) drive silent targets over random delays; after every step the
    pending accumulators must equal the brute-force sum over the raster's
    spikes, edge by edge, exactly."""
    n_src, n_tgt = 6, 9
    N = n_src + n_tgt
    rng = np.random.default_rng(spb)
    W = np.zeros((N, N))
    Dl = np.ones((N, N), dtype=np.int64)
    W[n_src:, :n_src] = synth.bf16_to_f64(synth.f64_to_bf16(rng.lognormal(-1, 0.5, (n_tgt, n_src))))
    Dl[n_src:, :n_src] = rng.integers(1, 13, (n_tgt, n_src))
    W[n_src + 2, 0] = 0.0  # a missing edge
    src = synth.default_region_params(I_ext=2.5, drive_rate_hz=0.0, Tref=2.0)
    fast = dict(src, Tref=0.0, I_ext=12.0)
    tgt = synth.default_region_params(I_ext=0.0, drive_rate_hz=0.0, g_u=(0.0, 0.0, 0.0, 0.0))
    # regions: the fast source, the other sources, the targets (half E, half I each)
    s = oracle.Sim(synth.graph_from_dense(W, Dl, [1, n_src - 1, n_tgt], 0.5), [fast, src, tgt],
                   dt_ms=dt, bin_ms=spb * dt, tr_ms=spb * dt * 4, precision=64, bin_spikes=True)
    g = s.graph
    D = s.info()["D"]
    S = s.info()["S"]
    dmax = int(Dl[n_src:, :n_src].max())
    assert D == dmax + spb
    ro = np.asarray(g.region_offsets)
    cls = np.zeros(N, dtype=np.int64)
    for r in range(3):
        cls[ro[r] + int(g.n_exc[r]):ro[r + 1]] = 1
    rp, col = np.asarray(g.row_ptr), np.asarray(g.col)
    wq = np.rint(np.ldexp(synth.bf16_to_f64(np.asarray(g.w_bf16)), S)).astype(np.int64)
    dly = np.asarray(g.delay).astype(np.int64)
    T = 40 * spb + 3
    twice = False
    for t in range(T):
        s.step(1)
        st, ids = s.raster()
        seen = set()
        want = np.zeros((D, N, 2), dtype=np.int64)
        for m, j in zip(st.tolist(), ids.tolist()):
            rel = (m // spb + 1) * spb - 1
            if (j, rel) in seen:
                twice = True
                continue
            seen.add((j, rel))
            for e in range(rp[j], rp[j + 1]):
                a = rel + dly[e]
                if a >= t + 1:   # not yet consumed
                    want[a % D, col[e], cls[j]] += wq[e]
        assert np.array_equal(s.ring(), want), t
        assert np.all(ids < n_src)   # the targets stay silent
    assert len(st) > 20
    assert twice == (spb > 1)       # the fast source fired twice within a bin
    # with one step per bin, binning changes nothing
    if spb == 1:
        s0 = oracle.Sim(s.graph, [fast, src, tgt], dt_ms=dt, bin_ms=dt, tr_ms=dt * 4,
                        precision=64)
        s0.step(T)
        assert np.array_equal(s0.raster()[1], s.raster()[1])
        assert np.array_equal(s0.state()[1], s.state()[1])


@pytest.mark.parametrize("precision", [32, 64])
def test_threaded_timing_variant_gives_identical_results(small_graph, precision):
    """The oracle's all-core timing variant (neuron ranges per thread, spike
    lists joined in order, exact integer accumulation with atomic adds) gives
    the single-threaded oracle's raster, state, accumulators and BOLD."""
    p = synth.default_region_params()
    a = oracle.Sim(small_graph, p, seed=5, tr_ms=20.0, precision=precision)
    b = oracle.Sim(small_graph, p, seed=5, tr_ms=20.0, precision=precision, threads=4)
    a.step(400)
    b.step(400)
    for x, y in zip(a.raster(), b.raster()):
        assert np.array_equal(x, y)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.ring(), b.ring())
    assert np.array_equal(a.bold(), b.bold())
    assert a.info() == b.info() and a.info()["spikes"] > 500
