"""HMDA ensemble on the GPU against the oracle.

Members share one graph and differ in their AMPA/GABA_A conductance scales
and Philox key, so each member must equal a single network built with the
scaled parameters.  The FP64 analysis (Supplementary Algorithm 3) is checked
against the numpy oracle applied to ensembles that the CPU oracle simulated
itself (no GPU value enters the oracle side); noise draws are passed to both.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import enkf as oenkf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LO, HI = np.log(0.5), np.log(2.0)


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _graph():
    return synth.make_graph([600, 500, 700, 400], 60, 31, k_within=48, d_within=(1, 20),
                            d_cross=(20, 60))


def _member_params(base, theta_m):
    out = []
    for r, p in enumerate(base):
        q = dict(p)
        g = list(q["g_u"])
        g[0] = g[0] * math.exp(theta_m[r, 0])   # the C library's exp, as the library uses
        g[2] = g[2] * math.exp(theta_m[r, 1])
        q["g_u"] = tuple(g)
        out.append(q)
    return out


def test_members_equal_single_networks():
    from paper_2211_15963_gb300 import dbnet
    g = _graph()
    base = [synth.default_region_params(I_ext=0.85 + 0.03 * r) for r in range(g.n_regions)]
    M = 3
    theta = np.random.default_rng(1).uniform(LO, HI, (M, g.n_regions, 2))
    opts = dict(seed=7, net_id=100, tr_ms=10.0, raster_capacity=1 << 20)
    ens = dbnet.Ensemble(g, base, M, theta, opts)
    ens.step(500)
    for m in range(M):
        net = dbnet.Network(g, _member_params(base, theta[m]), dict(opts, net_id=100 + m))
        net.step(500)
        a, b = ens.member_state(m), net.state()
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        assert np.array_equal(ens.member_bold(m), net.bold())
        sa, sb = ens.member_spikes(m), net.spikes()
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
        net.close()
    ens.close()


def test_two_weight_members_equal_single_networks():
    """Ensemble members over a graph with two weights per edge equal the
    same networks run alone."""
    from paper_2211_15963_gb300 import dbnet
    g = synth.with_second_weight(_graph(), 5)
    base = [synth.default_region_params(I_ext=0.85 + 0.03 * r) for r in range(g.n_regions)]
    M = 2
    theta = np.random.default_rng(2).uniform(LO, HI, (M, g.n_regions, 2))
    opts = dict(seed=8, net_id=200, tr_ms=10.0, raster_capacity=1 << 20)
    ens = dbnet.Ensemble(g, base, M, theta, opts)
    ens.step(400)
    for m in range(M):
        net = dbnet.Network(g, _member_params(base, theta[m]), dict(opts, net_id=200 + m))
        net.step(400)
        assert net.stats()["two_weights"] == 1
        for x, y in zip(ens.member_state(m), net.state()):
            assert np.array_equal(x, y)
        assert np.array_equal(ens.member_bold(m), net.bold())
        sa, sb = ens.member_spikes(m), net.spikes()
        assert len(sb[1]) > 100
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
        net.close()
    ens.close()


@pytest.mark.parametrize("mode", ["diffusion", "global"])
def test_analysis_matches_oracle_enkf(mode):
    from paper_2211_15963_gb300 import dbnet
    g = _graph()
    R = g.n_regions
    base = [synth.default_region_params(I_ext=0.85 + 0.03 * r) for r in range(R)]
    M, TR_STEPS = 8, 200
    rng = np.random.default_rng(2)
    theta = rng.uniform(LO, HI, (M, R, 2))
    obs_var, gamma, rw = 1e-8, 0.6, 0.05
    opts = dict(seed=9, net_id=40, tr_ms=20.0, z_scale=20.0)
    k = dict(obs_var=obs_var, gamma=gamma, rw_sigma=rw, theta_lo=LO, theta_hi=HI, floor=1e-2,
             mode=dbnet.DBENS_DIFFUSION if mode == "diffusion" else dbnet.DBENS_GLOBAL)
    ens = dbnet.Ensemble(g, base, M, theta, opts, k)
    ens.step(TR_STEPS)
    # oracle side: its own member simulations
    sims = [oracle.Sim(g, _member_params(base, theta[m]), seed=9, net_id=40 + m, tr_ms=20.0,
                       z_scale=20.0, precision=32) for m in range(M)]
    for s in sims:
        s.step(TR_STEPS)
    bw_o = np.stack([s.bw_state() for s in sims])
    y_o = np.stack([s.bold()[-1] for s in sims])
    X = oenkf.pack_state(theta, bw_o, y_o)
    y_obs = y_o.mean(0) * 1.3 + 1e-5
    eps = rng.normal(size=(M, R))
    xi = rng.normal(size=(M, R, 2))
    ypred = ens.assimilate(y_obs, eps, xi)
    assert np.allclose(ypred, y_o.mean(0), rtol=1e-9, atol=1e-15)
    Xa = oenkf.diffusion_enkf(X, y_obs, obs_var, gamma, eps, mode=mode)
    Xa = oenkf.constrain(Xa, LO, HI, 1e-2)
    Xa = oenkf.random_walk(Xa, rw, xi, LO, HI)
    th_o, bw_o2, _ = oenkf.unpack_state(Xa)
    th_g, bw_g, _ = ens.read()
    assert np.allclose(th_g, th_o, rtol=1e-8, atol=1e-11)
    assert np.allclose(bw_g, bw_o2, rtol=1e-8, atol=1e-13)
    assert np.abs(th_g - theta).max() > 1e-3  # the analysis moved the scales
    ens.close()


def test_twin_experiment_recovers_direction():
    """A hidden member generates the observations; the ensemble mean of the
    AMPA scales moves toward the hidden values over repeated analyses."""
    from paper_2211_15963_gb300 import dbnet
    g = _graph()
    R = g.n_regions
    base = [synth.default_region_params() for _ in range(R)]
    M, TR_STEPS = 24, 2000   # TR = 200 ms of biological time
    rng = np.random.default_rng(3)
    truth = np.zeros((1, R, 2))
    truth[0, :, 0] = np.log(1.6)
    opts = dict(seed=21, tr_ms=200.0, z_scale=50.0)
    hidden = dbnet.Network(g, _member_params(base, truth[0]), dict(opts, net_id=999))
    theta0 = rng.uniform(np.log(0.6), np.log(1.0), (M, R, 2))
    ens = dbnet.Ensemble(g, base, M, theta0, dict(opts, net_id=0),
                         dict(obs_var=1e-9, gamma=0.7, rw_sigma=0.01, theta_lo=LO, theta_hi=HI))
    start = theta0[:, :, 0].mean()
    for _ in range(12):
        hidden.step(TR_STEPS)
        ens.step(TR_STEPS)
        y = hidden.bold()[-1]
        ens.assimilate(y)
    th, _, _ = ens.read()
    end = th[:, :, 0].mean()
    assert abs(end - np.log(1.6)) < abs(start - np.log(1.6))
    hidden.close()
    ens.close()


def _scaled(base, theta_m, targets):
    """Region parameters with each target scaled by exp(theta) (math.exp, the
    C library's, as the library uses at create)."""
    from paper_2211_15963_gb300 import dbnet
    out = []
    for r, p in enumerate(base):
        q = dict(p)
        g = list(q["g_u"])
        for sl, t in enumerate(targets):
            f = math.exp(theta_m[r, sl])
            if t == dbnet.DBENS_T_IEXT:
                q["I_ext"] = q["I_ext"] * f
            elif t != dbnet.DBENS_T_NONE:
                g[t - dbnet.DBENS_T_AMPA] = g[t - dbnet.DBENS_T_AMPA] * f
        q["g_u"] = tuple(g)
        out.append(q)
    return out


def test_task_variant_members_equal_single_networks():
    """Task variant (Supp. Sec. 6): the scale multiplies the region's
    injected current, heterogeneous per neuron (Gamma, k = 3); each member
    (its own factors through its net_id) equals a single network."""
    from paper_2211_15963_gb300 import dbnet
    g = _graph()
    base = [synth.default_region_params(I_ext=0.8 + 0.03 * r, iext_shape=3.0)
            for r in range(g.n_regions)]
    M = 3
    targets = (dbnet.DBENS_T_IEXT, dbnet.DBENS_T_NONE)
    theta = np.random.default_rng(4).uniform(LO, HI, (M, g.n_regions, 2))
    opts = dict(seed=8, net_id=200, tr_ms=10.0, raster_capacity=1 << 20)
    ens = dbnet.Ensemble(g, base, M, theta, opts, dict(target=targets))
    ens.step(400)
    for m in range(M):
        net = dbnet.Network(g, _scaled(base, theta[m], targets), dict(opts, net_id=200 + m))
        net.step(400)
        for x, y in zip(ens.member_state(m), net.state()):
            assert np.array_equal(x, y)
        sa, sb = ens.member_spikes(m), net.spikes()
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
        net.close()
    ens.close()


def test_task_twin_experiment_recovers_injected_current():
    """A hidden member with every region's injected current scaled by 1.5
    makes the observations; assimilating the injected-current scale moves
    the ensemble toward it."""
    from paper_2211_15963_gb300 import dbnet
    g = _graph()
    R = g.n_regions
    base = [synth.default_region_params(I_ext=0.7) for _ in range(R)]
    targets = (dbnet.DBENS_T_IEXT, dbnet.DBENS_T_NONE)
    M, TR_STEPS = 24, 2000
    rng = np.random.default_rng(6)
    truth = np.zeros((R, 2))
    truth[:, 0] = np.log(1.5)
    opts = dict(seed=23, tr_ms=200.0, z_scale=50.0)
    hidden = dbnet.Network(g, _scaled(base, truth, targets), dict(opts, net_id=998))
    theta0 = rng.uniform(np.log(0.7), np.log(1.0), (M, R, 2))
    ens = dbnet.Ensemble(g, base, M, theta0, dict(opts, net_id=0),
                         dict(obs_var=1e-9, gamma=0.7, rw_sigma=0.01, theta_lo=LO, theta_hi=HI,
                              target=targets))
    start = theta0[:, :, 0].mean()
    for _ in range(12):
        hidden.step(TR_STEPS)
        ens.step(TR_STEPS)
        ens.assimilate(hidden.bold()[-1])
    th, _, _ = ens.read()
    assert abs(th[:, :, 0].mean() - np.log(1.5)) < abs(start - np.log(1.5))
    hidden.close()
    ens.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_failed_analysis_leaves_members_unchanged(mode):
    """An analysis whose forecast is not finite is refused (DBNET_EINVAL) and
    changes nothing: theta, the hemodynamic state and the members' region
    constants stay as they were.  A huge z_scale overflows every region's
    hemodynamic state within a few bins (FP64 overflow, not a fault); a later
    analysis on a healthy ensemble still runs."""
    from paper_2211_15963_gb300 import dbnet
    g = _graph()
    base = [synth.default_region_params(I_ext=0.9) for _ in range(g.n_regions)]
    M = 4
    theta = np.random.default_rng(3).uniform(LO, HI, (M, g.n_regions, 2))
    opts = dict(seed=9, net_id=300, tr_ms=10.0, z_scale=1e300)
    ens = dbnet.Ensemble(g, base, M, theta, opts, dict(mode=mode, obs_var=1e-6))
    ens.step(400)
    th0, bw0, y0 = ens.read()
    assert not np.all(np.isfinite(bw0))   # the forecast is broken
    with pytest.raises(dbnet.DbnetError) as ei:
        ens.assimilate(np.zeros(g.n_regions))
    assert ei.value.code == dbnet.DBNET_EINVAL and "unchanged" in str(ei.value)
    th1, bw1, y1 = ens.read()
    assert np.array_equal(th1, th0)
    assert np.array_equal(bw1, bw0, equal_nan=True)
    # the members' conductances were not rescaled: a member still equals a
    # single network with its initial scales
    ens.step(100)
    net = dbnet.Network(g, _member_params(base, theta[1]), dict(opts, net_id=301))
    net.step(500)
    a, b = ens.member_state(1), net.state()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    net.close()
    ens.close()
    # non-finite caller draws are refused on the host
    ens = dbnet.Ensemble(g, base, M, theta, dict(opts, z_scale=1.0), dict(mode=mode))
    ens.step(100)
    eps = np.zeros((M, g.n_regions))
    eps[2, 1] = np.nan
    with pytest.raises(dbnet.DbnetError):
        ens.assimilate(np.zeros(g.n_regions), eps_obs=eps)
    ens.assimilate(np.zeros(g.n_regions), eps_obs=np.zeros((M, g.n_regions)))
    ens.close()


def test_twin_experiment_recovers_one_scale_per_region():
    """Twin experiment (Supp. Alg. 3; Supp. Sec. 6, the resting-state fit of
    g_AMPA): a hidden member with its own AMPA scale per region generates
    the BOLD observations, one per TR of 800 ms; the ensemble analyses one
    log scale per region (the second slot carries nothing, so the data --
    one BOLD signal per region -- can fix the parameter).  Starting from a
    prior spread over [0.5, 2], after 20 TRs the ensemble mean of every
    region's scale lies within 0.25 (log units) of the hidden value, and
    within 0.08 on average over the regions (from 0.27 at the start)."""
    from paper_2211_15963_gb300 import dbnet
    R, size, kin, M = 10, 2000, 100, 48
    g = synth.make_graph([size] * R, kin, 5, k_within=80, d_within=(1, 30), d_cross=(30, 90))
    base = [synth.default_region_params() for _ in range(R)]
    rng = np.random.default_rng(6)
    truth = np.zeros((R, 2))
    truth[:, 0] = rng.uniform(LO, HI, R)
    theta0 = np.zeros((M, R, 2))
    theta0[:, :, 0] = rng.uniform(LO, HI, (M, R))
    opts = dict(seed=7, tr_ms=800.0, z_scale=50.0)
    hidden = dbnet.Network(g, _member_params(base, truth), dict(opts, net_id=1 << 20))
    ens = dbnet.Ensemble(g, base, M, theta0, dict(opts, net_id=0),
                         dict(obs_var=1e-8, gamma=1.0, rw_sigma=0.005, theta_lo=LO, theta_hi=HI,
                              target=(dbnet.DBENS_T_AMPA, dbnet.DBENS_T_NONE)))
    err0 = np.abs(theta0[:, :, 0].mean(0) - truth[:, 0])
    for _ in range(20):
        hidden.step(8000)
        ens.step(8000)
        ens.assimilate(hidden.bold()[-1])
    th, _, _ = ens.read()
    err = np.abs(th[:, :, 0].mean(0) - truth[:, 0])
    assert err.mean() < 0.08 and err.mean() < 0.3 * err0.mean(), (err.mean(), err0.mean())
    assert err.max() < 0.25, err
    hidden.close()
    ens.close()
