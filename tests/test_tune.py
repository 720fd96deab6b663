"""Conductance initialisation (Supplementary Algorithm 1), driven by the FP64
oracle on the CPU: the target channel currents obey the algorithm's
construction, and the iteration brings the measured currents to them."""
import numpy as np
import pytest

import oracle
import synth
from paper_2211_15963_gb300 import tune


def test_channel_targets_follow_the_construction():
    p = synth.default_region_params(I_ext=0.3)
    a, n, ga, gb = tune.channel_targets(p, 100.0, 10.0)
    assert a > 0 and n > 0 and ga < 0 and gb < 0      # excitatory in, inhibitory out
    assert abs(a / (a + n) - 0.3) < 1e-12 and abs(ga - gb) < 1e-15
    # a higher ceiling needs more excitation and then more inhibition
    a2, n2, ga2, _ = tune.channel_targets(p, 150.0, 10.0)
    assert a2 + n2 > a + n and ga2 < ga
    # a higher working rate needs less inhibition, the same excitation
    a3, n3, ga3, _ = tune.channel_targets(p, 100.0, 20.0)
    assert abs((a3 + n3) - (a + n)) < 1e-12 and ga3 > ga
    with pytest.raises(ValueError):
        tune.channel_targets(p, 600.0, 10.0)  # above 1 / T_ref


def _drive_dominated():
    """In-degree 10 with a strong Poisson drive: the regime in which the
    channel currents are close to linear in the conductances, as the
    algorithm assumes (a strongly recurrent network flips between silent
    and runaway under any conductance step)."""
    g = synth.make_graph([1600, 1400], 10, 91, d_within=(1, 20), d_cross=(20, 40))
    p = synth.default_region_params(I_ext=0.3, drive_K=20.0)
    p["g_u"] = tuple(x * 10 for x in p["g_u"])
    return g, p


def test_iteration_reaches_the_target_currents_with_the_oracle():
    """The paper's step (g_u times target / measured) with the FP64 oracle
    as the model brings every channel current within 5 % of its target."""
    g, p = _drive_dominated()

    def make(q):
        return oracle.Sim(g, q, seed=5, precision=64)

    gu, hist, target = tune.init_conductances(make, p, 60.0, 10.0, iters=16, tol=0.05,
                                              warm_steps=600, steps=600, every=20,
                                              step_exp=1.0, max_factor=4.0)
    first = np.abs(np.array(hist[0][1]) / np.array(target) - 1.0).max()
    last = np.abs(np.array(hist[-1][1]) / np.array(target) - 1.0).max()
    assert last < 0.05 < first and len(hist) < 16
    assert all(x > 0 for x in gu)


@pytest.mark.gpu
def test_iteration_with_the_library_as_the_model():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    from paper_2211_15963_gb300 import dbnet
    __graft_entry__.build()
    g, p = _drive_dominated()

    def make(q):
        return dbnet.Network(g, q, dict(seed=5))

    gu, hist, target = tune.init_conductances(make, p, 60.0, 10.0, iters=16, tol=0.05,
                                              warm_steps=600, steps=600, every=20,
                                              step_exp=1.0, max_factor=4.0)
    last = np.abs(np.array(hist[-1][1]) / np.array(target) - 1.0).max()
    assert last < 0.05 and len(hist) < 16
