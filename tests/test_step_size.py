"""The step-size study of Extended Data Fig. 1 through the matched-FP32
oracle, which performs the device's operations in the device's order (the
device equals it bit for bit on these networks:
`test_step_size_study_networks_bit_exact`).

One second of the 1,000-neuron study network at every step of the study,
V sampled every millisecond, compared with the finest step.  Forward Euler
is first order, so before the chaotic divergence takes over the error must
shrink with the step; over the second the dt = 1 ms error is of the size
the paper reports (about 5 %), the size any step reaches once the chaotic
network has parted from the reference.
"""
import numpy as np
import pytest

import bench
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.fixture(scope="module")
def table():
    seed = 4243
    runs = {}
    for dt in bench.DT_STUDY_MS:
        g, p, d = bench.dt_study_network(dt, seed)
        s = oracle.Sim(g, p, dt_ms=dt, bin_ms=1.0, seed=seed + 1, precision=32)
        V = np.empty((bench.DT_STUDY_STEPS, g.n_neurons))
        for ms in range(bench.DT_STUDY_STEPS):
            s.step(d)
            V[ms] = s.state()[0]
        st, ids = s.raster()
        runs[dt] = (V, (st.astype(np.int64) + 1) * dt, ids, 0.0)
    return {row["dt_ms"]: row for row in bench.dt_study_table(runs)}


def test_reference_row_is_exact(table):
    ref = table[bench.DT_STUDY_MS[-1]]
    assert ref["rel_err_mean_1s"] == 0.0
    assert ref["reference_spikes_matched_within_1ms"] == 1.0


def test_error_shrinks_with_the_step_before_divergence(table):
    """At the first sample (1 ms) no spike has yet parted the runs: the
    error falls with the step, by about the ratio of the steps (first
    order).  Later the network's chaos amplifies any difference, whatever
    the step, so later windows are not ordered."""
    first = [table[dt]["rel_err_at_1ms"] for dt in (1.0, 0.5, 0.2, 0.1)]
    assert first[0] > first[1] > first[2] > first[3] > 0.0
    assert first[0] / first[3] > 3.0


def test_one_millisecond_step_error_is_of_the_reported_size(table):
    one = table[1.0]
    assert 0.01 < one["rel_err_mean_1s"] < 0.2
    assert all(5.0 < row["rate_hz"] < 20.0 for row in table.values())
