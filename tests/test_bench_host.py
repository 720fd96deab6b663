"""Host logic of bench.py that needs no GPU: the replica combination over
ranks (run here as two gloo processes on the CPU), per-rank seeds, the
reference arm's rank rule, the serving drive interpolation, launch counts per
schedule and the hash gating of the profile figures."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per_rank = [(1000.0, 10.0, 2e6, 640.0), (3000.0, 30.0, 2e6, 655.5)][rank]
    res = bench.combine_ranks(*per_rank, world, "cpu")
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_combine_ranks_over_two_gloo_processes(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        e, s, n, ms = json.load(open(tmp_path / ("r%d.json" % r)))
        assert (e, s, n) == (4000.0, 40.0, 4e6)   # summed over the replicas
        assert ms == 655.5                         # the slowest replica


def test_single_rank_combination_is_identity():
    import bench
    assert bench.combine_ranks(7.0, 3.0, 5.0, 2.5, 1, "cpu") == (7.0, 3.0, 5.0, 2.5)


def test_rank_seeds_differ():
    import bench
    seeds = [bench.rank_seed(r) for r in range(8)]
    assert len(set(seeds)) == 8 and seeds[0] == 15973


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(bench.parse_from([]))
    assert capsys.readouterr().out == ""


def test_serving_drive_interpolation():
    import bench
    for k, v in bench.SERVE_DRIVE:
        assert abs(bench.serve_drive(k) - v) < 1e-12
    assert bench.SERVE_DRIVE[0][1] < bench.serve_drive(200) < bench.SERVE_DRIVE[1][1]
    assert bench.serve_drive(50) == bench.SERVE_DRIVE[0][1]


def test_step_size_study_networks_share_topology():
    """Every step of the study runs the same graph, weights and initial
    state; only the delay in steps (1 ms each) and dt change."""
    import bench
    g1, p1, d1 = bench.dt_study_network(1.0, 5)
    g2, p2, d2 = bench.dt_study_network(0.008, 5)
    assert (d1, d2) == (1, 125) and p1 == p2 and p1["drive_rate_hz"] == 0.0
    assert np.array_equal(g1.col, g2.col) and np.array_equal(g1.w_bf16, g2.w_bf16)
    assert np.all(np.asarray(g2.delay) == 125) and g2.max_delay == 125
    assert bench.DT_STUDY_MS[-1] * 250 >= p1["Tref"] - 1e-12   # refractory fits 8 bits


def test_matched_spikes_counts_reference_spikes_within_tolerance():
    import bench
    ref_t = np.array([1.0, 5.0, 9.0, 2.0, 3.0])
    ref_i = np.array([0, 0, 0, 1, 2])
    t = np.array([1.5, 7.0, 9.9, 4.0])
    i = np.array([0, 0, 0, 1])
    assert bench.matched_spikes(ref_t, ref_i, t, i, 1.0) == 2
    assert bench.matched_spikes(ref_t, ref_i, t, i, 2.0) == 4
    assert bench.matched_spikes(ref_t, ref_i, ref_t, ref_i, 0.0) == 5


def test_launch_count_per_schedule():
    """Kernels launched by one dbnet_step call of n steps: graph replays of
    64 steps (128 launches, 192 when pipelined, plus the long part launched
    ahead), direct steps for the rest, the base word and the bin close; on
    the persistent schedule one launch per 4,096 steps and the bin close."""
    import bench
    assert bench.launches_per_call(10_000, "sequential") == 156 * 128 + 16 * 2 + 2
    assert bench.launches_per_call(10_000, "pipelined") == 156 * 192 + 16 * 2 + 2 + 1
    assert bench.launches_per_call(63, "sequential") == 63 * 2 + 1
    assert bench.launches_per_call(10_000, "persistent") == 3 + 1
    assert bench.launches_per_call(4096, "persistent") == 1 + 1


def test_profile_figures_follow_the_kernel_source(tmp_path, monkeypatch):
    """The bench quotes traffic and occupancy from committed ncu summaries
    only while they carry the current kernels.cu hash."""
    import bench
    sha = bench.kernels_sha()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic_x.md").write_text(
        "kernels.cu sha256[:16]: %s\n\n| k_deliver | 123456 | a |\n" % sha)
    (tmp_path / "profiles" / "traffic_old.md").write_text(
        "kernels.cu sha256[:16]: 0000000000000000\n\n| k_deliver | 99 | a |\n")
    for name, what in (("k_deliver_400k_grid608.md", "d"), ("k_update_400k.md", "u")):
        (tmp_path / "profiles" / name).write_text(
            "kernels.cu sha256[:16] %s.\n\n| warps active (of peak) | 28.0 %% |\n"
            "| issue active | 27.1 %% (x) |\n" % sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernels_sha", lambda: sha)
    assert bench.measured_traffic("k_deliver", "traffic_x.md") == 123456
    assert bench.measured_traffic("k_deliver", "traffic_old.md") is None
    assert bench.measured_traffic("k_deliver", "missing.md") is None
    shape = bench.profiled_shape()
    assert shape["k_deliver"]["warps_active_pct"] == 28.0
    assert shape["k_update"]["issue_active_pct"] == 27.1
    monkeypatch.setattr(bench, "kernels_sha", lambda: "ffffffffffffffff")
    assert bench.profiled_shape() is None


def test_arm_cpu_part_names():
    import bench
    assert bench.ARM_PARTS["0xd4f"] == "Arm Neoverse V2"
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
