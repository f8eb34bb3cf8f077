"""CPU checks of bench.py's bookkeeping: the launch count it reports, the sampler
each workload uses by default, the figures it reads from the committed ncu
summaries and the bounded samples the CPU oracle is timed on."""
import types

import numpy as np
import pytest

import bench
from paper_1706_01094_gb300 import workloads

MODES = types.SimpleNamespace(MODE_AUTO=0, MODE_PLAIN=1, MODE_PERSISTENT=2, MODE_BATCHED=3)


def test_launch_counts_follow_the_library_schedule():
    single = workloads.single()
    batched = workloads.batched()
    # slice sampler: table kernel + heavy-node pass per step, one time-advance
    # kernel per 32-step graph and one time-set kernel per call
    assert bench.count_launches(10000, single, 0, False, False, MODES, True) == 20000 + 312 + 1
    assert bench.count_launches(31, single, 0, False, False, MODES, True) == 62   # no graph
    # statistics form: step kernel + heavy pass per step, a merge and a time
    # advance per graph, threshold set + time set + last partial + final merge
    assert bench.count_launches(64, single, 0, False, True, MODES, True) == 64 * 2 + 4 + 1 + 3
    assert bench.count_launches(70, single, 0, False, True, MODES, True) == 70 * 2 + 4 + 1 + 3
    assert bench.blocked_span({"stats_config": 2, "plain_variant": 14}, single, True) == 1
    # per-replica launches of the baseline mode
    assert bench.count_launches(3, batched, MODES.MODE_PLAIN, False, False, MODES, True) \
        == 3 * batched.replicas * 2
    assert bench.count_launches(3, batched, MODES.MODE_PLAIN, False, False, MODES) \
        == 3 * batched.replicas
    # sequential persistent: one launch per call of at most 65536 steps
    assert bench.count_launches(2000, batched, 0, True, False, MODES) == 1
    assert bench.count_launches(2000, batched, 0, True, False, MODES, True) == 1  # slice sampler
    uneven = workloads.uneven()
    assert bench.count_launches(64, uneven, 2, True, False, MODES, True) == 1 + 64 * 2 + 2 + 1
    # temporally blocked slice launches: 16, 8 or 4 steps each, 2, 4 or 8 per graph
    assert bench.blocked_span({"plain_variant": 14}, single, False) == 16
    assert bench.blocked_span({"plain_variant": 16}, single, False) == 4
    assert bench.blocked_span({"plain_variant": 15}, single, False) == 8
    assert bench.blocked_span({"plain_variant": 17}, single, False) == 8
    assert bench.blocked_span({"plain_variant": 4}, single, False) == 1
    assert bench.blocked_span({"plain_variant": 14}, batched, False) == 1   # several replicas
    assert bench.count_launches(10000, single, 0, False, False, MODES, True, 16) \
        == 312 * 2 + 312 + 1 + 1
    assert bench.count_launches(20, single, 0, False, False, MODES, True, 16) == 2
    assert bench.count_launches(64, single, 0, False, False, MODES, True, 8) == 8 + 2 + 1
    # the counts the GPU run of the 8-step windows reported: 10000 steps in 1563 launches
    # (1250 blocked launches, 312 time advances, one time set), 20 steps in 3 (8 + 8 + 4)
    assert bench.count_launches(10000, single, 0, False, False, MODES, True, 8) == 1563
    assert bench.count_launches(20, single, 0, False, False, MODES, True, 8) == 3


def test_default_sampler_per_workload():
    for name, want in (("single", "slice"), ("fluct", "slice"), ("batched", "slice"),
                       ("uneven", "slice"), ("small", "sequential")):
        args = types.SimpleNamespace(sampler="auto", workload=name)
        assert bench.pick_sampler(args) == want
    assert bench.pick_sampler(types.SimpleNamespace(sampler="sequential", workload="single")) \
        == "sequential"


def test_committed_profile_figures():
    # the blocked kernel moves the state through HBM once per 16-step launch
    traffic = bench.committed_figure("k_step_slice_tb", "single")
    assert traffic is not None and 1e8 < traffic < 4e8   # bytes per launch of 16 2^24-node steps
    for key in ("alu_pipe_pct", "issue_active_pct"):
        v = bench.committed_figure("k_step_slice_tb", "single", key)
        assert v is not None and 0 < v <= 100
    # the blocked kernel's summary holds for the variant it captured only
    assert bench.committed_figure("k_step_slice_tb", "single", variant=18) == traffic
    assert bench.committed_figure("k_step_slice_tb", "single", variant=15) is None
    assert bench.committed_figure("k_step_slice_tb", "single", "alu_pipe_pct", variant=15) is None
    # a summary whose kernel changed after its counters were taken reports null
    assert bench.committed_figure("k_step_slice", "single") is None
    assert bench.committed_figure("k_step_slice", "no_such_workload") is None
    assert bench.committed_figure("k_step_persistent", "batched") is not None
    assert bench.committed_figure("k_step_plain", "single", "alu_pipe_pct") is not None


@pytest.mark.parametrize("name", ["single", "batched", "uneven"])
def test_oracle_samples_are_bounded_slices_of_the_workload(name):
    wl = workloads.BY_NAME[name]()
    sw = bench.sample_workload(wl, 5000)
    assert 8 <= sw.nodes <= max(5000, int(wl.L.max())) and sw.nodes == int(sw.L.sum())
    assert sw.rho.size == sw.nodes and sw.u.size == sw.nodes
    if wl.replicas > 1:   # whole replicas from the front, same profiles
        k = sw.replicas
        assert np.array_equal(sw.L, wl.L[:k]) and np.array_equal(sw.rho, wl.rho[:sw.nodes])
    tiny = bench.sample_workload(wl, 1)
    assert tiny.nodes >= 8 or wl.replicas > 1


def test_op_tally_and_metric_follow_C():
    assert bench.int_ops_per_node_step(10) == 228
    assert bench.int_ops_per_node_step(1) == 98 + 13
    assert bench.int_ops_per_node_step(23) == 3 * 98 + 13 * 23
    assert "C=10" in bench.metric(10) and "C=1 " in bench.metric(1)
    args = types.SimpleNamespace(u=0.2, C=1)
    assert bench.make_workload("single", args).C == 1
    assert bench.make_workload("fluct", types.SimpleNamespace(u=0.0, C=10)).C == 10


def test_clock_samplers_fail_soft_without_a_gpu():
    """Without NVML or a GPU the NVML sampler reports itself unusable (the bench
    then falls back to nvidia-smi polling); with no samples the summary says so."""
    c = bench.NvmlClocks(0)
    if not c.ok:
        with c:
            pass
        s = c.summary()
        assert s["samples"] == 0 and s["sm_mhz"] is None
    smi = bench.ClockSampler(0)
    assert smi.summary()["samples"] == 0


def test_cpu_baseline_reports_all_cores_and_one():
    wl = workloads.small()
    cb = bench.cpu_baseline(wl, 0.6, "sequential")
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert cb["single_thread"]["cores"] == 1 and cb["single_thread"]["value"] > 0
    import oracle
    assert cb["cores"] == oracle.set_threads(0)
