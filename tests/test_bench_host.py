"""Host-side bookkeeping of bench.py on CPU: the variants' update and byte counts (against a
sub-step by sub-step count), the DRAM-traffic table's source hashes, and the sweep workloads."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_2601_14476_gb300 import inputs, pbit  # noqa: E402


def _count(g, T, Q, nu, state):
    """Due updates and their bytes, one sub-step at a time."""
    deg = np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
    upd = 0
    byt = 0
    for q in range(Q):
        due = (q % nu) == 0
        upd += T * int(due.sum())
        byt += T * int((deg[due] + 2 + state).sum())
    return upd, byt


@pytest.mark.parametrize("alg,state", [(pbit.ALG_PSA, 0), (pbit.ALG_SPSA, 8), (pbit.ALG_TAPSA, 8)])
def test_variant_work_timing_model_counts(alg, state):
    g = inputs.torus_2d(6, 7, 3, "pm1")
    dev = np.random.default_rng(1).normal(0, 0.3, g.n).astype(np.float32)
    v = {"algorithm": alg, "window": 4, "t_res": 10, "nu_dev": dev}
    nu = np.maximum(1, np.floor(10 * (1.0 + dev.astype(np.float64)) + 0.5)).astype(np.int64)
    for Q in (1, 2, 3, 37, 120):
        assert bench.variant_work(v, g, 8, Q) == _count(g, 8, Q, nu, state)


def test_variant_work_without_timing_is_every_node_every_step():
    g = inputs.erdos_renyi_gnm(50, 120, 2, "+1")
    upd, byt = bench.variant_work({"algorithm": pbit.ALG_SPSA}, g, 16, 9)
    assert upd == g.n * 16 * 9
    assert byt == 16 * 9 * (2 * g.m + g.n * (2 + 8))


def test_traffic_table_entries():
    """Each captured DRAM figure is reported only while its kernel's sources hash as they did at the
    capture (else null), and every source it hashes exists."""
    for key, entry in bench.TRAFFIC.items():
        assert bench.traffic_for(key) in (entry["bytes"], None), key
        for f in entry["files"]:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2601_14476_gb300", "csrc", f)), (key, f)
    assert bench.traffic_key("sparse_variant_words_kernel", {"algorithm": pbit.ALG_SPSA}) in bench.TRAFFIC
    assert bench.traffic_key("sparse_variant_words_kernel", {"algorithm": pbit.ALG_PSA, "t_res": 10}) is None
    assert bench.traffic_for(None) is None


def test_sweep_workloads_are_one_graph_many_points():
    ws = bench.sweep_workloads(seed=1, steps=50)
    assert len(ws) == 8
    assert all(w.graph is ws[0].graph and w.trials == 128 and w.steps == 50 for w in ws)
    assert [w.instance for w in ws] == list(range(8))
    assert ws[0].var is None and ws[-1].var is not None
    assert bench.multi_reference_workload("sweep").instance == 7
