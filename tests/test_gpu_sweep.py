"""Variability sweep as one batch: every grid point equals its plain anneal, and its cut trace ends
at the batch's final cuts."""
import numpy as np
import pytest

from paper_2601_14476_gb300 import inputs, pbit, sweep

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sweep_points_equal_plain_anneals_and_traces():
    g = inputs.erdos_renyi_gnm(400, 3000, 5, "+1")
    grid = [sweep.SweepPoint(), sweep.SweepPoint(s_intensity=0.1), sweep.SweepPoint(s_offset=0.1),
            sweep.SweepPoint(p_mean=0.9, s_p=0.05), sweep.SweepPoint(0.1, 0.1, 0.9, 0.05)]
    T, S = 32, 150
    recs = sweep.variability_sweep(g, grid, T, S, seed=3, trace_every=50)
    G = pbit.Graph.from_inputs(g)
    for k, (pt, rec) in enumerate(zip(grid, recs)):
        kw = sweep.point_kwargs(g, k, pt, T, S, 3, 0.1, 10.0)
        alone = G.anneal(kw.pop("trials"), kw.pop("steps"), **kw)
        assert np.array_equal(G.cut(alone), rec["cuts"]), k
        assert rec["trace"].shape == (3, T)
        assert np.array_equal(rec["trace"][-1], rec["cuts"]), k
    # the ideal point has no variability arrays; the mixed points differ from it
    assert sweep.point_variability(g.n, 1, grid[0]) is None
    assert not np.array_equal(recs[0]["cuts"], recs[4]["cuts"])
