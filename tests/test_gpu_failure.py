"""Failure detection without a GPU fault: a bounded device wait that runs out
is reported as PBIT_E_TIMEOUT, the flag clears, and the context stays usable."""
import numpy as np
import pytest

from paper_2601_14476_gb300 import inputs, pbit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_timeout_is_reported_and_recoverable():
    g = inputs.torus_2d(10, 10, 1)
    G = pbit.Graph.from_inputs(g)
    G.status()  # clean
    pbit.pbit_selftest_timeout(G.handle, 2000)
    with pytest.raises(pbit.PbitError) as ei:
        G.status()
    assert ei.value.code == pbit.PBIT_E_TIMEOUT
    G.status()  # cleared
    out = G.anneal(16, 20, seed=1)
    assert np.all(np.isin(out.cpu().numpy(), (-1, 1)))
    G.status()


def test_invalid_calls_fail_without_touching_the_device():
    g = inputs.torus_2d(10, 10, 1)
    G = pbit.Graph.from_inputs(g)
    bad = [dict(trials=0, steps=10), dict(trials=8, steps=10, step_begin=5, step_end=3),
           dict(trials=8, steps=10, offset_mode=7), dict(trials=8, steps=10, algorithm=9),
           dict(trials=8, steps=10, algorithm=pbit.ALG_TAPSA, window=0),
           dict(trials=8, steps=10, algorithm=pbit.ALG_SPSA, step_begin=2)]
    for kw in bad:
        out = torch.empty((g.n, max(kw["trials"], 1)), dtype=torch.int8, device="cuda")
        p, keep = pbit.make_params(**kw)
        with pytest.raises(pbit.PbitError) as ei:
            pbit.pbit_anneal(G.handle, p, None, out)
        assert ei.value.code == pbit.PBIT_E_INVALID, kw
    G.status()
