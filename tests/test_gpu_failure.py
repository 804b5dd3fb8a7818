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


# The persistent kernels' own waits, made to run out: PBIT_TEST_WITHHOLD names the kernel that then
# never publishes one progress signal (a software flag, counter or slice copy its peers poll; never a
# hardware barrier arrival), PBIT_TEST_WAIT_US shortens that kernel's waits to milliseconds.  The run
# reports PBIT_E_TIMEOUT; with the switch cleared the same process then anneals exactly as usual.
_FAULT_CHILD = r'''
import os, sys, numpy as np, torch
from paper_2601_14476_gb300 import inputs, pbit
kind, path = sys.argv[1], sys.argv[2]

def run():
    if kind == "flow":
        g = inputs.torus_2d(40, 50, 3, "pm1")
        G = pbit.Graph.from_inputs(g)
        out = G.anneal(1024, 30, seed=2, variability=inputs.variability(g.n, 3), kernel=pbit.KERNEL_SPARSE)
        return G, [out]
    if kind == "batch":
        gs = [inputs.erdos_renyi_gnm(800, 2400, 1, "+1"), inputs.rgg_knn(900, 2, 3, "pm1")]
        Gs = [pbit.Graph.from_inputs(x) for x in gs]
        B = pbit.Batch(Gs, [dict(trials=64, steps=40, seed=1), dict(trials=32, steps=40, seed=2, instance=1)])
        B.run(chunk_steps=16)
        torch.cuda.synchronize()
        outs = [B.spins(k) for k in range(2)]
        return Gs[0], outs
    if kind == "dense":
        g = inputs.complete_pm1(1000, 4)
        G = pbit.Graph.from_inputs(g, dense=True)
        out = G.anneal(128, 25, seed=3, i0_min=0.05, i0_max=5.0, kernel=pbit.KERNEL_DENSE)
        return G, [out]
    g = inputs.complete_pm1(300, 5)   # dense4: a cluster of three CTAs
    G = pbit.Graph.from_inputs(g, dense=True)
    out = G.anneal(32, 25, seed=4, i0_min=0.05, i0_max=5.0, kernel=pbit.KERNEL_DENSE)
    return G, [out]

G, _ = run()
try:
    G.status()
    code = 0
except pbit.PbitError as e:
    code = e.code
G.status()  # the flag is cleared
os.environ.pop("PBIT_TEST_WITHHOLD")
G, outs = run()
G.status()
np.savez(path, np.array([code]), *[o.cpu().numpy() for o in outs])
'''


@pytest.mark.parametrize("kind", ["flow", "batch", "dense", "dense4"])
def test_persistent_kernel_wait_runs_out(tmp_path, kind):
    import os
    import subprocess
    import sys
    path = str(tmp_path / f"{kind}.npz")
    env = dict(os.environ, PBIT_TEST_WITHHOLD=kind, PBIT_TEST_WAIT_US="2000")
    if kind == "flow":
        env["PBIT_SPARSE_FLOW"] = "always"
    if kind == "dense":
        env["PBIT_DENSE_E4M3"] = "1"
    subprocess.run([sys.executable, "-c", _FAULT_CHILD, kind, path], check=True, env=env, timeout=300)
    res = np.load(path)
    assert int(res["arr_0"][0]) == pbit.PBIT_E_TIMEOUT, int(res["arr_0"][0])
    # the clean run in the same process equals a run here without any switch
    clean_env = {k: v for k, v in env.items() if k not in ("PBIT_TEST_WITHHOLD", "PBIT_TEST_WAIT_US")}
    path2 = str(tmp_path / f"{kind}_ref.npz")
    ref_code = _FAULT_CHILD.replace('os.environ.pop("PBIT_TEST_WITHHOLD")', 'pass')
    subprocess.run([sys.executable, "-c", ref_code, kind, path2], check=True, env=clean_env, timeout=300)
    ref = np.load(path2)
    assert int(ref["arr_0"][0]) == 0
    for key in res.files[1:]:
        assert np.array_equal(res[key], ref[key]), key
