"""pbit_anneal_noalloc: the allocation-free variant of pbit_anneal.

It serves callers that cannot allocate device memory while they run:
applications whose own caching allocator has reserved nearly all of HBM,
processes under a fixed device-memory cap, and latency-bound loops that
cannot absorb an allocation's synchronisation.  (It still calls the CUDA
runtime, so it is not for stream callbacks or host functions.)  Its scratch
is a fixed 32 MiB array inside libpbit.so.  This file is named to be collected last, so
that a run stopping at its first failure has already run every other test;
it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2601_14476_gb300 import inputs, pbit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(fn, G, T, S, spins_in, **kw):
    out = torch.empty((G.n, T), dtype=torch.int8, device="cuda")
    p, keep = pbit.make_params(T, S, **kw)
    fn(G.handle, p, spins_in, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_anneal_on_two_calls_in_a_row():
    g = inputs.torus_2d(40, 50, 5, "pm1")
    var = inputs.variability(g.n, 5)
    G = pbit.Graph.from_inputs(g)
    T, S = 64, 120
    for seed in (3, 4):  # two calls in a row; the second reuses the array the first left behind
        kw = dict(seed=seed, variability=var, kernel=pbit.KERNEL_SPARSE)
        want = _run(pbit.pbit_anneal, G, T, S, None, **kw)
        got = _run(pbit.pbit_anneal_noalloc, G, T, S, None, **kw)
        assert np.array_equal(got, want)
    # a resumed range from a given state, odd step count, in place
    start = torch.from_numpy(inputs.random_spins(g.n, T, 1)).cuda()
    kw = dict(seed=9, variability=var, step_begin=7, step_end=40, kernel=pbit.KERNEL_SPARSE)
    want = _run(pbit.pbit_anneal, G, T, S, start.clone(), **kw)
    inplace = start.clone()
    p, keep = pbit.make_params(T, S, **kw)
    pbit.pbit_anneal_noalloc(G.handle, p, inplace, inplace)
    torch.cuda.synchronize()
    assert np.array_equal(inplace.cpu().numpy(), want)


def test_noalloc_rejects_sizes_beyond_its_array():
    g = inputs.torus_2d(100, 200, 1, "pm1")
    G = pbit.Graph.from_inputs(g)
    out = torch.empty((g.n, 2048), dtype=torch.int8, device="cuda")   # 40 MB of spins > 32 MiB
    p, keep = pbit.make_params(2048, 10, seed=1)
    with pytest.raises(pbit.PbitError) as ei:
        pbit.pbit_anneal_noalloc(G.handle, p, None, out)
    assert ei.value.code == pbit.PBIT_E_INVALID
    assert "scratch" in str(ei.value)


def test_noalloc_fresh_start_with_odd_step_count():
    """spins_in NULL with an odd number of steps: the initial state goes to the scratch buffer first
    and the Jacobi rotation must still end in spins_out."""
    g = inputs.rgg_knn(700, 3, 3, "pm1")
    var = inputs.variability(g.n, 3)
    G = pbit.Graph.from_inputs(g)
    for T, lo, hi in ((32, 0, 13), (48, 4, 21), (16, 0, 1)):
        kw = dict(seed=5, variability=var, step_begin=lo, step_end=hi, kernel=pbit.KERNEL_SPARSE)
        want = _run(pbit.pbit_anneal, G, T, 30, None, **kw)
        got = _run(pbit.pbit_anneal_noalloc, G, T, 30, None, **kw)
        assert np.array_equal(got, want), (T, lo, hi)


def test_noalloc_rejects_non_finite_parameters():
    g = inputs.torus_2d(10, 10, 1, "pm1")
    G = pbit.Graph.from_inputs(g)
    out = torch.empty((g.n, 16), dtype=torch.int8, device="cuda")
    for key in ("intensity", "offset"):
        var = inputs.variability(g.n, 1)
        var[key] = var[key].copy()
        var[key][5] = np.nan if key == "intensity" else np.inf
        p, keep = pbit.make_params(16, 10, seed=1, variability=var)
        with pytest.raises(pbit.PbitError) as ei:
            pbit.pbit_anneal_noalloc(G.handle, p, None, out)
        assert ei.value.code == pbit.PBIT_E_INVALID
