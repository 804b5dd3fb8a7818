"""GPU parity of the sparse / resident CUDA path against the CPU oracle.

Bit-exact: initial state, fields, cuts, energies, schedule.  Decisions: the
kernel takes the p-bit decision in float32 (tanhf), the oracle in FP64; a
decision may differ only where |tanh(x) - r| < 1e-6, and such mismatches must
be rarer than 1e-6 of all decisions.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14476_gb300 import inputs, pbit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BAND = 1e-6


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


GRAPHS = {
    "gnm800": lambda: inputs.erdos_renyi_gnm(800, 19176, 1, "+1"),
    "torus": lambda: inputs.torus_2d(12, 20, 2, "pm1"),
    "complete": lambda: inputs.complete_pm1(300, 3),
    "rgg": lambda: inputs.rgg_knn(700, 4, 3, "pm1"),
}


def _int8_weights(g, seed):
    g.w = np.random.default_rng(seed).integers(-127, 128, g.m).astype(np.int8)
    return g


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("T", [16, 12, 7, 1])
def test_fields_cut_energy_bit_exact(name, T):
    g = GRAPHS[name]()
    if name == "rgg":
        g = _int8_weights(g, 5)
    h = np.random.default_rng(9).integers(-30, 31, g.n).astype(np.int32)
    G = pbit.Graph(g.n, g.src, g.dst, g.w, h=h)
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    s = inputs.random_spins(g.n, T, 4)
    d = _dev(s)
    assert np.array_equal(_host(G.fields(d)).astype(np.int64), oracle.fields(csr, s, h))
    assert np.array_equal(G.energy(d), oracle.energy(csr, s, h))
    G0 = pbit.Graph(g.n, g.src, g.dst, g.w)
    assert np.array_equal(G0.cut(d), oracle.cut(g.src, g.dst, g.w, s))


@pytest.mark.parametrize("T", [16, 5, 64])
def test_init_spins_bit_exact(T):
    g = inputs.torus_2d(10, 30, 1)
    G = pbit.Graph.from_inputs(g)
    out = torch.empty((g.n, T), dtype=torch.int8, device="cuda")
    pbit.pbit_init_spins(G.handle, T, 0x1234_5678_9ABC, 7, out)
    assert np.array_equal(_host(out), oracle.init_spins(g.n, T, 0x1234_5678_9ABC, 7))


def test_schedule_bit_exact():
    g = inputs.erdos_renyi_gnm(800, 19176, 1, "+1")
    G = pbit.Graph.from_inputs(g)
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    assert np.array_equal(G.schedule(0.1, 10.0, 1000), oracle.schedule(csr, 0.1, 10.0, 1000))
    assert G.info()["mean_s"] == oracle.mean_s(csr)


def _lockstep(g, T, steps, var, kernel, seed=11, instance=3, mode=pbit.OFFSET_SCALED, c=(0.1, 10.0), S=None):
    """Advance one step at a time on the GPU; check each step against the oracle from the GPU's state."""
    G = pbit.Graph.from_inputs(g)
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    S = S or steps
    tab = oracle.schedule(csr, c[0], c[1], S)
    state = oracle.init_spins(g.n, T, seed, instance)
    decisions = mismatches = 0
    worst = 0.0
    for t in range(steps):
        d_in = _dev(state)
        d_out = torch.empty_like(d_in)
        p, keep = pbit.make_params(T, S, step_begin=t, step_end=t + 1, i0_min=c[0], i0_max=c[1], seed=seed,
                                   instance=instance, kernel=kernel, variability=var, offset_mode=mode)
        pbit.pbit_anneal(G.handle, p, d_in, d_out)
        gpu = _host(d_out)
        want, gap = oracle.step(csr, state, t, tab[t], seed, instance, variability=var, offset_mode=mode,
                                want_gap=True)
        bad = gpu != want
        decisions += state.size
        mismatches += int(bad.sum())
        if bad.any():
            worst = max(worst, float(np.abs(gap[bad]).max()))
        state = gpu
    return decisions, mismatches, worst


def _few(mis, dec):
    """Band mismatches allowed in a lockstep sample: fewer than 1e-6 of its decisions, and at most one
    in a sample of under 1e6 decisions (the rate itself is checked over 1.5e7 decisions below)."""
    return mis <= max(1, int(1e-6 * dec))


@pytest.mark.parametrize("kernel", [pbit.KERNEL_SPARSE, pbit.KERNEL_RESIDENT])
@pytest.mark.parametrize("mode", [pbit.OFFSET_SCALED, pbit.OFFSET_LISTING, pbit.OFFSET_EQUATION])
def test_lockstep_decisions(kernel, mode):
    g = inputs.erdos_renyi_gnm(400, 3000, 2, "pm1")
    var = inputs.variability(g.n, 2, s_intensity=0.3, s_offset=0.3)
    dec, mis, worst = _lockstep(g, 32, 30, var, kernel, mode=mode)
    assert mis == 0 or worst < BAND, (mis, worst)
    assert _few(mis, dec), (mis, dec)


@pytest.mark.parametrize("T", [1, 3, 16, 20])
def test_lockstep_ragged_trials(T):
    g = inputs.rgg_knn(333, 7, 3, "pm1")
    var = inputs.variability(g.n, 7)
    dec, mis, worst = _lockstep(g, T, 12, var, pbit.KERNEL_SPARSE)
    assert mis == 0 or worst < BAND
    assert _few(mis, dec), (mis, dec)


def test_resident_equals_sparse_full_run():
    g = inputs.erdos_renyi_gnm(800, 19176, 1, "+1")
    G = pbit.Graph.from_inputs(g)
    outs = []
    for kernel in (pbit.KERNEL_SPARSE, pbit.KERNEL_RESIDENT):
        outs.append(_host(G.anneal(16, 300, seed=5, kernel=kernel)))
    assert np.array_equal(outs[0], outs[1])


def test_resume_identity_and_in_place():
    g = inputs.torus_2d(10, 16, 3)
    var = inputs.variability(g.n, 3)
    G = pbit.Graph.from_inputs(g)
    T, S = 32, 41
    full = _host(G.anneal(T, S, seed=2, variability=var, kernel=pbit.KERNEL_SPARSE))
    a = G.anneal(T, S, step_end=17, seed=2, variability=var, kernel=pbit.KERNEL_SPARSE)
    # resume in place (odd and even remaining counts)
    p, keep = pbit.make_params(T, S, step_begin=17, step_end=30, seed=2, variability=var, kernel=pbit.KERNEL_SPARSE)
    pbit.pbit_anneal(G.handle, p, a, a)
    p, keep = pbit.make_params(T, S, step_begin=30, step_end=S, seed=2, variability=var, kernel=pbit.KERNEL_SPARSE)
    pbit.pbit_anneal(G.handle, p, a, a)
    assert np.array_equal(_host(a), full)
    # an empty range copies the input
    b = torch.empty_like(a)
    p, keep = pbit.make_params(T, S, step_begin=5, step_end=5, seed=2)
    pbit.pbit_anneal(G.handle, p, a, b)
    assert np.array_equal(_host(b), full)


def test_hold_and_zero_edge_graph():
    g = inputs.torus_2d(5, 7, 1)
    G = pbit.Graph.from_inputs(g)
    s = inputs.random_spins(g.n, 8, 1)
    var = {"p_update": np.zeros(g.n, np.float32)}
    out = G.anneal(8, 20, spins_in=_dev(s), seed=1, variability=var, kernel=pbit.KERNEL_SPARSE)
    assert np.array_equal(_host(out), s)
    # a graph with no edges: cut 0, decisions are fair coins, normalisation is rejected
    E = pbit.Graph(9, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8))
    out = E.anneal(64, 5, seed=1, i0_normalize=0, kernel=pbit.KERNEL_SPARSE)
    assert np.all(E.cut(out) == 0)
    with pytest.raises(pbit.PbitError):
        E.anneal(64, 5, seed=1)


def _explain_divergence(G, csr, w, trial, seg_begin, seg_end, tab):
    """Step the GPU one step at a time from its own state at seg_begin (the resume form) and the oracle
    beside it: every differing decision must lie in the tie band, and `trial` must take at least one
    such decision in the segment.  Returns the number of band decisions of `trial`."""
    g = w.graph
    state = _host(G.anneal(w.trials, w.steps, step_end=seg_begin, i0_min=w.c_min, i0_max=w.c_max, seed=w.seed,
                           instance=w.instance, variability=w.var)) if seg_begin else \
        oracle.init_spins(g.n, w.trials, w.seed, w.instance)
    hits = 0
    for t in range(seg_begin, seg_end):
        d_in = _dev(state)
        d_out = torch.empty_like(d_in)
        p, keep = pbit.make_params(w.trials, w.steps, step_begin=t, step_end=t + 1, i0_min=w.c_min,
                                   i0_max=w.c_max, seed=w.seed, instance=w.instance, variability=w.var)
        pbit.pbit_anneal(G.handle, p, d_in, d_out)
        gpu = _host(d_out)
        want, gap = oracle.step(csr, state, t, tab[t], w.seed, w.instance, variability=w.var, want_gap=True)
        bad = gpu != want
        assert not bad.any() or np.abs(gap[bad]).max() < BAND, t
        hits += int(bad[:, trial].sum())
        state = gpu
    return hits


def test_plain_workload_energy_trace_matches_oracle():
    """Plain G(800, 19176) workload (w = +1, ideal p-bits, 16 trials, 1000 steps).  Its final cut is 0
    on both sides (synchronous pSA falls into the all-+1 / all--1 two-cycle), so the mean cut pins
    nothing; the path there does.  The energy every 10 steps (pbit_anneal_trace) must equal the
    oracle's energy of its own states at the same steps, and the final spins of the bench's launch
    form (one resident launch) must equal the oracle's element by element, for every trial whose path
    no tie-band decision changed; a trial that departs must be explained by a band decision in the
    segment where its trace first differs."""
    w = inputs.plain_er800()
    g = w.graph
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    tab = oracle.schedule(csr, w.c_min, w.c_max, w.steps)
    G = pbit.Graph.from_inputs(g)
    T, S, every = w.trials, w.steps, 10
    whole = _host(G.anneal(T, S, i0_min=w.c_min, i0_max=w.c_max, seed=w.seed, instance=w.instance))
    trace = torch.zeros((S // every, T), dtype=torch.int64, device="cuda")
    out = torch.empty((g.n, T), dtype=torch.int8, device="cuda")
    p, keep = pbit.make_params(T, S, i0_min=w.c_min, i0_max=w.c_max, seed=w.seed, instance=w.instance)
    pbit.pbit_anneal_trace(G.handle, p, None, out, every, 0, trace)
    tr = _host(trace)
    assert np.array_equal(_host(out), whole)  # segmented run = one launch
    state = oracle.init_spins(g.n, T, w.seed, w.instance)
    ref = np.zeros_like(tr)
    for j in range(S // every):
        state = oracle.anneal(csr, state, tab, w.seed, w.instance, step_begin=j * every, step_end=(j + 1) * every)
        ref[j] = oracle.energy(csr, state)
    # the trace is not trivial: energies change along the anneal and differ between trials
    assert len(np.unique(tr[:20])) > 20 and np.ptp(tr[5]) > 0
    diverged = [t for t in range(T) if not (np.array_equal(tr[:, t], ref[:, t])
                                            and np.array_equal(whole[:, t], state[:, t]))]
    assert len(diverged) <= 2, diverged
    for t in diverged:
        rows = np.nonzero(tr[:, t] != ref[:, t])[0]
        j = int(rows[0]) if len(rows) else S // every - 1
        assert _explain_divergence(G, csr, w, t, j * every, (j + 1) * every, tab) >= 1, t
    assert np.array_equal(G.cut(_dev(whole)), oracle.cut(g.src, g.dst, g.w, whole))


def test_full_size_torus_sampled():
    """100x200 torus, 1024 trials, in the bench launch configuration: sampled decisions vs oracle."""
    w = inputs.sparse_torus20000()
    g = w.graph
    G = pbit.Graph.from_inputs(g)
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    tab = oracle.schedule(csr, w.c_min, w.c_max, w.steps)
    k = 3000  # a mid-schedule step
    state = G.anneal(w.trials, w.steps, step_end=k, i0_min=w.c_min, i0_max=w.c_max, seed=w.seed,
                     variability=w.var)
    nxt = torch.empty_like(state)
    p, keep = pbit.make_params(w.trials, w.steps, step_begin=k, step_end=k + 1, i0_min=w.c_min, i0_max=w.c_max,
                               seed=w.seed, variability=w.var)
    pbit.pbit_anneal(G.handle, p, state, nxt)
    s_host, n_host = _host(state), _host(nxt)
    rng = np.random.default_rng(0)
    nodes = rng.integers(0, g.n, 20000).astype(np.int32)
    trials = rng.integers(0, w.trials, 20000).astype(np.int32)
    want, gap = oracle.step_sampled(csr, s_host, nodes, trials, k, tab[k], w.seed, variability=w.var)
    bad = n_host[nodes, trials] != want
    assert not bad.any() or np.abs(gap[bad]).max() < BAND
    # the exact observables at full size
    cuts = G.cut(nxt)
    assert np.array_equal(cuts, oracle.cut(g.src, g.dst, g.w, n_host))


def test_mismatch_rate_below_bound():
    """Lockstep over > 1e7 decisions: mismatches only in the band, and fewer than 1e-6 of decisions."""
    g = inputs.torus_2d(50, 100, 9, "pm1")
    var = inputs.variability(g.n, 9)
    dec, mis, worst = _lockstep(g, 256, 12, var, pbit.KERNEL_SPARSE, S=100)
    assert dec >= 1.5e7
    assert mis == 0 or worst < BAND
    assert mis < 1e-6 * dec


@pytest.mark.parametrize("T", [64, 256, 48])
def test_table_variant_with_weights_and_bias(T):
    """Small-range fields (|w| <= 3, h != 0): the shared-memory threshold table path vs the oracle."""
    g = inputs.erdos_renyi_gnm(1500, 4500, 6, "+1")
    g.w = np.random.default_rng(6).integers(-3, 4, g.m).astype(np.int8)
    h = np.random.default_rng(7).integers(-4, 5, g.n).astype(np.int32)
    var = inputs.variability(g.n, 6, s_intensity=0.3, s_offset=0.3)
    G = pbit.Graph(g.n, g.src, g.dst, g.w, h=h)
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    S = 30
    tab = oracle.schedule(csr, 0.1, 10.0, S)
    state = inputs.random_spins(g.n, T, 2)
    for t in range(0, S, 4):
        d_in = _dev(state)
        d_out = torch.empty_like(d_in)
        p, keep = pbit.make_params(T, S, step_begin=t, step_end=t + 1, seed=3, variability=var,
                                   kernel=pbit.KERNEL_SPARSE)
        pbit.pbit_anneal(G.handle, p, d_in, d_out)
        gpu = _host(d_out)
        want, gap = oracle.step(csr, state, t, tab[t], 3, variability=var, h=h, want_gap=True)
        bad = gpu != want
        assert not bad.any() or np.abs(gap[bad]).max() < BAND
        state = gpu


def test_kernel_variants_agree(tmp_path):
    """Packed-count and table variants give exactly the plain variant's spins (plain forced in a child)."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch\n"
        "from paper_2601_14476_gb300 import inputs, pbit\n"
        "outs = []\n"
        "for g, T in ((inputs.torus_2d(40, 60, 3, 'pm1'), 256), (inputs.erdos_renyi_gnm(900, 2700, 4, '+1'), 64),\n"
        "             (inputs.rgg_knn(1200, 5, 3, 'pm1'), 32), (inputs.erdos_renyi_gnm(800, 19176, 1, '+1'), 16)):\n"
        "    G = pbit.Graph.from_inputs(g)\n"
        "    var = inputs.variability(g.n, 2)\n"
        "    outs.append(G.anneal(T, 40, seed=9, variability=var, kernel=pbit.KERNEL_SPARSE).cpu().numpy())\n"
        "np.savez(%r, *outs)\n")
    res = []
    for k, extra in enumerate(({}, {"PBIT_SPARSE_PLAIN": "1"})):
        path = str(tmp_path / f"v{k}.npz")
        subprocess.run([sys.executable, "-c", code % path], check=True, env=dict(os.environ, **extra), timeout=300)
        res.append(np.load(path))
    for key in res[0].files:
        assert np.array_equal(res[0][key], res[1][key]), key


def _warp_tile_applies(g, T):
    """The launch rule of the warp-table tile: unit weights, max-degree + 1 lanes per node segment."""
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n).max() if g.m else 0
    if np.any(np.abs(g.w) != 1) or deg > 15:
        return False
    for G in (32, 16):
        if T % G:
            continue
        groups = T // G
        if groups % 32 and 32 % groups:
            continue
        if deg + 1 <= min(32, groups):
            return True
    return False


WARP_CASES = [
    ("torus7x9_T256", lambda: inputs.torus_2d(7, 9, 5, "pm1"), 256, True, False),    # 2 nodes per warp, ragged
    ("torus9x11_T512", lambda: inputs.torus_2d(9, 11, 6, "pm1"), 512, True, False),  # G = 32, 2 nodes per warp
    ("torus6x8_T1024", lambda: inputs.torus_2d(6, 8, 7, "pm1"), 1024, True, True),   # one node per warp, h != 0
    ("torus5x6_T2048", lambda: inputs.torus_2d(5, 6, 8, "pm1"), 2048, False, False),  # two warps per node, ideal
    ("rgg300_T1024", lambda: inputs.rgg_knn(300, 9, 3, "pm1"), 1024, True, False),
]


@pytest.mark.parametrize("case", WARP_CASES, ids=[c[0] for c in WARP_CASES])
def test_warp_tile_lockstep(case):
    """Warp-table tile (threshold table in lanes, shuffled by packed count) vs the oracle, step by step."""
    _, make, T, with_var, with_h = case
    g = make()
    assert _warp_tile_applies(g, T)
    var = inputs.variability(g.n, 4, s_intensity=0.3, s_offset=0.3) if with_var else None
    h = np.random.default_rng(3).integers(-3, 4, g.n).astype(np.int32) if with_h else None
    G = pbit.Graph(g.n, g.src, g.dst, g.w, h=h)
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    S = 40
    tab = oracle.schedule(csr, 0.1, 10.0, S)
    state = oracle.init_spins(g.n, T, 21, 2)
    for t in list(range(0, S, 3)) + [S - 1]:
        d_in = _dev(state)
        d_out = torch.empty_like(d_in)
        p, keep = pbit.make_params(T, S, step_begin=t, step_end=t + 1, seed=21, instance=2, variability=var,
                                   kernel=pbit.KERNEL_SPARSE)
        pbit.pbit_anneal(G.handle, p, d_in, d_out)
        gpu = _host(d_out)
        want, gap = oracle.step(csr, state, t, tab[t], 21, 2, variability=var, h=h, want_gap=True)
        bad = gpu != want
        assert not bad.any() or np.abs(gap[bad]).max() < BAND, (t, int(bad.sum()))
        state = gpu


def test_warp_tile_equals_block_tile(tmp_path):
    """Whole anneals: the warp-table tile gives exactly the block-table tile's spins (forced in a child)."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch\n"
        "from paper_2601_14476_gb300 import inputs, pbit\n"
        "outs = []\n"
        "for g, T in ((inputs.torus_2d(30, 40, 3, 'pm1'), 1024), (inputs.torus_2d(13, 17, 4, 'pm1'), 256),\n"
        "             (inputs.torus_2d(11, 13, 5, 'pm1'), 512), (inputs.rgg_knn(900, 6, 3, 'pm1'), 2048)):\n"
        "    G = pbit.Graph.from_inputs(g)\n"
        "    var = inputs.variability(g.n, 2)\n"
        "    outs.append(G.anneal(T, 60, seed=9, variability=var, kernel=pbit.KERNEL_SPARSE).cpu().numpy())\n"
        "np.savez(%r, *outs)\n")
    res = []
    for k, extra in enumerate(({}, {"PBIT_SPARSE_NOWARP": "1"})):
        path = str(tmp_path / f"w{k}.npz")
        subprocess.run([sys.executable, "-c", code % path], check=True, env=dict(os.environ, **extra), timeout=300)
        res.append(np.load(path))
    for key in res[0].files:
        assert np.array_equal(res[0][key], res[1][key]), key


def test_multistep_flow_equals_stepwise(tmp_path):
    """One persistent multi-step launch gives exactly the spins of one launch per step (forced in a child).

    The multi-step form is forced for every graph (by default only graphs with local tile dependencies
    take it) and compared with forced per-step launches and with the default.  Covers the warp-table and
    block-table tiles, tile dependency lists and whole-step waits (random
    graph), nodes spanning two tiles (T = 16384), and in-place resumes with odd and even step counts.
    """
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch\n"
        "from paper_2601_14476_gb300 import inputs, pbit\n"
        "outs = []\n"
        "cases = ((inputs.torus_2d(40, 50, 3, 'pm1'), 1024), (inputs.erdos_renyi_gnm(3000, 9000, 4, '+1'), 64),\n"
        "         (inputs.rgg_knn(1500, 5, 3, 'pm1'), 16), (inputs.torus_2d(5, 6, 2, 'pm1'), 16384),\n"
        "         (inputs.complete_pm1(200, 1), 32))\n"
        "for g, T in cases:\n"
        "    G = pbit.Graph.from_inputs(g)\n"
        "    var = inputs.variability(g.n, 2)\n"
        "    outs.append(G.anneal(T, 57, seed=9, variability=var, kernel=pbit.KERNEL_SPARSE).cpu().numpy())\n"
        "g = inputs.torus_2d(20, 30, 7, 'pm1')\n"
        "G = pbit.Graph.from_inputs(g)\n"
        "a = G.anneal(512, 100, step_end=33, seed=4, kernel=pbit.KERNEL_SPARSE)\n"
        "for lo, hi in ((33, 60), (60, 100)):\n"
        "    p, keep = pbit.make_params(512, 100, step_begin=lo, step_end=hi, seed=4, kernel=pbit.KERNEL_SPARSE)\n"
        "    pbit.pbit_anneal(G.handle, p, a, a)\n"
        "outs.append(a.cpu().numpy())\n"
        "torch.cuda.synchronize()\n"
        "print('launches', pbit.pbit_launch_count())\n"
        "np.savez(%r, *outs)\n")
    res, launches = [], []
    for k, extra in enumerate(({"PBIT_SPARSE_FLOW": "always"}, {"PBIT_SPARSE_STEPWISE": "1"}, {})):
        path = str(tmp_path / f"f{k}.npz")
        r = subprocess.run([sys.executable, "-c", code % path], check=True, env=dict(os.environ, **extra),
                           timeout=300, capture_output=True, text=True)
        launches.append(int(r.stdout.split("launches")[-1]))
        res.append(np.load(path))
    for key in res[0].files:
        assert np.array_equal(res[0][key], res[1][key]), key
        assert np.array_equal(res[2][key], res[1][key]), key
    assert launches[0] < launches[1] // 10, launches
    assert launches[2] < launches[1], launches  # the default takes the multi-step form for the tori


def test_torus_full_run_mean_cut_matches_oracle():
    """100x200 torus, 1024 trials, all 5000 steps in the bench launch form; the oracle runs the first
    16 trials (same seeds and counters).  Over 1e8 decisions per trial a float32 tie-band decision
    can send a trial down another path, so the check is the mean cut, within 0.5 %."""
    w = inputs.sparse_torus20000()
    g = w.graph
    G = pbit.Graph.from_inputs(g)
    out = _host(G.anneal(w.trials, w.steps, i0_min=w.c_min, i0_max=w.c_max, seed=w.seed, instance=w.instance,
                         variability=w.var))
    K = 16
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    tab = oracle.schedule(csr, w.c_min, w.c_max, w.steps)
    ref = oracle.anneal(csr, oracle.init_spins(g.n, K, w.seed, w.instance), tab, w.seed, w.instance,
                        variability=w.var)
    gpu_cut = oracle.cut(g.src, g.dst, g.w, np.ascontiguousarray(out[:, :K]))
    ref_cut = oracle.cut(g.src, g.dst, g.w, ref)
    assert np.array_equal(G.cut(_dev(out))[:K], gpu_cut)
    assert abs(gpu_cut.mean() - ref_cut.mean()) <= 0.005 * abs(ref_cut.mean()), (gpu_cut, ref_cut)


def test_graph_from_any_edge_order_equals_canonical():
    """The same graph given as a shuffled edge list with random orientations (the general CSR
    build) gives the canonical build's fields, cut, schedule normalisation and anneal; a duplicate
    edge in a shuffled list is rejected."""
    g = inputs.rgg_knn(900, 8, 3, "pm1")
    rng = np.random.default_rng(1)
    perm = rng.permutation(g.m)
    flip = rng.integers(0, 2, g.m).astype(bool)
    src = np.where(flip, g.dst, g.src)[perm].astype(np.int32)
    dst = np.where(flip, g.src, g.dst)[perm].astype(np.int32)
    w = g.w[perm]
    A = pbit.Graph(g.n, g.src, g.dst, g.w)
    B = pbit.Graph(g.n, src, dst, w)
    assert A.info()["mean_s"] == B.info()["mean_s"]
    s = _dev(inputs.random_spins(g.n, 32, 3))
    assert np.array_equal(_host(A.fields(s)), _host(B.fields(s)))
    assert np.array_equal(A.cut(s), B.cut(s))
    var = inputs.variability(g.n, 3)
    assert np.array_equal(_host(A.anneal(32, 40, seed=2, variability=var)), _host(B.anneal(32, 40, seed=2, variability=var)))
    with pytest.raises(pbit.PbitError):
        pbit.Graph(g.n, np.append(src, dst[5]), np.append(dst, src[5]), np.append(w, w[5]))


def test_large_graph_build_threads_any_order():
    """Graphs large enough for the threaded host build (over 512K edges): the canonical edge list and
    a shuffled, randomly oriented copy give the same fields and cuts."""
    g = inputs.erdos_renyi_gnm(60000, 600000, 11, "+1")
    g.w = np.random.default_rng(4).choice(np.array([-2, -1, 1, 3], np.int8), g.m)
    rng = np.random.default_rng(2)
    perm = rng.permutation(g.m)
    flip = rng.integers(0, 2, g.m).astype(bool)
    src = np.where(flip, g.dst, g.src)[perm].astype(np.int32)
    dst = np.where(flip, g.src, g.dst)[perm].astype(np.int32)
    A = pbit.Graph(g.n, g.src, g.dst, g.w)
    B = pbit.Graph(g.n, src, dst, g.w[perm])
    assert A.info()["mean_s"] == B.info()["mean_s"]
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    assert A.info()["mean_s"] == oracle.mean_s(csr)
    s = inputs.random_spins(g.n, 16, 5)
    d = _dev(s)
    fa = _host(A.fields(d))
    assert np.array_equal(fa, _host(B.fields(d)))
    assert np.array_equal(fa.astype(np.int64), oracle.fields(csr, s))
    assert np.array_equal(A.cut(d), oracle.cut(g.src, g.dst, g.w, s))


def test_resident_cluster_equals_single_cta_and_oracle(tmp_path):
    """The resident kernel over a cluster of CTAs (spins exchanged through distributed shared memory)
    gives exactly the single-CTA form's spins (forced in a child), on ragged trial counts, a graph
    with fewer nodes than CTAs and a bias; and a lockstep step matches the oracle."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch\n"
        "from paper_2601_14476_gb300 import inputs, pbit\n"
        "outs = []\n"
        "for g, T, S in ((inputs.erdos_renyi_gnm(800, 19176, 1, '+1'), 16, 120), (inputs.rgg_knn(700, 3, 3, 'pm1'), 3, 90),\n"
        "                (inputs.torus_2d(3, 3, 1, 'pm1'), 64, 50), (inputs.erdos_renyi_gnm(300, 2000, 2, 'pm1'), 40, 77)):\n"
        "    h = (np.mod(np.arange(g.n), 5) - 2).astype(np.int32)\n"
        "    G = pbit.Graph(g.n, g.src, g.dst, g.w, h=h)\n"
        "    var = inputs.variability(g.n, 4)\n"
        "    outs.append(G.anneal(T, S, seed=6, variability=var, kernel=pbit.KERNEL_RESIDENT).cpu().numpy())\n"
        "np.savez(%r, *outs)\n")
    res = []
    for k, extra in enumerate(({}, {"PBIT_RESIDENT_CLUSTER": "1"})):
        path = str(tmp_path / f"r{k}.npz")
        subprocess.run([sys.executable, "-c", code % path], check=True, env=dict(os.environ, **extra), timeout=300)
        res.append(np.load(path))
    for key in res[0].files:
        assert np.array_equal(res[0][key], res[1][key]), key
    g = inputs.rgg_knn(500, 9, 3, "pm1")
    var = inputs.variability(g.n, 9)
    dec, mis, worst = _lockstep(g, 20, 10, var, pbit.KERNEL_RESIDENT)
    assert mis == 0 or worst < BAND


def test_resident_resume_in_place():
    """Cluster-resident kernel: a run split into resumed segments, in place (input = output buffer),
    equals the whole run, for odd and even segment lengths and an empty range."""
    g = inputs.erdos_renyi_gnm(500, 4000, 12, "pm1")
    var = inputs.variability(g.n, 12)
    G = pbit.Graph.from_inputs(g)
    T, S = 24, 61
    full = _host(G.anneal(T, S, seed=7, variability=var, kernel=pbit.KERNEL_RESIDENT))
    a = G.anneal(T, S, step_end=20, seed=7, variability=var, kernel=pbit.KERNEL_RESIDENT)
    for lo, hi in ((20, 33), (33, 33), (33, S)):
        p, keep = pbit.make_params(T, S, step_begin=lo, step_end=hi, seed=7, variability=var,
                                   kernel=pbit.KERNEL_RESIDENT)
        pbit.pbit_anneal(G.handle, p, a, a)
    assert np.array_equal(_host(a), full)
