"""CPU-only checks of the C-ABI library: it builds, loads, exports every
declared symbol, and its host-side logic (edge-list validation, mean_s, the
float32 I0 schedule) equals the oracle's bit for bit.  No device calls."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2601_14476_gb300 import inputs, pbit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(pbit_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = pbit.lib()
    names = _declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version():
    assert pbit.pbit_version() >= 100


@pytest.mark.parametrize("lo,hi,S", [(0.1, 10.0, 1000), (0.05, 5.0, 2000), (0.1, 10.0, 5000), (1e-3, 3.0, 1),
                                     (0.013, 1.7, 7)])
def test_i0_table_bit_exact_vs_oracle(lo, hi, S):
    assert np.array_equal(pbit.pbit_i0_table(lo, hi, S), oracle.i0_table(lo, hi, S))


@pytest.mark.parametrize("make", [
    lambda: inputs.erdos_renyi_gnm(800, 19176, 1, "+1"),
    lambda: inputs.torus_2d(10, 20, 2, "pm1"),
    lambda: inputs.complete_pm1(60, 3),
    lambda: inputs.rgg_knn(500, 4, 3, "pm1"),
])
def test_mean_s_and_schedule_match_oracle(make):
    g = make()
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    ms = pbit.pbit_mean_s(g.n, g.src, g.dst, g.w)
    assert ms == oracle.mean_s(csr)
    for (c0, c1, S) in [(0.1, 10.0, 1000), (0.05, 5.0, 2000)]:
        assert np.array_equal(pbit.pbit_i0_table(c0 / ms, c1 / ms, S), oracle.schedule(csr, c0, c1, S))


def test_validation_rejects_bad_edge_lists():
    bad = [
        (4, [0], [0], [1]),          # self loop
        (4, [0, 1], [1, 0], [1, 1]),  # duplicate
        (4, [0], [4], [1]),          # out of range
        (4, [0], [1], [-128]),       # J = -w overflows int8
        (0, [], [], []),             # empty node set
    ]
    for n, s, d, w in bad:
        with pytest.raises(pbit.PbitError) as ei:
            pbit.pbit_mean_s(n, s, d, w)
        assert ei.value.code == pbit.PBIT_E_INVALID
    with pytest.raises(pbit.PbitError):
        pbit.pbit_i0_table(0.0, 1.0, 10)
    with pytest.raises(pbit.PbitError):
        pbit.pbit_i0_table(0.1, 1.0, 0)


def test_generators_shapes():
    g = inputs.erdos_renyi_gnm(800, 19176, 1, "+1")
    assert g.m == 19176 and np.all(g.src < g.dst) and len(set(zip(g.src.tolist(), g.dst.tolist()))) == g.m
    t = inputs.torus_2d(100, 200, 1)
    assert t.n == 20000 and t.m == 40000 and set(np.unique(t.w)) == {-1, 1}
    deg = np.bincount(np.concatenate([t.src, t.dst]), minlength=t.n)
    assert np.all(deg == 4)
    k = inputs.complete_pm1(50, 1)
    assert k.m == 50 * 49 // 2
    r = inputs.rgg_knn(1000, 1, 3)
    deg = np.bincount(np.concatenate([r.src, r.dst]), minlength=r.n)
    assert deg.min() >= 3
    v = inputs.variability(1000, 1)
    assert abs(v["intensity"].mean() - 1) < 0.02 and abs(v["intensity"].std() - 0.1) < 0.02
    assert np.all((v["p_update"] >= 0) & (v["p_update"] <= 1)) and abs(v["p_update"].mean() - 0.9) < 0.01
    b = inputs.batch64(1, count=8, steps=10)
    assert [w.trials for w in b] == [32, 64, 128, 256, 32, 64, 128, 256]


def test_sweep_grid_points_draw_the_stated_spreads():
    """Host side of the variability sweep: ideal points carry no arrays; others draw Eq. 7's spreads."""
    import numpy as np

    from paper_2601_14476_gb300 import sweep

    assert sweep.point_variability(100, 1, sweep.SweepPoint()) is None
    v = sweep.point_variability(40000, 2, sweep.SweepPoint(s_intensity=0.2, s_offset=0.05, p_mean=0.8, s_p=0.1))
    assert abs(v["intensity"].mean() - 1.0) < 0.01 and abs(v["intensity"].std() - 0.2) < 0.01
    assert abs(v["offset"].mean()) < 0.005 and abs(v["offset"].std() - 0.05) < 0.005
    assert v["p_update"].min() >= 0.0 and v["p_update"].max() <= 1.0 and abs(v["p_update"].mean() - 0.8) < 0.01
    grid = sweep.default_grid()
    assert grid[0].ideal and len(set(grid)) == len(grid)
