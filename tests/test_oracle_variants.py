"""Pins of the oracle's pSA variants (Eq. SpSA, Eq. TApSA) and the period
timing model (T_res sub-steps per cycle) to special cases and closed forms."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2601_14476_gb300 import inputs


def _setup(n=60, m=300, T=24, seed=3):
    g = inputs.erdos_renyi_gnm(n, m, seed, "pm1")
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    s0 = oracle.init_spins(n, T, seed)
    var = inputs.variability(n, seed, s_intensity=0.3, s_offset=0.3)
    return g, csr, s0, var


def test_spsa_without_stalls_is_psa():
    g, csr, s, var = _setup()
    tab = oracle.schedule(csr, 0.1, 10.0, 12)
    st = oracle.VariantState(g.n, s.shape[1])
    a, b = s.copy(), s.copy()
    for q in range(12):
        a = oracle.step_variant(csr, a, q, tab, 5, algorithm=oracle.ALG_SPSA, stall_prob=0.0, variability=var,
                                state=st)
        b = oracle.step(csr, b, q, tab[q], 5, variability=var)
        assert np.array_equal(a, b), q


@pytest.mark.parametrize("mode", [oracle.OFFSET_SCALED, oracle.OFFSET_LISTING, oracle.OFFSET_EQUATION])
def test_tapsa_window_one_is_psa(mode):
    g, csr, s, var = _setup()
    tab = oracle.schedule(csr, 0.1, 10.0, 10)
    st = oracle.VariantState(g.n, s.shape[1], window=1)
    a, b = s.copy(), s.copy()
    for q in range(10):
        a = oracle.step_variant(csr, a, q, tab, 7, algorithm=oracle.ALG_TAPSA, window=1, variability=var,
                                offset_mode=mode, state=st)
        b = oracle.step(csr, b, q, tab[q], 7, variability=var, offset_mode=mode)
        assert np.array_equal(a, b), q


def test_timing_unit_period_is_psa():
    g, csr, s, var = _setup()
    tab = oracle.schedule(csr, 0.1, 10.0, 8)
    a, b = s.copy(), s.copy()
    for q in range(8):
        a = oracle.step_variant(csr, a, q, tab, 9, t_res=1, nu_dev=np.zeros(g.n, np.float32), variability=var)
        b = oracle.step(csr, b, q, tab[q], 9, variability=var)
        assert np.array_equal(a, b)


def test_timing_period_mapping():
    assert oracle.timing_period(10, 0.0) == 10
    assert oracle.timing_period(10, 0.25) == 13     # 12.5 rounds away from zero
    assert oracle.timing_period(10, -0.25) == 8     # 7.5 -> 8
    assert oracle.timing_period(10, 0.75) == 18     # 17.5 -> 18
    assert oracle.timing_period(10, -1.2) == 1      # clamped to one sub-step
    assert oracle.timing_period(10, 0.26) == 13


def test_timing_nodes_update_only_on_their_period():
    g, csr, s, _ = _setup(T=16)
    nu_dev = np.random.default_rng(1).normal(0, 0.5, g.n).astype(np.float32)
    periods = np.array([oracle.timing_period(10, v) for v in nu_dev])
    tab = np.full(5, 1e30, np.float32)  # deterministic decisions: sgn(field)
    state = s.copy()
    for q in range(45):
        nxt = oracle.step_variant(csr, state, q, tab, 2, t_res=10, nu_dev=nu_dev)
        idle = (q % periods) != 0
        assert np.array_equal(nxt[idle], state[idle]), q
        D = oracle.fields(csr, state)
        due = ~idle
        nz = D[due] != 0
        assert np.array_equal(nxt[due][nz], np.sign(D[due][nz]).astype(np.int8))
        state = nxt


def test_tapsa_average_includes_zero_history():
    """Frozen spins: at sub-step q the TApSA input is I0 * D * min(q+1, alpha) / alpha (TI(t<0) = 0)."""
    g, csr, s, _ = _setup(T=8)
    lam = np.full(g.n, 1.0, np.float32)
    var = {"intensity": lam, "offset": np.zeros(g.n, np.float32), "p_update": np.zeros(g.n, np.float32)}
    tab = oracle.i0_table(0.2, 0.9, 6)
    st = oracle.VariantState(g.n, 8, window=4)
    D = oracle.fields(csr, s)
    for q in range(6):
        out, gap = oracle.step_variant(csr, s, q, tab, 4, algorithm=oracle.ALG_TAPSA, window=4, variability=var,
                                       state=st, want_gap=True)
        assert np.array_equal(out, s)  # p = 0: nothing moves, inputs still enter the ring
        r = np.array([[oracle.draw_ru(4, 0, i, q, t)[0] for t in range(8)] for i in range(g.n)])
        x = np.arctanh(np.clip(gap + r, -1 + 1e-15, 1 - 1e-15))
        want = float(tab[q]) * D * min(q + 1, 4) / 4.0
        ok = np.abs(want) < 5  # away from tanh saturation the inversion is accurate
        assert np.allclose(x[ok], want[ok], rtol=1e-7, atol=1e-9), q


def test_spsa_stall_rate_and_full_stall():
    g, csr, s, var = _setup(T=64)
    tab = oracle.schedule(csr, 0.1, 10.0, 6)
    st = oracle.VariantState(g.n, 64)
    prev = None
    same = total = 0
    for q in range(6):
        s = oracle.step_variant(csr, s, q, tab, 11, algorithm=oracle.ALG_SPSA, stall_prob=0.5, state=st)
        if prev is not None:
            same += int((st.Iprev == prev).sum())
            total += st.Iprev.size
        prev = st.Iprev.copy()
    # kept inputs: stalls plus the rare fresh input equal to the old one (only possible when D = 0 twice)
    assert abs(same / total - 0.5) < 0.05
    # p = 1: the input stays at its initial 0 -> x = I0 * delta; with delta = 0 a fair coin
    st = oracle.VariantState(g.n, 64)
    ups = 0
    for q in range(4):
        out = oracle.step_variant(csr, s, q, tab, 13, algorithm=oracle.ALG_SPSA, stall_prob=1.0, state=st)
        ups += int((out == 1).sum())
    assert np.all(st.Iprev == 0)
    tot = 4 * out.size
    assert abs(ups / tot - 0.5) < 5 * 0.5 / np.sqrt(tot)


def test_spsa_stall_draw_against_triton_philox():
    """The SpSA stall draw (reading: word t mod 4 of Philox at counter (node, q, instance xor 2^31,
    t / 4), stall iff its top 24 bits / 2^24 < p) pinned to Triton's independent Philox.  A stalled
    (node, trial) keeps its previous input, so with every previous input set to NaN the NaNs left
    after one sub-step mark exactly the stalls; at p = 1/2 a stall is a word whose top bit is 0."""
    pytest.importorskip("triton")
    g, csr, s, _ = _setup(n=5, m=8, T=12)
    seed, instance, q = 0x7777_0000_1234, 6, 3
    tab = oracle.schedule(csr, 0.1, 10.0, 8)
    st = oracle.VariantState(g.n, 12)
    st.Iprev[:] = np.nan
    oracle.step_variant(csr, s, q, tab, seed, instance, algorithm=oracle.ALG_SPSA, stall_prob=0.5, state=st)
    stalled = np.isnan(st.Iprev)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    cases = [([i, q, instance ^ 0x80000000, c], key) for i in range(g.n) for c in range(3)]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = os.path.join(root, "tests", "golden", "triton_philox.py")
    res = subprocess.run([sys.executable, script], input=json.dumps(cases), capture_output=True, text=True,
                         env=dict(os.environ, TRITON_INTERPRET="1"), timeout=600)
    if res.returncode != 0:
        pytest.skip(f"triton interpreter unavailable: {res.stderr[-300:]}")
    words = json.loads(res.stdout)
    for i in range(g.n):
        for t in range(12):
            w = words[3 * i + t // 4][t % 4]
            assert stalled[i, t] == ((w >> 31) == 0), (i, t)
    assert 0 < stalled.sum() < stalled.size
