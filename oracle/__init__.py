"""ctypes front end of the plain CPU pSA oracle (``pbit_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product package never
imports it.  The C source is compiled with gcc on first use (or by
``__graft_entry__.build``) into ``oracle/_build/``.

Every function mirrors one C entry point; arrays are numpy, spins are
trial-major int8 ``sigma[i, t]`` (node i, trial t).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbit_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libpbit_oracle.so")
_LOCK = threading.Lock()
_LIB = None

ALG_PSA, ALG_SPSA, ALG_TAPSA = 0, 1, 2
OFFSET_SCALED = 0
OFFSET_LISTING = 1
OFFSET_EQUATION = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so both ISAs agree)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i32, i64, u32, u64, f64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_draw_ru.argtypes = [u64, u32, i32, u32, i32, P, P]
            lib.orc_build_csr.argtypes = [i32, i64, P, P, P, P, P, P]
            lib.orc_build_csr.restype = C.c_int
            lib.orc_mean_s.argtypes = [i32, P, P]
            lib.orc_mean_s.restype = f64
            lib.orc_i0_table.argtypes = [f64, f64, i32, P]
            lib.orc_fields.argtypes = [i32, P, P, P, P, P, i32, P]
            lib.orc_energy.argtypes = [i32, P, P, P, P, P, i32, P]
            lib.orc_cut.argtypes = [i64, P, P, P, P, i32, P]
            lib.orc_bruteforce_maxcut.argtypes = [i32, i64, P, P, P, P]
            lib.orc_bruteforce_maxcut.restype = i64
            lib.orc_step.argtypes = [i32, P, P, P, P, i32, P, P, P, i32, u64, u32, u32, C.c_float, P, P, P]
            lib.orc_step_sampled.argtypes = [i32, P, P, P, P, i32, P, P, P, i32, u64, u32, u32, C.c_float, P,
                                             i64, P, P, P, P]
            lib.orc_init_spins.argtypes = [i32, i32, u64, u32, P]
            lib.orc_init_spins_trials.argtypes = [i32, i32, i32, u64, u32, P]
            lib.orc_anneal.argtypes = [i32, P, P, P, P, i32, P, P, P, i32, u64, u32, P, i32, i32, P]
            lib.orc_anneal.restype = C.c_int
            lib.orc_anneal_trials.argtypes = [i32, P, P, P, P, i32, i32, P, P, P, i32, u64, u32, P, i32, i32, P]
            lib.orc_anneal_trials.restype = C.c_int
            lib.orc_timing_period.argtypes = [i32, C.c_float]
            lib.orc_timing_period.restype = i32
            lib.orc_step_variant.argtypes = [i32, P, P, P, P, i32, P, P, P, i32, u64, u32, i32, f64, i32, i32, P,
                                             u32, P, P, P, P, P, P]
            _LIB = lib
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def philox4x32_10(ctr, key) -> np.ndarray:
    ctr = _c(ctr, np.uint32)
    key = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _lib().orc_philox4x32_10(_p(ctr), _p(key), _p(out))
    return out


def draw_ru(seed: int, instance: int, node: int, step: int, trial: int):
    r, u = C.c_double(), C.c_double()
    _lib().orc_draw_ru(seed, instance, node, step & 0xFFFFFFFF, trial, C.byref(r), C.byref(u))
    return r.value, u.value


class Csr:
    """The oracle's own CSR of J = -w (both directions, sorted columns)."""

    def __init__(self, n, src, dst, w):
        src, dst, w = _c(src, np.int32), _c(dst, np.int32), _c(w, np.int8)
        m = len(src)
        self.n = int(n)
        self.row_ptr = np.zeros(self.n + 1, np.int32)
        self.col = np.zeros(max(2 * m, 1), np.int32)
        self.J = np.zeros(max(2 * m, 1), np.int8)
        rc = _lib().orc_build_csr(self.n, m, _p(src), _p(dst), _p(w), _p(self.row_ptr), _p(self.col), _p(self.J))
        if rc != 0:
            raise ValueError(f"oracle rejected the edge list (code {rc})")
        self.src, self.dst, self.w = src, dst, w

    def args(self):
        return self.n, _p(self.row_ptr), _p(self.col), _p(self.J)


def mean_s(csr: Csr) -> float:
    return _lib().orc_mean_s(csr.n, _p(csr.row_ptr), _p(csr.J))


def i0_table(i0min: float, i0max: float, steps: int) -> np.ndarray:
    out = np.zeros(max(steps, 1), np.float32)
    _lib().orc_i0_table(float(i0min), float(i0max), int(steps), _p(out))
    return out[:steps]


def schedule(csr: Csr, c_min: float, c_max: float, steps: int, normalize: bool = True) -> np.ndarray:
    """I0 table of the Methods section: c/mean(s_i) when normalize, else absolute."""
    if normalize:
        ms = mean_s(csr)
        return i0_table(c_min / ms, c_max / ms, steps)
    return i0_table(c_min, c_max, steps)


def fields(csr: Csr, sigma, h=None) -> np.ndarray:
    sigma = _c(sigma, np.int8)
    T = sigma.shape[1]
    out = np.zeros((csr.n, T), np.int64)
    _lib().orc_fields(*csr.args(), _p(_c(h, np.int32)), _p(sigma), T, _p(out))
    return out


def energy(csr: Csr, sigma, h=None) -> np.ndarray:
    sigma = _c(sigma, np.int8)
    T = sigma.shape[1]
    out = np.zeros(T, np.int64)
    _lib().orc_energy(*csr.args(), _p(_c(h, np.int32)), _p(sigma), T, _p(out))
    return out


def cut(src, dst, w, sigma) -> np.ndarray:
    src, dst, w, sigma = _c(src, np.int32), _c(dst, np.int32), _c(w, np.int8), _c(sigma, np.int8)
    T = sigma.shape[1]
    out = np.zeros(T, np.int64)
    _lib().orc_cut(len(src), _p(src), _p(dst), _p(w), _p(sigma), T, _p(out))
    return out


def bruteforce_maxcut(n, src, dst, w):
    src, dst, w = _c(src, np.int32), _c(dst, np.int32), _c(w, np.int8)
    best = np.zeros(n, np.int8)
    val = _lib().orc_bruteforce_maxcut(int(n), len(src), _p(src), _p(dst), _p(w), _p(best))
    return int(val), best


def init_spins(n: int, T: int, seed: int, instance: int = 0, trial_base: int = 0) -> np.ndarray:
    """Initial state of trials trial_base .. trial_base + T - 1 (column t is trial trial_base + t)."""
    out = np.zeros((n, T), np.int8)
    _lib().orc_init_spins_trials(int(n), int(T), int(trial_base), seed, instance, _p(out))
    return out


def _var(v):
    if v is None:
        return None, None, None
    return _c(v.get("intensity"), np.float32), _c(v.get("offset"), np.float32), _c(v.get("p_update"), np.float32)


def step(csr: Csr, sigma, step_idx: int, I0: float, seed: int, instance: int = 0, variability=None, h=None,
         offset_mode: int = OFFSET_SCALED, want_gap: bool = False):
    sigma = _c(sigma, np.int8)
    T = sigma.shape[1]
    lam, dlt, pu = _var(variability)
    out = np.zeros_like(sigma)
    gap = np.zeros(sigma.shape, np.float64) if want_gap else None
    _lib().orc_step(*csr.args(), _p(_c(h, np.int32)), T, _p(lam), _p(dlt), _p(pu), offset_mode, seed, instance,
                    step_idx & 0xFFFFFFFF, float(I0), _p(sigma), _p(out), _p(gap))
    return (out, gap) if want_gap else out


def step_sampled(csr: Csr, sigma, nodes, trials, step_idx: int, I0: float, seed: int, instance: int = 0,
                 variability=None, h=None, offset_mode: int = OFFSET_SCALED):
    sigma = _c(sigma, np.int8)
    T = sigma.shape[1]
    nodes, trials = _c(nodes, np.int32), _c(trials, np.int32)
    lam, dlt, pu = _var(variability)
    out = np.zeros(len(nodes), np.int8)
    gap = np.zeros(len(nodes), np.float64)
    _lib().orc_step_sampled(*csr.args(), _p(_c(h, np.int32)), T, _p(lam), _p(dlt), _p(pu), offset_mode, seed,
                            instance, step_idx & 0xFFFFFFFF, float(I0), _p(sigma), len(nodes), _p(nodes),
                            _p(trials), _p(out), _p(gap))
    return out, gap


def anneal(csr: Csr, sigma0, table, seed: int, instance: int = 0, variability=None, h=None,
           offset_mode: int = OFFSET_SCALED, step_begin: int = 0, step_end: int | None = None,
           trial_base: int = 0) -> np.ndarray:
    """Schedule steps [step_begin, step_end) of the trials whose columns sigma0 holds: column t is
    trial trial_base + t (the trials are independent, so any range of them can run alone)."""
    sigma = np.array(sigma0, dtype=np.int8, order="C", copy=True)
    T = sigma.shape[1]
    table = _c(table, np.float32)
    if step_end is None:
        step_end = len(table)
    lam, dlt, pu = _var(variability)
    rc = _lib().orc_anneal_trials(*csr.args(), _p(_c(h, np.int32)), T, int(trial_base), _p(lam), _p(dlt), _p(pu),
                                  offset_mode, seed, instance, _p(table), int(step_begin), int(step_end), _p(sigma))
    if rc != 0:
        raise MemoryError("oracle anneal failed")
    return sigma


def anneal_cuts(job: dict) -> np.ndarray:
    """Final cuts of a whole anneal of trials [base, base + trials) of one instance, from a picklable job
    (keys n, src, dst, w, trials, steps, c_min, c_max, seed, instance, var, optional base), so that a
    spawned process pool can share out the trials of a large instance."""
    csr = Csr(job["n"], job["src"], job["dst"], job["w"])
    tab = schedule(csr, job["c_min"], job["c_max"], job["steps"])
    base = int(job.get("base", 0))
    s0 = init_spins(job["n"], job["trials"], job["seed"], job["instance"], trial_base=base)
    out = anneal(csr, s0, tab, job["seed"], job["instance"], variability=job["var"], trial_base=base)
    return cut(job["src"], job["dst"], job["w"], out)


def timing_period(t_res: int, nu_dev: float) -> int:
    return int(_lib().orc_timing_period(int(t_res), float(nu_dev)))


class VariantState:
    """Per-(node, trial) state of SpSA (last input) and TApSA (last `window` fields)."""

    def __init__(self, n, T, window=4):
        self.Iprev = np.zeros((n, T), np.float64)
        self.ring = np.zeros((max(window, 1), n, T), np.int64)
        self.window = window


def step_variant(csr: Csr, sigma, q: int, table, seed: int, instance: int = 0, algorithm: int = ALG_PSA,
                 stall_prob: float = 0.5, window: int = 4, t_res: int = 0, nu_dev=None, variability=None, h=None,
                 offset_mode: int = OFFSET_SCALED, state: VariantState | None = None, want_gap: bool = False):
    """One sub-step q of pSA / SpSA / TApSA with the optional period timing model; updates `state`."""
    sigma = _c(sigma, np.int8)
    T = sigma.shape[1]
    lam, dlt, pu = _var(variability)
    state = state or VariantState(csr.n, T, window)
    out = np.zeros_like(sigma)
    gap = np.zeros(sigma.shape, np.float64) if want_gap else None
    tab = _c(table, np.float32)
    _lib().orc_step_variant(*csr.args(), _p(_c(h, np.int32)), T, _p(lam), _p(dlt), _p(pu), offset_mode, seed,
                            instance, algorithm, float(stall_prob), int(window), int(t_res),
                            _p(_c(nu_dev, np.float32)), q & 0xFFFFFFFF, _p(tab), _p(sigma), _p(out),
                            _p(state.Iprev), _p(state.ring), _p(gap))
    return (out, gap) if want_gap else out


def anneal_variant(csr: Csr, sigma0, table, seed: int, instance: int = 0, algorithm: int = ALG_PSA,
                   stall_prob: float = 0.5, window: int = 4, t_res: int = 0, nu_dev=None, variability=None,
                   h=None, offset_mode: int = OFFSET_SCALED, q_begin: int = 0, q_end: int | None = None,
                   state: VariantState | None = None):
    """Sub-steps [q_begin, q_end) (q_end default: len(table) * max(t_res, 1))."""
    sigma = np.array(sigma0, dtype=np.int8, order="C", copy=True)
    state = state or VariantState(csr.n, sigma.shape[1], window)
    if q_end is None:
        q_end = len(table) * max(t_res, 1)
    for q in range(q_begin, q_end):
        sigma = step_variant(csr, sigma, q, table, seed, instance, algorithm, stall_prob, window, t_res, nu_dev,
                             variability, h, offset_mode, state)
    return sigma, state
