"""Thin ctypes binding of ``libpbit.so`` (include/pbit.h).

Each function has the C entry point's name and only marshals arguments:
numpy arrays become host pointers, torch CUDA tensors become device
pointers, ``torch.cuda.Stream`` objects become ``cudaStream_t``.  Every step
of the annealing path runs inside the library's CUDA kernels; there is no
Python or CPU fallback, and a missing library raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

PBIT_OK = 0
PBIT_PENDING = 1
PBIT_E_INVALID = -1
PBIT_E_NOMEM = -2
PBIT_E_CUDA = -3
PBIT_E_TIMEOUT = -4
PBIT_E_BUDGET = -5
PBIT_E_UNSUPPORTED = -6
PBIT_E_NOTFOUND = -7

PBIT_GRAPH_DENSE = 1

OFFSET_SCALED, OFFSET_LISTING, OFFSET_EQUATION = 0, 1, 2
KERNEL_AUTO, KERNEL_SPARSE, KERNEL_DENSE, KERNEL_RESIDENT = 0, 1, 2, 3
ALG_PSA, ALG_SPSA, ALG_TAPSA = 0, 1, 2

_STATUS = {0: "PBIT_OK", 1: "PBIT_PENDING", -1: "PBIT_E_INVALID", -2: "PBIT_E_NOMEM", -3: "PBIT_E_CUDA",
           -4: "PBIT_E_TIMEOUT", -5: "PBIT_E_BUDGET", -6: "PBIT_E_UNSUPPORTED", -7: "PBIT_E_NOTFOUND"}


class PbitError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class pbit_graph_info_t(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_edges", C.c_int64), ("max_degree", C.c_int32), ("unit_weights", C.c_int32),
                ("has_dense", C.c_int32), ("device", C.c_int32), ("mean_s", C.c_double),
                ("total_weight", C.c_int64), ("device_bytes", C.c_size_t), ("has_dense_fp4", C.c_int32)]


class pbit_anneal_params(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("trials", C.c_int32), ("steps", C.c_int32),
                ("step_begin", C.c_int32), ("step_end", C.c_int32), ("i0_min", C.c_double),
                ("i0_max", C.c_double), ("i0_normalize", C.c_int32), ("offset_mode", C.c_int32),
                ("seed", C.c_uint64), ("instance", C.c_uint32), ("kernel", C.c_int32),
                ("intensity", C.c_void_p), ("offset", C.c_void_p), ("p_update", C.c_void_p),
                ("stream", C.c_void_p), ("algorithm", C.c_int32), ("stall_prob", C.c_float),
                ("window", C.c_int32), ("t_res", C.c_int32), ("nu_dev", C.c_void_p), ("state", C.c_void_p)]


class pbit_batch_tuning(C.Structure):
    _fields_ = [("chunk_steps", C.c_int32), ("ctas_per_sm", C.c_int32), ("ms_per_step", C.c_float)]


class pbit_server_stats_t(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("queued", C.c_uint64), ("resident", C.c_int32),
                ("peak_resident", C.c_int32), ("chunks", C.c_uint64), ("spin_updates", C.c_double),
                ("busy_seconds", C.c_double), ("hbm_in_use", C.c_size_t)]


_LIB = None
_LOCK = threading.Lock()
_P = C.c_void_p


def _declare(lib):
    i32, i64, u32, u64, f64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
    sig = {
        "pbit_last_error": ([], C.c_char_p),
        "pbit_version": ([], i32),
        "pbit_launch_count": ([], i64),
        "pbit_graph_create": ([i32, i64, _P, _P, _P, _P, u32, _P], C.c_int),
        "pbit_graph_destroy": ([_P], None),
        "pbit_graph_info": ([_P, _P], C.c_int),
        "pbit_schedule": ([_P, f64, f64, i32, i32, _P], C.c_int),
        "pbit_i0_table": ([f64, f64, i32, _P], C.c_int),
        "pbit_mean_s": ([i32, i64, _P, _P, _P, _P], C.c_int),
        "pbit_anneal_params_default": ([_P], None),
        "pbit_anneal": ([_P, _P, _P, _P], C.c_int),
        "pbit_anneal_noalloc": ([_P, _P, _P, _P], C.c_int),
        "pbit_anneal_trace": ([_P, _P, _P, _P, i32, i32, _P], C.c_int),
        "pbit_variant_state_bytes": ([i32, i32, i32, i32], C.c_size_t),
        "pbit_init_spins": ([_P, i32, u64, u32, _P, _P], C.c_int),
        "pbit_select_kernel": ([_P, i32, i32, _P], C.c_int),
        "pbit_fields": ([_P, _P, i32, _P, _P], C.c_int),
        "pbit_fields_dense": ([_P, _P, i32, _P, _P], C.c_int),
        "pbit_graph_status": ([_P, _P], C.c_int),
        "pbit_selftest_timeout": ([_P, i32, _P], C.c_int),
        "pbit_cut": ([_P, _P, i32, _P, i32, _P], C.c_int),
        "pbit_energy": ([_P, _P, i32, _P, i32, _P], C.c_int),
        "pbit_batch_create": ([i32, _P, _P, _P], C.c_int),
        "pbit_batch_destroy": ([_P], None),
        "pbit_batch_set_spins": ([_P, i32, _P, _P], C.c_int),
        "pbit_batch_run": ([_P, i32, i32, _P], C.c_int),
        "pbit_batch_progress": ([_P, i32, _P], C.c_int),
        "pbit_batch_spins": ([_P, i32, _P, _P], C.c_int),
        "pbit_batch_cuts": ([_P, i32, _P, _P], C.c_int),
        "pbit_batch_autotune": ([_P, _P, _P], C.c_int),
        "pbit_batch_set_tuning": ([_P, i32, i32], C.c_int),
        "pbit_server_create": ([C.c_size_t, i32, i32, _P], C.c_int),
        "pbit_server_destroy": ([_P], None),
        "pbit_server_submit": ([_P, _P, _P, _P], C.c_int),
        "pbit_server_poll": ([_P, u64, _P, _P], C.c_int),
        "pbit_server_wait": ([_P, u64, f64, _P, _P], C.c_int),
        "pbit_server_stats": ([_P, _P], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def lib():
    """Load (building first if needed) the in-tree libpbit.so."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libpbit.so is missing and could not be built")
            _LIB = _declare(C.CDLL(path))
    return _LIB


def _check(code):
    if code not in (PBIT_OK, PBIT_PENDING):
        raise PbitError(code, lib().pbit_last_error().decode(errors="replace"))
    return code


def _host(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(_P)


def _dev(t):
    """Device pointer of a CUDA tensor (or an int already holding one)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(s):
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # noqa: BLE001
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---------------------------------------------------------------- entries ---

def pbit_version() -> int:
    return int(lib().pbit_version())


def pbit_launch_count() -> int:
    return int(lib().pbit_launch_count())


def pbit_graph_create(n, src, dst, w, h=None, flags=0):
    src_a, src_p = _host(src, np.int32)
    dst_a, dst_p = _host(dst, np.int32)
    w_a, w_p = _host(w, np.int8)
    h_a, h_p = _host(h, np.int32)
    out = _P()
    _check(lib().pbit_graph_create(int(n), len(src_a), src_p, dst_p, w_p, h_p, int(flags), C.byref(out)))
    return out


def pbit_graph_destroy(g):
    if g:
        lib().pbit_graph_destroy(g)


def pbit_graph_info(g) -> dict:
    info = pbit_graph_info_t()
    _check(lib().pbit_graph_info(g, C.byref(info)))
    return {k: getattr(info, k) for k, _ in info._fields_}


def pbit_schedule(g, i0_min, i0_max, normalize, steps) -> np.ndarray:
    out = np.zeros(int(steps), np.float32)
    _check(lib().pbit_schedule(g, float(i0_min), float(i0_max), int(normalize), int(steps),
                               out.ctypes.data_as(_P)))
    return out


def pbit_i0_table(i0_min, i0_max, steps) -> np.ndarray:
    out = np.zeros(int(steps), np.float32)
    _check(lib().pbit_i0_table(float(i0_min), float(i0_max), int(steps), out.ctypes.data_as(_P)))
    return out


def pbit_mean_s(n, src, dst, w) -> float:
    src_a, src_p = _host(src, np.int32)
    dst_a, dst_p = _host(dst, np.int32)
    w_a, w_p = _host(w, np.int8)
    out = C.c_double()
    _check(lib().pbit_mean_s(int(n), len(src_a), src_p, dst_p, w_p, C.byref(out)))
    return out.value


def make_params(trials, steps, step_begin=0, step_end=0, i0_min=0.1, i0_max=10.0, i0_normalize=1,
                offset_mode=OFFSET_SCALED, seed=1, instance=0, kernel=KERNEL_AUTO, variability=None,
                stream=None, algorithm=ALG_PSA, stall_prob=0.5, window=4, t_res=0, nu_dev=None, state=None):
    """Build a pbit_anneal_params; returns (params, keepalive) - keep both alive during the call."""
    p = pbit_anneal_params()
    lib().pbit_anneal_params_default(C.byref(p))
    p.trials, p.steps, p.step_begin, p.step_end = int(trials), int(steps), int(step_begin), int(step_end)
    p.i0_min, p.i0_max, p.i0_normalize = float(i0_min), float(i0_max), int(i0_normalize)
    p.offset_mode, p.seed, p.instance, p.kernel = int(offset_mode), int(seed) & (2**64 - 1), int(instance), \
        int(kernel)
    keep = []
    if variability is not None:
        for field in ("intensity", "offset", "p_update"):
            arr, ptr = _host(variability.get(field), np.float32)
            keep.append(arr)
            setattr(p, field, ptr.value if ptr is not None else None)
    p.stream = _stream(stream)
    p.algorithm, p.stall_prob, p.window, p.t_res = int(algorithm), float(stall_prob), int(window), int(t_res)
    if nu_dev is not None:
        arr, ptr = _host(nu_dev, np.float32)
        keep.append(arr)
        p.nu_dev = ptr.value
    p.state = _dev(state)
    return p, keep


def pbit_anneal(g, params, spins_in, spins_out):
    _check(lib().pbit_anneal(g, C.byref(params), _dev(spins_in), _dev(spins_out)))


def pbit_anneal_noalloc(g, params, spins_in, spins_out):
    """pbit_anneal with its scratch in the library's fixed device array (no allocation)."""
    _check(lib().pbit_anneal_noalloc(g, C.byref(params), _dev(spins_in), _dev(spins_out)))


def pbit_select_kernel(g, requested, trials) -> int:
    out = C.c_int32()
    _check(lib().pbit_select_kernel(g, int(requested), int(trials), C.byref(out)))
    return out.value


def pbit_anneal_trace(g, params, spins_in, spins_out, every, what, trace):
    """`trace`: CUDA int64 tensor [ceil(steps/every), T]; what 0 = energy, 1 = cut."""
    _check(lib().pbit_anneal_trace(g, C.byref(params), _dev(spins_in), _dev(spins_out), int(every), int(what),
                                   _dev(trace)))


def pbit_variant_state_bytes(n, trials, algorithm, window=4) -> int:
    return int(lib().pbit_variant_state_bytes(int(n), int(trials), int(algorithm), int(window)))


def pbit_init_spins(g, trials, seed, instance, spins, stream=None):
    _check(lib().pbit_init_spins(g, int(trials), int(seed) & (2**64 - 1), int(instance), _dev(spins),
                                 _stream(stream)))


def pbit_fields(g, spins, trials, fields, stream=None):
    _check(lib().pbit_fields(g, _dev(spins), int(trials), _dev(fields), _stream(stream)))


def pbit_fields_dense(g, spins, trials, fields, stream=None):
    _check(lib().pbit_fields_dense(g, _dev(spins), int(trials), _dev(fields), _stream(stream)))


def pbit_selftest_timeout(g, budget_us, stream=None):
    _check(lib().pbit_selftest_timeout(g, int(budget_us), _stream(stream)))


def pbit_graph_status(g, stream=None):
    _check(lib().pbit_graph_status(g, _stream(stream)))


def pbit_cut(g, spins, trials, stream=None) -> np.ndarray:
    out = np.zeros(int(trials), np.int64)
    _check(lib().pbit_cut(g, _dev(spins), int(trials), out.ctypes.data_as(_P), 1, _stream(stream)))
    return out


def pbit_energy(g, spins, trials, stream=None) -> np.ndarray:
    out = np.zeros(int(trials), np.int64)
    _check(lib().pbit_energy(g, _dev(spins), int(trials), out.ctypes.data_as(_P), 1, _stream(stream)))
    return out


def pbit_cut_device(g, spins, trials, out, stream=None):
    _check(lib().pbit_cut(g, _dev(spins), int(trials), _dev(out), 0, _stream(stream)))


def pbit_batch_create(graphs, params):
    """graphs: list of handles; params: list of pbit_anneal_params (host arrays kept alive by the caller)."""
    n = len(graphs)
    garr = (C.c_void_p * n)(*[g.value if isinstance(g, C.c_void_p) else g for g in graphs])
    parr = (pbit_anneal_params * n)(*params)
    out = _P()
    _check(lib().pbit_batch_create(n, garr, parr, C.byref(out)))
    return out


def pbit_batch_destroy(b):
    if b:
        lib().pbit_batch_destroy(b)


def pbit_batch_set_spins(b, k, spins, stream=None):
    _check(lib().pbit_batch_set_spins(b, int(k), _dev(spins), _stream(stream)))


def pbit_batch_run(b, chunk_steps=0, max_chunks=0, stream=None):
    _check(lib().pbit_batch_run(b, int(chunk_steps), int(max_chunks), _stream(stream)))


def pbit_batch_progress(b, k) -> int:
    out = C.c_int32()
    _check(lib().pbit_batch_progress(b, int(k), C.byref(out)))
    return out.value


def pbit_batch_spins(b, k, out, stream=None):
    _check(lib().pbit_batch_spins(b, int(k), _dev(out), _stream(stream)))


def pbit_batch_cuts(b, k, trials, stream=None) -> np.ndarray:
    out = np.zeros(int(trials), np.int64)
    _check(lib().pbit_batch_cuts(b, int(k), out.ctypes.data_as(_P), _stream(stream)))
    return out


def pbit_batch_autotune(b, stream=None) -> dict:
    t = pbit_batch_tuning()
    _check(lib().pbit_batch_autotune(b, _stream(stream), C.byref(t)))
    return {"chunk_steps": t.chunk_steps, "ctas_per_sm": t.ctas_per_sm, "ms_per_step": t.ms_per_step}


def pbit_batch_set_tuning(b, chunk_steps, ctas_per_sm=0):
    _check(lib().pbit_batch_set_tuning(b, int(chunk_steps), int(ctas_per_sm)))


def pbit_server_create(hbm_budget, max_slots, chunk_steps):
    out = _P()
    _check(lib().pbit_server_create(int(hbm_budget), int(max_slots), int(chunk_steps), C.byref(out)))
    return out


def pbit_server_destroy(s):
    if s:
        lib().pbit_server_destroy(s)


def pbit_server_submit(s, g, params) -> int:
    rid = C.c_uint64()
    _check(lib().pbit_server_submit(s, g, C.byref(params), C.byref(rid)))
    return rid.value


def pbit_server_poll(s, req_id, trials):
    """(status, cuts or None, latency seconds or None)."""
    cuts = np.zeros(int(trials), np.int64)
    lat = C.c_double()
    code = _check(lib().pbit_server_poll(s, int(req_id), cuts.ctypes.data_as(_P), C.byref(lat)))
    if code == PBIT_PENDING:
        return code, None, None
    return code, cuts, lat.value


def pbit_server_wait(s, req_id, trials, timeout_s=0.0):
    cuts = np.zeros(int(trials), np.int64)
    lat = C.c_double()
    code = _check(lib().pbit_server_wait(s, int(req_id), float(timeout_s), cuts.ctypes.data_as(_P), C.byref(lat)))
    if code == PBIT_PENDING:
        return code, None, None
    return code, cuts, lat.value


def pbit_server_stats(s) -> dict:
    st = pbit_server_stats_t()
    _check(lib().pbit_server_stats(s, C.byref(st)))
    return {k: getattr(st, k) for k, _ in st._fields_}


# ------------------------------------------------------------ convenience ---

class Batch:
    """Owning wrapper of a pbit_batch over Graph objects and per-instance keyword parameters."""

    def __init__(self, graphs, kwargs_list):
        self.graphs = list(graphs)
        self._keep = []
        params = []
        for kw in kwargs_list:
            p, keep = make_params(**kw)
            params.append(p)
            self._keep.append(keep)
        self.trials = [int(kw["trials"]) for kw in kwargs_list]
        self.handle = pbit_batch_create([g.handle for g in self.graphs], params)

    def run(self, chunk_steps=0, max_chunks=0, stream=None):
        pbit_batch_run(self.handle, chunk_steps, max_chunks, stream)

    def autotune(self, stream=None):
        return pbit_batch_autotune(self.handle, stream)

    def spins(self, k, stream=None):
        import torch
        out = torch.empty((self.graphs[k].n, self.trials[k]), dtype=torch.int8, device="cuda")
        pbit_batch_spins(self.handle, k, out, stream)
        return out

    def cuts(self, k, stream=None):
        return pbit_batch_cuts(self.handle, k, self.trials[k], stream)

    def progress(self, k):
        return pbit_batch_progress(self.handle, k)

    def close(self):
        if self.handle:
            pbit_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Graph:
    """Owning wrapper of a pbit_graph handle."""

    def __init__(self, n, src, dst, w, h=None, dense=False):
        self.handle = pbit_graph_create(n, src, dst, w, h, PBIT_GRAPH_DENSE if dense else 0)
        self.n = int(n)

    @classmethod
    def from_inputs(cls, g, dense=False):
        return cls(g.n, g.src, g.dst, g.w, dense=dense)

    def info(self):
        return pbit_graph_info(self.handle)

    def close(self):
        if self.handle:
            pbit_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def anneal(self, trials, steps, spins_in=None, out=None, **kw):
        import torch
        if out is None:
            out = torch.empty((self.n, trials), dtype=torch.int8, device="cuda")
        p, keep = make_params(trials, steps, **kw)
        pbit_anneal(self.handle, p, spins_in, out)
        del keep
        return out

    def cut(self, spins, stream=None):
        return pbit_cut(self.handle, spins, spins.shape[1], stream)

    def energy(self, spins, stream=None):
        return pbit_energy(self.handle, spins, spins.shape[1], stream)

    def fields(self, spins, stream=None):
        import torch
        out = torch.empty(spins.shape, dtype=torch.int32, device=spins.device)
        pbit_fields(self.handle, spins, spins.shape[1], out, stream)
        return out

    def fields_dense(self, spins, stream=None):
        import torch
        out = torch.empty(spins.shape, dtype=torch.int32, device=spins.device)
        pbit_fields_dense(self.handle, spins, spins.shape[1], out, stream)
        return out

    def status(self, stream=None):
        pbit_graph_status(self.handle, stream)

    def schedule(self, i0_min, i0_max, steps, normalize=True):
        return pbit_schedule(self.handle, i0_min, i0_max, 1 if normalize else 0, steps)
