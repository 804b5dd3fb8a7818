"""Seeded synthetic workloads shaped like the paper's MAX-CUT benchmarks.

This module only draws inputs: graphs (edge lists with MAX-CUT weights) and
per-node device-variability parameters.  It holds none of the annealing
arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it.

The paper evaluates on G-set graphs (Table "tb:graph": "random" graphs with
weights +1 and "toroidal" graphs with weights +-1, 800 to 20000 nodes).
Those files are not available here; these generators produce graphs with the
same node counts, edge counts, structure and weight alphabets:

* ``erdos_renyi_gnm``  uniform G(n, m) edge set ("random", e.g. G1: n=800,
  m=19176, w=+1);
* ``torus_2d``         2-D grid wrapped on both axes ("toroidal", e.g. G81:
  100 x 200, m=40000, w in {-1,+1});
* ``complete_pm1``     the complete graph with w in {-1,+1} (dense workload);
* ``rgg_knn``          random geometric graph: points uniform in the unit
  square, each linked to its k nearest neighbours (union of directed kNN).

Variability follows Eq. (7) of the paper: intensity ~ N(1, s_lambda^2),
offset ~ N(0, s_delta^2); timing is drawn as a per-node update probability
p ~ clip(N(p_mean, s_p^2), 0, 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    """An undirected MAX-CUT instance: edge list (src < dst) and int8 weights."""
    n: int
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(len(self.src))


def _weights(rng: np.random.Generator, m: int, kind: str) -> np.ndarray:
    if kind == "+1":
        return np.ones(m, np.int8)
    if kind == "pm1":
        return (rng.integers(0, 2, size=m, dtype=np.int8) * 2 - 1).astype(np.int8)
    raise ValueError(f"unknown weight alphabet {kind!r}")


def _pairs_from_index(n: int, idx: np.ndarray):
    """Map linear indices of the strict upper triangle (row-major) to (i, j)."""
    idx = idx.astype(np.int64)
    # row i starts at offset i*n - i*(i+1)/2; invert by the quadratic formula, then fix rounding
    b = 2 * n - 1
    i = np.floor((b - np.sqrt(np.maximum(b * b - 8.0 * idx, 0.0))) / 2.0).astype(np.int64)
    start = i * n - i * (i + 1) // 2
    over = start > idx
    while over.any():
        i[over] -= 1
        start = i * n - i * (i + 1) // 2
        over = start > idx
    nxt = (i + 1) * n - (i + 1) * (i + 2) // 2
    under = nxt <= idx
    while under.any():
        i[under] += 1
        start = i * n - i * (i + 1) // 2
        nxt = (i + 1) * n - (i + 1) * (i + 2) // 2
        under = nxt <= idx
    j = idx - start + i + 1
    return i.astype(np.int32), j.astype(np.int32)


def erdos_renyi_gnm(n: int, m: int, seed: int, weights: str = "+1") -> Graph:
    """G(n, m): exactly m distinct undirected edges chosen uniformly."""
    total = n * (n - 1) // 2
    if m > total:
        raise ValueError("too many edges")
    rng = np.random.default_rng([0x6E72, seed])
    chosen = np.empty(0, np.int64)
    while len(chosen) < m:
        draw = rng.integers(0, total, size=2 * (m - len(chosen)) + 16, dtype=np.int64)
        chosen = np.unique(np.concatenate([chosen, draw]))
    chosen = rng.permutation(chosen)[:m]
    chosen.sort()
    i, j = _pairs_from_index(n, chosen)
    return Graph(n, i, j, _weights(rng, m, weights), name=f"gnm_{n}_{m}", meta={"kind": "gnm", "seed": seed})


def torus_2d(rows: int, cols: int, seed: int, weights: str = "pm1") -> Graph:
    """rows x cols grid with wrap-around on both axes: n = rows*cols, m = 2n."""
    if rows < 3 or cols < 3:
        raise ValueError("torus needs at least 3 rows and 3 columns")
    rng = np.random.default_rng([0x7472, seed])
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    node = (r * cols + c).ravel()
    right = (r * cols + (c + 1) % cols).ravel()
    down = (((r + 1) % rows) * cols + c).ravel()
    a = np.concatenate([node, node])
    b = np.concatenate([right, down])
    src = np.minimum(a, b).astype(np.int32)
    dst = np.maximum(a, b).astype(np.int32)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    n = rows * cols
    return Graph(n, src, dst, _weights(rng, len(src), weights), name=f"torus_{rows}x{cols}",
                 meta={"kind": "torus", "seed": seed})


def complete_pm1(n: int, seed: int) -> Graph:
    """Complete graph K_n with weights uniform in {-1, +1}."""
    rng = np.random.default_rng([0x636F, seed])
    i, j = np.triu_indices(n, k=1)
    m = len(i)
    return Graph(n, i.astype(np.int32), j.astype(np.int32), _weights(rng, m, "pm1"), name=f"complete_{n}",
                 meta={"kind": "complete", "seed": seed})


def rgg_knn(n: int, seed: int, k: int = 3, weights: str = "pm1") -> Graph:
    """Random geometric graph: uniform points, each joined to its k nearest."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng([0x7267, seed])
    pts = rng.random((n, 2))
    _, nb = cKDTree(pts).query(pts, k=k + 1)
    a = np.repeat(np.arange(n), k)
    b = nb[:, 1:].reshape(-1)
    src = np.minimum(a, b)
    dst = np.maximum(a, b)
    key = np.unique(src.astype(np.int64) * n + dst)
    src = (key // n).astype(np.int32)
    dst = (key % n).astype(np.int32)
    return Graph(n, src, dst, _weights(rng, len(src), weights), name=f"rgg{k}_{n}",
                 meta={"kind": "rgg", "seed": seed})


def variability(n: int, seed: int, s_intensity: float = 0.1, s_offset: float = 0.1, p_mean: float = 0.9,
                s_p: float = 0.05) -> dict:
    """Per-node intensity, offset and update probability (Eq. 7, timing as p)."""
    rng = np.random.default_rng([0x7661, seed])
    return {
        "intensity": (1.0 + s_intensity * rng.standard_normal(n)).astype(np.float32),
        "offset": (s_offset * rng.standard_normal(n)).astype(np.float32),
        "p_update": np.clip(p_mean + s_p * rng.standard_normal(n), 0.0, 1.0).astype(np.float32),
    }


def timing_deviation(n: int, seed: int, s_nu: float = 0.1) -> np.ndarray:
    """Per-node deviation of the update period for the paper's timing model: nu_i ~ N(0, s_nu^2)."""
    rng = np.random.default_rng([0x6E75, seed])
    return (s_nu * rng.standard_normal(n)).astype(np.float32)


def random_spins(n: int, T: int, seed: int) -> np.ndarray:
    """Uniform +-1 trial-major spins, for tests that start from a given state."""
    rng = np.random.default_rng([0x7370, seed])
    return (rng.integers(0, 2, size=(n, T), dtype=np.int8) * 2 - 1).astype(np.int8)


# --------------------------------------------------------------------------
# The five benchmark workloads (sizes as the method's evaluation uses them)
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    graph: Graph
    trials: int
    steps: int
    c_min: float
    c_max: float
    var: dict | None
    seed: int
    instance: int = 0


def plain_er800(graph_seed: int = 1, anneal_seed: int = 1) -> Workload:
    """G(800, 19176), w=+1, 16 trials, 1000 steps, I0 0.1->10, ideal p-bits."""
    g = erdos_renyi_gnm(800, 19176, graph_seed, "+1")
    return Workload("gnm800_T16_S1000_ideal", g, 16, 1000, 0.1, 10.0, None, anneal_seed)


def dense_k2000(graph_seed: int = 1, anneal_seed: int = 1) -> Workload:
    """K_2000 with w in {-1,+1}, 256 trials, 2000 steps, I0 0.05->5, variability on."""
    g = complete_pm1(2000, graph_seed)
    return Workload("complete2000_T256_S2000_var", g, 256, 2000, 0.05, 5.0, variability(2000, graph_seed),
                    anneal_seed)


def sparse_torus20000(graph_seed: int = 1, anneal_seed: int = 1) -> Workload:
    """100x200 torus, w in {-1,+1}, 1024 trials, 5000 steps, I0 0.1->10, variability on."""
    g = torus_2d(100, 200, graph_seed, "pm1")
    return Workload("torus100x200_T1024_S5000_var", g, 1024, 5000, 0.1, 10.0, variability(g.n, graph_seed),
                    anneal_seed)


def batch64(seed: int = 1, count: int = 64, steps: int = 2000, n_lo: int = 800, n_hi: int = 10000):
    """64 uneven instances: N log-uniform, half G(n, 3n) w=+1, half 3-NN RGG w=+-1.

    Trials per instance cycle through {32, 64, 128, 256}; variability on.
    """
    rng = np.random.default_rng([0x6261, seed])
    out = []
    for k in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        gs = seed * 1000 + k + 1
        if k % 2 == 0:
            g = erdos_renyi_gnm(n, 3 * n, gs, "+1")
        else:
            g = rgg_knn(n, gs, 3, "pm1")
        T = (32, 64, 128, 256)[k % 4]
        out.append(Workload(f"batch{k}_{g.name}_T{T}", g, T, steps, 0.1, 10.0, variability(n, gs), seed, k))
    return out


def serving_request(req_id: int, seed: int = 1, n_lo: int = 800, n_hi: int = 20000, t_lo: int = 16,
                    t_hi: int = 256, s_lo: int = 1000, s_hi: int = 10000) -> Workload:
    """One solve request of the Poisson serving stream (request seed = id)."""
    rng = np.random.default_rng([0x7271, seed, req_id])
    n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
    gs = seed * 1_000_000 + req_id
    g = erdos_renyi_gnm(n, 3 * n, gs, "+1") if rng.integers(0, 2) == 0 else rgg_knn(n, gs, 3, "pm1")
    T = int(rng.integers(t_lo, t_hi + 1))
    S = int(rng.integers(s_lo, s_hi + 1))
    var = variability(n, gs) if rng.integers(0, 2) == 1 else None
    return Workload(f"req{req_id}_{g.name}_T{T}_S{S}", g, T, S, 0.1, 10.0, var, seed, req_id)


def serving_draw(req_id: int, seed: int = 1, t_lo: int = 16, t_hi: int = 256, s_lo: int = 1000,
                 s_hi: int = 10000):
    """Trials, steps and variability flag of one serving request (no graph)."""
    rng = np.random.default_rng([0x7264, seed, req_id])
    T = int(rng.integers(t_lo, t_hi + 1))
    S = int(rng.integers(s_lo, s_hi + 1))
    return T, S, bool(rng.integers(0, 2) == 1)


def poisson_arrivals(rate: float, duration_s: float, seed: int = 1) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng([0x706F, seed])
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        out.append(t)
    return np.asarray(out)
