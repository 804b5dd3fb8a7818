"""Variability sweeps run as one batch: the cut-versus-variability study of the Results section
(the paper's figures of mean cut and energy against the intensity, offset and timing spreads of
Eq. 7), on synthetic graphs.

Each grid point is one instance of the same graph with its own variability draw and its own
instance number; the whole grid runs through the batched persistent kernel, and each point's
result is exactly the plain `pbit_anneal` result of that point (same seeds and counters).
Optional per-point energy or cut traces come from `pbit_anneal_trace`.

    python -m paper_2601_14476_gb300.sweep --graph gnm800 --trials 64 --steps 1000
"""
from __future__ import annotations

import argparse
from dataclasses import asdict, dataclass

import numpy as np

from . import inputs, pbit


@dataclass(frozen=True)
class SweepPoint:
    """Spreads of the per-node device parameters (Eq. 7): intensity ~ N(1, s_intensity^2),
    offset ~ N(0, s_offset^2), update probability ~ clip(N(p_mean, s_p^2), 0, 1)."""
    s_intensity: float = 0.0
    s_offset: float = 0.0
    p_mean: float = 1.0
    s_p: float = 0.0

    @property
    def ideal(self) -> bool:
        return self.s_intensity == 0.0 and self.s_offset == 0.0 and self.p_mean >= 1.0 and self.s_p == 0.0


def point_variability(n: int, seed: int, pt: SweepPoint) -> dict | None:
    """The per-node parameters of one grid point (None for ideal p-bits)."""
    if pt.ideal:
        return None
    return inputs.variability(n, seed, s_intensity=pt.s_intensity, s_offset=pt.s_offset, p_mean=pt.p_mean,
                              s_p=pt.s_p)


def point_kwargs(graph: inputs.Graph, k: int, pt: SweepPoint, trials: int, steps: int, seed: int, c_min: float,
                 c_max: float, **extra) -> dict:
    """Anneal keyword arguments of grid point k (instance k, variability seed derived from seed and k)."""
    return dict(trials=trials, steps=steps, i0_min=c_min, i0_max=c_max, seed=seed, instance=k,
                variability=point_variability(graph.n, seed * 1000 + k, pt), **extra)


def variability_sweep(graph: inputs.Graph, points, trials: int, steps: int, seed: int = 1, c_min: float = 0.1,
                      c_max: float = 10.0, trace_every: int = 0, trace_what: int = 1, **extra) -> list[dict]:
    """Anneal every grid point of `points` on `graph` as one batch.

    Returns one record per point: the point, its per-trial final cuts, their mean and best, and,
    with trace_every > 0, the [ceil(steps / trace_every), trials] trace of cuts (trace_what = 1) or
    energies (0) from a separate traced anneal of the same point.
    """
    import torch

    points = list(points)
    G = pbit.Graph.from_inputs(graph)
    kws = [point_kwargs(graph, k, pt, trials, steps, seed, c_min, c_max, **extra) for k, pt in enumerate(points)]
    B = pbit.Batch([G] * len(points), kws)
    try:
        B.run()
        out = []
        for k, pt in enumerate(points):
            cuts = B.cuts(k)
            rec = {"point": pt, "cuts": cuts, "mean_cut": float(cuts.mean()), "best_cut": int(cuts.max())}
            if trace_every > 0:
                p, keep = pbit.make_params(**kws[k])
                spins = torch.empty((graph.n, trials), dtype=torch.int8, device="cuda")
                rows = -(-steps // trace_every)
                trace = torch.empty((rows, trials), dtype=torch.int64, device="cuda")
                pbit.pbit_anneal_trace(G.handle, p, None, spins, trace_every, trace_what, trace)
                torch.cuda.synchronize()
                rec["trace"] = trace.cpu().numpy()
            out.append(rec)
    finally:
        B.close()
    return out


def default_grid() -> list[SweepPoint]:
    """Ideal p-bits, each variability kind alone at 5 % and 10 %, and all three together."""
    grid = [SweepPoint()]
    for s in (0.05, 0.1):
        grid += [SweepPoint(s_intensity=s), SweepPoint(s_offset=s), SweepPoint(p_mean=1.0 - s, s_p=s / 2)]
    grid.append(SweepPoint(s_intensity=0.1, s_offset=0.1, p_mean=0.9, s_p=0.05))
    return grid


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--graph", default="gnm800", choices=["gnm800", "torus"])
    ap.add_argument("--trials", type=int, default=64)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--algorithm", default="psa", choices=["psa", "spsa", "tapsa"],
                    help="pSA, SpSA (stall probability 0.5) or TApSA (window 4) at every grid point")
    args = ap.parse_args(argv)
    g = (inputs.erdos_renyi_gnm(800, 19176, args.seed, "+1") if args.graph == "gnm800"
         else inputs.torus_2d(100, 200, args.seed, "pm1"))
    extra = {"algorithm": {"psa": pbit.ALG_PSA, "spsa": pbit.ALG_SPSA, "tapsa": pbit.ALG_TAPSA}[args.algorithm]}
    for rec in variability_sweep(g, default_grid(), args.trials, args.steps, seed=args.seed, **extra):
        print({**asdict(rec["point"]), "mean_cut": round(rec["mean_cut"], 2), "best_cut": rec["best_cut"]})


if __name__ == "__main__":
    main()
