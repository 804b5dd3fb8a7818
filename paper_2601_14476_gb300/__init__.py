"""GB300-native p-bit simulated annealing (pSA) with device variability.

The compute path is the C-ABI library ``libpbit.so`` (hand-written sm_103a
CUDA behind ``include/pbit.h``); :mod:`.pbit` is its thin ctypes binding,
:mod:`.inputs` draws seeded synthetic workloads and :mod:`.sweep` runs grids
of variability settings as one batch.  Importing the package loads nothing;
the library is loaded on first use and the binding raises if it is missing.

Example: anneal a 100 x 200 torus (1024 trials, 5000 steps, variability on)
and read the per-trial cuts::

    from paper_2601_14476_gb300 import inputs, pbit
    w = inputs.sparse_torus20000()
    G = pbit.Graph.from_inputs(w.graph)
    spins = G.anneal(w.trials, w.steps, i0_min=w.c_min, i0_max=w.c_max, seed=w.seed,
                     variability=w.var)          # torch int8 [n][T] on the GPU
    cuts = G.cut(spins)                          # numpy int64 [T]
"""
__all__ = ["inputs", "pbit", "sweep"]
