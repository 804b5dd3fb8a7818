"""Benchmark: spin-updates/s of the p-bit annealing hot path on GB300.

Default (``--config headline``): the uneven batch of 64 MAX-CUT instances
(n log-uniform in [800, 10000], half G(n, 3n) with w = +1, half 3-NN random
geometric graphs with w in {-1,+1}; 32/64/128/256 trials; 2000 steps;
variability on), one "step" being one complete batched anneal of all 64
instances followed by their exact cuts, on inputs already resident in HBM.
The same line carries the plain one-instance-per-launch form of the same
work on the same GPU (identical cuts), the oracle's whole-anneal mean cut of
the two smallest instances on the same seeds (the "equal mean cut" check),
the Poisson serving sweep (p50/p99 latency per arrival rate, saturation
rate) and two single-instance components with their own rooflines: the dense
K_2000 anneal on the tensor cores and the sparse 100x200 torus anneal.

Other workloads: --config dense | sparse | plain | batch | serve | sweep.
Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle as
the reference arm on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2601_14476_gb300 import inputs  # noqa: E402

L2_FLUSH_BYTES = 512 << 20

# DRAM bytes (read + write) per launch of each dominant kernel from one ncu capture, valid only while
# the kernel's sources hash to the recorded value; otherwise the bench reports traffic null.
TRAFFIC = {
    # one persistent launch: K_2000 +-1, 256 trials, 2000 steps, e4m3 kernel (forced; weights outside e2m1)
    "dense_persistent_kernel": {"bytes": 4828928 + 403456, "files": ["pbit_dense.cu", "pbit_device.cuh"],
                                "sha": "89e83f860105013d"},
    # one cluster-resident FP4 launch: K_2000 +-1, 256 trials, 2000 steps
    "dense4_cluster_kernel": {"bytes": 3026944 + 0, "files": ["pbit_dense4.cu", "pbit_device.cuh"],
                              "sha": "c0bd8b766236d721"},
    # one multi-step launch: 100x200 torus, 1024 trials, 5000 steps
    "sparse_flow_kernel": {"bytes": 25699840 + 608477696,
                           "files": ["pbit_tile.cuh", "pbit_flow.cu", "pbit_device.cuh"],
                           "sha": "44d9ecba49512c4c"},
    # per one-step launch of SpSA / TApSA (window 4) on the 100x200 torus, T = 1024
    "sparse_variant_words_kernel:spsa": {"bytes": 103571456 + 41346304,
                                         "files": ["pbit_variant.cu", "pbit_tile.cuh", "pbit_device.cuh"],
                                         "sha": "96ab07d6c8cac8ed"},
    "sparse_variant_words_kernel:tapsa": {"bytes": 144523264 + 35471531,
                                          "files": ["pbit_variant.cu", "pbit_tile.cuh", "pbit_device.cuh"],
                                          "sha": "96ab07d6c8cac8ed"},
    # per launch of a 64-step chunk of all 64 instances of the uneven batch
    "batch_chunk_kernel": {"bytes": 1474757376 + 2120900608, "files": ["pbit_tile.cuh", "pbit_batch.cu", "pbit_device.cuh"],
                           "sha": "189392b7e0472f25", "chunk_steps": 64},
}


def batch_traffic(tuning, steps: int):
    """DRAM bytes of one batched run, scaled from the capture of one 64-step chunk by the number of
    steps (the traffic is per step: the spin buffers' write-back and re-read), whatever chunk length
    the autotuner picked."""
    per_chunk = traffic_for("batch_chunk_kernel")
    chunk = TRAFFIC["batch_chunk_kernel"]["chunk_steps"]
    if per_chunk is None:
        return None
    return int(per_chunk * steps / chunk)


def sparse_tile_kernel(g, T: int, launches_per_anneal: float, steps: int) -> str:
    """Name of the sparse kernel the library launched: the multi-step kernel when an anneal took far
    fewer launches than steps, else the one-step kernel of the graph's tile form.

    Same rule as the library's tile choice: the warp-table tile needs unit weights and
    max degree + 1 lanes per node segment of min(32, T / G) lanes (G = 32 or 16).
    """
    if steps >= 2 and launches_per_anneal < steps / 2:
        return "sparse_flow_kernel"
    deg = int(np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n).max()) if g.m else 0
    if np.all(np.abs(g.w) == 1) and deg <= 15:
        for G in (32, 16):
            groups = T // G
            if T % G == 0 and (groups % 32 == 0 or 32 % groups == 0) and deg + 1 <= min(32, groups):
                return "sparse_warp_kernel"
    return "sparse_step_kernel"


def traffic_for(kernel):
    import hashlib
    t = TRAFFIC.get(kernel) if kernel else None
    if not t:
        return None
    m = hashlib.sha256()
    for f in t["files"]:
        with open(os.path.join(ROOT, "paper_2601_14476_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return t["bytes"] if t["bytes"] is not None and m.hexdigest()[:16] == t["sha"] else None


def workload(name: str):
    if name == "dense":
        return inputs.dense_k2000()
    if name == "sparse":
        return inputs.sparse_torus20000()
    if name == "plain":
        return inputs.plain_er800()
    raise SystemExit(f"unknown config {name}")


def variant_args(args, w) -> dict:
    """make_params keywords of the pSA variant / timing model selected on the command line (empty for
    plain pSA); the workload's name records the choice."""
    from paper_2601_14476_gb300 import pbit
    alg = {"psa": pbit.ALG_PSA, "spsa": pbit.ALG_SPSA, "tapsa": pbit.ALG_TAPSA}[args.algorithm]
    if alg == pbit.ALG_PSA and args.t_res <= 0:
        return {}
    if args.config not in ("sparse", "plain"):
        raise SystemExit("the pSA variants and the timing model run on the sparse configs")
    out = {"algorithm": alg, "stall_prob": args.stall_prob, "window": args.window}
    if alg != pbit.ALG_PSA:
        w.name += f"_{args.algorithm}" + (f"_w{args.window}" if alg == pbit.ALG_TAPSA else f"_p{args.stall_prob:g}")
    if args.t_res > 0:
        out["t_res"] = args.t_res
        out["nu_dev"] = inputs.timing_deviation(w.graph.n, w.seed, args.s_nu)
        w.name += f"_tres{args.t_res}_snu{args.s_nu:g}"
        w.updates = variant_work(out, w.graph, w.trials, w.steps * args.t_res)[0]
    return out


def variant_work(variant: dict, g, T: int, Q: int):
    """(spin updates, algorithmic bytes) of the first Q (sub-)steps of a variant on graph g with T trials.

    An update of node i reads deg_i neighbour bytes and its own, writes one, and carries its state
    (SpSA: the float32 input read and written, 8 B; TApSA: window - 1 int16 fields read, one written,
    2 window B).  Timing model (period nu_i = max(1, round(t_res (1 + nu_dev_i)))): node i updates at
    the sub-steps q % nu_i == 0 only and an idle node costs nothing (the parity form copies no spins
    between sub-steps; its two placement passes per call are not counted)."""
    from paper_2601_14476_gb300 import pbit
    alg = variant.get("algorithm", pbit.ALG_PSA)
    state = 8 if alg == pbit.ALG_SPSA else (2 * variant.get("window", 4) if alg == pbit.ALG_TAPSA else 0)
    deg = (np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)).astype(np.int64)
    t_res = variant.get("t_res", 0)
    if t_res <= 0:
        return g.n * T * Q, T * Q * float(deg.sum() + g.n * (2 + state))
    dev = np.zeros(g.n) if variant.get("nu_dev") is None else np.asarray(variant["nu_dev"], np.float32)
    nu = np.maximum(1, np.floor(t_res * (1.0 + dev.astype(np.float64)) + 0.5)).astype(np.int64)
    due = (Q + nu - 1) // nu
    return T * int(due.sum()), T * float((due * (deg + 2 + state)).sum())


def traffic_key(kname: str, variant: dict):
    """TRAFFIC entry of a launch: per kernel; the variants' one-step launches per algorithm (the timing
    model's launches vary in size with the due nodes, so they have none)."""
    if not variant:
        return kname
    if variant.get("t_res", 0) > 0 or variant.get("algorithm", 0) not in (1, 2) or variant.get("window", 4) != 4:
        return None
    return f"{kname}:{'spsa' if variant['algorithm'] == 1 else 'tapsa'}"


def workload_config(w) -> dict:
    """The keys that name a single-instance workload, shared by both bench arms."""
    g = w.graph
    return {"workload": w.name, "n": g.n, "edges": g.m, "trials": w.trials, "anneal_steps": w.steps,
            "variability": w.var is not None, "updates_per_step": getattr(w, "updates", g.n * w.trials * w.steps)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "source": "measured"}
    except Exception:  # noqa: BLE001
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
                "source": "fallback"}


# ----------------------------------------------------------------- clocks ----

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        # raw samples: PBIT_BENCH_OUT if set, else the system temporary directory
        import tempfile
        out_dir = os.environ.get("PBIT_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{device_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)  # let the sampler start before the timed region
        except Exception:  # noqa: BLE001
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        busy = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle ----

_ORACLE_CASE = {}


def _oracle_sample(job):
    """One process's copy of the oracle sample: (workload kind, k steps) -> seconds for the k steps."""
    import oracle
    kind, k = job
    if _ORACLE_CASE.get("kind") != kind:
        w = multi_reference_workload(kind) if kind in ("batch", "sweep", "headline") else workload(kind)
        g = w.graph
        csr = oracle.Csr(g.n, g.src, g.dst, g.w)
        _ORACLE_CASE.update(kind=kind, w=w, csr=csr, tab=oracle.schedule(csr, w.c_min, w.c_max, w.steps),
                            s0=oracle.init_spins(g.n, w.trials, w.seed, w.instance))
    c = _ORACLE_CASE
    w = c["w"]
    t0 = time.perf_counter()
    oracle.anneal(c["csr"], c["s0"], c["tab"], w.seed, w.instance, variability=w.var, step_end=k)
    return time.perf_counter() - t0


def cpu_baseline(w, budget_s: float = 12.0, kind: str | None = None, all_cores: bool = True, variant=None):
    """Time the oracle (single-threaded FP64) on a bounded sample: all trials, first k schedule steps.

    With all_cores, every host core also runs its own copy of the same sample at once (spawned
    processes, the oracle as it stands): the aggregate rate is all their updates over the wall time.
    """
    import oracle
    g = w.graph
    csr = oracle.Csr(g.n, g.src, g.dst, g.w)
    tab = oracle.schedule(csr, w.c_min, w.c_max, w.steps)
    s0 = oracle.init_spins(g.n, w.trials, w.seed, w.instance)
    v = dict(variant or {})

    def run(k):  # the first k (sub-)steps
        if v:
            oracle.anneal_variant(csr, s0, tab, w.seed, w.instance, algorithm=v.get("algorithm", 0),
                                  stall_prob=v.get("stall_prob", 0.5), window=v.get("window", 4),
                                  t_res=v.get("t_res", 0), nu_dev=v.get("nu_dev"), variability=w.var, q_end=k)
        else:
            oracle.anneal(csr, s0, tab, w.seed, w.instance, variability=w.var, step_end=k)

    total = w.steps * max(1, v.get("t_res", 0))
    t0 = time.perf_counter()
    run(1)
    one = max(time.perf_counter() - t0, 1e-6)
    k = int(max(1, min(total, budget_s / one)))
    t0 = time.perf_counter()
    run(k)
    dt = time.perf_counter() - t0
    upd = variant_work(v, g, w.trials, k)[0] if v else g.n * w.trials * k
    out = {"value": upd / dt, "unit": "spin-updates/s", "cores": 1, "kind": "oracle",
           "sample": f"{w.name}: all {w.trials} trials, (sub-)steps [0,{k}) of {total} "
                     f"({upd:.3g} updates, {dt:.1f} s)"}
    ncores = os.cpu_count() or 1
    if all_cores and kind and ncores > 1 and not v:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(ncores) as pool:
            pool.map(_oracle_sample, [(kind, 1)] * ncores)  # build each process's case, warm up
            t0 = time.perf_counter()
            pool.map(_oracle_sample, [(kind, k)] * ncores)
            wall = time.perf_counter() - t0
        out["all_cores"] = {"value": ncores * upd / wall, "unit": "spin-updates/s", "cores": ncores,
                            "sample": f"each of {ncores} processes runs the same sample at once ({wall:.1f} s wall)"}
    return out


def run_reference(args, w, variant=None, config=None):
    """The reference arm: the oracle as it stands, each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t_all = []
    base = None
    for it in range(args.warmup + args.steps):
        b = cpu_baseline(w, budget_s=max(2.0, 60.0 / max(1, args.steps + args.warmup)), variant=variant)
        if it >= args.warmup:
            t_all.append(b["value"])
            base = b
    val = float(np.mean(t_all))
    upd_run = (config or {}).get("updates_per_step") or getattr(w, "updates", w.graph.n * w.trials * w.steps)
    line = {"impl": "reference", "metric": "spin-updates/s", "value": val, "unit": "spin-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * upd_run / val, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config or workload_config(w),
            "cpu_baseline": {**base, "value": val},
            "e2e": {"value": val, "unit": "spin-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- plumbing ----

def _dist_setup():
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local, dist


def _max_over_ranks(dist, x, device="cuda"):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(dist, units_per_rank: float, ms_local: float, world: int, device="cuda"):
    """Whole-job rate: all ranks' units (each rank runs the same per-rank work: weak scaling)
    divided by the slowest rank's time.  Returns (value per second, max ms)."""
    ms = _max_over_ranks(dist, ms_local, device)
    return world * units_per_rank / (ms * 1e-3), ms


def sweep_workloads(seed: int = 1, steps: int = 1000):
    """The variability sweep of the Results section on the G81-shaped 100x200 torus (w in {-1,+1}),
    128 trials: one instance per point of the default grid (its own variability draw and instance
    number), all run as one batch."""
    from paper_2601_14476_gb300 import sweep
    g = inputs.torus_2d(100, 200, seed, "pm1")
    return [inputs.Workload(f"sweep_point{k}_torus100x200_T128_S{steps}", g, 128, steps, 0.1, 10.0,
                            sweep.point_variability(g.n, seed * 1000 + k, pt), seed, k)
            for k, pt in enumerate(sweep.default_grid())]


def multi_reference_workload(config: str):
    """The single instance the oracle times for the multi-instance configs: the first batch instance
    (batch, headline, serve: requests come from the same generators) or the sweep point with all three
    spreads."""
    return sweep_workloads()[-1] if config == "sweep" else inputs.batch64(count=1)[0]


def batch_config(ws, wname):
    """The keys that name the batched workload, shared by both bench arms."""
    return {"workload": wname, "instances": len(ws),
            "n_range": [min(w.graph.n for w in ws), max(w.graph.n for w in ws)],
            "trials": sorted(set(w.trials for w in ws)), "anneal_steps": ws[0].steps, "variability": True,
            "updates_per_step": sum(w.graph.n * w.trials * w.steps for w in ws)}


# ------------------------------------------------------ oracle mean cut ----

def oracle_mean_cut_check(ws, gpu_cuts, count: int = 2):
    """The "equal mean cut" condition: the oracle anneals every trial of the `count` smallest
    instances (by n*T) on the same seeds and counters; their mean cut must be within 0.5 % of the
    GPU's mean cut over the same trials.  Trials whose cuts differ are those where a float32/FP64
    tie-band decision sent the trial down another path."""
    order = sorted(range(len(ws)), key=lambda k: ws[k].graph.n * ws[k].trials)[:count]
    jobs = [dict(n=ws[k].graph.n, src=ws[k].graph.src, dst=ws[k].graph.dst, w=ws[k].graph.w, trials=ws[k].trials,
                 steps=ws[k].steps, c_min=ws[k].c_min, c_max=ws[k].c_max, seed=ws[k].seed,
                 instance=ws[k].instance, var=ws[k].var) for k in order]
    import multiprocessing as mp

    import oracle
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        ref = pool.map(oracle.anneal_cuts, jobs)
    secs = time.perf_counter() - t0
    gpu = [np.asarray(gpu_cuts[k])[:len(r)] for k, r in zip(order, ref)]
    mg = float(np.mean(np.concatenate(gpu)))
    mo = float(np.mean(np.concatenate(ref)))
    rel = abs(mg - mo) / max(1.0, abs(mo))
    return {"instances": [ws[k].name for k in order], "trials": [len(r) for r in ref],
            "mean_cut_gpu": mg, "mean_cut_oracle": mo, "rel_diff": rel, "within_0p5pct": bool(rel <= 0.005),
            "trials_identical": float(np.mean(np.concatenate([a == b for a, b in zip(gpu, ref)]))),
            "oracle_seconds": secs}


# ------------------------------------------------------ single instance ----

def run_single(args, w, variant, kernel, dense, steps, warmup, e2e_reps, dist, world, local):
    """Time whole anneals (+ exact cuts) of one instance: device time with CUDA events on the launching
    stream, L2 flushed between timed anneals; the dominant kernel's roofline; the same anneal end to end
    through the C ABI from host buffers."""
    import torch
    from paper_2601_14476_gb300 import pbit
    g = w.graph
    G = pbit.Graph.from_inputs(g, dense=dense)
    T, S = w.trials, w.steps
    stream = torch.cuda.current_stream()
    spins = torch.empty((g.n, T), dtype=torch.int8, device="cuda")
    cuts = torch.empty(T, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    params, keep = pbit.make_params(T, S, i0_min=w.c_min, i0_max=w.c_max, seed=w.seed, instance=w.instance,
                                    kernel=kernel, variability=w.var, stream=stream, **variant)
    sub = max(1, variant.get("t_res", 0))  # updates per cycle and node-trial (timing model: sub-steps)

    def one_run():
        pbit.pbit_anneal(G.handle, params, None, spins)
        pbit.pbit_cut_device(G.handle, spins, T, cuts, stream)

    for _ in range(warmup):
        one_run()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = pbit.pbit_launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()                     # L2 flushed between timed steps (not timed)
            a.record(stream)
            one_run()
            b.record(stream)
        torch.cuda.synchronize()
    launches = pbit.pbit_launch_count() - launches0
    ms = [a.elapsed_time(b) for a, b in ev]
    upd_run = getattr(w, "updates", g.n * T * S)  # the timing model counts the updates of due nodes only
    value, ms_step = job_throughput(dist, upd_run, float(np.mean(ms)), world)

    # dominant kernel: the anneal itself (one persistent launch for the dense path and the multi-step
    # sparse form, one launch per step otherwise); its average launch duration from CUDA events on the
    # launching stream
    chosen = pbit.pbit_select_kernel(G.handle, kernel, T)
    ka, kb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    l0 = pbit.pbit_launch_count()
    ka.record(stream)
    pbit.pbit_anneal(G.handle, params, None, spins)
    kb.record(stream)
    torch.cuda.synchronize()
    G.status()
    anneal_ms = ka.elapsed_time(kb)
    anneal_launches = pbit.pbit_launch_count() - l0
    pk = peaks()
    if chosen == pbit.KERNEL_DENSE:
        # 2 n^2 T flops per step (algorithmic, unpadded); the anneal is one kernel timed alone, so the
        # peak is the burst one, scaled from the measured bf16 burst peak by the nominal dense ratio of
        # the contraction's own type: packed e2m1 (FP4) 6x for the cluster-resident kernel, e4m3 2x
        fp4 = (G.info()["has_dense_fp4"] == 1 and T % 16 == 0 and not os.environ.get("PBIT_DENSE_E4M3"))
        flops = 2.0 * g.n * g.n * T * S
        achieved = flops / (anneal_ms * 1e-3) / 1e12
        ratio, kname = (6.0, "dense4_cluster_kernel") if fp4 else (2.0, "dense_persistent_kernel")
        peak = ratio * pk["bf16_tflops"]
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic_for(kname),
                    "kernel": kname,
                    "peak_source": f"{pk['source']} bf16 burst x{ratio:g} ({'e2m1' if fp4 else 'e4m3'} nominal ratio)",
                    "per_launch": "2*n^2*T*S flops over one launch (includes the spin layout kernel)"}
    else:
        kname = sparse_tile_kernel(g, T, anneal_launches, S) if chosen == pbit.KERNEL_SPARSE else "resident_kernel"
        if variant:
            kname = "sparse_variant_words_kernel" if T % 128 == 0 else "sparse_variant_kernel"
        launches_main = S if kname in ("sparse_warp_kernel", "sparse_step_kernel") else 1
        if variant:
            launches_main = anneal_launches
        per_launch_ms = anneal_ms / launches_main
        mean_deg = 2.0 * g.m / g.n
        # algorithmic bytes per spin-update of the sparse gather: deg neighbour bytes + own + write
        # (variants: plus their carried state and the timing model's copies, see variant_work)
        if variant:
            alg_bytes = variant_work(variant, g, T, S * sub)[1] / launches_main
        else:
            alg_bytes = g.n * T * (mean_deg + 2.0) * (S / launches_main)
        achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"],
                    "traffic": traffic_for(traffic_key(kname, variant)) if g.n == 20000 and T == 1024 else None,
                    "kernel": kname, "peak_source": pk["source"],
                    "per_launch": (f"variant bytes of the whole run (deg+2+state per update) / "
                                   f"{launches_main} launches" if variant else
                                   f"(deg+2) bytes x n*T updates per step; {launches_main} launches"),
                    "note": "algorithmic gather bytes; the spin buffers largely stay in L2 (DRAM bytes in traffic)"}
    roofline["kernel_ms_per_anneal"] = anneal_ms

    # end to end through the C ABI from host buffers: graph upload, anneal, cut to host
    e2e_ms = []
    h2d = g.m * (4 + 4 + 1) + (3 * g.n * 4 if w.var else 0) + S * 4 + (4 * g.n if "nu_dev" in variant else 0)
    d2h = T * 8
    host_cuts = None
    for it in range(0 if args.no_e2e else 1 + e2e_reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = pbit.Graph.from_inputs(g, dense=dense)
        out = torch.empty((g.n, T), dtype=torch.int8, device="cuda")
        p2, keep2 = pbit.make_params(T, S, i0_min=w.c_min, i0_max=w.c_max, seed=w.seed, instance=w.instance,
                                     kernel=kernel, variability=w.var, stream=stream, **variant)
        pbit.pbit_anneal(G2.handle, p2, None, out)
        host_cuts = pbit.pbit_cut(G2.handle, out, T, stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        G2.close()
        if it >= 1:
            e2e_ms.append(dt * 1e3)
    e2e_val = world * upd_run / (np.mean(e2e_ms) * 1e-3) if e2e_ms else None
    if host_cuts is None:
        host_cuts = cuts.cpu().numpy()
    return {"value": value, "ms_per_anneal": ms_step, "roofline": roofline,
            "kernel": {0: "auto", 1: "sparse", 2: "dense", 3: "resident"}[chosen],
            "mean_cut": float(host_cuts.mean()), "launches": int(launches),
            "e2e": {"value": e2e_val, "unit": "spin-updates/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "clocks": clk.summary(), "updates_per_anneal": upd_run}


# ---------------------------------------------------------------- batch ----

def batch_variant_kw(args, w) -> dict:
    """make_params keywords of the pSA variant / timing model chosen on the command line for one batch
    instance (empty for plain pSA)."""
    from paper_2601_14476_gb300 import pbit
    alg = {"psa": pbit.ALG_PSA, "spsa": pbit.ALG_SPSA, "tapsa": pbit.ALG_TAPSA}[args.algorithm]
    if alg == pbit.ALG_PSA and args.t_res <= 0:
        return {}
    out = {"algorithm": alg, "stall_prob": args.stall_prob, "window": args.window}
    if args.t_res > 0:
        out["t_res"] = args.t_res
        out["nu_dev"] = inputs.timing_deviation(w.graph.n, w.seed * 1000 + w.instance, args.s_nu)
    return out


def run_batch(args, ws, Gs, wname, dist, world, local):
    """The batched persistent form (timed `args.steps` times) against the plain one-instance-per-launch
    form of the same work on the same GPU; results must be identical per trial.  With a pSA variant
    chosen, every instance runs it, and the batched form is also timed with the variants kept in the
    group tile (the word tile's gain)."""
    import torch
    from paper_2601_14476_gb300 import pbit
    pk = peaks()
    stream = torch.cuda.current_stream()
    vkw = [batch_variant_kw(args, w) for w in ws]
    kws = [dict(trials=w.trials, steps=w.steps, seed=w.seed, instance=w.instance, variability=w.var,
                i0_min=w.c_min, i0_max=w.c_max, **v) for w, v in zip(ws, vkw)]
    work = [variant_work(v, w.graph, w.trials, w.steps * max(1, v.get("t_res", 0))) if v else
            (w.graph.n * w.trials * w.steps, w.graph.n * w.trials * w.steps * (2.0 * w.graph.m / w.graph.n + 2.0))
            for w, v in zip(ws, vkw)]
    upd_run = sum(x[0] for x in work)
    bytes_run = sum(x[1] for x in work)
    B0 = pbit.Batch(Gs, kws)
    tuning = B0.autotune(stream)
    B0.close()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def batched_run():
        B = pbit.Batch(Gs, kws)
        pbit.pbit_batch_set_tuning(B.handle, tuning["chunk_steps"], tuning["ctas_per_sm"])
        return B

    for _ in range(args.warmup):
        B = batched_run()
        B.run(stream=stream)
        torch.cuda.synchronize()
        B.close()
    if dist:
        dist.barrier()
    times = []
    launches = 0                       # kernels launched inside the timed regions only
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            B = batched_run()          # instance setup is outside the timed region
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = pbit.pbit_launch_count()
            a.record(stream)
            B.run(stream=stream)
            b.record(stream)
            launches += pbit.pbit_launch_count() - l0
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
            batched_cuts = [B.cuts(k) for k in range(len(ws))]
            B.close()
    value, ms = job_throughput(dist, upd_run, float(np.mean(times)), world)
    # plain form: one instance after another through pbit_anneal (AUTO: the cluster-resident kernel for
    # the small instances, the sparse path otherwise); one untimed pass builds the per-graph tables
    outs = [torch.empty((w.graph.n, w.trials), dtype=torch.int8, device="cuda") for w in ws]
    plist = [pbit.make_params(stream=stream, **kw) for kw in kws]
    plain_ms_all = []
    for it in range(1 + max(1, args.plain_reps)):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for G, o, (p, keep) in zip(Gs, outs, plist):
            pbit.pbit_anneal(G.handle, p, None, o)
        b.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            plain_ms_all.append(a.elapsed_time(b))
    plain_value, plain_ms = job_throughput(dist, upd_run, float(np.mean(plain_ms_all)), world)
    plain_cuts = [G.cut(o) for G, o in zip(Gs, outs)]
    same = all(np.array_equal(x, y) for x, y in zip(batched_cuts, plain_cuts))
    group = None
    if any(vkw):
        # the same batch with the variants kept in the group tile (the switch is read at instance setup)
        os.environ["PBIT_BATCH_GROUP_TILE"] = "1"
        try:
            gms = []
            for it in range(1 + max(1, args.plain_reps)):
                B = batched_run()
                flush.zero_()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                B.run(stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if it >= 1:
                    gms.append(a.elapsed_time(b))
                gcuts = [B.cuts(k) for k in range(len(ws))]
                B.close()
        finally:
            os.environ.pop("PBIT_BATCH_GROUP_TILE", None)
        group = {"group_tile_ms": float(np.mean(gms)), "word_tile_over_group_tile": float(np.mean(gms)) / ms,
                 "cuts_identical": all(np.array_equal(x, y) for x, y in zip(batched_cuts, gcuts))}
    # end to end: graphs from host arrays, batch setup, run, cuts back to host
    e2e = []
    for it in range(0 if args.no_e2e else 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = ([pbit.Graph.from_inputs(w.graph) for w in ws] if wname.startswith("batch")
              else [pbit.Graph.from_inputs(ws[0].graph)] * len(ws))
        B2 = pbit.Batch(G2, kws)
        pbit.pbit_batch_set_tuning(B2.handle, tuning["chunk_steps"], tuning["ctas_per_sm"])
        B2.run(stream=stream)
        host_cuts = [B2.cuts(k) for k in range(len(ws))]
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
        B2.close()
        for G in set(G2):
            G.close()
    one_graph = not wname.startswith("batch")
    h2d = sum((w.graph.m * 9 if (not one_graph or k == 0) else 0) + (12 * w.graph.n if w.var else 0)
              + 4 * w.steps for k, w in enumerate(ws))
    d2h = sum(8 * w.trials for w in ws)
    achieved = bytes_run / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"],
                "traffic": batch_traffic(tuning, ws[0].steps) if wname.startswith("batch") and not any(vkw) else None,
                "kernel": "batch_chunk_kernel", "peak_source": pk["source"],
                "per_launch": "sum over instances of (deg+2) bytes x n*T updates per step, over the "
                              "batched run's chunk launches",
                "note": "algorithmic gather bytes; DRAM bytes of the whole run in traffic"}
    return {"value": value, "ms": ms, "upd_run": upd_run, "tuning": tuning, "plain_value": plain_value,
            "plain_ms": plain_ms, "batched_over_plain": plain_ms / ms, "cuts_identical_to_plain": bool(same),
            "mean_cut_batched": float(np.mean([c.mean() for c in batched_cuts])),
            "mean_cut_plain": float(np.mean([c.mean() for c in plain_cuts])),
            "batched_cuts": batched_cuts, "roofline": roofline, "launches": int(launches), "group_tile": group,
            "e2e": {"value": world * upd_run / float(np.mean(e2e)) if e2e else None, "unit": "spin-updates/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "clocks": clk.summary()}


# ---------------------------------------------------------------- serve ----

def run_serve(args, rank, local):
    """Poisson request streams through the continuous-batching server, one per arrival rate: p50/p99
    latency from submission to result, and the aggregate spin-updates/s."""
    from paper_2601_14476_gb300 import pbit
    rates = [float(r) for r in args.serve_rates.split(",")]
    # a pool of request graphs (n log-uniform in [800, 20000], G(n,3n) w=+1 or 3-NN RGG w=+-1) built
    # before the sweep; every request draws its own trials, steps, variability and seed
    pool = []
    for r in range(48):
        w = inputs.serving_request(r, seed=1 + rank)
        pool.append((pbit.Graph.from_inputs(w.graph), w, inputs.variability(w.graph.n, r)))
    sweep = []
    total_upd, total_wall = 0.0, 0.0
    launches0 = pbit.pbit_launch_count()
    with ClockSampler(local) as clk:
        for ri, rate in enumerate(rates):
            arrivals = inputs.poisson_arrivals(rate, args.serve_seconds, seed=100 + ri + 1000 * rank)
            srv = pbit.pbit_server_create(64 << 30, 64, 64)
            pending = {}
            t_start = time.perf_counter()
            upd = 0.0
            for k, t_arr in enumerate(arrivals):
                now = time.perf_counter() - t_start
                if t_arr > now:
                    time.sleep(t_arr - now)
                T, S, with_var = inputs.serving_draw(k, seed=7 + ri)
                G, w, var = pool[k % len(pool)]
                p, keep = pbit.make_params(T, S, seed=k + 1, instance=k, variability=var if with_var else None)
                t_sub = time.perf_counter()
                rid = pbit.pbit_server_submit(srv, G.handle, p)
                pending[rid] = (T, w.graph.n * T * S, keep, t_sub)
            # drain for up to serve_drain s; a request still unfinished then counts with its age so far as a
            # lower bound of its latency (censored)
            lat, censored = [], 0
            deadline = time.perf_counter() + args.serve_drain
            for rid, (T, u, keep, t_sub) in list(pending.items()):
                left = deadline - time.perf_counter()
                code = pbit.PBIT_PENDING
                if left > 0:
                    code, cuts, l = pbit.pbit_server_wait(srv, rid, T, timeout_s=left)
                if code == pbit.PBIT_OK:
                    lat.append(l)
                    upd += u
                else:
                    lat.append(time.perf_counter() - t_sub)
                    censored += 1
            wall = time.perf_counter() - t_start
            st = pbit.pbit_server_stats(srv)
            pbit.pbit_server_destroy(srv)
            total_upd += upd
            total_wall += wall
            sweep.append({"rate": rate, "submitted": len(arrivals), "completed": len(arrivals) - censored,
                          "censored": censored,
                          "p50_s": float(np.percentile(lat, 50)) if lat else None,
                          "p99_s": float(np.percentile(lat, 99)) if lat else None,
                          "updates_per_s": upd / wall, "peak_resident": st["peak_resident"]})
    launches = pbit.pbit_launch_count() - launches0
    for G, _, _ in pool:
        G.close()
    return {"rates": rates, "window_s": args.serve_seconds, "drain_s": args.serve_drain, "sweep": sweep,
            "saturation_updates_per_s": max(x["updates_per_s"] for x in sweep),
            "aggregate_updates_per_s": total_upd / total_wall, "request_pool": len(pool),
            "budget_bytes": 64 << 30, "max_slots": 64, "chunk_steps": 64,
            "latency": "submit to result; unfinished after the drain enter with their age (censored)",
            "launches": int(launches), "clocks": clk.summary()}


# ------------------------------------------------------------- headline ----

def bench_headline(args):
    """The headline line: batched spin-updates/s on the uneven 64-instance batch, beside the plain form,
    the oracle's mean cut, the serving sweep and the dense / sparse single-instance components."""
    import torch
    from paper_2601_14476_gb300 import pbit
    rank, world, local, dist = _dist_setup()
    ws = inputs.batch64(seed=1 + rank, steps=args.anneal_steps or 2000)
    Gs = [pbit.Graph.from_inputs(w.graph) for w in ws]
    wname = f"batch64_uneven_S{ws[0].steps}"
    b = run_batch(args, ws, Gs, wname, dist, world, local)
    components = {}
    if not args.no_components:
        for name in ("dense", "sparse"):
            w = workload(name)
            w.instance = rank
            r = run_single(args, w, {}, pbit.KERNEL_AUTO, name == "dense", steps=max(3, min(args.steps, 5)),
                           warmup=3, e2e_reps=1, dist=dist, world=world, local=local)
            components[name] = {"workload": w.name, "n": w.graph.n, "edges": w.graph.m, "trials": w.trials,
                                "anneal_steps": w.steps, "value": r["value"], "unit": "spin-updates/s",
                                "ms_per_anneal": r["ms_per_anneal"], "kernel": r["kernel"],
                                "kernel_ms_per_anneal": r["roofline"]["kernel_ms_per_anneal"],
                                "roofline": r["roofline"], "e2e": r["e2e"], "mean_cut": r["mean_cut"],
                                "clocks": r["clocks"]}
    serve = run_serve(args, rank, local) if not args.no_serve else None
    if serve:
        serve["served_over_plain"] = serve["saturation_updates_per_s"] / (b["plain_value"] / world)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    check = None if args.no_oracle_check else oracle_mean_cut_check(ws, b["batched_cuts"])
    cb = None
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_baseline(multi_reference_workload("batch"), kind="headline")
    cfg = batch_config(ws, wname)
    cfg.update({"l2": "flushed between timed steps", "tuning": b["tuning"],
                "plain_value": b["plain_value"], "plain_ms": b["plain_ms"],
                "plain_form": "each instance in turn through pbit_anneal (AUTO kernel)",
                "batched_over_plain": b["batched_over_plain"], "cuts_identical_to_plain": b["cuts_identical_to_plain"],
                "mean_cut_batched": b["mean_cut_batched"], "mean_cut_plain": b["mean_cut_plain"],
                "oracle_mean_cut": check, "serve": serve, "components": components})
    line = {
        "metric": "spin-updates/s", "value": b["value"], "unit": "spin-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i8/f32", "data": "synthetic", "config": cfg,
        "roofline": b["roofline"], "cpu_baseline": cb, "e2e": b["e2e"], "gpu_launches": b["launches"],
        "clocks": b["clocks"],
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------- other configurations ----

def bench_multi(args):
    """config batch / sweep: the batched persistent form vs the plain form; config serve: the Poisson
    serving sweep alone."""
    import torch  # noqa: F401
    from paper_2601_14476_gb300 import pbit
    rank, world, local, dist = _dist_setup()
    if args.config in ("batch", "sweep"):
        if args.config == "batch":
            ws = inputs.batch64(seed=1 + rank, steps=args.anneal_steps or 2000)
            Gs = [pbit.Graph.from_inputs(w.graph) for w in ws]
            wname = f"batch64_uneven_S{ws[0].steps}"
        else:
            ws = sweep_workloads(seed=1 + rank, steps=args.anneal_steps or 1000)
            Gs = [pbit.Graph.from_inputs(ws[0].graph)] * len(ws)
            wname = f"sweep{len(ws)}_torus100x200_T128_S{ws[0].steps}"
        b = run_batch(args, ws, Gs, wname, dist, world, local)
        if rank == 0:
            cfg = batch_config(ws, wname)
            cfg.update({"tuning": b["tuning"], "l2": "flushed between timed steps", "plain_value": b["plain_value"],
                        "plain_ms": b["plain_ms"], "batched_over_plain": b["batched_over_plain"],
                        "cuts_identical_to_plain": b["cuts_identical_to_plain"],
                        "mean_cut_batched": b["mean_cut_batched"], "mean_cut_plain": b["mean_cut_plain"],
                        "variant": {k: v for k, v in batch_variant_kw(args, ws[0]).items() if k != "nu_dev"} or None,
                        "group_tile": b["group_tile"]})
            line = {"metric": "spin-updates/s", "value": b["value"], "unit": "spin-updates/s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms"], "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "i8/f32", "data": "synthetic", "config": cfg,
                    "roofline": b["roofline"], "cpu_baseline": None, "e2e": b["e2e"],
                    "gpu_launches": b["launches"], "clocks": b["clocks"]}
            if world == 1 and not args.no_cpu_baseline:
                line["cpu_baseline"] = cpu_baseline(multi_reference_workload(args.config), kind=args.config)
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    serve = run_serve(args, rank, local)
    if rank == 0:
        line = {"metric": "spin-updates/s", "value": world * serve["aggregate_updates_per_s"], "unit": "spin-updates/s",
                "n_gpus": world, "steps": len(serve["rates"]), "warmup": args.warmup,
                "ms_per_step": 1e3 * args.serve_seconds, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "i8/f32", "data": "synthetic",
                "config": {"workload": "poisson_serving", **{k: v for k, v in serve.items() if k != "clocks"},
                           "l2": "inputs larger than L2 in aggregate"},
                "roofline": None, "cpu_baseline": None,
                "e2e": {"value": world * serve["aggregate_updates_per_s"], "unit": "spin-updates/s",
                        "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
                "gpu_launches": serve["launches"], "clocks": serve["clocks"]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def bench_one(args):
    """A single-instance workload (dense, sparse, plain; optionally a pSA variant)."""
    from paper_2601_14476_gb300 import pbit
    w = workload(args.config)
    if args.anneal_steps > 0:
        w.steps = args.anneal_steps
        w.name += f"_first{args.anneal_steps}steps"
    variant = variant_args(args, w)
    if args.impl == "reference":
        return run_reference(args, w, variant)
    rank, world, local, dist = _dist_setup()
    # each rank anneals its own instance of the workload (weak scaling, no data-path collective)
    w.instance = rank
    kernel = {"auto": pbit.KERNEL_AUTO, "sparse": pbit.KERNEL_SPARSE, "dense": pbit.KERNEL_DENSE,
              "resident": pbit.KERNEL_RESIDENT}[args.kernel]
    r = run_single(args, w, variant, kernel, args.config == "dense", steps=args.steps, warmup=args.warmup,
                   e2e_reps=args.steps, dist=dist, world=world, local=local)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cb = None
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_baseline(w, kind=args.config, variant=variant)
    line = {
        "metric": "spin-updates/s", "value": r["value"], "unit": "spin-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_anneal"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i8/f32", "data": "synthetic",
        "config": {**workload_config(w), "l2": "flushed between timed steps", "kernel": r["kernel"],
                   "mean_cut": r["mean_cut"]},
        "roofline": r["roofline"], "cpu_baseline": cb, "e2e": r["e2e"], "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ main ----

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="headline",
                    choices=["headline", "dense", "sparse", "plain", "batch", "serve", "sweep"])
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="arrival window per rate (serving)")
    ap.add_argument("--serve-drain", type=float, default=15.0, help="longest wait for a rate's last results")
    ap.add_argument("--serve-rates", default="10,30,100,300,1000")
    ap.add_argument("--plain-reps", type=int, default=2, help="timed passes of the plain form")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "sparse", "dense", "resident"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="headline: leave out the serving sweep")
    ap.add_argument("--no-components", action="store_true", help="headline: leave out the dense/sparse lines")
    ap.add_argument("--no-oracle-check", action="store_true", help="headline: leave out the oracle's mean cut")
    ap.add_argument("--anneal-steps", type=int, default=0,
                    help="shorten the schedule (profiling captures only; such a line is not a bench value)")
    ap.add_argument("--algorithm", default="psa", choices=["psa", "spsa", "tapsa"],
                    help="pSA variant of the Methods section (sparse / plain configs)")
    ap.add_argument("--stall-prob", type=float, default=0.5, help="SpSA stall probability")
    ap.add_argument("--window", type=int, default=4, help="TApSA window")
    ap.add_argument("--t-res", type=int, default=0, help="timing model: sub-steps per cycle (0: off)")
    ap.add_argument("--s-nu", type=float, default=0.1, help="timing model: spread of the period deviation")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.config == "headline":
        if args.impl == "reference":
            ws = inputs.batch64(steps=args.anneal_steps or 2000)
            return run_reference(args, multi_reference_workload("batch"),
                                 config=batch_config(ws, f"batch64_uneven_S{ws[0].steps}"))
        return bench_headline(args)
    if args.config in ("batch", "serve", "sweep"):
        if args.impl == "reference":
            return run_reference(args, multi_reference_workload(args.config))
        return bench_multi(args)
    return bench_one(args)


if __name__ == "__main__":
    main()
