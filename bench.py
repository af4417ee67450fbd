"""Benchmark of the adaptive ray trace on one GB300 (and one problem split by source over N
GPUs under torchrun).

Workload (default): the coupled trace + ionization-balance step on a 512^3 lognormal grid
(sigma_ln = 2.0, k^-4 power spectrum, mean n_H = 100 in code units) with 1024 power-law
sources: one step = one batched persistent trace of all sources + the Eq. e:xn3 update of the
neutral fraction, whose result feeds the next step's neutral density. Metric: cell-segment
crossings per second. Inputs (512 MB density, 2 GB accumulator) exceed the 129 MB L2, so no
L2 flush is needed between steps.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle on a bounded
sample of the same workload instead. Under torchrun (N > 1) each rank traces its share of the
sources and one all-reduce per step sums gamma and force; the total work is fixed, so the
scaling is strong.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1711_06277_gb300 import synth  # noqa: E402

BYTES_PER_CROSSING = 20  # 4 B opacity gather + 16 B deposit reduction

# reverse sweep, per forward crossing: the cell record gathered in each of the two passes
# ({chi, w}: 8 B for a loss on gamma without dust) and one 4-byte gradient reduction
BYTES_PER_CROSSING_ADJ = 2 * 8 + 4

CONFIGS = {
    # name: grid side, log-density spread, sources, seed, mean n_H, sigma_H, alpha_B, x_n(0)
    "c5_512_1024src": dict(n=512, sigma_ln=2.0, nsrc=1024, seed=5, nbar=100.0, sigma_H=0.1,
                           alpha=2e-4, x0=1e-3),
    "c1_32_uniform": dict(n=32, sigma_ln=None, nsrc=1, seed=None, nbar=1.0, sigma_H=5.0,
                          alpha=None, x0=1.0),
    "c2_128_1src": dict(n=128, sigma_ln=1.5, nsrc=1, seed=1, nbar=1.0, sigma_H=10.0,
                        alpha=None, x0=1.0),
    "c3_256_64src": dict(n=256, sigma_ln=2.0, nsrc=64, seed=3, nbar=1.0, sigma_H=10.0,
                         alpha=None, x0=1.0),
    "c4_128_16src": dict(n=128, sigma_ln=1.5, nsrc=16, seed=4, nbar=1.0, sigma_H=10.0,
                         alpha=None, x0=1.0),
    # smaller cases of the same kernels (ncu captures keep a few GB on the device at most)
    "c5_512_8src": dict(n=512, sigma_ln=2.0, nsrc=8, seed=5, nbar=100.0, sigma_H=0.1,
                        alpha=2e-4, x0=1e-3),
    "c3_256_8src": dict(n=256, sigma_ln=2.0, nsrc=8, seed=3, nbar=1.0, sigma_H=10.0,
                        alpha=None, x0=1.0),
}


def kernel_sources_digest() -> str:
    """SHA-256 over the sources the forward trace kernel is compiled from (its translation
    unit art_api.cu and every header), to tell whether a stored ncu capture of it still
    applies; the reverse sweep, x_n and work-estimate units do not enter."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1711_06277_gb300", "csrc")
    files = [os.path.join(csrc, "art_api.cu")] + glob.glob(os.path.join(csrc, "*.cuh")) \
        + glob.glob(os.path.join(csrc, "*.h")) + [os.path.join(ROOT, "include", "art.h")]
    for path in sorted(files):
        with open(path, "rb") as f:
            h.update(os.path.basename(path).encode() + b"\0" + f.read())
    return h.hexdigest()


def captured_traffic(crossings_per_launch: float):
    """DRAM bytes of one trace launch, scaled from the committed ncu capture of a smaller case
    of the same workload (bytes per crossing x crossings); None if the kernels changed since."""
    path = os.path.join(ROOT, "profiles", "trace_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None, "no capture"
    if d.get("sources_sha256") != kernel_sources_digest():
        return None, "kernel changed since the capture"
    per = float(d["dram_bytes"]) / float(d["crossings"])
    return per * crossings_per_launch, f"scaled from {d['case']} ({per:.2f} B/crossing)"


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def make_workload(cfg: dict):
    """Total H density (float32, (n, n, n)), source positions and luminosities of a config."""
    n = cfg["n"]
    if cfg["sigma_ln"] is None:  # config 1: uniform grid, one source at the box centre
        return (np.full((n, n, n), cfg["nbar"], dtype=np.float32), np.array([[0.5, 0.5, 0.5]]),
                np.array([1.0]))
    rho = synth.lognormal_field(n, cfg["sigma_ln"], seed=cfg["seed"])
    nH = (cfg["nbar"] * rho).astype(np.float32)
    if cfg["nsrc"] == 1:  # config 2: one source at a seeded cell centre
        return nH, synth.cell_centre_position(n, seed=cfg["seed"]), np.array([1.0])
    pos = synth.uniform_positions(cfg["nsrc"], seed=cfg["seed"])
    L = synth.power_law_luminosities(cfg["nsrc"], seed=cfg["seed"])
    return nH, pos, L


def _params(A, cfg, args=None, **kw):
    p = A.Params(level0=4, m_ray=4.0, tau_max=30.0, sigma_H=cfg["sigma_H"], **kw)
    if args is not None:
        p.schedule, p.chunk, p.block_threads = args.schedule, args.chunk, args.block_threads
    return p


def run_ours(args, rank, world, local_rank):
    """The timed coupled step. With world > 1 the one problem is split by source over the
    ranks (paper_1711_06277_gb300.shard): each rank traces its share, one all-reduce sums
    gamma and force, every rank updates x_n."""
    import torch
    from paper_1711_06277_gb300 import art as A

    dev = torch.device("cuda", local_rank % torch.cuda.device_count())
    torch.cuda.set_device(dev)
    cfg = CONFIGS[args.config]
    n = cfg["n"]
    nH_h, pos, L = make_workload(cfg)
    x0 = cfg["x0"]
    nH = torch.from_numpy(nH_h).to(dev)
    xn = torch.full_like(nH, x0)
    nH0 = (xn * nH).contiguous()
    stream = torch.cuda.Stream(dev)
    p = _params(A, cfg, args)
    sharded = None
    mine = np.arange(len(L))
    if world > 1:
        from paper_1711_06277_gb300 import shard
        with torch.cuda.stream(stream):
            sharded = shard.ShardedTrace(nH0, 1.0 / n, pos, L, p, stream=stream)
        mine = sharded.mine
    tuned = None
    if args.tune and args.schedule == "persistent" and not args.chunk and not args.block_threads \
            and len(mine):
        from paper_1711_06277_gb300 import autotune
        with torch.cuda.stream(stream):
            p = autotune.tune(nH0, 1.0 / n, pos[mine], L[mine], p)
        tuned = {"chunk": p.chunk, "block_threads": p.block_threads,
                 "queue_capacity": p.queue_capacity}
    if sharded is not None:
        sharded.params = p
        grid = sharded.grid
        gamma, force = sharded.out[0], sharded.out[1:4]
    else:
        with torch.cuda.stream(stream):
            grid = A.Grid(nH0, 1.0 / n, stream=stream)
            grid.add_sources(pos, L)
        gamma = torch.empty_like(nH)
        force = torch.empty((3,) + tuple(nH.shape), device=dev, dtype=torch.float32)
    alpha = cfg["alpha"]
    dt = 0.1 / (alpha * cfg["nbar"]) if alpha else 0.0

    def enqueue_step():
        if sharded is not None:
            sharded.trace(stats=False)
        else:
            grid.trace(p, force=True, stats=False, out={"gamma": gamma, "force": force})
        if alpha:
            A.xn_update(gamma, nH, xn, alpha, dt, nH0_out=nH0, stream=stream)

    def local_crossings():
        return grid.stats()["crossings"] if len(mine) else 0

    def check_status():
        if len(mine):
            st = grid.stats()
            if st["status"] != 0:
                raise RuntimeError(f"trace status {st['status']}")
            return st["crossings"]
        return 0

    # warm-up (the first trace allocates ray buffers and direction tables)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            enqueue_step()
            check_status()
    graph = None
    graph_note = None
    if args.graph and sharded is None:
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                enqueue_step()
            torch.cuda.synchronize(dev)
        except Exception as e:  # report and run eagerly
            graph, graph_note = None, f"capture failed: {type(e).__name__}: {e}"[:200]
    elif sharded is not None:
        graph_note = "eager: a step holds a collective all-reduce"

    def step():
        with torch.cuda.stream(stream):
            if graph is not None:
                graph.replay()
            else:
                enqueue_step()

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    cross = 0
    step_ms = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(dev.index) as clk:
        ev[0].record(stream)
        for _ in range(args.steps):
            sev[0].record(stream)
            step()
            sev[1].record(stream)
            cross += check_status()  # synchronizes; the counters of this step's trace
            step_ms.append(sev[0].elapsed_time(sev[1]))
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = ev[0].elapsed_time(ev[1])
    ms_all, cross_all = reduce_over_ranks(ms, cross, dev if world > 1 else None)
    value = cross_all / (ms_all / 1e3)

    # dominant kernel: the persistent trace. Its launch time is taken from events around
    # each step on the trace's stream; the other kernels of a step (opacity, injection,
    # finalize, x_n update: ~5 GB of streaming traffic at 512^3) add well under 0.1 %.
    peak, peak_kind = _measured_peaks()
    trace_s = statistics.mean(step_ms) / 1e3
    per_launch_cross = cross / args.steps
    achieved = per_launch_cross * BYTES_PER_CROSSING / trace_s / 1e9
    traffic, traffic_note = captured_traffic(per_launch_cross)

    # end to end through the public API with host buffers (pinned), over as many steps as
    # the device-timed run: H2D of the neutral density, trace + update, D2H of the updated
    # neutral fraction
    e2e = None
    e2e_steps = args.steps if args.e2e_steps is None else args.e2e_steps
    if e2e_steps > 0:
        h_in = torch.empty(nH0.shape, dtype=torch.float32, pin_memory=True)
        h_in.copy_(nH0.cpu())
        h_out = torch.empty_like(h_in, pin_memory=True)
        e_cross = 0
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(e2e_steps):
                nH0.copy_(h_in, non_blocking=True)
                enqueue_step()
                h_out.copy_(xn, non_blocking=True)
                e_cross += local_crossings()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        e_ms, e_cross = reduce_over_ranks(e0.elapsed_time(e1), e_cross, dev if world > 1 else None)
        nbytes = nH0.numel() * 4
        e2e = {"value": e_cross / (e_ms / 1e3), "unit": "crossings/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": e2e_steps}

    extra = {}
    if rank == 0 and args.compare_plain:
        extra["plain_vs_persistent"] = compare_schedules(A, dev)
    if rank == 0 and args.adjoint:
        extra["adjoint"] = adjoint_ratio(A, dev, "c4_128_16src")
        extra["adjoint_512"] = adjoint_ratio(A, dev, "c5_512_8src")
    if rank == 0 and args.per_config:
        extra["per_config"] = per_config(A, dev)
    if sharded is not None:
        extra["shard"] = {"sources_this_rank": int(len(mine)),
                          "estimated_load": [float(v) for v in sharded.load]}
        sharded.close()
    else:
        grid.close()
    launches = 5 if alpha else 4
    return {
        "value": value, "ms": ms_all, "cross": cross_all, "clocks": clk.summary(),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                     "peak_kind": peak_kind,
                     "kernel": "k_trace_persistent",
                     "bytes_per_crossing": BYTES_PER_CROSSING,
                     "crossings_per_launch": per_launch_cross,
                     "launch_ms": trace_s * 1e3},
        "e2e": e2e, "extra": extra, "tuned": tuned,
        "graph": graph is not None, "graph_note": graph_note,
        "gpu_launches": launches * args.steps,
    }


def reduce_over_ranks(ms: float, crossings: float, device=None):
    """Whole-job timing: the slowest rank's time and every rank's crossings. Without an
    initialised process group it returns its inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(crossings)
    t = torch.tensor([ms, float(crossings)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def _time(fn, stream, reps=3):
    import torch
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def adjoint_ratio(A, dev, name="c4_128_16src"):
    """Forward trace vs hand-written adjoint (loss = sum w gamma, no dust), and the adjoint's
    roofline at 20 algorithmic bytes per forward crossing (two 8-byte record gathers and a
    4-byte gradient reduction)."""
    import torch
    cfg = CONFIGS[name]
    nH_h, pos, L = make_workload(cfg)
    nH0 = torch.from_numpy((cfg["x0"] * nH_h).astype(np.float32)).to(dev)
    w = torch.from_numpy(synth.uniform_weights(cfg["n"], seed=cfg["seed"]).astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    g = A.Grid(nH0, 1.0 / cfg["n"], stream=stream)
    g.add_sources(pos, L)
    p = _params(A, cfg)
    g.trace(p, force=False)
    g.trace_backward(p, w)
    tf, tb = [], []
    for _ in range(3):
        tf.append(_time(lambda: g.trace(p, force=False, stats=False), stream, 1))
        tb.append(_time(lambda: g.trace_backward(p, w, stats=False), stream, 1))
    st = g.stats()
    g.close()
    peak, kind = _measured_peaks()
    achieved = st["crossings"] * BYTES_PER_CROSSING_ADJ / (min(tb) / 1e3) / 1e9
    return {"workload": f"{cfg['n']}^3 lognormal sigma_ln={cfg['sigma_ln']}, {cfg['nsrc']} "
                        f"sources, loss = sum w gamma",
            "forward_ms": min(tf), "backward_ms": min(tb), "ratio": min(tb) / min(tf),
            "crossings": st["crossings"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": kind,
                         "kernel": "k_backward_persistent",
                         "bytes_per_crossing": BYTES_PER_CROSSING_ADJ}}


def compare_schedules(A, dev):
    """Persistent batched trace vs the plain one-source-per-launch trace, 256^3 / 64 sources."""
    import torch
    cfg = CONFIGS["c3_256_64src"]
    nH_h, pos, L = make_workload(cfg)
    nH0 = torch.from_numpy(nH_h).to(dev)
    stream = torch.cuda.current_stream(dev)
    g = A.Grid(nH0, 1.0 / cfg["n"], stream=stream)
    g.add_sources(pos, L)
    res = {}
    for sched in ("persistent", "plain"):
        p = _params(A, cfg, schedule=sched)
        st = g.trace(p, force=False)["stats"]
        res[sched] = {"ms": _time(lambda: g.trace(p, force=False, stats=False), stream),
                      "crossings": st["crossings"]}
        res[sched]["crossings_per_s"] = st["crossings"] / (res[sched]["ms"] / 1e3)
    res["speedup"] = res["plain"]["ms"] / res["persistent"]["ms"]
    g.close()
    return res


def per_config(A, dev):
    """Crossings/s and the trace's roofline fraction (20 B per crossing) on configs 1-4:
    the persistent schedule writing gamma and force, best of 3 after a warm-up trace;
    configs 2-4 with autotuned launch knobs (config 1 is bound by its launch latency)."""
    import torch
    peak, _ = _measured_peaks()
    out = {}
    stream = torch.cuda.current_stream(dev)
    for name in ("c1_32_uniform", "c2_128_1src", "c3_256_64src", "c4_128_16src"):
        cfg = CONFIGS[name]
        nH_h, pos, L = make_workload(cfg)
        nH0 = torch.from_numpy(nH_h).to(dev)
        p = _params(A, cfg)
        if name != "c1_32_uniform":
            from paper_1711_06277_gb300 import autotune
            p = autotune.tune(nH0, 1.0 / cfg["n"], pos, L, p)
        g = A.Grid(nH0, 1.0 / cfg["n"], stream=stream)
        g.add_sources(pos, L)
        gam = torch.empty_like(nH0)
        frc = torch.empty((3,) + tuple(nH0.shape), device=dev, dtype=torch.float32)
        st = g.trace(p, force=True, out={"gamma": gam, "force": frc})["stats"]
        ms = _time(lambda: g.trace(p, force=True, stats=False, out={"gamma": gam, "force": frc}),
                   stream)
        g.close()
        rate = st["crossings"] / (ms / 1e3)
        out[name] = {"crossings": st["crossings"], "ms": ms, "crossings_per_s": rate,
                     "roofline_frac": rate * BYTES_PER_CROSSING / 1e9 / peak,
                     "knobs": {"chunk": p.chunk, "block_threads": p.block_threads,
                               "queue_capacity": p.queue_capacity}}
    return out


# --------------------------------------------------------------------------------------
# FP64 oracle on the host cores (the CPU baseline and the reference arm)
# --------------------------------------------------------------------------------------
# Bounded samples of one source of a workload: the base rays whose pixel index is a
# multiple of the stride, with all their descendants (every ray is traced as in the full
# trace; only the set of base rays is thinned). The strides keep one sample near 1-3 s.
STRIDE_ONE_THREAD = 64
STRIDE_ALL_CORES = 4


def _oracle_sample(cfg, k, nthreads, stride):
    from oracle import oracle as O
    nH_h, pos, L = make_workload(cfg)
    nH0 = (cfg["x0"] * nH_h.astype(np.float64)).astype(np.float32)
    s = k % len(L)
    prob = O.Problem(nH0=nH0, pos=pos[s:s + 1], L=L[s:s + 1], dx=1.0 / cfg["n"],
                     sigma_H=cfg["sigma_H"], level0=4, m_ray=4.0, tau_max=30.0)
    t0 = time.perf_counter()
    r = O.trace(prob, nthreads=nthreads, pix_stride=stride)
    return r.crossings, time.perf_counter() - t0


def cpu_baseline(name, reps=5):
    """The oracle as it stands on one bounded sample of the workload, at 1 thread and at all
    host cores: median of ``reps`` timed runs after one untimed run each."""
    cfg = CONFIGS[name]
    cores = os.cpu_count() or 1
    rates = {}
    for threads, stride in ((1, STRIDE_ONE_THREAD), (cores, STRIDE_ALL_CORES)):
        _oracle_sample(cfg, 0, threads, stride)
        runs = [_oracle_sample(cfg, 0, threads, stride) for _ in range(reps)]
        rates[threads] = statistics.median(c / t for c, t in runs)
    return {"value": rates[cores], "unit": "crossings/s", "cores": cores, "kind": "oracle",
            "value_1thread": rates[1], "speedup_all_cores": rates[cores] / rates[1],
            "sample": (f"source 0 of the {cfg['n']}^3 / {cfg['nsrc']}-source workload at its "
                       f"initial neutral fraction, base rays with pixel index a multiple of "
                       f"{STRIDE_ONE_THREAD} (1 thread) or {STRIDE_ALL_CORES} ({cores} threads) "
                       f"and all their descendants; median of {reps}")}


def run_reference(args):
    """FP64 CPU oracle on all host cores, one bounded sample of the workload per step."""
    cfg = CONFIGS[args.config]
    threads = os.cpu_count() or 1
    for k in range(args.warmup):
        _oracle_sample(cfg, k, threads, STRIDE_ALL_CORES)
    cross, dt = 0, 0.0
    for k in range(args.steps):
        c, t = _oracle_sample(cfg, args.warmup + k, threads, STRIDE_ALL_CORES)
        cross += c
        dt += t
    sample = (f"per step one source of the {cfg['n']}^3 / {cfg['nsrc']}-source workload at its "
              f"initial neutral fraction (sources {args.warmup}..{args.warmup + args.steps - 1} "
              f"mod {cfg['nsrc']}), base rays with pixel index a multiple of {STRIDE_ALL_CORES} "
              f"and all their descendants")
    return {"value": cross / dt, "ms": dt * 1e3 / args.steps, "threads": threads, "sample": sample}


def oracle_table():
    """Oracle crossings/s per config at 1 thread and at all cores (median of 5), for the
    results table: configs 1-2 whole, configs 3-4 on their first 8 sources, config 5 on 8
    sources; thinned base rays where a whole run would take minutes."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    plan = {"c1_32_uniform": (1, 1, 1), "c2_128_1src": (1, 2, 1), "c3_256_64src": (8, 64, 4),
            "c4_128_16src": (8, 8, 1), "c5_512_1024src": (8, 512, 32)}
    out = {}
    for name, (nsrc, s1, sn) in plan.items():
        cfg = CONFIGS[name]
        nH_h, pos, L = make_workload(cfg)
        nH0 = (cfg["x0"] * nH_h.astype(np.float64)).astype(np.float32)
        prob = O.Problem(nH0=nH0, pos=pos[:nsrc], L=L[:nsrc], dx=1.0 / cfg["n"],
                         sigma_H=cfg["sigma_H"], level0=4, m_ray=4.0, tau_max=30.0)
        row = {"sources": nsrc}
        for threads, stride in ((1, s1), (cores, sn)):
            O.trace(prob, nthreads=threads, pix_stride=stride)
            runs = []
            for _ in range(5):
                t0 = time.perf_counter()
                r = O.trace(prob, nthreads=threads, pix_stride=stride)
                runs.append(r.crossings / (time.perf_counter() - t0))
            row[f"threads_{threads}"] = {"crossings_per_s": statistics.median(runs),
                                         "pix_stride": stride}
        out[name] = row
    return {"oracle_table": out, "cores": cores}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c5_512_1024src", choices=sorted(CONFIGS))
    ap.add_argument("--schedule", default="persistent", choices=["persistent", "plain"])
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end measurement (default: --steps)")
    ap.add_argument("--no-e2e", dest="e2e_steps", action="store_const", const=0)
    ap.add_argument("--graph", action="store_true", default=True)
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--tune", action="store_true", default=True)
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--adjoint", action="store_true", default=True)
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the forward/backward timing of the adjoint cases")
    ap.add_argument("--adjoint-cases", default="c4_128_16src,c5_512_8src",
                    help="configs timed by the adjoint comparison (comma-separated)")
    ap.add_argument("--per-config", action="store_true", default=True)
    ap.add_argument("--no-per-config", dest="per_config", action="store_false")
    ap.add_argument("--oracle-table", action="store_true",
                    help="only the oracle's rates per config (1 thread and all cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-plain", action="store_true", default=True)
    ap.add_argument("--no-compare-plain", dest="compare_plain", action="store_false")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = CONFIGS[args.config]
    config = {"workload": f"{cfg['n']}^3 lognormal sigma_ln={cfg['sigma_ln']}, {cfg['nsrc']} "
                          f"power-law sources, l0=4, m_ray=4, tau_max=30, gamma and force"
                          + (", trace + Eq. e:xn3 update per step" if cfg["alpha"] else ""),
              "grid": cfg["n"], "sources": cfg["nsrc"], "schedule": args.schedule,
              "cuda_graph": args.graph,
              "parallelism": (f"sources split over {world} GPUs, one all-reduce of gamma and "
                              f"force per step" if world > 1 else "one GPU"),
              "l2": (f"inputs larger than L2 ({cfg['n'] ** 3 * 4 >> 20} MB density, "
                     f"{cfg['n'] ** 3 * 16 >> 20} MB accumulator; L2 is 129 MB)")}

    if args.oracle_table:
        if rank == 0:
            print(json.dumps(oracle_table()), flush=True)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        r = run_reference(args)
        line = {"impl": "reference", "metric": "cell-segment crossings/s", "value": r["value"],
                "unit": "crossings/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config,
                "cpu_baseline": {"value": r["value"], "unit": "crossings/s", "cores": r["threads"],
                                 "kind": "oracle", "sample": r["sample"]},
                "e2e": {"value": r["value"], "unit": "crossings/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if args.adjoint_only:
        if rank == 0:
            import torch
            from paper_1711_06277_gb300 import art as A
            dev = torch.device("cuda", local_rank)
            print(json.dumps({name: adjoint_ratio(A, dev, name)
                              for name in args.adjoint_cases.split(",")}))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank % torch.cuda.device_count())
        # NCCL across the node's GPUs; ART_BENCH_BACKEND=gloo runs the same split path with
        # host-side collectives (e.g. several ranks sharing one GPU to check the path)
        dist.init_process_group(os.environ.get("ART_BENCH_BACKEND", "nccl"))
    r = run_ours(args, rank, world, local_rank)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(args.config)
    config["cuda_graph"] = r["graph"]
    if r["graph_note"]:
        config["cuda_graph_note"] = r["graph_note"]
    if r["tuned"]:
        config["autotuned"] = r["tuned"]
    line = {"metric": "cell-segment crossings/s", "value": r["value"], "unit": "crossings/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
            "clocks": r["clocks"], "roofline": r["roofline"], "cpu_baseline": cpu,
            "e2e": r["e2e"], "gpu_launches": r["gpu_launches"]}
    line.update(r["extra"])
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
