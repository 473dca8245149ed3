#!/usr/bin/env python
"""Benchmark of the domain wall fermion hot path on one GB300 (per rank).

Workload (default): the paper's per-GPU volume, Moebius DWF on 32^4 x Ls=16
(b5=1.5, c5=0.5, M5=1.8, m_f=0.005), links U = exp(i 0.3 H) from seed 1003,
one Gaussian source.  One step = the whole hot path on that source:

  * mixed-precision CGNE of D x = b to |b - D x|/|b| <= 1e-10 (FP32 operator,
    FP32 vectors, FP64 reliable updates, FP64 reductions and solution);
  * the same solve with the Dirichlet block operator D_Omega of the 30^4
    interior box left by a band of width 2 in all four directions.

The printed value is the Dslash-model throughput of the step: every Wilson
hop the step applies counts 1320 flops per 5D site of its checkerboard,
divided by the step time (CUDA events).  Beside it, measured once: the same
solves with plain FP64 CG, D_Omega for bands of width 1 and 4, the bare-hop
roofline (FP32 at 32^4 x 16, L2 flushed between launches), the earlier
16^4 x Ls=12 workload, and the CPU oracle on the host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DWF Dslash TFLOP/s & HBM GB/s; time-to-1e-10 residual vs plain FP64 CG"
DIMS, LS = (32, 32, 32, 32), 16
M5, MF, B5, C5 = 1.8, 0.005, 1.5, 0.5
EPS, SEED = 0.3, 1003
BANDS = {1: ((0, 0, 0, 0), (31, 31, 31, 31)), 2: ((1, 1, 1, 1), (30, 30, 30, 30)),
         4: ((2, 2, 2, 2), (28, 28, 28, 28))}
STEP_BAND = 2
FLOPS_PER_SITE = 1320
WORKLOAD = ("Moebius DWF 32^4 x Ls=16 (b5=1.5, c5=0.5, M5=1.8, m_f=0.005, exp(i 0.3 H) links); "
            "mixed FP32/FP64 CGNE to 1e-10 of D and of D_Omega (w=2 band, 30^4 interior box)")
# the earlier, smaller workload (Moebius 16^4 x Ls=12, m_f = 0.01), reported as extra keys
SMALL_DIMS, SMALL_LS, SMALL_MF, SMALL_SEED = (16, 16, 16, 16), 12, 0.01, 1001
SMALL_BAND = ((1, 1, 1, 1), (14, 14, 14, 14))
SMALL_WORKLOAD = "Moebius DWF 16^4 x Ls=12 (b5=1.5, c5=0.5, M5=1.8, m_f=0.01, exp(i 0.3 H) links)"
# CPU oracle sample: one M_pc^+ M_pc application (the operator work of one CG
# iteration) on an 8^4 x Ls=16 lattice per worker
ORACLE_SAMPLE_DIMS = (8, 8, 8, 8)


def hop_bytes_per_site(Ls, word):
    """Algorithmic bytes per 5D output site of one hop: spinor in + out
    (24 reals each) and the site's share of the 4V links (144/Ls reals)."""
    return (48.0 + 144.0 / Ls) * word


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"dwf_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- our arm
def job_time_ms(local_ms, world, device=None):
    """The job's time for the timed steps: the slowest rank's (the ranks meet at
    a barrier on both sides of the timed region).  world = 1: local_ms."""
    if world == 1:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, flops_per_rank, job_ms):
    """Whole-job throughput (TFLOP/s): every rank's work over the slowest rank's time."""
    return world * flops_per_rank / (job_ms * 1e-3) / 1e12


def _event_ms(fn, stream):
    """Run fn() between two CUDA events on `stream`; returns (result, ms)."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    r = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return r, a.elapsed_time(b)


def _bare_hop(G, h, prec, configs, flush, stream, reps, tc=False):
    """Mean time (ms) of the bare hop Dh into the even checkerboard (CUDA
    events on the launching stream, L2 flushed before every launch) for each
    kernel configuration (tile, lanes, chunk) or None (the handle's current
    one); returns the best as (ms, config)."""
    import torch
    h.set_hop_kernel(1, 1 if tc else 0)
    inp = torch.randn(h.cb_shape(1), device=stream.device).to(G._DTYPE[prec])
    out = h.empty_cb(0, 1, prec)
    saved = h.tuning(1)
    best = None
    for cfg in configs:
        if cfg is not None:
            h.set_tile(1, cfg[0], cfg[1])
            h.set_hop_chunk(1, cfg[2])
        for _ in range(3):
            h.hop(out, inp, 0, prec=prec)
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            ts.append(_event_ms(lambda: h.hop(out, inp, 0, prec=prec), stream)[1])
        m = statistics.mean(ts)
        if best is None or m < best[0]:
            best = (m, list(cfg) if cfg is not None else list(h.tuning(1)[:3]))
    h.set_tile(1, saved[0], saved[1])
    h.set_hop_chunk(1, saved[2])
    h.set_hop_kernel(1, 0)
    del inp, out
    return best


def _box_source(src, box):
    o, e = box
    sub = src[o[3]:o[3] + e[3], o[2]:o[2] + e[2], o[1]:o[1] + e[1], o[0]:o[0] + e[0]]
    return sub.reshape(-1)


def _solve_flops(st, sites):
    """Dslash-model flops of one CGNE solve: 2 hops per M_pc application, plus
    b' (1 hop), x_e (1 hop) and the final D x (2 hops)."""
    return (2 * st["op_applies"] + 4) * FLOPS_PER_SITE * sites


def _small_workload(G, inputs, dev, stream, flush):
    """The earlier workload, Moebius 16^4 x Ls=12, m_f = 0.01: one mixed solve
    of D and of D_Omega (w = 2, 14^4 box) after a warm-up solve, and the bare
    FP32 hop (autotuned configuration)."""
    import numpy as np
    import torch
    act = G.Action(M5, SMALL_MF, B5, C5)
    rng = np.random.default_rng(SMALL_SEED)
    U = inputs.gauge_field(SMALL_DIMS, "exp", eps=EPS, rng=rng)
    src = inputs.gaussian_source(SMALL_DIMS, SMALL_LS, rng=rng)
    Ut = torch.from_numpy(U.reshape(-1)).to(dev)
    res = {"workload": "Moebius DWF 16^4 x Ls=12 (m_f=0.01, exp(i 0.3 H) links, seed 1001): "
                       "mixed CGNE to 1e-10 of D and of D_Omega (w=2, 14^4 box)"}
    for name, box in (("D", None), ("D_Omega", SMALL_BAND)):
        h = G.Handle(SMALL_DIMS, SMALL_LS, act, boxes=[box] if box else None)
        h.set_gauge(Ut)
        h.autotune(1, G.FP32)
        canon = src.reshape(-1) if box is None else _box_source(src, box)
        b = h.pack(torch.from_numpy(np.ascontiguousarray(canon)).to(dev))
        x = torch.zeros_like(b)
        for _ in range(2):
            x.zero_()
            (st, _), ms = _event_ms(lambda: h.cgne_solve(x, b, tol=1e-10, inner=G.FP32), stream)
        res[name] = {"ms": round(ms, 3), "iters": st[0]["iters"], "true_resid": st[0]["true_resid"]}
        if box is None:
            sites = SMALL_DIMS[0] ** 4 // 2 * SMALL_LS
            ms_hop, cfg = _bare_hop(G, h, G.FP32, [None], flush, stream, 10)
            nbytes = hop_bytes_per_site(SMALL_LS, 4) * sites
            res["dslash_f32"] = {"ms": round(ms_hop, 4), "config": cfg,
                                 "tflops": round(FLOPS_PER_SITE * sites / (ms_hop * 1e-3) / 1e12, 3),
                                 "gbs": round(nbytes / (ms_hop * 1e-3) / 1e9, 1)}
        del h, b, x
    torch.cuda.empty_cache()
    return res


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs

    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    act = G.Action(M5, MF, B5, C5)
    t_setup = time.time()
    rng = np.random.default_rng(SEED)
    U = inputs.gauge_field(DIMS, "exp", eps=EPS, rng=rng)
    src = inputs.gaussian_source(DIMS, LS, rng=rng)
    Ut = torch.from_numpy(U.reshape(-1)).to(dev)
    del U
    box = BANDS[STEP_BAND]
    hD = G.Handle(DIMS, LS, act)
    hD.set_gauge(Ut)
    hO = G.Handle(DIMS, LS, act, boxes=[box])
    hO.set_gauge(Ut)
    canonD = torch.from_numpy(src.reshape(-1)).to(dev)
    canonO = torch.from_numpy(np.ascontiguousarray(_box_source(src, box))).to(dev)
    if args.config:   # a fixed kernel configuration (e.g. to replay a tuned run under a profiler)
        for hh in (hD, hO):
            hh.set_tile(1, args.config[0], args.config[1])
            hh.set_hop_chunk(1, args.config[2])
    else:
        hD.autotune(1, G.FP32)
        hO.autotune(1, G.FP32)
    tiles = {"D": list(hD.tuning(1)[:3]), "D_Omega": list(hO.tuning(1)[:3])}
    bD, bO = hD.pack(canonD), hO.pack(canonO)
    xD, xO = torch.zeros_like(bD), torch.zeros_like(bO)
    sitesD = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2 * LS
    e = box[1]
    sitesO = (e[0] * e[1] * e[2] * e[3]) // 2 * LS
    del canonD, canonO
    print(f"[bench] set-up {time.time() - t_setup:.1f} s", file=sys.stderr)

    def step(host=None):
        stats = []
        for h, x, b, hb, hx in ((hD, xD, bD, host and host[0], host and host[1]),
                                (hO, xO, bO, host and host[2], host and host[3])):
            if hb is not None:
                b.copy_(hb, non_blocking=True)
            x.zero_()
            st, _ = h.cgne_solve(x, b, tol=1e-10, inner=G.FP32)
            if hx is not None:
                hx.copy_(x, non_blocking=True)
            stats.append(st[0])
        return stats

    def flops(stats):
        return sum(_solve_flops(s, n) for s, n in zip(stats, (sitesD, sitesO)))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = G.launch_count()
    print(f"[bench] launches before timed region: {l0}", file=sys.stderr)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    all_stats = []
    torch.cuda.synchronize()
    for k in range(args.steps):
        ev[k][0].record(stream)
        all_stats.append(step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = G.launch_count() - l0
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    times = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(times)
    tot_flops = sum(flops(s) for s in all_stats)
    tot_ms = job_time_ms(tot_ms, world, dev)
    value = job_value(world, tot_flops, tot_ms)
    last = all_stats[-1]
    mixed_ms = {"D": last[0]["seconds"] * 1e3, "D_Omega": last[1]["seconds"] * 1e3}

    # ---- end to end: host (pinned) sources in and solutions out for every
    # step, timed over a block of steps.  The copies run on a side stream
    # beside the solves: the D_Omega source goes in during the D solve, x_D
    # comes out and the next step's D source goes in during the D_Omega solve,
    # x_Omega comes out during the next step's D solve; the block ends when the
    # last copy has landed.
    n_e2e = max(1, min(args.steps, 3))
    hb = [bD.cpu().pin_memory(), None, bO.cpu().pin_memory(), None]
    hb[1] = torch.empty_like(hb[0]).pin_memory()
    hb[3] = torch.empty_like(hb[2]).pin_memory()
    side = torch.cuda.Stream(device=dev)

    def e2e_block(n):
        # the copies are dwf_copy calls (the GPU's own loads and stores to pinned
        # host memory), on the side stream
        out = []
        side.wait_stream(stream)          # nothing on the side stream before the start event
        G.copy(bD, hb[0], stream=side)
        ready_D = side.record_event()
        for k in range(n):
            G.copy(bO, hb[2], stream=side)
            ready_O = side.record_event()
            stream.wait_event(ready_D)
            xD.zero_()
            stD, _ = hD.cgne_solve(xD, bD, tol=1e-10, inner=G.FP32)
            side.wait_stream(stream)
            G.copy(hb[1], xD, stream=side)
            if k + 1 < n:
                G.copy(bD, hb[0], stream=side)
            ready_D = side.record_event()
            stream.wait_event(ready_O)
            xO.zero_()
            stO, _ = hO.cgne_solve(xO, bO, tol=1e-10, inner=G.FP32)
            side.wait_stream(stream)
            G.copy(hb[3], xO, stream=side)
            out.append([stD[0], stO[0]])
        stream.wait_stream(side)
        return out

    e2e_block(1)    # warm-up: the first transfers into freshly pinned buffers touch their pages
    sts, e2e_ms = _event_ms(lambda: e2e_block(n_e2e), stream)
    e2e_flops = sum(flops(st) for st in sts)
    h2d = (bD.numel() + bO.numel()) * bD.element_size()
    d2h = (xD.numel() + xO.numel()) * xD.element_size()
    # the copy bandwidth of this machine, for reading the e2e figure: dwf_copy and
    # the copy engines (cudaMemcpyAsync through torch)
    nbD = bD.numel() * bD.element_size()
    copy_gbs = {}
    for name, fn in (("h2d_dwf_copy", lambda: G.copy(bD, hb[0])), ("d2h_dwf_copy", lambda: G.copy(hb[1], xD)),
                     ("h2d_copy_engine", lambda: bD.copy_(hb[0], non_blocking=True)),
                     ("d2h_copy_engine", lambda: hb[1].copy_(xD, non_blocking=True))):
        fn()
        _, ms = _event_ms(fn, stream)
        copy_gbs[name] = round(nbD / (ms * 1e-3) / 1e9, 1)
    del hb

    # ---- plain FP64 CG on the same two systems (time to 1e-10), once
    fp64 = {}
    if not args.no_fp64_cg:
        for name, h, x, b in (("D", hD, xD, bD), ("D_Omega", hO, xO, bO)):
            x.zero_()
            (st, _), ms = _event_ms(lambda: h.cgne_solve(x, b, tol=1e-10, inner=G.FP64), stream)
            fp64[name] = {"ms": round(ms, 1), "iters": st[0]["iters"], "true_resid": st[0]["true_resid"]}

    # ---- D_Omega for the other band widths, once each (one warm-up solve)
    bands = {}
    for w in sorted(BANDS):
        if w == STEP_BAND:
            continue
        h = G.Handle(DIMS, LS, act, boxes=[BANDS[w]])
        h.set_gauge(Ut)
        h.set_tile(1, tiles["D_Omega"][0], tiles["D_Omega"][1])
        h.set_hop_chunk(1, tiles["D_Omega"][2])
        b = h.pack(torch.from_numpy(np.ascontiguousarray(_box_source(src, BANDS[w]))).to(dev))
        x = torch.zeros_like(b)
        for _ in range(2):
            x.zero_()
            (st, _), ms = _event_ms(lambda: h.cgne_solve(x, b, tol=1e-10, inner=G.FP32), stream)
        bands[f"w{w}"] = {"box": [list(BANDS[w][0]), list(BANDS[w][1])], "ms": round(ms, 3),
                          "iters": st[0]["iters"], "true_resid": st[0]["true_resid"]}
        del h, b, x
    torch.cuda.empty_cache()
    del src

    # ---- bare hop (dominant kernel) at 32^4 x 16: CUDA events per launch, L2 flushed
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    reps = max(args.steps, 10)
    hop = {}
    for name, prec, word, tc in (("f32", G.FP32, 4, False), ("bf16", G.BF16, 2, False),
                                 ("bf16_tc", G.BF16, 2, True), ("f64", G.FP64, 8, False)):
        cfgs = [None]
        if prec == G.FP32:
            cfgs += [(64, 2, 8), (64, 2, 1), (32, 2, 8)]
        ms, cfg = _bare_hop(G, hD, prec, cfgs, flush, stream, reps if prec != G.FP64 else 3, tc)
        nbytes = hop_bytes_per_site(LS, word) * sitesD
        hop[name] = {"ms": round(ms, 4), "config": cfg,
                     "tflops": round(FLOPS_PER_SITE * sitesD / (ms * 1e-3) / 1e12, 3),
                     "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1), "bytes": nbytes}
    small = None if args.no_small else _small_workload(G, inputs, dev, stream, flush)
    del flush
    # the batched workload (6 uneven Dirichlet boxes x 16 right-hand sides at 24^4 x 16), once
    batched = None if args.no_batched else batched_result(16, "f32", args.steps)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    for v in hop.values():
        v["frac_hbm"] = round(v["gbs"] / peak, 3)
    # DRAM bytes per launch from the committed ncu capture of the same kernel
    # configuration (tile, lanes, chunk, tile order), while hop.cu is unchanged
    traffic = None
    order = list(hD.tile_order())
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "hop_f32_traffic.json")))
        src_hash = hashlib.sha256(open(os.path.join(ROOT, "paper_2203_17119_gb300", "csrc", "hop.cu"),
                                       "rb").read()).hexdigest()[:16]
        if prof.get("hop_cu_sha256_16") == src_hash and prof.get("lattice") == list(DIMS) \
                and prof.get("Ls") == LS:
            for cap in prof["captures"]:
                if cap["config_tile_lanes_chunk"] == list(hop["f32"]["config"]) and cap["tile_order"][0] == order[0] \
                        and (order[0] == 0 or cap["tile_order"] == order):
                    traffic = cap["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError, TypeError):
        pass
    roof = {"bound": "hbm", "kernel": "k_hop<float> (bare Wilson hop, FP32, 32^4 x Ls=16)",
            "config_tile_lanes_chunk": hop["f32"]["config"], "tile_order": order,
            "achieved": hop["f32"]["gbs"], "peak": peak, "unit": "GB/s",
            "frac": round(hop["f32"]["gbs"] / peak, 3), "traffic": traffic,
            "algorithmic_bytes_per_launch": hop["f32"]["bytes"],
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
            else "fallback 6800 GB/s"}

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded exp(i 0.3 H) SU(3) links, Gaussian source)",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "Ls": LS, "mf": MF,
                   "inner": "FP32 operator + FP32 vectors; FP64 reliable updates/reductions/x",
                   "l2": "inputs larger than L2 (one FP32 checkerboard field is 0.8 GB; solver "
                         "state ~20 GB per solve)",
                   "parallelism": f"replicas x{world}", "tile_sites_lanes_chunk": tiles},
        "time_to_solution_ms": {k: round(v, 3) for k, v in mixed_ms.items()},
        "iters": {"D": last[0]["iters"], "D_Omega": last[1]["iters"]},
        "reliable_updates": {"D": last[0]["reliable_updates"], "D_Omega": last[1]["reliable_updates"]},
        "true_resid": {"D": last[0]["true_resid"], "D_Omega": last[1]["true_resid"]},
        "fp64_cg": fp64,
        "speedup_vs_fp64_cg": {k: round(fp64[k]["ms"] / mixed_ms[k], 2) for k in fp64},
        "d_omega_other_bands": bands,
        "dslash": hop,
        "roofline": roof,
        "small_16x12": small,
        "batched_24x16": batched,
        "e2e": {"value": round(world * e2e_flops / (e2e_ms * 1e-3) / 1e12, 3), "unit": "TFLOP/s",
                "steps": n_e2e, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "copies": "every step's sources in and solutions out by dwf_copy on a side stream beside "
                          "the solves; the block of steps is timed whole",
                "pinned_copy_gbs": copy_gbs},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    return result


# --------------------------------------------------------- CPU oracle leg
def _oracle_mpc_normal(seed):
    """One M_pc^+ M_pc application of the oracle (the operator work of one CG
    iteration) on the sample lattice; returns its wall time in seconds.  Runs
    in a spawned worker with one thread."""
    import numpy as np
    from oracle import dwf as O
    from paper_2203_17119_gb300 import inputs
    rng = np.random.default_rng(seed)
    # Haar links: the oracle's work does not depend on the link values
    U = inputs.gauge_field(ORACLE_SAMPLE_DIMS, "haar", rng=rng)
    psi = O.parity_part(inputs.gaussian_source(ORACLE_SAMPLE_DIMS, LS, rng=rng), 1)
    prm = O.DWFParams(M5=M5, mf=MF, b5=B5, c5=C5)
    t = time.perf_counter()
    O.mpc(U, O.mpc(U, psi, prm), prm, True)
    return time.perf_counter() - t


def _sample_flops():
    """Dslash-model flops of one M_pc^+ M_pc (4 hops) on the sample lattice."""
    V = 1
    for d in ORACLE_SAMPLE_DIMS:
        V *= d
    return 4 * FLOPS_PER_SITE * (V // 2) * LS


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """Spawned single-threaded worker processes that run the oracle sample
    (spawn: no fork after CUDA initialisation)."""

    def __init__(self, n):
        self.n = n
        keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                "MKL_NUM_THREADS")}
        for k in keep:
            os.environ[k] = "1"
        self.pool = multiprocessing.get_context("spawn").Pool(n)
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def run(self, workers, seed):
        """`workers` samples at once; returns the time of the slowest sample's
        operator application (the samples run concurrently; their set-up is
        not timed)."""
        return max(self.pool.map(_oracle_mpc_normal, [seed + i for i in range(workers)]))

    def close(self):
        self.pool.close()
        self.pool.join()


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(iters_D):
    """The oracle timed on the host cores: one M_pc^+ M_pc application of the
    8^4 x 16 sample per worker, on all cores at once and on one core, in the
    Dslash-model TFLOP/s of `value`; plus the oracle's time to 1e-10 for the D
    solve extrapolated from it (per-iteration time scaled by volume, times the
    GPU's iteration count)."""
    cores = _host_cores()
    pool = OraclePool(cores)
    pool.run(cores, 7)                                  # warm-up: imports, first touch
    wall_all = pool.run(cores, 11)
    wall_1 = pool.run(1, 13)
    pool.close()
    f = _sample_flops()
    scale = 1.0
    for a, b in zip(DIMS, ORACLE_SAMPLE_DIMS):
        scale *= a / b
    per_iter_1 = wall_1 * scale
    return {
        "value": cores * f / wall_all / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
        "sample": (f"one oracle M_pc^+ M_pc (4 Wilson hops, the operator of one CG iteration) on a "
                   f"{'x'.join(map(str, ORACLE_SAMPLE_DIMS))} x Ls={LS} Moebius lattice per worker, "
                   f"{cores} single-threaded workers at once ({wall_all:.1f} s), numpy FP64; "
                   "same flop model as value"),
        "cpu_model": _cpu_model(),
        "one_core": {"value": f / wall_1 / 1e12, "unit": "TFLOP/s", "seconds": round(wall_1, 2)},
        "extrapolated_time_to_solution_s": {
            "D": round(per_iter_1 * iters_D / cores, 1) if iters_D else None,
            "how": "one-core sample time x (32^4 / sample volume) x GPU iteration count / cores "
                   "(extrapolated, not run)"},
    }


def run_reference(args):
    """The reference arm: the CPU oracle as it stands on the host cores.  Each
    step is one M_pc^+ M_pc application of the 8^4 x 16 sample per core, all
    cores at once; value = Dslash-model TFLOP/s over the timed steps."""
    cores = _host_cores()
    pool = OraclePool(cores)
    walls = []
    for k in range(args.warmup + args.steps):
        wall = pool.run(cores, 100 + k * cores)
        if k >= args.warmup:
            walls.append(wall)
    pool.close()
    f = _sample_flops() * cores
    value = f * len(walls) / sum(walls) / 1e12
    sample = (f"per step one oracle M_pc^+ M_pc (4 Wilson hops) on a "
              f"{'x'.join(map(str, ORACLE_SAMPLE_DIMS))} x Ls={LS} Moebius lattice on each of "
              f"{cores} single-threaded workers at once, numpy FP64")
    return {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "Ls": LS}, "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_hop(args):
    """Bare Wilson hop at a chosen size: --hop L Ls prec [nrhs] (CUDA events
    per launch, L2 flushed between launches).  Used for the Dslash sweep and
    as the command the hop profiles are captured from."""
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    L, Ls, prec_name = int(args.hop[0]), int(args.hop[1]), args.hop[2]
    nrhs = int(args.hop[3]) if len(args.hop) > 3 else 1
    prec = G.PREC[prec_name]
    word = {G.FP64: 8, G.FP32: 4, G.BF16: 2}[prec]
    dims = (L, L, L, L)
    U = inputs.gauge_field(dims, "exp", eps=EPS, seed=SMALL_SEED)
    h = G.Handle(dims, Ls, G.Action(M5, SMALL_MF, B5, C5), nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    del U
    if args.hop_config:
        T, vl = args.hop_config
        h.set_tile(nrhs, T, vl)
    if args.tc:
        h.set_hop_kernel(nrhs, 1)
    if args.chunk:
        h.set_hop_chunk(nrhs, args.chunk)
    else:
        T = h.autotune(nrhs, prec) if not args.no_autotune else None
    if args.tile_order:
        h.set_tile_order(1, *args.tile_order)
    inp = torch.randn(h.cb_shape(1, nrhs), device="cuda").to(G._DTYPE[prec])
    out = h.empty_cb(0, nrhs, prec)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        h.hop(out, inp, 0, prec=prec, nrhs=nrhs)
    ts = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.hop(out, inp, 0, prec=prec, nrhs=nrhs)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.mean(ts)
    sites = L ** 4 // 2 * Ls * nrhs
    nbytes = (48.0 + 144.0 / (Ls * nrhs)) * word * sites
    peak = 6800.0
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, ValueError, KeyError):
        pass
    print(json.dumps({"kernel": "hop", "lattice": [L] * 4, "Ls": Ls, "nrhs": nrhs, "prec": prec_name,
                      "tile_sites": T, "config": args.hop_config, "tensor_cores": bool(args.tc), "chunk": args.chunk or None, "tile_order": args.tile_order, "ms": ms, "tflops": FLOPS_PER_SITE * sites / (ms * 1e-3) / 1e12,
                      "gbs": nbytes / (ms * 1e-3) / 1e9, "frac_hbm": nbytes / (ms * 1e-3) / 1e9 / peak,
                      "algorithmic_bytes": nbytes}))


def run_multishift(args):
    """Multi-shift CG (--multishift NSHIFT [f64|f32]) on the default 16^4 x Ls=12
    Moebius lattice to 1e-10: NSHIFT log-spaced shifts 1e-4 .. 1 (the poles of a
    rational approximation), against NSHIFT single-shift solves of the same
    systems (f32: FP32 operator plus FP64 defect correction)."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    ns = int(args.multishift[0])
    prec = G.PREC[args.multishift[1]] if len(args.multishift) > 1 else G.FP64
    tol = 1e-10
    rng = np.random.default_rng(SMALL_SEED)
    U = inputs.gauge_field(SMALL_DIMS, "exp", eps=EPS, rng=rng)
    h = G.Handle(SMALL_DIMS, SMALL_LS, G.Action(M5, SMALL_MF, B5, C5))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    h.autotune(1, G.FP32)
    full = h.pack(torch.from_numpy(inputs.gaussian_source(SMALL_DIMS, SMALL_LS, rng=rng).reshape(-1)).cuda())
    b = full[h.nsite[0]:].contiguous()
    shifts = list(np.logspace(-4, 0, ns))
    x = torch.zeros((ns,) + tuple(b.shape), dtype=torch.float64, device="cuda")
    h.multishift_solve(x, b, shifts, tol=tol, inner=prec)   # warm-up
    torch.cuda.synchronize()
    t = time.time()
    st, rc = h.multishift_solve(x, b, shifts, tol=tol, inner=prec)
    torch.cuda.synchronize()
    t_ms = time.time() - t
    t = time.time()
    singles = []
    for sig in shifts:
        st1, _ = h.multishift_solve(x[:1], b, [sig], tol=tol, inner=prec)
        singles.append(st1[0][0]["iters"])
    torch.cuda.synchronize()
    t_single = time.time() - t
    print(json.dumps({"workload": f"multi-shift CG on M_pc^+ M_pc, {SMALL_WORKLOAD}",
                      "nshift": ns, "prec": args.multishift[1] if len(args.multishift) > 1 else "f64",
                      "tol": tol, "seconds": t_ms, "seconds_single_shift_solves": t_single,
                      "speedup": t_single / t_ms,
                      "iters": [s[0]["iters"] for s in st], "iters_single": singles,
                      "max_true_resid": max(s[0]["true_resid"] for s in st)}))


def run_force(args):
    """Link force of Re <X, D Y> (--force [f64|f32] [L] [Ls]) on an L^4 x Ls
    Moebius lattice (default the 16^4 x 12 workload): the whole dwf_force call
    (the two site-local B = b5 + c5 S5 launches and the force kernel), CUDA
    events per call, L2 flushed between calls; the oracle's time per site on an
    8^4 sample beside it."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    prec_name = args.force[0] if args.force else "f64"
    L = int(args.force[1]) if len(args.force) > 1 else SMALL_DIMS[0]
    Ls = int(args.force[2]) if len(args.force) > 2 else SMALL_LS
    prec = G.PREC[prec_name]
    word = {G.FP64: 8, G.FP32: 4}[prec]
    dims = (L, L, L, L)
    rng = np.random.default_rng(SMALL_SEED)
    U = inputs.gauge_field(dims, "exp", eps=EPS, rng=rng)
    h = G.Handle(dims, Ls, G.Action(M5, SMALL_MF, B5, C5))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    n = 2 * 12 * Ls * L ** 4
    X = torch.randn(n, dtype=torch.float64, device="cuda").to(G._DTYPE[prec])
    Y = torch.randn(n, dtype=torch.float64, device="cuda").to(G._DTYPE[prec])
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    del U
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        h.force(out, X, Y, prec=prec)
    ts = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.force(out, X, Y, prec=prec)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.mean(ts)
    V = L ** 4
    # per site: X and Y once, four forward links, four FP64 forces written
    nbytes = V * (2 * 24 * Ls * word + 4 * 18 * word + 4 * 18 * 8)
    # per site, direction and lane: four half-spinor projections (12 flops
    # each) and two rank-2 outer products (2 x 9 complex multiply-adds)
    flops = V * 4 * Ls * (4 * 12 + 2 * 2 * 9 * 8)
    peak = 6800.0
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, ValueError, KeyError):
        pass
    from oracle import dwf as O
    from oracle.force import force_bilinear
    sd = (8, 8, 8, 8)
    Us = inputs.gauge_field(sd, "exp", eps=EPS, rng=rng)
    Xs, Ys = (inputs.gaussian_source(sd, Ls, rng=rng) for _ in range(2))
    prm = O.DWFParams(M5=M5, mf=SMALL_MF, b5=B5, c5=C5)
    t = time.time()
    force_bilinear(Us, Xs, Ys, prm)
    oracle_s_per_site = (time.time() - t) / 8 ** 4
    print(json.dumps({"kernel": "force", "lattice": list(dims), "Ls": Ls, "prec": prec_name,
                      "ms": ms, "gflops": flops / (ms * 1e-3) / 1e9,
                      "gbs": nbytes / (ms * 1e-3) / 1e9, "frac_hbm": nbytes / (ms * 1e-3) / 1e9 / peak,
                      "algorithmic_bytes": nbytes, "flops": flops,
                      "oracle_ms_scaled": oracle_s_per_site * V * 1e3,
                      "oracle_sample": "8^4 x Ls, one call, time per site scaled to the lattice"}))


def run_one_flavour(args):
    """One-flavour DD-RHMC boundary term (--one-flavour [f64|f32] [N]) on the
    16^4 x 12 Moebius workload cut into two t-slabs of 16^3 x 8 (Omega and
    Omega-bar: D_dirichlet = D_Omega (+) D_Omega-bar): the type (N, N) fits of
    x^(1/4), x^(-1/2) and x^(-1/4) (dwf_rational_power) on [1e-6, 1.1 lam_max],
    then the heat bath phi = A_d^(-1/4) A^(1/4) eta, the action (checked:
    S(phi) = |eta|^2 up to the fits) and the link force, wall-clock per call
    with the multi-shift solves to 1e-10 (f32: FP32 operator with FP64 defect
    correction)."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    opt = args.one_flavour
    prec_name = opt[0] if opt else "f32"
    n = int(opt[1]) if len(opt) > 1 else 20
    inner = G.PREC[prec_name]
    tol = 1e-10
    dims, Ls = SMALL_DIMS, SMALL_LS
    rng = np.random.default_rng(SMALL_SEED)
    U = inputs.gauge_field(dims, "exp", eps=EPS, rng=rng)
    act = G.Action(M5, SMALL_MF, B5, C5)
    cut = [((0, 0, 0, 0), (dims[0], dims[1], dims[2], dims[3] // 2))]
    h = G.Handle(dims, Ls, act)
    hd = G.Handle(dims, Ls, act, cut=cut)
    Ut = torch.from_numpy(U.reshape(-1)).cuda()
    h.set_gauge(Ut)
    hd.set_gauge(Ut)
    for hh in (h, hd):
        hh.autotune(1, G.FP32)

    def lam_max(hh, iters=40):
        x = torch.randn(hh.cb_shape(1), dtype=torch.float64, device="cuda")
        t, y = torch.empty_like(x), torch.empty_like(x)
        lam = 0.0
        for _ in range(iters):
            x /= x.norm()
            hh.mpc(t, x)
            hh.mpc(y, t, dagger=True)
            lam = float((x * y).sum())
            x, y = y, x
        return lam

    hi = 1.1 * max(lam_max(h), lam_max(hd))
    lo = 1e-6
    t = time.time()
    fits = {a: G.rational_power(a, n, lo, hi) for a in (0.25, -0.25, -0.5)}
    fit_s = time.time() - t
    rat = {a: (f[0], f[1], f[2]) for a, f in fits.items()}
    eta = torch.empty(h.cb_shape(1), dtype=torch.float64, device="cuda")
    eta.normal_()
    phi = torch.empty_like(eta)
    out = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    del U

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.time()
        r = fn()
        torch.cuda.synchronize()
        return time.time() - t0, r

    # warm-up of every path, then one timed call each
    h.one_flavour_heatbath(hd, phi, eta, rat[-0.25], rat[0.25], tol=tol, inner=inner)
    t_hb, st_hb = timed(lambda: h.one_flavour_heatbath(hd, phi, eta, rat[-0.25], rat[0.25], tol=tol, inner=inner))
    t_act, (S, st_act) = timed(lambda: h.one_flavour_action(hd, phi, rat[0.25], rat[-0.5], tol=tol, inner=inner))
    h.one_flavour_force(hd, out, phi, rat[0.25], rat[-0.5], tol=tol, inner=inner)
    t_f, st_f = timed(lambda: h.one_flavour_force(hd, out, phi, rat[0.25], rat[-0.5], tol=tol, inner=inner))
    e2 = float((eta * eta).sum())

    def iters(st, counts):
        out_, k = [], 0
        for c in counts:
            out_.append(max(s["iters"] for s in st[k:k + c]))
            k += c
        return out_

    print(json.dumps({
        "workload": f"one-flavour DD-RHMC term, {SMALL_WORKLOAD}, Omega / Omega-bar the two 16^3 x 8 t-slabs",
        "prec": prec_name, "poles": n, "spectrum": [lo, hi], "fit_seconds": fit_s,
        "fit_delta": {str(a): f[3] for a, f in fits.items()},
        "heatbath_s": t_hb, "action_s": t_act, "force_s": t_f,
        "action_over_eta2_minus_1": S[0] / e2 - 1.0,
        "cg_iters": {"heatbath": iters(st_hb, [n, n]), "action": iters(st_act, [n, n]),
                     "force": iters(st_f, [n, n, n])},
        "max_true_resid": max(s["true_resid"] for s in st_f),
        "force_norm": float(out.norm())}))


def run_boundary(args):
    """DD-HMC boundary operator at the default workload (--boundary [f32|f64]):
    Omega = the interior 14^4 box of the width-2 band.  Times the projector P,
    R^-1 phi (one D solve) and the force of |R^-1 phi|^2 (two solves, two force
    insertions), each after one warm-up call, solves to 1e-10 with the given
    inner precision; then R phi once (two FP64 Dirichlet CGNR solves)."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    prec_name = args.boundary[0] if args.boundary else "f32"
    prec = G.PREC[prec_name]
    rng = np.random.default_rng(SMALL_SEED)
    U = inputs.gauge_field(SMALL_DIMS, "exp", eps=EPS, seed=SMALL_SEED)
    h = G.Handle(SMALL_DIMS, SMALL_LS, G.Action(M5, SMALL_MF, B5, C5))
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    h.autotune(1, G.FP32)
    phi = h.pack(torch.from_numpy(inputs.gaussian_source(SMALL_DIMS, SMALL_LS, rng=rng).reshape(-1)).cuda())
    out = torch.empty_like(phi)
    force = torch.zeros(U.size * 2, dtype=torch.float64, device="cuda")
    del U
    res = {}

    def timed(name, fn):
        fn()
        torch.cuda.synchronize()
        t = time.time()
        r = fn()
        torch.cuda.synchronize()
        res[name + "_ms"] = (time.time() - t) * 1e3
        return r

    timed("project", lambda: h.boundary_project(out, phi, SMALL_BAND))
    st = timed("rinv", lambda: h.boundary_rinv(out, phi, SMALL_BAND, tol=1e-10, inner=prec))
    res["rinv_iters"] = st[0]["iters"]
    res["rinv_true_resid"] = st[0]["true_resid"]
    st = timed("force", lambda: h.boundary_force(force, phi, SMALL_BAND, tol=1e-10, inner=prec))
    res["force_iters"] = [s["iters"] for s in st]
    res["force_true_resid"] = max(s["true_resid"] for s in st)
    # the Hasenbusch ratio force against the Pauli-Villars (m_f = 1) boundary operator
    hp = G.Handle(SMALL_DIMS, SMALL_LS, G.Action(M5, 1.0, B5, C5))
    hp.set_gauge(torch.from_numpy(inputs.gauge_field(SMALL_DIMS, "exp", eps=EPS, seed=SMALL_SEED).reshape(-1)).cuda())
    st = timed("ratio_force", lambda: h.boundary_ratio_force(hp, force, phi, SMALL_BAND, tol=1e-10, inner=prec))
    res["ratio_force_iters"] = [s["iters"] for s in st]
    res["ratio_force_true_resid"] = max(s["true_resid"] for s in st)
    del hp
    # R itself: two FP64 Dirichlet CGNR solves (Omega-bar, then Omega), timed once
    torch.cuda.synchronize()
    t = time.time()
    st = h.boundary_r(out, phi, SMALL_BAND, tol=1e-10)
    torch.cuda.synchronize()
    res["r_ms"] = (time.time() - t) * 1e3
    res["r_iters"] = [s["iters"] for s in st]
    res["r_true_resid"] = max(s["true_resid"] for s in st)
    print(json.dumps({"workload": "DD-HMC boundary operator, " + SMALL_WORKLOAD
                      + f", Omega = {SMALL_BAND}", "inner": prec_name, **res}))


def run_chebyshev(args):
    """Chebyshev filter (--chebyshev ORDER [f32|f64]) of the Shamir D_Omega
    normal Schur operator on the 14^4 interior box of the 16^4 x Ls=12 lattice
    (the local-solve setting of Sec. 4), applied to 8 Gaussian vectors at once:
    hi = 1.05 x the top of the spectrum from 30 power iterations, lo = hi / 50.
    Reports the time per filter and the drop of the Rayleigh quotient
    <v, A v> / <v, v> (mean over the vectors)."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    order = int(args.chebyshev[0]) if args.chebyshev else 30
    prec_name = args.chebyshev[1] if len(args.chebyshev) > 1 else "f32"
    prec = G.PREC[prec_name]
    nvec = 8
    from paper_2203_17119_gb300 import inputs
    U = inputs.gauge_field(SMALL_DIMS, "exp", eps=EPS, seed=SMALL_SEED)
    h = G.Handle(SMALL_DIMS, SMALL_LS, G.Action(M5, SMALL_MF, 1.0, 0.0), boxes=[SMALL_BAND], nrhs_max=nvec)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    del U
    h.autotune(nvec, G.FP32)
    g = torch.Generator(device="cuda").manual_seed(SMALL_SEED)
    v = torch.randn(h.cb_shape(1, nvec), dtype=torch.float64, device="cuda", generator=g).to(G._DTYPE[prec])
    t1, t2 = torch.empty_like(v), torch.empty_like(v)

    def A(dst, src):
        h.mpc(t1, src, prec=prec, nrhs=nvec)
        h.mpc(dst, t1, dagger=True, prec=prec, nrhs=nvec)

    def rq(x):
        A(t2, x)
        xr, ar = x.double().view(-1, 12, nvec, SMALL_LS, 2), t2.double().view(-1, 12, nvec, SMALL_LS, 2)
        num = (xr * ar).sum(dim=(0, 1, 3, 4))
        den = (xr * xr).sum(dim=(0, 1, 3, 4))
        return (num / den).cpu().numpy()

    x = v.clone()
    for _ in range(30):
        A(t2, x)
        x = t2 / t2.double().norm().to(t2.dtype)
    lam_max = float(rq(x).max())
    hi, lo = 1.05 * lam_max, 1.05 * lam_max / 50.0
    out = torch.empty_like(v)
    h.chebyshev_filter(out, v, order, lo, hi, prec=prec, nrhs=nvec)   # warm-up
    torch.cuda.synchronize()
    t = time.time()
    h.chebyshev_filter(out, v, order, lo, hi, prec=prec, nrhs=nvec)
    torch.cuda.synchronize()
    sec = time.time() - t
    rq0, rq1 = rq(v), rq(out)
    print(json.dumps({"workload": "Chebyshev filter of the Shamir D_Omega normal Schur operator, 16^4 x Ls=12, "
                      f"Omega = {SMALL_BAND}, {nvec} vectors", "prec": prec_name, "order": order,
                      "lo": lo, "hi": hi, "ms": sec * 1e3,
                      "ms_per_A_per_vector": sec * 1e3 / order / nvec,
                      "rayleigh_before": float(np.mean(rq0)), "rayleigh_after": float(np.mean(rq1))}))


def run_large(args):
    """The paper's per-GPU volume (--large): Moebius 32^4 x Ls=16, m_f = 0.005,
    exp(i 0.3 H) links; mixed FP32/FP64 CGNE to 1e-10 of D and of D_Omega for
    Dirichlet bands of width 1, 2 and 4 (the interior boxes), one solve each
    (graph capture included), default kernel configuration.  One JSON line per
    solve, flushed as it completes."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    dims, Ls, mf = (32, 32, 32, 32), 16, 0.005
    rng = np.random.default_rng(SEED)
    U = inputs.gauge_field(dims, "exp", eps=EPS, rng=rng)
    src = inputs.gaussian_source(dims, Ls, rng=rng)
    Ut = torch.from_numpy(U.reshape(-1)).cuda()
    del U
    act = G.Action(M5, mf, B5, C5)
    for name, w in (("D", 0), ("D_Omega_w1", 1), ("D_Omega_w2", 2), ("D_Omega_w4", 4)):
        box = ((w // 2,) * 4, (32 - w,) * 4) if w else None
        h = G.Handle(dims, Ls, act, boxes=[box] if box else None)
        h.set_gauge(Ut)
        if box:
            o, e = box
            canon = np.ascontiguousarray(src[o[3]:o[3] + e[3], o[2]:o[2] + e[2], o[1]:o[1] + e[1],
                                             o[0]:o[0] + e[0]])
        else:
            canon = src
        b = h.pack(torch.from_numpy(canon.reshape(-1)).cuda())
        del canon
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t = time.time()
        st, rc = h.cgne_solve(x, b, tol=1e-10, inner=G.FP32, allow_fail=True)
        torch.cuda.synchronize()
        sec = time.time() - t
        print(json.dumps({"workload": "Moebius DWF 32^4 x Ls=16, m_f=0.005, exp(i 0.3 H) links, mixed "
                          "FP32/FP64 CGNE to 1e-10", "operator": name, "box": box, "ms": sec * 1e3,
                          "iters": st[0]["iters"], "reliable_updates": st[0]["reliable_updates"],
                          "true_resid": st[0]["true_resid"], "status": rc}), flush=True)
        del h, b, x
        torch.cuda.empty_cache()


def run_mg(args):
    """Two-level multigrid for the local solves (--mg [NVEC] [ORDER] [BLOCK] [STEPS]):
    Shamir D_Omega of the 14^4 interior box of the 16^4 x Ls=12 lattice (the
    setting of Sec. 4).  Set-up = Chebyshev filter of NVEC Gaussian vectors
    (ORDER applications of A, [hi/50, hi], hi = 1.05 x the top of the spectrum
    from power iteration) + block aggregation (blocks BLOCK^4) + Galerkin
    coarse operator; solve = flexible GCR with the V-cycle (Chebyshev
    smoother, STEPS steps on [hi/10, hi]) to 1e-10.  Against one red-black solve:
    the mixed-precision CGNE and plain FP64 CG of the same system."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    nvec = int(args.mg[0]) if args.mg else 12
    order = int(args.mg[1]) if len(args.mg) > 1 else 30
    blk = int(args.mg[2]) if len(args.mg) > 2 else 7
    rng = np.random.default_rng(SMALL_SEED)
    U = inputs.gauge_field(SMALL_DIMS, "exp", eps=EPS, rng=rng)
    src = inputs.gaussian_source(SMALL_DIMS, SMALL_LS, rng=rng)
    h = G.Handle(SMALL_DIMS, SMALL_LS, G.Action(M5, SMALL_MF, 1.0, 0.0), boxes=[SMALL_BAND], nrhs_max=nvec)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    h.autotune(1, G.FP32)
    b = h.pack(torch.from_numpy(np.ascontiguousarray(_box_source(src, SMALL_BAND))).cuda())
    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda").manual_seed(SMALL_SEED)
    # top of the spectrum of A (FP32 power iteration)
    x = torch.randn(h.cb_shape(1), device="cuda", generator=g)
    t, y = torch.empty_like(x), torch.empty_like(x)
    lam = 0.0
    for _ in range(30):
        x /= x.norm()
        h.mpc(t, x, prec=G.FP32)
        h.mpc(y, t, dagger=True, prec=G.FP32)
        lam = float((x * y).sum())
        x, y = y, x
    hi = 1.05 * lam
    res = {"workload": "Shamir DWF D_Omega, 16^4 x Ls=12 (M5=1.8, m_f=0.01), Omega = the 14^4 interior box",
           "nvec": nvec, "filter_order": order, "block": [blk] * 4, "lam_max": lam,
           "smoother": f"Chebyshev iteration, {int(args.mg[3]) if len(args.mg) > 3 else 3} steps on [hi/10, hi]"}

    steps = int(args.mg[3]) if len(args.mg) > 3 else 3

    def setup():
        V0 = torch.randn(h.cb_shape(1, nvec), device="cuda", generator=g)
        V = torch.empty_like(V0)
        h.chebyshev_filter(V, V0, order, hi / 50, hi, prec=G.FP32, nrhs=nvec)
        mg = G.MG(h, (blk,) * 4, nvec)
        mg.setup(V)
        mg.set_smoother("chebyshev", steps, hi / 10, hi)
        return mg

    mg = setup()                       # warm-up (kernels, workspaces)
    (mg, ms) = _event_ms(setup, stream)
    res["setup_ms"] = round(ms, 2)
    res["coarse_unknowns"] = mg.sizes()[1]
    for name, fn in (("gcr_mg", lambda xx: h.gcr_solve_mg(xx, b, mg, tol=1e-10)),
                     ("gcr_plain", lambda xx: h.gcr_solve(xx, b, tol=1e-10)),
                     ("cgne_mixed", lambda xx: h.cgne_solve(xx, b, tol=1e-10, inner=G.FP32)),
                     ("cgne_fp64", lambda xx: h.cgne_solve(xx, b, tol=1e-10, inner=G.FP64))):
        xx = torch.zeros_like(b)
        fn(xx)
        xx.zero_()
        (st, ms) = _event_ms(lambda: fn(xx), stream)
        res[name] = {"ms": round(ms, 2), "iters": st[0][0]["iters"], "true_resid": st[0][0]["true_resid"],
                     "fallback_to_cg": st[0][0]["recorded"] == -1}
    res["setup_plus_solve_ms"] = round(res["setup_ms"] + res["gcr_mg"]["ms"], 2)
    res["vs_one_red_black_solve"] = round(res["cgne_mixed"]["ms"] / res["setup_plus_solve_ms"], 3)
    print(json.dumps(res))


def run_learned(args):
    """The learned preconditioner at the configuration it is quoted on
    (--learned [SOURCES] [ITERATES]): K trained on the GPU (library kernels)
    on (residual, error) pairs from FP64 solves at 16^4 x Ls=12, m_f = 0.005,
    then used at 24^4 x Ls=16, m_f = 0.005: GCR with K, GCR without it, GCR
    with the two-level multigrid (Chebyshev smoother / K as smoother), mixed
    CG and FP64 CG to 1e-10 on a held-out source."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    from paper_2203_17119_gb300 import train as TR
    sources = int(args.learned[0]) if args.learned else 16
    iterates = int(args.learned[1]) if len(args.learned) > 1 else 64
    act = G.Action(M5, 0.005, B5, C5)
    dims, Ls, batch = SMALL_DIMS, SMALL_LS, 4
    rng = np.random.default_rng(1004)
    U = inputs.gauge_field(dims, "exp", eps=EPS, rng=rng)
    Ut = torch.from_numpy(U.reshape(-1)).cuda()
    h1 = G.Handle(dims, Ls, act, nrhs_max=1)
    h1.set_gauge(Ut)
    hb = G.Handle(dims, Ls, act, nrhs_max=batch)
    hb.set_gauge(Ut)
    K = TR.initial_network(B5 * (4 - M5) + 1)
    t0 = time.time()
    npairs, loss0, loss1 = 0, None, None
    for s in range(sources):
        b = inputs.gaussian_source(dims, Ls, rng=rng)
        r, e = TR.make_pairs(h1, torch.from_numpy(b.reshape(-1)).cuda(), iterates, record_every=4)
        npairs += r.shape[0]
        losses = TR.train(K, hb, r, e, steps=16, batch=batch, lr=1e-3, seed=s, loss_kind="a2")
        loss0 = losses[0] if loss0 is None else loss0
        loss1 = losses[-1]
        del r, e
    train_s = time.time() - t0
    del h1, hb, Ut
    torch.cuda.empty_cache()
    ev = TR.evaluate(K, (24, 24, 24, 24), 16, act)
    print(json.dumps({"workload": "learned preconditioner: trained at 16^4 x Ls=12, used at 24^4 x Ls=16, "
                                  "Moebius m_f=0.005, exp(i 0.3 H) links",
                      "train_pairs": npairs, "train_seconds": round(train_s, 1),
                      "train_loss_first_last": [loss0, loss1], "eval": ev}))


def run_nn(args):
    """One application of the learned preconditioner K (dwf_nn_apply, the form
    GCR and the multigrid smoother use): --nn L Ls [nrhs], random BF16-exact
    weights, CUDA events around each application on the launching stream.  The
    network's intermediate fields (11 transported and 11 mixed fields of the
    whole lattice) are larger than L2 at the sizes it is timed on, so no flush.
    mix_tflops counts the folded mixes' multiply-adds: per (site, colour, lane)
    32 x 32 complex on even sites and 12 x 12 on odd sites."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    L, Ls = int(args.nn[0]), int(args.nn[1])
    nrhs = int(args.nn[2]) if len(args.nn) > 2 else 1
    dims = (L, L, L, L)
    U = inputs.gauge_field(dims, "exp", eps=EPS, seed=SMALL_SEED)
    h = G.Handle(dims, Ls, G.Action(M5, MF, B5, C5), nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    del U
    rng = np.random.default_rng(1005)

    def bf16(a):
        return torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).double().numpy()

    W1 = bf16(rng.standard_normal((11, 16, 1, 4, 4)) * 0.1) + 1j * bf16(rng.standard_normal((11, 16, 1, 4, 4)) * 0.1)
    W2 = bf16(rng.standard_normal((11, 1, 16, 4, 4)) * 0.1) + 1j * bf16(rng.standard_normal((11, 1, 16, 4, 4)) * 0.1)
    K = G.NN()
    K.set_weights(W1, W2)
    x = torch.randn(h.cb_shape(1, nrhs), dtype=torch.float32, device="cuda")
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        K.apply(h, out, x, nrhs, stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(max(1, args.steps)):
        _, ms = _event_ms(lambda: K.apply(h, out, x, nrhs, stream), stream)
        times.append(ms)
    ms = float(np.median(times))
    half = L ** 4 // 2
    flops = 8.0 * (32 * 32 + 12 * 12) * half * 3 * Ls * nrhs
    print(json.dumps({"workload": f"learned preconditioner K applied on {L}^4 x Ls={Ls}, nrhs={nrhs}",
                      "ms": ms, "ms_all": times, "mix_gflop": flops / 1e9,
                      "mix_tflops": flops / (ms * 1e-3) / 1e12, "l2_flush": "none (fields > L2)"}))


BATCH_BOXES = [((0, 0, 0, 0), (8, 8, 8, 8)), ((0, 0, 0, 0), (8, 8, 12, 12)),
               ((0, 0, 0, 0), (12, 12, 12, 12)), ((0, 0, 0, 0), (12, 12, 16, 16)),
               ((0, 0, 0, 0), (16, 16, 16, 12)), ((0, 0, 0, 0), (16, 16, 16, 16))]


def batched_result(nrhs, prec_name="f32", steps=5, seed=1002):
    """Six standalone Dirichlet boxes of uneven extents (8^4 ... 16^4) inside a
    24^4 x Ls=16 Moebius lattice, nrhs right-hand sides each: the hop and a
    mixed-precision CGNE of all 6 * nrhs systems in one persistent launch per
    kernel, autotuned; returns the result dict."""
    import numpy as np
    import torch
    from paper_2203_17119_gb300 import dwf as G
    from paper_2203_17119_gb300 import inputs
    prec = G.PREC[prec_name]
    dims, Ls = (24, 24, 24, 24), 16
    rng = np.random.default_rng(seed)
    U = inputs.gauge_field(dims, "exp", eps=EPS, rng=rng)
    h = G.Handle(dims, Ls, G.Action(M5, SMALL_MF, B5, C5), boxes=BATCH_BOXES, nrhs_max=nrhs)
    h.set_gauge(torch.from_numpy(U.reshape(-1)).cuda())
    del U
    T = h.autotune(nrhs, prec)
    vol = sum(int(np.prod(e)) for _, e in BATCH_BOXES)
    # sources: per box and rhs, Gaussian on the box sites (canonical layout)
    canon = torch.from_numpy(inputs.gaussian_source((vol * nrhs, 1, 1, 1), Ls, rng=rng).reshape(-1)).cuda()
    b = h.pack(canon, nrhs)
    del canon
    word = {G.FP64: 8, G.FP32: 4, G.BF16: 2}[prec]
    inp = b[h.nsite[0]:].to(G._DTYPE[prec]).contiguous()
    out = h.empty_cb(0, nrhs, prec)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(3):
        h.hop(out, inp, 0, prec=prec, nrhs=nrhs)
    ts = []
    for _ in range(max(steps, 5)):
        flush.fill_(1.0)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.hop(out, inp, 0, prec=prec, nrhs=nrhs)
        e.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(e))
    ms = statistics.mean(ts)
    sites = h.nsite[0] * Ls * nrhs     # output 5D sites of one hop (all boxes, all rhs)
    nbytes = (48.0 + 144.0 / (Ls * nrhs)) * word * sites
    del inp, out, flush
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    t0 = time.time()
    st, rc = h.cgne_solve(x, b, nrhs=nrhs, tol=1e-10, inner=prec, allow_fail=True)
    torch.cuda.synchronize()
    secs = time.time() - t0
    res = {"workload": "6 Dirichlet boxes 8^4..16^4 in 24^4 x Ls=16, Moebius m_f=0.01", "nrhs": nrhs,
           "prec": prec_name, "tile_sites": T, "systems": len(st), "hop_ms": round(ms, 4),
           "hop_tflops": round(FLOPS_PER_SITE * sites / (ms * 1e-3) / 1e12, 3),
           "hop_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1), "solve_seconds": round(secs, 3),
           "solve_status": rc, "max_iters": max(s["iters"] for s in st),
           "max_true_resid": max(s["true_resid"] for s in st),
           "seconds_per_system": round(secs / len(st), 4)}
    del h, b, x
    torch.cuda.empty_cache()
    return res


def run_batched(args):
    """--batched NRHS [f32|bf16]: batched_result as one JSON line."""
    print(json.dumps(batched_result(int(args.batched[0]), args.batched[1] if len(args.batched) > 1 else "f32",
                                    args.steps)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batched", nargs="+", metavar="ARG",
                    help="six uneven Dirichlet boxes in 24^4 x 16: NRHS [f32|bf16]")
    ap.add_argument("--multishift", nargs="+", metavar="ARG",
                    help="NSHIFT [f64|f32]: multi-shift CG against single-shift solves")
    ap.add_argument("--learned", nargs="*", metavar="ARG",
                    help="train K at 16^4 x 12, evaluate at 24^4 x 16: [SOURCES] [ITERATES]")
    ap.add_argument("--mg", nargs="*", metavar="ARG",
                    help="multigrid local solve: [NVEC] [ORDER] [BLOCK] (Sec. 4 setting)")
    ap.add_argument("--large", action="store_true",
                    help="32^4 x 16 m_f = 0.005 solves of D and of D_Omega, bands 1, 2, 4")
    ap.add_argument("--chebyshev", nargs="*", metavar="ARG",
                    help="Chebyshev filter of the local normal operator: [ORDER] [f32|f64]")
    ap.add_argument("--boundary", nargs="*", metavar="ARG",
                    help="boundary operator P, R^-1 and the boundary-action force: [f32|f64]")
    ap.add_argument("--one-flavour", nargs="*", metavar="ARG",
                    help="[f64|f32] [N]: the one-flavour DD-RHMC heat bath, action and force")
    ap.add_argument("--force", nargs="*", metavar="ARG",
                    help="link force of Re <X, D Y>: [f64|f32] [L] [Ls]")
    ap.add_argument("--nn", nargs="+", metavar="ARG",
                    help="L Ls [nrhs]: time one application of the learned preconditioner K")
    ap.add_argument("--hop", nargs="+", metavar="ARG",
                    help="bare hop only: L Ls prec(f64|f32|bf16) [nrhs]")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tc", action="store_true", help="--hop bf16: the tensor-core kernel")
    ap.add_argument("--chunk", type=int, default=0, help="--hop: consecutive tiles per CTA")
    ap.add_argument("--tile-order", nargs=2, type=int, metavar=("BZ", "BT"),
                    help="--hop: tiles blocked in (z, t) by BZ x BT planes")
    ap.add_argument("--hop-config", nargs=2, type=int, metavar=("TILE", "VL"),
                    help="--hop: fixed sites per tile and lanes per thread instead of autotuning")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-cg", action="store_true", help="skip the plain FP64 CG solves")
    ap.add_argument("--no-small", action="store_true", help="skip the 16^4 x 12 extra keys")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 24^4 x 16 extra key")
    ap.add_argument("--config", nargs=3, type=int, metavar=("TILE", "VL", "CHUNK"),
                    help="default workload: fixed kernel configuration instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    if args.multishift:
        run_multishift(args)
        return
    if args.force is not None:
        run_force(args)
        return
    if args.one_flavour is not None:
        run_one_flavour(args)
        return
    if args.boundary is not None:
        run_boundary(args)
        return
    if args.chebyshev is not None:
        run_chebyshev(args)
        return
    if args.large:
        run_large(args)
        return
    if args.mg is not None:
        run_mg(args)
        return
    if args.learned is not None:
        run_learned(args)
        return
    if args.nn:
        run_nn(args)
        return
    if args.hop:
        run_hop(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(env_int("LOCAL_RANK", 0))
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = cpu_baseline(res["iters"]["D"])
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
