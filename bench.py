#!/usr/bin/env python
"""Benchmark: delivered bubble points/s of the one-loop Keldysh bubble in all three
channels on the mixed-precision workload (K1 401, K2 101x101, K3 51^3, 4001
Gauss-Lobatto nodes, complex64 vertex storage; U/Delta = 2, T = 0.05).

One step = one bubble B_r(Gamma, Gamma) (Pi = G G) for r = a, p, t, every class
(K1, K2, K2', K3) of each channel, from the seeded SIAM-shaped vertex resident in HBM.
A delivered point is one (w, v, v') x one of the 16 Keldysh components of one class of
one channel: 7,365,792 per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64] [--impl reference]
                 [--channels apt] [--no-e2e] [--no-cpu-baseline] [--workload step|points32|vjp]

--channels and --no-e2e narrow a run to one channel's kernels for profiling captures; the
default line is the three-channel step.

Under torchrun (N > 1) every rank runs its own independent parameter point (weak
scaling, no data-path collective); value = points of all ranks / max-over-ranks time.
--impl reference times the FP64 CPU oracle (the reference arm of this method) on a
bounded sample of the same workload.
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRIDS = dict(n1=401, n2w=101, n2v=101, n3w=51, n3v=51)
NQ, U, DELTA, T = 4001, 2.0, 1.0, 0.05
WORKLOAD = "one-loop bubble a,p,t; K1 401, K2 101x101, K3 51^3, 16 Keldysh comps, Nq 4001, c64 vertex"
METRIC = "bubble points/s (w.v.v'.Keldysh) at <=1e-6 rel err vs plain FP64 GPU"


def class_points(g):
    return {"K1": g["n1"] * 16, "K2": g["n2w"] * g["n2v"] * 16, "K2p": g["n2w"] * g["n2v"] * 16,
            "K3": g["n3w"] * g["n3v"] ** 2 * 16}


POINTS_PER_STEP = 3 * sum(class_points(GRIDS).values())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# FP64 FMA pipe: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (max SM clock);
# measured 1.20 TFLOP/s with a register-resident FMA loop on this GPU model.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 pipe: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz; measured 70 TFLOP/s.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# TF32 tensor peak: measured dense bf16 (MEASURED_PEAKS.json) x the nominal tf32/bf16 ratio
# (1.1 / 2.25 PFLOP/s dense).
TF32_OVER_BF16 = 1.1 / 2.25


def mixed_kernel_work(channels=(0, 1, 2), t_su2=False):
    """Algorithmic work per step of the symmetric mixed path, by kernel (flops).
    Gather kernels: every interpolation corner adds 16 complex values times a real weight
    (64 flops); a record (one (w, v, node) of one spin term) has nominally 44 corners in
    the up-down component (own K3 8 + two other channels x (K1 2 + K2 4 + K2' 4 + K3 8));
    the up-up one adds the exchanged term (each lookup again at the exchanged legs: 44 more),
    so a t record, which needs both spin components, has 88; the fused K2 kernel
    adds the 4x4x4 complex contraction (512 flops), the K3 tile kernel the Pi fold of the
    right record (512 flops; p folds two, the record and its crossing image) and the own K2
    class (4 corners).  Symmetric mode: a, t compute w >= 0, p computes v >= 0 of K2 and K3.
    K3 contraction: 8 M N K useful flops per bosonic frequency (M = N = 4 n3v, K = 4 ns nq);
    the 3xTF32 split issues three times that on the tensor pipe."""
    g = GRIDS
    nq = NQ
    half = lambda n: n - n // 2
    w = {}
    # k_mx_k2 (K2 only; K2' is filled by symmetry)
    rec_a = half(g["n2w"]) * g["n2v"] * (nq - 2)
    rec_p = g["n2w"] * half(g["n2v"]) * (nq - 2)
    rec_t = half(g["n2w"]) * g["n2v"] * (nq - 2)
    # the own K3 lookups (8 corners of 44) are taken through node-weighted sums outside the
    # node loop, so a record gathers 36 corners (t: 72)
    w["k_mx_k2"] = ((0 in channels) * rec_a + (1 in channels) * rec_p) * (36 * 64 + 512) + \
        (2 in channels) * rec_t * ((36 + 36) * 64 + 2 * 512)
    # k_mx_tile3_both
    r3a = half(g["n3w"]) * g["n3v"] * nq
    r3p = g["n3w"] * half(g["n3v"]) * nq
    r3t = half(g["n3w"]) * g["n3v"] * nq
    # t in its SU(2) form: one density record per side (both lookups, one Pi fold)
    w["k_mx_tile3_both"] = (0 in channels) * r3a * (48 * 64 + 512) + (1 in channels) * r3p * (48 * 64 + 2 * 512) + \
        (2 in channels) * r3t * ((48 + 48) * 64 + (1 if t_su2 else 2) * 512)
    # k_tc_k3 (useful): 8 flops per complex multiply-add of the points the method needs, i.e.
    # a, t: the pairs v <= v' (the others are conjugation images, and the contraction skips
    # the output blocks that hold only v > v'; the diagonal blocks it computes in full are
    # not credited); p: rows v >= 0 (the rest by crossing), all v'
    N = 4 * g["n3v"]
    n3 = g["n3v"]
    tc = 0.0
    for r, nw in ((0, half(g["n3w"])), (1, g["n3w"]), (2, half(g["n3w"]))):
        if r not in channels:
            continue
        ns = 2 if (r == 2 and not t_su2) else 1      # the SU(2) form contracts one density record
        MN = 4 * half(n3) * N if r == 1 else 16 * n3 * (n3 + 1) // 2
        tc += 8.0 * MN * (4 * ns * nq) * nw
    w["k_tc_k3"] = tc
    return w


# DRAM bytes (read + write) of one launch of each timed kernel, from ncu captures of the
# a-channel bubble of this workload (dram__bytes_read.sum + dram__bytes_write.sum; the
# commands are in profiles/).  The K3 kernels' traffic grows with the bosonic frequencies of
# a launch; these are the figures of the captured launches (26 frequencies).
NCU_TRAFFIC = {"k_mx_k2": 79.61e6, "k_mx_tile3_both": 2.830e9, "k_tc_k3": 3.463e9}


def roofline_entry(name, ms_total, steps, work, bf16_peak, traffic=None):
    if name not in work or ms_total <= 0:
        return None
    if traffic is None:
        traffic = NCU_TRAFFIC.get(name)
    flops = work[name] * steps
    if name == "k_tc_k3":
        peak = bf16_peak * TF32_OVER_BF16
        issued = 3.0 * flops / (ms_total / 1e3) / 1e12
        return {"kernel": name, "bound": "tensor", "achieved": issued, "peak": peak, "unit": "TFLOP/s",
                "frac": issued / peak, "traffic": traffic,
                "note": "issued TF32 flops (3 MMAs per useful product); useful = achieved / 3; peak = measured "
                        "bf16 x nominal tf32/bf16 ratio"}
    ach = flops / (ms_total / 1e3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP32_PEAK_TFLOPS, "traffic": traffic,
            "note": "algorithmic interpolation + contraction flops (see mixed_kernel_work); peak = FP32 pipe "
                    "152 SMs x 128 lanes x 2 x 2.07 GHz"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def weak_scaling_value(points_per_rank, ms_local, dist=None, device="cpu"):
    """Whole-job throughput of a weak-scaling run: every rank processes points_per_rank
    points per step; the job's step time is the maximum of the ranks' times.  Returns
    (points/s over all ranks, max step time in ms)."""
    import torch
    ws = dist.get_world_size() if dist is not None else 1
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ws * points_per_rank / (ms_max / 1e3), ms_max


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# --------------------------------------------------------------------------------------
def oracle_rate(budget_s=12.0, seed=0, nthreads=0):
    """Oracle points/s on a stratified sample of the workload (all channels and classes,
    sample sizes scaled to roughly budget_s of CPU time) on nthreads threads (0: all host
    cores); returns (rate, threads, description, elapsed)."""
    import seeded as S
    from oracle import oracle as O
    ch = S.seeded_vertex(GRIDS, U, seed=seed)
    c64 = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    V = O.Vertex(GRIDS, U=U, has_R=True, channels=c64)
    P = O.Prop(Delta=DELTA, T=T)
    rng = np.random.default_rng(seed)
    shapes = {"K1": (GRIDS["n1"],), "K2": (GRIDS["n2w"], GRIDS["n2v"]), "K2p": (GRIDS["n2w"], GRIDS["n2v"]),
              "K3": (GRIDS["n3w"], GRIDS["n3v"], GRIDS["n3v"])}
    cores = nthreads or os.cpu_count() or 1
    # calibrate on a few K3 points
    idx = [tuple(int(rng.integers(0, n)) for n in shapes["K3"]) for _ in range(max(4, cores))]
    t0 = time.perf_counter()
    O.bubble_class(V, V, P, 0, "K3", NQ, idx=idx, nthreads=nthreads)
    per_pt = (time.perf_counter() - t0) / len(idx)
    n_k3 = int(max(cores, min(4096, budget_s / 3 / 1.6 / max(per_pt, 1e-6))))
    n_small = max(cores, n_k3 // 4)
    est, sampled, elapsed = 0.0, 0, 0.0
    for r in range(3):
        for cls, n in (("K1", n_small), ("K2", n_small), ("K2p", n_small), ("K3", n_k3)):
            idx = [tuple(int(rng.integers(0, m)) for m in shapes[cls]) for _ in range(n)]
            t0 = time.perf_counter()
            O.bubble_class(V, V, P, r, cls, NQ, idx=idx, nthreads=nthreads)
            dt = time.perf_counter() - t0
            elapsed += dt
            sampled += n
            est += dt / n * int(np.prod(shapes[cls]))
    rate = POINTS_PER_STEP / est
    desc = ("stratified random sample of %d output points (%d per K3, %d per K1/K2/K2' class, 3 channels), "
            "%.1f s CPU wall; whole-step time extrapolated per class" % (sampled, n_k3, n_small, elapsed))
    return rate, cores, desc, elapsed


def oracle_loop_rate(grids, channels, budget_s=10.0, seed=0):
    """Oracle self-energy loop rate (integrand evaluations/s) on a random sample of the loop
    workload's frequencies (the K1 grid), sized to about budget_s of CPU time; returns (rate,
    cores, description)."""
    import seeded as S
    from oracle import oracle as O
    V = O.Vertex(grids, U=U, has_R=True, channels=channels)
    P = O.Prop(Delta=DELTA, T=T)
    nus = S.grid_freqs(grids["n1"])
    rng = np.random.default_rng(seed)
    cores = os.cpu_count() or 1
    m = min(cores, len(nus))
    t0 = time.perf_counter()
    O.loop(V, P, NQ, nus[rng.integers(0, len(nus), size=m)])          # one frequency per thread
    per = (time.perf_counter() - t0) / m
    n = int(max(1, min(len(nus), budget_s / max(per, 1e-9))))
    pick = nus if n == len(nus) else nus[rng.integers(0, len(nus), size=n)]
    t0 = time.perf_counter()
    O.loop(V, P, NQ, pick)
    el = time.perf_counter() - t0
    desc = ("%s of the K1 grid x %d interior nodes, %.1f s CPU wall"
            % ("all %d frequencies" % n if n == len(nus) else "%d random frequencies" % n, NQ - 2, el))
    return n * (NQ - 2) / el, cores, desc


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    times = []
    for _ in range(args.warmup):
        oracle_rate(budget_s=3.0)
    vals = []
    for _ in range(args.steps):
        rate, cores, desc, el = oracle_rate(budget_s=args.ref_budget)
        vals.append(rate)
        times.append(el)
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * POINTS_PER_STEP / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points_per_step": POINTS_PER_STEP},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------
def contraction_flops(prec):
    """Useful (complex-as-real) flops of the contractions per step by kernel family."""
    g = GRIDS
    out = {}
    for r in range(3):
        ns = 2 if r == 2 else 1
        K = 4 * ns * NQ
        for cls, nw, nL, nR in (("K1", g["n1"], 1, 1), ("K2", g["n2w"], g["n2v"], 1),
                                ("K2p", g["n2w"], 1, g["n2v"]), ("K3", g["n3w"], g["n3v"], g["n3v"])):
            out[(r, cls)] = 8.0 * nw * (4 * nL) * (4 * nR) * K
    return out


# --------------------------------------------------------------------------------------
# Secondary workloads (not the default line): the batching and the adjoint paths
# --------------------------------------------------------------------------------------
def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def run_points32(args):
    """32 independent parameter points of uneven grid sizes (U/Delta ~ U[0.5, 3], T ~ log-
    uniform in [0.005, 0.5], K3 n^3 with n in {21, 31, 41, 51, 61}, K2 (2n-1)^2, K1 5n-4,
    Nq 4001), the one-loop bubble of all three channels of each, mixed precision: one step
    graph with one branch per point, against the same bubbles launched eagerly."""
    import torch
    import seeded as S
    from paper_2405_20996_gb300.engine import Engine, StepGraph
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(2024)
    pts, points, sizes = [], 0, []
    for i in range(32):
        n = int(rng.choice([21, 31, 41, 51, 61]))
        Ui = float(rng.uniform(0.5, 3.0))
        Ti = float(10 ** rng.uniform(np.log10(0.005), np.log10(0.5)))
        g = dict(n1=5 * n - 4, n2w=2 * n - 1, n2v=2 * n - 1, n3w=n, n3v=n)
        e = Engine(g, NQ, device=0)
        e.set_model(DELTA, Ti)
        e.set_workspace_limit(2 << 30)
        e.set_vertex(0, U=Ui, has_R=True, channels=S.seeded_vertex(g, Ui, seed=3000 + i), dtype=torch.complex64,
                     symmetric=True)
        e.alloc_out(1, dtype=torch.complex64)
        pts.append(e)
        sizes.append(n)
        points += 3 * sum(class_points(g).values())
    stream = torch.cuda.current_stream(dev)
    su2 = not args.no_t_su2          # each point's t bubble in its SU(2) form (its own a bubble's K3)
    descs = []
    for e in pts:
        descs += [e.desc(0, 0, 0, 1, precision="mixed"), e.desc(1, 0, 0, 1, precision="mixed")]
        descs += [e.desc_t_su2(0, 1), e.desc_t_su2_finish(1, e, 1)] if su2 else [e.desc(2, 0, 0, 1, precision="mixed")]
    graph = StepGraph(descs, device=dev)
    n0 = sum(e.launches() for e in pts)
    ms_graph = _timed(lambda: graph.launch(stream), args.steps, args.warmup, stream)
    launches = (sum(e.launches() for e in pts) - n0) // (args.steps + args.warmup)

    def eager():
        for e in pts:
            e.bubble(0, 0, 0, 1, precision="mixed", stream=stream)
            e.bubble(1, 0, 0, 1, precision="mixed", stream=stream)
            if su2:
                e.bubble_t_su2(0, 1, stream=stream)
                e.t_su2_finish(1, e.out(1, 0)["K3"], stream=stream)
            else:
                e.bubble(2, 0, 0, 1, precision="mixed", stream=stream)

    ms_eager = _timed(eager, args.steps, args.warmup, stream)
    line = {"metric": METRIC, "value": points / (ms_graph / 1e3), "unit": "points/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "32 parameter points, K3 n^3 n in {21..61}, K2 (2n-1)^2, K1 5n-4, Nq 4001, a,p,t",
                       "n3": sizes, "points_per_step": points, "launch": "one CUDA graph, one branch per point",
                       "t_channel": "SU(2) form" if su2 else "both spin terms contracted"},
            "eager": {"value": points / (ms_eager / 1e3), "ms_per_step": ms_eager}, "gpu_launches": launches}
    print(json.dumps(line))
    return 0


ML_SIZES = {
    # K1 201, K2 81^2, K3 41^3, Nq 4001, U/Delta = 2, T = 0.05
    "multiloop": (dict(n1=201, n2w=81, n2v=81, n3w=41, n3v=41), 4001, 2.0, 0.05),
    # the largest instance: K1 801, K2 201^2, K3 101^3, Nq 8001, U/Delta = 3, T = 0.01
    "multiloop-large": (dict(n1=801, n2w=201, n2v=201, n3w=101, n3v=101), 8001, 3.0, 0.01),
}


def run_multiloop(args):
    """Right-hand side of the six-loop flow for the vertex (Sec. III.C): per channel one
    one-loop bubble with the single-scale pair, then left / central / right parts up to
    l = 6 (15 bubbles per channel, 45 per step) plus the slot additions, mixed precision,
    one step graph with the channels as parallel branches and a join between loop orders;
    against the same entries launched eagerly on one stream."""
    import torch
    import seeded as S
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.multiloop import MultiloopStep
    g, nq, Ui, Ti = ML_SIZES[args.workload]
    dev = torch.device("cuda", 0)
    ml = MultiloopStep(g, nq, Ui, DELTA, Ti, S.seeded_vertex(g, Ui, seed=4242), n_loops=6, precision="mixed",
                       cache={"off": False, "auto": "auto", "all": True}[args.ml_cache])
    for e in ml.e.values():
        e.set_workspace_limit(args.ws_gb << 30)
        e.set_autotune(not args.no_autotune)
    stream = torch.cuda.current_stream(dev)
    nb = ml.parts_per_step()                 # delivered parts (order 2's right parts as symmetry images)
    points = nb * sum(class_points(g).values())
    graph = ml.build()

    def launches():
        return sum(e.launches() for e in ml.e.values())

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # 256 MB > 129 MB L2

    def timed(fn, steps, warmup, clk=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        c = ClockSampler(0) if clk else None
        evs = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / steps, (c.stop() if c else None)

    n0 = launches()
    ms_graph, clocks = timed(lambda: graph.launch(stream), args.steps, args.warmup, clk=True)
    per_step = (launches() - n0) // (args.steps + args.warmup)
    ms_eager, _ = timed(lambda: ml.run_eager(stream), args.steps, min(args.warmup, 1))
    for e in ml.e.values():
        kb.kb_profile_enable(e.ctx, True)
    flush.zero_()
    ml.run_eager(stream)
    torch.cuda.synchronize()
    prof = {}
    for e in ml.e.values():
        for k, (t, c) in kb.kb_profile_read(e.ctx).items():
            p0 = prof.get(k, (0.0, 0))
            prof[k] = (p0[0] + t, p0[1] + c)
        kb.kb_profile_enable(e.ctx, False)
    for e in ml.e.values():
        kb.kb_check_device(e.ctx)
    tot = max(sum(v[0] for v in prof.values()), 1e-30)
    # K3 contraction work of one step (useful flops; 3xTF32 issues three times that): the
    # one-loop bubble of the symmetric vertex computes the independent half (a, t: w >= 0;
    # p: rows v >= 0), every other part the full K3 (M = N = 4 n3v, K = 4 ns nq per w)
    half = lambda n: n - n // 2
    tc_useful = 0.0
    for x in ml.descs:
        if x.op != kb.KB_OP_BUBBLE:
            continue
        r, ns = x.channel, (2 if x.channel == 2 else 1)
        N = 4 * g["n3v"]
        M, nw = N, g["n3w"]
        if x.slot_left == x.slot_right:
            M, nw = (4 * half(g["n3v"]), g["n3w"]) if r == 1 else (N, half(g["n3w"]))
        tc_useful += 8.0 * M * N * 4 * ns * nq * nw
    roof = None
    if "k_tc_k3" in prof:
        _, bf16, _ = peaks()
        peak = bf16 * TF32_OVER_BF16
        issued = 3.0 * tc_useful / (prof["k_tc_k3"][0] / 1e3) / 1e12
        roof = {"kernel": "k_tc_k3", "bound": "tensor", "achieved": issued, "peak": peak, "unit": "TFLOP/s",
                "frac": issued / peak, "traffic": None, "share": prof["k_tc_k3"][0] / tot,
                "note": "issued TF32 flops of the step's K3 contractions / their CUDA-event time in one profiled "
                        "eager step; peak = measured bf16 x nominal tf32/bf16 ratio"}
    line = {"metric": METRIC, "value": points / (ms_graph / 1e3), "unit": "points/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "six-loop vertex flow step, a,p,t, K1 %d, K2 %dx%d, K3 %d^3, Nq %d, c64"
                                   % (g["n1"], g["n2w"], g["n2v"], g["n3w"], nq),
                       "bubbles_per_step": nb, "bubble_calls_per_step": ml.bubbles_per_step(),
                       "points_per_step": points, "U": Ui, "T": Ti,
                       "record_cache": {r: ml.cached[r] for r in ml.cached} or "off",
                       "l2": "flushed (256 MB write) before every timed step",
                       "launch": "one CUDA graph per step, channels as branches, a join per loop order"},
            "eager": {"value": points / (ms_eager / 1e3), "ms_per_step": ms_eager}, "gpu_launches": per_step,
            "roofline": roof, "clocks": clocks,
            "kernels_ms": {k: round(v[0], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}}
    print(json.dumps(line))
    ml.close()
    return 0


def run_parquet(args):
    """Parquet-approximation solve (Sec. III.B) at K1 201, K2 81^2, K3 41^3, Nq 4001,
    U/Delta = 2, T = 0.05 to a 1e-8 relative residual: Newton-Krylov with mixed-precision
    Jacobian products and FP64 residuals, beside the damped fixed point (mixing 0.5, FP64
    bubbles) capped at --fp-maxit iterations (its remaining iterations extrapolated from its
    measured contraction factor when the cap is reached), and Anderson acceleration of that
    iteration (memory 5) under the same cap."""
    import torch
    from paper_2405_20996_gb300.parquet import ParquetPA
    g = dict(n1=201, n2w=81, n2v=81, n3w=41, n3v=41)
    Ui, Ti, tol = 2.0, 0.05, 1e-8
    pa = ParquetPA(g, NQ, Ui, DELTA, Ti, jvp_precision="mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_nk, h_nk, lin = pa.newton_krylov(tol=tol, gmres_m=40, gmres_maxit=400)
    torch.cuda.synchronize()
    t_nk = time.perf_counter() - t0
    nk = {"seconds": t_nk, "newton_steps": len(h_nk) - 1, "gmres_products": lin, "residuals": h_nk,
          "fp64_bubbles": pa.bubbles, "mixed_bubbles": pa.mixed_bubbles}
    pa.bubbles = pa.mixed_bubbles = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_fp, h_fp = pa.fixed_point(mix=0.5, tol=tol, maxit=args.fp_maxit)
    torch.cuda.synchronize()
    t_fp = time.perf_counter() - t0
    fp = {"seconds": t_fp, "iterations": len(h_fp), "residual": h_fp[-1], "fp64_bubbles": pa.bubbles}
    if h_fp[-1] > tol and len(h_fp) > 10:
        rho = (h_fp[-1] / h_fp[-11]) ** 0.1               # contraction factor over the last 10
        more = float(np.log(tol / h_fp[-1]) / np.log(rho)) if rho < 1 else float("inf")
        fp["contraction_factor"] = rho
        fp["extrapolated_iterations"] = len(h_fp) + more
        fp["extrapolated_seconds"] = t_fp * (len(h_fp) + more) / len(h_fp)
    agree = pa.rel(g_fp - g_nk, g_nk) if h_fp[-1] <= tol else None
    pa.bubbles = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_aa, h_aa = pa.anderson(mix=0.5, m=5, tol=tol, maxit=args.fp_maxit)
    torch.cuda.synchronize()
    t_aa = time.perf_counter() - t0
    aa = {"seconds": t_aa, "iterations": len(h_aa), "residual": h_aa[-1], "fp64_bubbles": pa.bubbles,
          "memory": 5, "rel_diff_to_newton_krylov": pa.rel(g_aa - g_nk, g_nk) if h_aa[-1] <= tol else None}
    line = {"metric": "parquet solve time to 1e-8 relative residual", "value": t_nk, "unit": "s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 residual, f32 Jacobian products", "data": "synthetic",
            "config": {"workload": "parquet approximation, K1 201, K2 81x81, K3 41^3, Nq 4001, U/Delta 2, T 0.05",
                       "solver": "Newton-Krylov (GMRES(40)), mixed-precision Jacobian products, FP64 residual"},
            "newton_krylov": nk, "fixed_point": fp, "anderson": aa, "solutions_rel_diff": agree}
    print(json.dumps(line))
    pa.close()
    return 0


def run_vjp(args):
    """Adjoint of the one-loop bubble of all three channels (K1 201, K2 81^2, K3 41^3,
    Nq 4001, U/Delta = 2, T = 0.05): kb_bubble_vjp with respect to the vertex (both sides,
    one gradient slot) and G^R, beside the forward bubble of the same precision; mixed
    (complex64 vertex, FP32 records and GEMMs, FP64 accumulation of the scatter) unless
    --precision fp64.  Points: output points whose gradient is pulled back per second."""
    import torch
    import seeded as S
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    prec = "fp64" if args.precision == "fp64" else "mixed"
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    large = args.workload == "vjp-large"
    if large:      # the largest single-instance workload
        g, nq, u, temp = dict(n1=801, n2w=201, n2v=201, n3w=101, n3v=101), 8001, 3.0, 0.01
    else:
        g, nq, u, temp = dict(n1=201, n2w=81, n2v=81, n3w=41, n3v=41), NQ, U, T
    dev = torch.device("cuda", 0)
    e = Engine(g, nq, device=0)
    e.set_model(DELTA, temp)
    e.set_workspace_limit(args.ws_gb << 30)
    e.set_vertex(0, U=u, has_R=True, channels=S.seeded_vertex(g, u, seed=77), dtype=dt)
    e.alloc_out(1, dtype=dt)
    rng = np.random.default_rng(5)
    for t in e.tensors[1].values():
        t.copy_(torch.from_numpy(rng.standard_normal(t.shape) + 1j * rng.standard_normal(t.shape)))
    e.alloc_out(2)                                  # gradient slot (complex128, zeroed)
    e.alloc_out(3, dtype=dt)                        # forward output slot
    tabs = e.gr_tables()
    stream = torch.cuda.current_stream(dev)
    points = 3 * sum(class_points(g).values())

    def vjp():
        for r in range(3):
            e.bubble_vjp(r, 0, 0, 1, grad_left=2, grad_right=2, grad_gr=tabs, precision=prec, stream=stream)

    def fwd():
        for r in range(3):
            e.bubble(r, 0, 0, 3, precision=prec, stream=stream)

    ms_vjp = _timed(vjp, args.steps, min(args.warmup, 1), stream)
    ms_fwd = _timed(fwd, args.steps, min(args.warmup, 1), stream)
    kb.kb_profile_enable(e.ctx, True)
    vjp()
    torch.cuda.synchronize()
    prof = kb.kb_profile_read(e.ctx)
    kb.kb_profile_enable(e.ctx, False)
    kb.kb_check_device(e.ctx)
    line = {"metric": "adjoint bubble points/s (w.v.v'.Keldysh, vertex + G^R gradients)",
            "value": points / (ms_vjp / 1e3), "unit": "points/s", "n_gpus": 1, "steps": args.steps,
            "warmup": min(args.warmup, 1), "ms_per_step": ms_vjp, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": "VJP of the one-loop bubble a,p,t; K1 %d, K2 %dx%d, K3 %d^3, Nq %d"
                                   % (g["n1"], g["n2w"], g["n2v"], g["n3w"], nq),
                       "precision": prec, "points_per_step": points},
            "forward": {"precision": prec, "value": points / (ms_fwd / 1e3), "ms_per_step": ms_fwd},
            "kernels_ms": {k: round(v[0], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}}
    print(json.dumps(line))
    return 0


def run_loop(args):
    """Self-energy loop (kb_loop, plain FP64) of the full vertex at the step's sizes (K1 401,
    K2 101^2, K3 51^3 in all three channels with the bare part, Nq 4001, U/Delta = 2,
    T = 0.05) at 401 frequencies (the K1 grid).  Unit: integrand evaluations (frequency x
    interior node) per second.  Algorithmic work per evaluation: the interpolated reads of
    both spin components of the v'-dependent vertex part (144 class corners of 16 complex
    values, 64 flops each) and the two Keldysh contractions (288 flops); corners that fall
    outside a grid are counted too, so `achieved` is an upper bound."""
    import torch
    import seeded as S
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    g = dict(n1=401, n2w=101, n2v=101, n3w=51, n3v=51)
    dev = torch.device("cuda", 0)
    e = Engine(g, NQ, device=0)
    e.set_model(DELTA, T)
    e.set_vertex(0, U=U, has_R=True, channels=S.seeded_vertex(g, U, seed=91))
    nus = torch.from_numpy(S.grid_freqs(g["n1"])).to(dev)
    out = torch.empty((nus.numel(), 2, 2), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        kb.kb_loop(e.ctx, 0, 0, nus.numel(), nus.data_ptr(), out.data_ptr(), stream.cuda_stream)

    ms = _timed(step, args.steps, max(args.warmup, 3), stream)
    kb.kb_check_device(e.ctx)
    cpu = None
    if not args.no_cpu_baseline:
        rate, cores, desc = oracle_loop_rate(g, S.seeded_vertex(g, U, seed=91))
        cpu = {"value": rate, "unit": "evaluations/s", "cores": cores, "kind": "oracle", "sample": desc}
    evals = nus.numel() * (NQ - 2)
    flops = evals * (144 * 64 + 288)
    ach = flops / (ms / 1e3) / 1e12
    line = {"metric": "self-energy loop integrand evaluations/s", "value": evals / (ms / 1e3),
            "unit": "evaluations/s", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "loop of the full vertex, K1 401, K2 101x101, K3 51^3, Nq 4001, 401 frequencies",
                       "evaluations_per_step": evals, "l2": "vertex 17 MB per K3 channel, L2-resident"},
            "roofline": {"kernel": "k_loop", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                         "note": "upper-bound flop count; FP64 peak derived from SM count and clock"},
            "cpu_baseline": cpu}
    print(json.dumps(line))
    e.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "mixed", "fp64"])
    ap.add_argument("--ref-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--channels", default="apt", help="subset of a, p, t (profiling captures)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling captures)")
    ap.add_argument("--no-fp64-check", action="store_true",
                    help="skip the plain-FP64 step behind per_class_err and fp64_gpu (profiling captures)")
    ap.add_argument("--no-graph", action="store_true", help="eager launches instead of one step graph")
    ap.add_argument("--no-t-su2", action="store_true",
                    help="the t bubble's two spin terms contracted directly instead of its SU(2) form")
    ap.add_argument("--ws-gb", type=int, default=8, help="device workspace limit per context (GiB)")
    ap.add_argument("--ml-cache", default="auto", choices=["off", "auto", "all"],
                    help="multiloop workloads: record cache of the full vertex (off, the useful sides, all sides)")
    ap.add_argument("--fp-maxit", type=int, default=40, help="parquet workload: iteration cap of the fixed point and of Anderson acceleration")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the wave-model split-K factors instead of timing candidates before the step graph")
    ap.add_argument("--workload", default="step",
                    choices=["step", "points32", "vjp", "vjp-large", "multiloop", "multiloop-large", "parquet",
                             "loop"],
                    help="step: the default three-channel line; points32 / vjp / multiloop: the batching, "
                         "adjoint and multiloop paths")
    args = ap.parse_args()
    if args.workload != "step" and args.impl == "ours":
        if args.workload.startswith("multiloop"):
            return run_multiloop(args)
        if args.workload == "parquet":
            return run_parquet(args)
        if args.workload == "loop":
            return run_loop(args)
        return run_points32(args) if args.workload == "points32" else run_vjp(args)
    chans = tuple(sorted({"apt".index(c) for c in args.channels}))
    if not chans:
        ap.error("--channels needs at least one of a, p, t")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import seeded as S
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine, StepGraph

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    prec = args.precision
    if prec == "auto":
        prec = "mixed"
    ch = S.seeded_vertex(GRIDS, U, seed=1000 + rank)        # each rank: its own parameter point
    out_dt = torch.complex64 if prec == "mixed" else torch.complex128
    # one context per channel: the channels' bubbles are independent branches of the step
    # graph (each context has its own workspace); all read the one vertex in HBM
    engs = {}
    for r in chans:
        e = Engine(GRIDS, NQ, device=local)
        e.set_model(DELTA, T)
        e.set_workspace_limit(args.ws_gb << 30)
        e.set_autotune(not args.no_autotune)
        if not engs:
            # the seeded vertex is conjugation- and crossing-symmetric by construction
            e.set_vertex(0, U=U, has_R=True, channels=ch, dtype=torch.complex64, symmetric=True)
        else:
            e.share_slot(0, next(iter(engs.values())), 0, U=U, has_R=True, symmetric=True)
        e.alloc_out(1, channels=(r,), dtype=out_dt)
        engs[r] = e
    eng = next(iter(engs.values()))
    stream = torch.cuda.current_stream(dev)

    points = POINTS_PER_STEP * len(chans) // 3

    # the t bubble in its SU(2) form (mixed precision, with the a bubble in the same step):
    # its K3 from the density contraction (half the quadrature length) and the a bubble's K3
    su2 = prec == "mixed" and 0 in chans and 2 in chans and not args.no_t_su2

    def step_eager():
        for r in chans:
            if r == 2 and su2:
                engs[2].bubble_t_su2(0, 1, stream=stream)
            else:
                engs[r].bubble(r, 0, 0, 1, precision=prec, stream=stream)
        if su2:
            engs[2].t_su2_finish(1, engs[0].out(1, 0)["K3"], stream=stream)

    graph = None
    if not args.no_graph:
        descs = [engs[r].desc_t_su2(0, 1) if (r == 2 and su2) else engs[r].desc(r, 0, 0, 1, precision=prec)
                 for r in chans]
        if su2:
            descs.append(engs[2].desc_t_su2_finish(1, engs[0], 1))
        graph = StepGraph(descs, device=dev)

    def step():
        if graph is not None:
            graph.launch(stream)
        else:
            step_eager()

    def launches():
        return sum(e.launches() for e in engs.values())

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # 256 MB > 129 MB L2
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each, events on the launching stream ----
    n0 = launches()
    clk = ClockSampler(local) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop() if clk else None
    launches_timed = launches() - n0

    # ---- per-kernel CUDA-event times: the same K steps run eagerly with the library's
    # timing hook (a graph replay has no per-launch events) ----
    for e in engs.values():
        kb.kb_profile_enable(e.ctx, True)
    for _ in range(args.steps):
        flush.zero_()
        step_eager()
    torch.cuda.synchronize()
    prof = {}
    for e in engs.values():
        for k, (t, c) in kb.kb_profile_read(e.ctx).items():
            p0 = prof.get(k, (0.0, 0))
            prof[k] = (p0[0] + t, p0[1] + c)
        kb.kb_profile_enable(e.ctx, False)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms_median = float(np.median([a.elapsed_time(b) for a, b in evs]))
    value, ms_step = weak_scaling_value(points, ms / args.steps, dist, dev)

    # ---- end to end through the public API: pinned host inputs -> device -> bubbles -> host ----
    e2e = None
    if not args.no_e2e:
        host_in = {k: v.to("cpu").pin_memory() for k, v in eng.tensors[0].items()}
        dev_out = {(r, k): v for r, e in engs.items() for k, v in e.tensors[1].items()}
        host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in dev_out.items()}
        h2d = sum(v.numel() * v.element_size() for v in host_in.values())
        d2h = sum(v.numel() * v.element_size() for v in host_out.values())
        e2e_ms = []
        for it in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k, v in host_in.items():
                eng.tensors[0][k].copy_(v, non_blocking=True)
            step()
            for k, v in host_out.items():
                v.copy_(dev_out[k], non_blocking=True)
            torch.cuda.synchronize()
            if it >= args.warmup:
                e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_val, _ = weak_scaling_value(points, sum(e2e_ms) / len(e2e_ms), dist, dev)
        e2e = {"value": e2e_val, "unit": "points/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- roofline of the dominant kernel (its CUDA-event time in the profiled eager pass) ----
    hbm, bf16, src = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    name, (dms, dcnt) = dom
    share = dms / max(sum(v[0] for v in prof.values()), 1e-30)
    fl = contraction_flops(prec)
    roof = None
    if name in ("k_zgemm_f64", "k_zgemm_skinny_f64"):
        sel = [k for k in fl if (k[1] in ("K3", "K2p")) == (name == "k_zgemm_f64")]
        work = sum(fl[k] for k in sel) * args.steps
        ach = work / (dms / 1e3) / 1e12
        roof = {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "share": share,
                "note": "FP64 FMA pipe peak derived from 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    else:
        work = mixed_kernel_work(chans, t_su2=su2) if prec == "mixed" else {}
        roof = roofline_entry(name, dms, args.steps, work, bf16) or {
            "kernel": name, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None}
        roof["share"] = share
        others = []
        for k in ("k_mx_tile3_both", "k_tc_k3"):
            if k in prof and k != name:
                e = roofline_entry(k, prof[k][0], args.steps, work, bf16)
                if e:
                    e["share"] = prof[k][0] / max(sum(v[0] for v in prof.values()), 1e-30)
                    others.append(e)
        roof["others"] = others

    # ---- the error clause of the metric: one plain-FP64 step of the same bubbles on the same
    # (complex64) vertex; per channel and class the relative max-norm error of the mixed
    # outputs (the last timed step's) against it, and the FP64 step's own rate ----
    per_class_err, fp64_gpu = None, None
    if prec == "mixed" and not args.no_fp64_check:
        CN = ("K1", "K2", "K2p", "K3")
        for r, e in engs.items():
            e.alloc_out(2, channels=(r,), dtype=torch.complex128)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        for r in chans:
            engs[r].bubble(r, 0, 0, 2, precision="fp64", stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        fp64_gpu = {"value": points / (ms64 / 1e3), "ms_per_step": ms64, "steps": 1,
                    "note": "plain FP64 path (FP64 gather and FP64 SIMT contraction), same vertex and outputs, "
                            "one step after the mixed ones"}
        per_class_err = {}
        worst = 0.0
        for r in chans:
            mx, fp = engs[r].out(1, r), engs[r].out(2, r)
            d = {}
            for k in CN:
                num = float((mx[k].to(torch.complex128) - fp[k]).abs().max())
                den = float(fp[k].abs().max())
                d[k] = num / den if den > 0 else num
                worst = max(worst, d[k])
            per_class_err["apt"[r]] = d
        per_class_err["max"] = worst
        per_class_err["tolerance"] = 1e-6

    # ---- the dominant kernel counted by output points alone: 32 Nq real flops per output
    # point it computes (4 Nq complex multiply-adds), against the FP32 pipe ----
    if roof is not None and roof.get("kernel") == "k_mx_k2":
        half = lambda n: n - n // 2
        comp = {0: half(GRIDS["n2w"]) * GRIDS["n2v"], 1: GRIDS["n2w"] * half(GRIDS["n2v"]),
                2: half(GRIDS["n2w"]) * GRIDS["n2v"]}
        f8 = sum(comp[r] * 16 * 32.0 * NQ for r in chans) * args.steps
        a8 = f8 / (dms / 1e3) / 1e12
        roof["frac_s8d"] = a8 / FP32_PEAK_TFLOPS
        roof["achieved_s8d"] = a8
        roof["note_s8d"] = ("32 Nq flops per computed K2 point (the independent half), i.e. the contraction's "
                            "4 Nq complex multiply-adds per point without the gather, against the same FP32 pipe peak")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and len(chans) == 3:
        rate, cores, desc, _ = oracle_rate(budget_s=args.ref_budget)
        rate1, _, desc1, _ = oracle_rate(budget_s=4.0, seed=1, nthreads=1)
        cpu = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle", "sample": desc,
               "single_thread": {"value": rate1, "unit": "points/s", "cores": 1, "sample": desc1}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "ms_per_step_median": ms_median,
                "vs_baseline": None, "dtype": "f32" if prec == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD if len(chans) == 3 else WORKLOAD.replace("a,p,t", args.channels),
                           "precision": prec, "points_per_step": points,
                           "l2": "flushed (256 MB write) before every timed step", "parallelism": "weak: one "
                           "independent parameter point per GPU",
                           "launch": "one CUDA graph per step (channels as parallel branches)" if graph is not None
                           else "eager, one stream",
                           "t_channel": "SU(2) form: K3 from the density contraction and the a bubble" if su2
                           else "both spin terms contracted"},
                "e2e": e2e,
                "gpu_launches": int(launches_timed), "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
                "per_class_err": per_class_err, "fp64_gpu": fp64_gpu,
                "kernels_ms": {k: round(v[0] / args.steps, 4) for k, v in prof.items()},
                "kernels_ms_note": "per-kernel CUDA-event times of the same steps run eagerly (sum %.3f ms/step)"
                                   % (sum(v[0] for v in prof.values()) / args.steps),
                "peaks_source": src}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
