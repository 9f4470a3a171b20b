"""Benchmark of the Quantization Tree forward step (Algorithm III of Pages &
Wilbertz, arXiv:1101.3228) on GB300.

Metric: certified sample.layers/s -- M pairs per layer times n layers divided
by the device time of one qt_transitions call (counts exact under the FP64
contract, ready on the device).  A step is one whole forward step over all
layers.  Default workload: the largest one whose step is a few seconds, the
8-d AR(1) chain at full size (d = 8, n = 50, N_k = 4000, M = 10^8 pairs per
layer), in the automatic form (the tensor-core screen).  Extra keys: the 10-d
365-layer chain at full size (M = 10^8, two timed steps), the 4-d basket at
full size, the 2-factor OU workload (the FP32 screen, Algorithm II, the swing
option's backward induction) and the paper's own scenario.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME] [--impl ours|reference]
                    [--no-extras]

Prints one JSON line on rank 0.  With torchrun, every rank runs an independent
replica with its own seed (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import qt_workloads as W  # noqa: E402

FP32_LANES_PER_SM = 128
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="ar8", choices=list(W.BUILDERS))
    ap.add_argument("--form", default="auto")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--no-extras", action="store_true", help="skip the extra workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--M", type=int, default=0, help="override samples per layer")
    ap.add_argument("--layers", type=int, default=0, help="first n layers only (small profiling cases)")
    ap.add_argument("--hist", default="auto", choices=["auto", "smem", "global"],
                    help="count histogram: library choice, shared-memory privatised, or L2 reductions")
    ap.add_argument("--spt", type=int, default=0, help="samples per thread (0 = library choice)")
    ap.add_argument("--tc-draw", type=int, default=0, choices=[0, 1, 2],
                    help="tensor-core form's sample-draw layout: 0 autotuned, 1 draw pass, 2 in the screen kernel")
    ap.add_argument("--router-samples", type=int, default=10**7, help="labelled pairs for the router form")
    return ap.parse_args()


def workload(name, M=0):
    model = W.get(name)
    if M:
        model = W.get(name, M=M) if name != "paper" else W.paper(M=M)
    return model


def grid_method(model):
    from paper_1101_3228_gb300 import binding as B
    return {"lloyd1d": B.GRID_LLOYD1D, "product": B.GRID_PRODUCT, "kmeans": B.GRID_KMEANS}[model.grid_kind]


def default_form(model, B):
    # the fastest certified form measured for each dimension class: the FP32 screen
    # for d <= 2, the tensor-core screen for 3 <= d <= 10 (both exact through their
    # certificates)
    return B.FORM_TC_RECHECK if 3 <= model.d <= 10 else B.FORM_F32_RECHECK


def plain_form(model, B):
    # the plain GPU comparator: exact FP64 brute force for d <= 2, FP32 brute force
    # with FP64 recheck for d >= 4 (the path the learned and tensor forms are compared with)
    return B.FORM_PLAIN_F64 if model.d <= 2 else B.FORM_F32_RECHECK


def candidates_per_sample_layer(model, pathwise=False):
    """Brute-force candidate distances per sample.layer, averaged over layers:
    N_k + N_{k+1} for Algorithm III (both points of a pair are searched), N_{k+1}
    for Algorithm II (one search per path and layer)."""
    N = np.asarray(model.N, dtype=np.float64)
    return float(np.sum(N[1:] if pathwise else N[:-1] + N[1:]) / model.n)


def flops_per_sample_layer(model, pathwise=False):
    """Algorithmic work of the search: per candidate distance d subtractions (or
    the expanded form's d multiply-adds) and d multiply-adds, 2d flops (Sec. 4
    counts 6 operations for a 2-d distance including its comparison; the
    comparison is not counted here)."""
    return candidates_per_sample_layer(model, pathwise) * 2 * model.d


def tc_pipe_flops_per_sample_layer(model):
    """Work the tensor pipe does for the tensor-core screen: per candidate a dot
    product over all K operand columns (the FP16 head/tail split of sample and grid
    point, the squared norm, zero padding), 2 flops each."""
    dm = 2 if model.d <= 2 else (4 if model.d <= 4 else (6 if model.d <= 6 else (8 if model.d <= 8 else 10)))
    K = 16 if dm <= 4 else 32
    return candidates_per_sample_layer(model) * 2 * K


def replica_seed(model, rank: int) -> int:
    """Every rank runs an independent replica (weak scaling): its own Philox key."""
    return int(model.seed) + 7919 * int(rank)


def max_over_ranks(ms: float, dist, device=None) -> float:
    """The slowest rank's time; the whole job waits for it."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: int, ms: float) -> float:
    """Whole-job throughput: the sample.layers of all ranks over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def source_hash():
    h = hashlib.sha256()
    for d in ("paper_1101_3228_gb300/csrc", "include"):
        for f in sorted(os.listdir(os.path.join(ROOT, d))):
            if f.endswith((".cu", ".cuh", ".h")):
                h.update(open(os.path.join(ROOT, d, f), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sms.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return None
        load = [s for s in sms if mx and s > 0.5 * mx] or sms
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def cpu_baseline(model, grids_np, seconds):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload."""
    import oracle
    oracle.build()
    prec = model.prec
    Ms = 20000 if model.d <= 2 else 4000
    # size the sample from one probe layer so that the run takes about `seconds`
    t = time.perf_counter()
    mdl = model.restrict(n=1, M=Ms)
    oracle.transitions(mdl, grids_np[: int(model.N[0] + model.N[1])], Ms, model.seed, prec)
    dt = time.perf_counter() - t
    per_sl = dt / Ms
    layers = max(1, min(model.n, int(seconds / max(per_sl * Ms, 1e-9))))
    M = int(max(1000, min(model.M, seconds / max(per_sl * layers, 1e-12))))
    mdl = model.restrict(n=layers, M=M)
    off = model.offsets()
    t = time.perf_counter()
    oracle.transitions(mdl, grids_np[: off[layers + 1]], M, model.seed, prec)
    el = time.perf_counter() - t
    return {"value": layers * M / el, "unit": "sample*layers/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {layers} of {model.n} layers x {M} pairs per layer (FP64 brute force, {el:.1f} s)"}


def run_reference(args, model, rank, world):
    """Reference arm: the CPU oracle, timed as it stands on the host cores."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    g = W.layer_grids(model, samples=20000, iters=5) if model.grid_kind == "kmeans" else W.layer_grids(model)
    probe = cpu_baseline(model, g, 2.0)
    rate = probe["value"]
    # each step: a bounded sample of the workload sized to ~ a few seconds
    budget = max(1.0, 90.0 / max(1, args.steps + args.warmup))
    layers = max(1, min(model.n, 4))
    M = int(max(1000, min(model.M, budget * rate / layers)))
    mdl = model.restrict(n=layers, M=M)
    off = model.offsets()
    gg = g[: off[layers + 1]]
    for _ in range(args.warmup):
        oracle.transitions(mdl, gg, M, model.seed, model.prec)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.transitions(mdl, gg, M, model.seed, model.prec)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = layers * M / (ms / 1e3)
    sample = f"first {layers} of {model.n} layers x {M} pairs per layer per step"
    line = {"impl": "reference", "metric": "certified sample*layers/s (exact counts)", "value": value,
            "unit": "sample*layers/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": model.name, "d": model.d, "n": model.n,
                                            "N": int(model.N[-1]), "M": model.M},
            "cpu_baseline": {"value": value, "unit": "sample*layers/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "sample*layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_grids(ctx, B, model):
    """The benchmark's grids, built by the library: product grids of 1-d stationary
    quantizers for the 2-factor model, sample Lloyd on seeded Gaussian draws otherwise."""
    return ctx.build_grids(model, grid_method(model), samples=max(20 * int(np.max(model.N)), 200000), iters=20,
                           seed=W.GRID_SEED_BASE + W.CONFIG_INDEX.get(model.name, 9))


def counts_type_for(B, model, dev):
    """int64 counts unless they would take more than a quarter of the device (then uint32)."""
    import torch
    big = model.count_entries * 8 > torch.cuda.get_device_properties(dev).total_memory // 4
    return B.COUNTS_U32 if big else B.COUNTS_I64


def tensor_roofline(model, units, kern_ms, peaks):
    """Tensor-core screen against the measured dense 16-bit tensor rate (FP16 runs at
    the bf16 rate on this part), sustained figure: the algorithmic work (2d flops per
    candidate) and, beside it, the pipe's share (K operand columns per candidate)."""
    tpeak = peaks.get("bf16_tflops_sustained", 1700.0)
    sec = kern_ms / 1e3
    ach = flops_per_sample_layer(model) * units / sec / 1e12
    pipe = tc_pipe_flops_per_sample_layer(model) * units / sec / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s", "frac": ach / tpeak,
            "mma_frac": pipe / tpeak, "kernel_ms": kern_ms,
            "work": f"{flops_per_sample_layer(model):.0f} flops per sample.layer "
                    f"(2d per candidate, {candidates_per_sample_layer(model):.0f} candidates)",
            "peak_basis": "measured dense bf16 GEMM, sustained (of measured)"
            if "bf16_tflops_sustained" in peaks else "fallback 1.7 PFLOP/s sustained (of fallback)"}


def alu_roofline(model, units, kern_ms, peaks, n_sm, pathwise=False):
    """FP32 screen against the FP32 FMA lanes (SMs x 128 lanes x 2 flops x max clock)."""
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    peak = 2.0 * FP32_LANES_PER_SM * n_sm * sm_max * 1e6 / 1e12
    work = flops_per_sample_layer(model, pathwise)
    ach = work * units / (kern_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "kernel_ms": kern_ms,
            "work": f"{work:.0f} flops per sample.layer (2d per candidate, "
                    f"{candidates_per_sample_layer(model, pathwise):.0f} candidates)",
            "peak_basis": f"FP32 FMA lanes: {n_sm} SMs x {FP32_LANES_PER_SM} x 2 flops x {sm_max:.0f} MHz"}


def timed_steps(ctx, step, K, W_, flush, stream, dist=None):
    """W_ untimed steps, then K steps each between CUDA events on the launching stream
    (a buffer larger than L2 written between steps, outside the events).  Returns
    the mean step time, the library's per-step forward-region times and the stats."""
    import torch
    for _ in range(W_):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    kern = []
    for i in range(K):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        torch.cuda.synchronize()
        kern.append(ctx.status()[1].ms)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    return sum(ms) / K, kern, ctx.status()[1]


def extra_workloads(ctx, B, dev, stream, flush, peaks, n_sm):
    """Further workloads, each timed on its own (one replica, this GPU)."""
    import torch
    out = {}

    def run(name, model, K, W_, o=None, pathwise=False, grids=None):
        g = grids if grids is not None else bench_grids(ctx, B, model)
        ct = counts_type_for(B, model, dev)
        o = o or B.options(prec=model.prec, counts_type=ct)
        o.counts_type = ct
        counts = torch.empty(model.count_entries, dtype=torch.int64 if ct == B.COUNTS_I64 else torch.int32,
                             device=dev)
        f = ctx.transitions_pathwise if pathwise else ctx.transitions

        def step():
            f(model, g, model.M, model.seed, o, counts=counts, want_stats=False, stream=stream)
        ms, kern, st = timed_steps(ctx, step, K, W_, flush, stream)
        units = model.n * model.M
        kmean = statistics.mean(kern) if kern and all(k > 0 for k in kern) else ms
        r = {"workload": model.name, "d": model.d, "n": model.n, "N": int(model.N[-1]), "M": model.M,
             "value": units / (ms / 1e3), "unit": "sample*layers/s", "ms_per_step": ms, "steps": K, "warmup": W_,
             "form": "pathwise_f32" if pathwise else B.FORM_NAMES.get(st.form_used, "?"),
             "counts": "int64" if ct == B.COUNTS_I64 else "uint32", "launches_per_step": st.launches,
             "rechecks_per_step": st.rechecks}
        if st.form_used == B.FORM_ROUTER_CERT:
            r["candidates_per_search"] = st.candidates / (2 * units)
        if st.form_used == B.FORM_TC_RECHECK and not pathwise:
            r["tc_draw"] = {1: "draw pass", 2: "in the screen kernel"}.get(st.tc_draw)
            r["roofline"] = tensor_roofline(model, units, kmean, peaks)
        else:
            r["roofline"] = alu_roofline(model, units, kmean, peaks, n_sm, pathwise)
        del counts
        torch.cuda.empty_cache()
        return r, g

    # the 10-d, 365-layer chain at full size (uint32 counts: 93 GB); one warm-up at M = 10^6
    m5 = W.maxcall10()
    _, _ = run("warm", W.maxcall10(M=10**6).restrict(n=4), 1, 1)
    out["maxcall10_full"], _ = run("maxcall10", m5, 2, 0)
    # the 4-d basket at full size
    out["basket4_full"], _ = run("basket4", W.basket4(), 2, 1)
    # the 2-factor OU workload: Algorithm III (FP32 screen) and Algorithm II (path-wise)
    m2 = W.ou2()
    out["ou2_alg3"], g2 = run("ou2", m2, 5, 3, B.options(form=B.FORM_F32_RECHECK, prec=m2.prec))
    out["ou2_alg2_pathwise"], _ = run("ou2", m2, 5, 3, B.options(prec=m2.prec), pathwise=True)
    out["ou2_alg2_pathwise"]["vs_alg3"] = out["ou2_alg2_pathwise"]["value"] / out["ou2_alg3"]["value"]
    # Algorithm II on the 8-d chain (grids streamed through shared memory), M = 10^7
    m8 = W.ar8(M=10**7)
    out["ar8_alg2_pathwise_M1e7"], _ = run("ar8", m8, 2, 1, B.options(prec=m8.prec), pathwise=True)
    # the learned router (MLP on the tensor cores) with the Elkan certificate on the
    # 8-d chain at M = 10^7, trained on 10^7 labelled pairs, beside the FP32 screen
    # on the same grids
    m8r = W.ar8(M=10**7)
    g8 = bench_grids(ctx, B, m8r)
    t0 = time.perf_counter()
    rt = ctx.router_train(m8r, g8, samples=10**7, layers=8, epochs=4, seed=7 + W.CONFIG_INDEX["ar8"])
    ri = rt.info()
    rr, _ = run("ar8", m8r, 2, 1, B.options(form=B.FORM_ROUTER_CERT, prec=m8r.prec, router=rt.handle), grids=g8)
    rr["router"] = {"train_samples": 10**7, "train_accuracy": ri.train_accuracy, "train_loss": ri.train_loss,
                    "build_s": time.perf_counter() - t0, "neighbours": ri.neighbours}
    rf, _ = run("ar8", m8r, 2, 1, B.options(form=B.FORM_F32_RECHECK, prec=m8r.prec), grids=g8)
    rr["f32_screen_value"] = rf["value"]
    rr["vs_f32_screen"] = rr["value"] / rf["value"]
    out["ar8_router_M1e7"] = rr
    rt.close()
    # the paper's scenario (d = 2, n = 365, M = 10^5, N = 500): Algorithm III and II
    mp = W.paper(N=500)
    out["paper_alg3"], _ = run("paper", mp, 5, 3, B.options(prec=mp.prec))
    out["paper_alg2_pathwise"], _ = run("paper", mp, 5, 3, B.options(prec=mp.prec), pathwise=True)
    # the swing option's backward induction on the 2-factor tree (100 dates, N = 500)
    counts, _, _ = ctx.transitions(m2, g2, m2.M, m2.seed, B.options(prec=m2.prec), stream=stream)
    v = torch.from_numpy(W.payoff_values(m2, g2.cpu().numpy()) - 0.004).to(dev)
    sw = {}
    for qmin, qmax in ((0, 1), (20, 60), (0, 100)):
        ctx.swing(m2.N, counts, v, qmin, qmax, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P_, price = ctx.swing(m2.N, counts, v, qmin, qmax, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sw[f"Q[{qmin},{qmax}]"] = {"ms": e0.elapsed_time(e1), "price": price}
    out["ou2_swing"] = sw
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    model = workload(args.config, args.M)
    if args.layers:
        model = model.restrict(n=min(args.layers, model.n))
    if args.impl == "reference":
        run_reference(args, model, rank, world)
        return

    import torch
    from paper_1101_3228_gb300 import binding as B
    from paper_1101_3228_gb300 import build as libbuild
    if rank == 0:
        libbuild.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = B.Context(local)
    stream = torch.cuda.current_stream()
    seed = replica_seed(model, rank)          # independent replica per rank
    grids = bench_grids(ctx, B, model)
    form = {"auto": B.FORM_AUTO, "plain_f64": B.FORM_PLAIN_F64, "f32_recheck": B.FORM_F32_RECHECK,
            "tc_recheck": B.FORM_TC_RECHECK, "router_cert": B.FORM_ROUTER_CERT}.get(args.form, B.FORM_AUTO)
    if form == B.FORM_AUTO:
        form = default_form(model, B)
    prec = model.prec
    entries = model.count_entries
    ctype = counts_type_for(B, model, dev)
    router = None
    router_info = None
    if form == B.FORM_ROUTER_CERT:
        # trained before the timed region, on pairs the method itself labels
        router = ctx.router_train(model, grids, samples=args.router_samples, layers=8, epochs=4, seed=7 +
                                  W.CONFIG_INDEX[model.name])
        ri = router.info()
        router_info = {"train_samples": args.router_samples, "train_accuracy": ri.train_accuracy,
                       "train_loss": ri.train_loss, "build_ms": ri.build_ms, "neighbours": ri.neighbours}
    hist_flags = {"auto": 0, "smem": B.FLAG_SMEM_HIST, "global": B.FLAG_GLOBAL_HIST}[args.hist]
    opts = B.options(form=form, prec=prec, samples_per_thread=args.spt, counts_type=ctype, flags=hist_flags,
                     router=router.handle if router else None, tc_draw=args.tc_draw)
    counts = torch.empty(entries, dtype=torch.int64 if ctype == B.COUNTS_I64 else torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # larger than the 129 MB L2
    units = model.n * model.M

    def step(o=opts):
        ctx.transitions(model, grids, model.M, seed, o, counts=counts, want_stats=False, stream=stream)

    with ClockSampler(local) as clk:
        ms_step, kern_ms, st = timed_steps(ctx, step, args.steps, max(3, args.warmup), flush, stream, dist)
    clocks = clk.summary()
    ms_step = max_over_ranks(ms_step, dist, dev) if dist else ms_step
    value = job_value(world, units, ms_step)

    # plain GPU comparator (exact FP64 brute force for d <= 2, FP32 screen otherwise)
    plain = None
    pform = plain_form(model, B)
    if args.plain_steps > 0 and pform != form:
        po = B.options(form=pform, prec=prec, counts_type=ctype)
        pms, pkern, _ = timed_steps(ctx, lambda: step(po), args.plain_steps, 1, flush, stream, dist)
        plain = {"form": B.FORM_NAMES[pform], "value": world * units / (pms / 1e3), "ms_per_step": pms}
        if pform == B.FORM_F32_RECHECK:
            pk = statistics.mean(pkern) if pkern and all(k > 0 for k in pkern) else pms
            n_sm_p = torch.cuda.get_device_properties(dev).multi_processor_count
            pk_peaks = json.load(open(MEASURED)) if os.path.exists(MEASURED) else {}
            plain["roofline"] = alu_roofline(model, units, pk, pk_peaks, n_sm_p)

    # end to end through the public API: host grids and payoff in, price out
    del counts
    torch.cuda.empty_cache()
    gh = grids.cpu().numpy()
    phi = W.payoff_values(model, gh)
    gpin = torch.from_numpy(gh).pin_memory()
    ppin = torch.from_numpy(phi).pin_memory()
    e2e_ms = []
    for i in range(max(1, min(args.steps, 3)) + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        price, _ = ctx.price(model, gpin.numpy(), model.M, seed, ppin.numpy(), opts, stream=stream)
        if i > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e = {"value": world * units / (statistics.mean(e2e_ms) / 1e3), "unit": "sample*layers/s",
           "h2d_bytes_per_step": int(gh.nbytes + phi.nbytes), "d2h_bytes_per_step": 8,
           "ms_per_step": statistics.mean(e2e_ms), "price": price}

    # roofline of the dominant kernel: the forward region (screen launches and, with
    # the draw-pass layout, the draw passes), timed by the library's CUDA events on
    # the launching stream at every timed step
    peaks = json.load(open(MEASURED)) if os.path.exists(MEASURED) else {}
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    kmean = statistics.mean(kern_ms) if kern_ms and all(k > 0 for k in kern_ms) else ms_step
    if form == B.FORM_TC_RECHECK:
        roofline = tensor_roofline(model, units, kmean, peaks)
    else:
        roofline = alu_roofline(model, units, kmean, peaks, n_sm)
    layout = {1: "draw pass", 2: "in the screen kernel"}.get(st.tc_draw)
    traffic = None
    if os.path.exists(TRAFFIC):
        # DRAM bytes of one ncu capture of this kernel, kept only while the sources,
        # the form and the sample-draw layout are those it was taken on
        ent = json.load(open(TRAFFIC)).get(model.name)
        if ent and ent.get("source_hash") == source_hash() and ent.get("form") == B.FORM_NAMES[form] and \
                ent.get("layout") == layout and model.M == W.get(model.name).M and model.n == W.get(model.name).n:
            traffic = ent.get("bytes_per_launch")
    roofline["traffic"] = traffic

    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = extra_workloads(ctx, B, dev, stream, flush, peaks, n_sm)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(model, gh, args.cpu_seconds)

    if rank == 0:
        line = {"metric": "certified sample*layers/s (exact counts)", "value": value, "unit": "sample*layers/s",
                "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {B.FORM_PLAIN_F64: "f64", B.FORM_TC_RECHECK: "f16x3+f32"}.get(form, "f32"),
                "data": "synthetic",
                "config": {"workload": model.name, "d": model.d, "n": model.n, "N": int(model.N[-1]),
                           "M": model.M, "form": B.FORM_NAMES[form],
                           "tc_draw": layout,
                           "counts": "int64" if ctype == B.COUNTS_I64 else "uint32",
                           "sample_prec": "f32" if prec == 1 else "f64",
                           "l2": "256 MiB buffer written between timed steps",
                           "rechecks_per_step": st.rechecks,
                           "uncertified_by_cause": list(st.diag) if form == B.FORM_TC_RECHECK else None,
                           "router": router_info,
                           "candidates_per_search": (st.candidates / (2 * units)) if router else None},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": st.launches * args.steps, "clocks": clocks, "plain": plain, "extras": extras}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
