#!/usr/bin/env python3
"""Benchmark: normalized Lomb-Scargle periodogram throughput on GB300.

Workload (one step = one lsp_periodogram call = prep + main + finalize):
``gapped_100k`` -- 100,000 samples over 1000 d with nightly gaps, three
sinusoids + noise, oversampling 4, 200,000 frequencies (2e10 terms).  Inputs
are resident in HBM when the timed region starts; the L2 is flushed between
timed steps (inputs are 2.4 MB, smaller than L2).  Metric: L-S terms/s
(N_t * N_f per second), whole job.

With --gpus N (launched by torchrun) every rank evaluates its own block of
200,000 frequencies of one longer grid (rank r starts at f_0 + r N_f df): the
frequencies are independent, so there is no data-path collective and the
scaling is weak.

``--impl reference`` times the FP64 CPU oracle (the only other implementation
this project has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "L-S terms/s (N_t·N_f) & % SFU/FMA peak; batched MC curves/s vs plain"
UNIT = "terms/s"
WORKLOAD = "gapped_100k"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


MAIN_SOURCES = ("ls_main.cu", "ls_device.cuh", "lsp_kernels.cuh")
GLS_SOURCES = ("gls.cu", "ls_device.cuh", "lsp_kernels.cuh")


def _kernel_sha(files=MAIN_SOURCES):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1007_1658_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _recorded_traffic(kernel: str, profile="ls_main_gapped_100k.md", files=MAIN_SOURCES):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"traffic_record:\s*(\{.*?\})", txt)
    if not m:
        return None
    rec = json.loads(m.group(1))
    if rec.get("kernel_sha") != _kernel_sha(files) or rec.get("kernel") != kernel:
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        exe = shutil.which("nvidia-smi")
        if exe:
            self.proc = subprocess.Popen([exe, "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_median": float(np.median(pw)) if pw else None}


def cpu_baseline_sample(c, n_bins: int):
    """Oracle (as it stands) on the first n_bins frequencies of the workload."""
    import oracle
    fr = c.f0 + np.arange(n_bins) * c.df
    t0 = time.perf_counter()
    oracle.periodogram_at(c.t, c.X, fr)
    dt = time.perf_counter() - t0
    terms = c.t.size * n_bins
    return {"value": terms / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%s: all %d samples x first %d of %d frequencies (%.3g terms), FP64 two-pass Eq. 1-2"
                      % (WORKLOAD, c.t.size, n_bins, c.nf, terms),
            "seconds": dt}


def run_reference(args, rank, world):
    from paper_1007_1658_gb300 import synth
    if rank != 0:
        return 0
    c = synth.gapped_100k()
    n_bins = args.ref_bins
    for _ in range(args.warmup):
        cpu_baseline_sample(c, max(8, n_bins // 16))
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_baseline_sample(c, n_bins)
        vals.append(r["value"])
        secs.append(r["seconds"])
    terms = c.t.size * n_bins * args.steps
    value = terms / sum(secs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "N_t": int(c.t.size), "N_f": int(c.nf),
                                            "sample_bins": n_bins},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args, rank, world, dist):
    import torch
    from paper_1007_1658_gb300 import lsp, shard, synth

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c = synth.gapped_100k()
    if args.nf:
        c.nf = int(args.nf)  # smaller case of the same kernel (profiling captures)
    f0, _, _ = shard.weak_block(c.f0, c.df, c.nf, rank, world)  # this rank's block of the grid
    terms = c.t.size * c.nf
    t_d = torch.from_numpy(c.t).to(dev)
    X_d = torch.from_numpy(c.X).to(dev)
    P_d = torch.empty(c.nf, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.Stream(device=dev)
    ctx = lsp.Context(local, stream=stream, timing=1, sincos_mode=args.mode, freqs_per_thread=args.F)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx.periodogram(t_d, X_d, f0, c.df, c.nf, out=P_d)
        ctx.sync(120.0)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    main_ms, launches = [], 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                ctx.periodogram(t_d, X_d, f0, c.df, c.nf, out=P_d)
                ev[i][1].record(stream)
            _, m, fin = ctx.last_timing()
            main_ms.append(m)
            launches += ctx.last_launch_count()
        ctx.sync(120.0)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    total_ms = shard.max_over_ranks(total_ms, dist, dev)
    value = world * terms * args.steps / (total_ms * 1e-3)

    # latency of one small call (plain_1k: 1000 x 2000, device pointers)
    small = synth.plain_1k()
    ts_d, Xs_d = torch.from_numpy(small.t).to(dev), torch.from_numpy(small.X).to(dev)
    Ps_d = torch.empty(small.nf, dtype=torch.float32, device=dev)
    lat_fn = lambda: ctx.periodogram(ts_d, Xs_d, small.f0, small.df, small.nf, out=Ps_d)
    lat_ms = _time_calls(torch, stream, lat_fn, 5, 20, flush)

    # end to end through the C ABI with pinned host buffers (copies inside)
    e2e_val = None
    if args.e2e:
        e2e_val = _e2e(lsp, torch, c, f0, local, stream, args, world)

    if rank != 0:
        ctx.close()
        return 0
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # the library's AUTO choice is the packed three-term strip
    mode = args.mode if args.mode else lsp.SINCOS_RECUR3_X2
    F = args.F if args.F else {lsp.SINCOS_MUFU: 8, lsp.SINCOS_RECUR: 16, lsp.SINCOS_RECUR3: 24,
                               lsp.SINCOS_RECUR3_X2: 24}[mode]
    # algorithmic work per term on the bounding pipe (roof in terms per clock per SM)
    roof = {lsp.SINCOS_MUFU: (2, "SFU (MUFU): 2 sin/cos ops per term, 16 ops/clk/SM", 16.0 / 2),
            lsp.SINCOS_RECUR: (8, "FMA pipe: 4 accumulate + 4 rotation FP32 ops per term, 128/clk/SM", 128.0 / 8),
            lsp.SINCOS_RECUR3: (6, "FMA pipe: 4 accumulate + 2 three-term FP32 ops per term, 128/clk/SM",
                                128.0 / 6),
            lsp.SINCOS_RECUR3_X2: (6, "FMA pipe: 4 accumulate + 2 three-term FP32 lane ops per term (3 FFMA2), "
                                      "128/clk/SM", 128.0 / 6)}[mode]
    terms_per_clk = roof[2]
    peak = terms_per_clk * sms * peaks["sm_max_mhz"] * 1e6
    achieved = terms / (float(np.mean(main_ms)) * 1e-3)
    kernel = "ls_main_kernel<%d,%d>" % (F, {1: 1, 2: 2, 3: 4, 4: 5}[mode])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N_t": int(c.t.size), "N_f": int(c.nf), "terms_per_step": terms,
                   "sincos": {1: "mufu", 2: "recurrence", 3: "three-term recurrence",
                              4: "three-term recurrence, packed FP32x2"}[mode], "F": F,
                   "phase": "fixed64",
                   "l2": "flushed between steps (256 MB write)", "parallelism": "frequency shards x%d" % world},
        "roofline": {"bound": "alu", "kernel": kernel, "achieved": achieved / 1e9, "peak": peak / 1e9,
                     "unit": "Gterms/s", "frac": achieved / peak, "traffic": _recorded_traffic(kernel),
                     "peak_basis": "%s: %.2f terms/clk/SM x %d SMs x %.0f MHz (%s sm_max_mhz)" % (
                         roof[1], terms_per_clk, sms, peaks["sm_max_mhz"], peak_src),
                     "main_ms": float(np.mean(main_ms))},
        "e2e": None if e2e_val is None else {
            "value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(c.t.nbytes + c.X.nbytes),
            "d2h_bytes_per_step": int(c.nf * 4)},
        "gpu_launches": int(launches),
        "latency": {"workload": "plain_1k: 1000 x 2000", "us_per_call": lat_ms * 1e3,
                    "note": "prep + main (+ finalize), device pointers, median of 20"},
        "clocks": clk.summary(),
    }
    if args.cpu_baseline and world == 1:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline_sample(c, args.cpu_bins).items() if k != "seconds"}
    # the legs below are ordered so that the last ones (the Monte-Carlo batch,
    # the 65k-cadence precision comparison and the pipe rates) close the line
    if args.gls:
        line["floating_mean"] = _compact(run_gls_bench(torch, dev, stream, args, peaks, peak_src, sms))
    if args.paper:
        line["paper_shape"] = _compact(run_paper_shape(torch, dev, stream, args, peaks, sms))
    if args.batch:
        line["multi_rhs"] = _compact(run_mrhs_bench(torch, dev, stream, args.mrhs_patterns, args.mrhs_real,
                                                    tuple(int(g) for g in args.mrhs_groups.split(",")),
                                                    sms * peaks["sm_max_mhz"] * 1e6))
    if args.probe:
        line["pipe_rates"] = _compact(pipe_rates(ctx, sms, peaks["sm_max_mhz"]))
    if args.cadence:
        line["cadence_65k"] = _compact(run_cadence_bench(torch, dev, stream, args, peaks, peak_src, sms,
                                                         args.cpu_baseline and world == 1))
    if args.batch and args.mc:
        mc = run_batch_bench(ctx, torch, dev, stream, args)
        if args.cpu_baseline and world == 1:
            cb = batch_cpu_sample()
            # kept before the graph-vs-plain figures, which close the line
            mc = dict([("cpu_baseline", {"curves_per_s": cb["value"], "terms_per_s": cb["terms_per_s"],
                                         "cores": cb["cores"], "kind": cb["kind"], "sample": cb["sample"]})]
                      + list(mc.items()))
        line["batched_mc"] = _compact(mc)
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _compact(v, digits=4):
    """Floats rounded to `digits` significant digits (keeps the line short
    enough that its last legs survive a log tail)."""
    if isinstance(v, float):
        return float("%.*g" % (digits, v)) if np.isfinite(v) else v
    if isinstance(v, dict):
        return {k: _compact(x, digits) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [_compact(x, digits) for x in v]
    return v


def run_cadence_bench(torch, dev, stream, args, peaks, peak_src, sms, with_oracle):
    """Satellite-cadence precision stress (cadence_65k: 65,536 samples over
    1300 d, 1e-3 sinusoids near 20 c/d, 318,500 frequencies, f t up to 3.2e4
    turns): throughput of the default exact-phase kernel and of the paper's
    single-precision phase (f*t - rintf(f*t), Sec. 4.3, hardware sin/cos), and
    -- with the CPU baseline -- the error of each against the FP64 oracle on
    sampled bins (256 random + 49 around each injected line), the oracle's
    time on those bins being the CPU baseline of this workload."""
    from paper_1007_1658_gb300 import lsp, synth
    c = synth.cadence_65k()
    terms = c.t.size * c.nf
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    t_d, X_d = d(c.t), d(c.X)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"workload": "cadence_65k: N_t = %d, N_f = %d (%.3g terms)" % (c.t.size, c.nf, terms)}
    res = {}
    with ClockSampler(dev.index or 0) as clk:
        for name, opts, per_clk, basis in (
                ("fixed64", dict(), 128.0 / 6, "FMA pipe, 6 ops/term"),
                ("naive_fp32", dict(phase_mode=lsp.PHASE_NAIVE_FP32), 16.0 / 2, "SFU, 2 ops/term")):
            cctx = lsp.Context(dev.index or 0, stream=stream, timing=1, **opts)
            P_d = torch.empty(c.nf, dtype=torch.float32, device=dev)
            main = []

            def fn():
                cctx.periodogram(t_d, X_d, c.f0, c.df, c.nf, out=P_d)
                main.append(cctx.last_timing()[1])
            ms = _time_calls(torch, stream, fn, 2, max(3, args.steps // 2), flush)
            cctx.sync(120.0)
            main_ms = float(np.median(main[2:]))
            peak = per_clk * sms * peaks["sm_max_mhz"] * 1e6
            res[name] = P_d.cpu().numpy().astype(np.float64)
            out[name] = {"ms": ms, "terms_per_s": terms / (ms * 1e-3), "main_ms": main_ms,
                         "frac_of_roof": terms / (main_ms * 1e-3) / peak,
                         "roof": "%s, %s sm_max_mhz" % (basis, peak_src)}
            cctx.close()
    out["clocks"] = clk.summary()
    if with_oracle:
        import oracle
        rng = np.random.default_rng(99)
        ks = set(rng.integers(0, c.nf, 256).tolist())
        for f in c.signal_freqs:
            k = int(round((f - c.f0) / c.df))
            ks.update(range(max(0, k - 24), min(c.nf, k + 25)))
        ks = np.array(sorted(ks), dtype=np.int64)
        t0 = time.perf_counter()
        ref = oracle.periodogram_at(c.t, c.X, c.f0 + ks * c.df)
        sec = time.perf_counter() - t0
        top = ks[np.argsort(-ref)[:10]]
        rtop = np.sort(ref)[::-1][:10]
        for name in ("fixed64", "naive_fp32"):
            got = res[name][ks]
            out[name]["max_abs_dP_over_maxP"] = float(np.max(np.abs(got - ref)) / ref.max())
            out[name]["max_rel_err_top10"] = float(np.max(np.abs(res[name][top] - rtop) / rtop))
        out["tolerance"] = 1e-4
        out["cpu_baseline"] = {"terms_per_s": c.t.size * ks.size / sec, "cores": oracle.num_threads(),
                               "kind": "oracle", "sample": "%d sampled bins x all samples" % ks.size}
    return out


def pipe_rates(ctx, sms, sm_max_mhz):
    """lsp_probe_pipes on this GPU (after the timed region): the measured
    per-SM, per-clock rates behind the roofline denominators, and the roofs
    they imply for each sin/cos mode at the SM count and maximum clock."""
    r = ctx.probe_pipes()
    g = sms * sm_max_mhz * 1e6 / 1e9
    # roofs (Gterms/s) these rates imply: 1 sin/cos pair, 8 and 6 FMA-pipe ops per term
    r["roof_Gterms"] = {"mufu": r["sincos_per_clk_sm"] * g, "recur": r["ffma_per_clk_sm"] / 8 * g,
                        "recur3": r["ffma_per_clk_sm"] / 6 * g}
    return r


def _e2e(lsp, torch, c, f0, local, stream, args, world):
    """Same metric through the C ABI with pinned host buffers: every step copies
    t and X in and P out inside the timed region (the call blocks on P)."""
    terms = c.t.size * c.nf
    t_h = torch.from_numpy(c.t).pin_memory()
    X_h = torch.from_numpy(c.X).pin_memory()
    P_h = torch.empty(c.nf, dtype=torch.float32).pin_memory()
    ctx_h = lsp.Context(local, stream=stream, sincos_mode=args.mode, freqs_per_thread=args.F)
    ctx_h.periodogram(t_h, X_h, f0, c.df, c.nf, out=P_h)
    e2e_s = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        ctx_h.periodogram(t_h, X_h, f0, c.df, c.nf, out=P_h)  # blocks until P_h is written
        e2e_s.append(time.perf_counter() - t0)
    ctx_h.close()
    return world * terms * len(e2e_s) / sum(e2e_s)


def _time_calls(torch, stream, fn, warmup, steps, flush):
    """Median device time (ms) of fn() over `steps` calls after `warmup`, L2
    flushed before each, CUDA events on the launching stream."""
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        ms = []
        for i in range(steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def run_paper_shape(torch, dev, stream, args, peaks, sms):
    """The paper's benchmark shape (Sec. 5.2-5.3) on synthetic data: N_t =
    382,003 samples over 150 d, N_f = 1,528,064 (5.84e11 terms), one call, and
    the N_t sweep of its Fig. 4 (uniform down-sampling by 2^k, N_f = 4 N_t
    rounded up to 256), with the oracle timed on the host cores at the small
    end.  The paper's Tesla C1060 took 20.3 s for its 382,003-sample curve
    (another machine and FP32 phases: context, not a target)."""
    from paper_1007_1658_gb300 import lsp, synth
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = lsp.Context(dev.index or 0, stream=stream)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sweep = []
    with ClockSampler(dev.index or 0) as clk:
        for step in (256, 128, 64, 32, 16, 8, 4, 2, 1):
            c = synth.corot_382k(step=step)
            t_d, X_d = d(c.t), d(c.X)
            P_d = torch.empty(c.nf, dtype=torch.float32, device=dev)
            fn = lambda: ctx.periodogram(t_d, X_d, c.f0, c.df, c.nf, out=P_d)
            ms = _time_calls(torch, stream, fn, 2, 3, flush)
            row = {"N_t": int(c.t.size), "gpu_ms": ms, "gpu_terms_per_s": c.terms / (ms * 1e-3)}
            if args.cpu_baseline and c.terms <= 2e8:
                import oracle
                t0 = time.perf_counter()
                oracle.periodogram(c.t, c.X, c.f0, c.df, c.nf)
                row["cpu_oracle_ms"] = 1e3 * (time.perf_counter() - t0)
            sweep.append(row)
        ctx.sync(120.0)
        # Press-Rybicki approximation of the full-size curve (the last one above)
        fn = lambda: ctx.press_rybicki(t_d, X_d, c.f0, c.df, c.nf, macc=4, out=Q_d)
        Q_d = torch.empty(c.nf, dtype=torch.float32, device=dev)
        pr_ms = _time_calls(torch, stream, fn, 2, 3, flush)
        pr_launches = ctx.last_launch_count()
        ctx.sync(120.0)
        pr_err = float((Q_d - P_d).abs().max() / P_d.max())
    ctx.close()
    full = sweep[-1]
    big = sweep[-4:]
    slope = float(np.polyfit(np.log([r["N_t"] for r in big]), np.log([r["gpu_ms"] for r in big]), 1)[0])
    import oracle
    return {"workload": "corot_382k: N_t = 382,003 over 150 d (32-s slots, orbit gaps), N_f = 1,528,064, "
                        "f_0 = df = 1/(4T); sweep by uniform down-sampling",
            "t_calc_s": full["gpu_ms"] * 1e-3, "terms_per_s": full["gpu_terms_per_s"],
            "paper_c1060_t_calc_s": 20.3, "paper_8core_cpu_t_calc_s": 566.0,
            "slope_dlog_t_dlog_Nt_top4": slope,
            "press_rybicki": {"macc": 4, "ms": pr_ms, "launches": pr_launches,
                              "speedup_vs_exact": full["gpu_ms"] / pr_ms,
                              "max_abs_dP_over_maxP_vs_exact": pr_err},
            "sweep": sweep,
            "cpu_cores": oracle.num_threads() if args.cpu_baseline else None, "clocks": clk.summary()}


def run_gls_bench(torch, dev, stream, args, peaks, peak_src, sms):
    """Floating-mean (generalized, weighted) periodogram on gapped_100k with
    per-sample errors (same times and grid): device-resident inputs, L2
    flushed between steps, CUDA events on the launching stream."""
    from paper_1007_1658_gb300 import lsp, synth
    c = synth.with_errors(synth.gapped_100k)
    if args.nf:
        c.nf = int(args.nf)
    terms = c.t.size * c.nf
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    t_d, X_d, dy_d = d(c.t), d(c.X), d(c.dy)
    P_d = torch.empty(c.nf, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    mode = args.mode if args.mode else lsp.SINCOS_RECUR3_X2
    gctx = lsp.Context(dev.index or 0, stream=stream, timing=1, sincos_mode=mode,
                       freqs_per_thread=args.F if args.F in (8, 16) else 0)
    F = args.F if args.F in (8, 16) else (8 if mode == lsp.SINCOS_MUFU else 16)
    steps = max(3, args.steps)
    with torch.cuda.stream(stream), ClockSampler(dev.index or 0) as clk:
        for _ in range(args.warmup):
            gctx.periodogram_gls(t_d, X_d, c.f0, c.df, c.nf, dy=dy_d, out=P_d)
        gctx.sync(120.0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        main_ms = []
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            gctx.periodogram_gls(t_d, X_d, c.f0, c.df, c.nf, dy=dy_d, out=P_d)
            ev[i][1].record(stream)
            main_ms.append(gctx.last_timing()[1])
        gctx.sync(120.0)
    torch.cuda.synchronize(dev)
    gctx.close()
    step_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    # bounding pipe per term: 6 accumulating FMA + the sin/cos of the mode
    roof = {lsp.SINCOS_MUFU: ("SFU (MUFU): 2 sin/cos ops per term, 16 ops/clk/SM", 16.0 / 2),
            lsp.SINCOS_RECUR: ("FMA pipe: 6 accumulate + 4 rotation FP32 ops per term, 128/clk/SM", 128.0 / 10),
            lsp.SINCOS_RECUR3: ("FMA pipe: 6 accumulate + 2 three-term FP32 ops per term, 128/clk/SM",
                                128.0 / 8),
            lsp.SINCOS_RECUR3_X2: ("FMA pipe: 6 accumulate + 2 three-term FP32 lane ops per term (4 FFMA2), "
                                   "128/clk/SM", 128.0 / 8)}[mode]
    peak = roof[1] * sms * peaks["sm_max_mhz"] * 1e6
    achieved = terms / (float(np.mean(main_ms)) * 1e-3)
    kernel = "gls_main_kernel<%d,%d>" % (F, {1: 1, 2: 2, 3: 4, 4: 5}[mode])
    # many curves: the Monte-Carlo batch's 4096 sampling patterns as measured curves with errors
    b = synth.noise_batch(n_curves=args.batch_curves)
    rng = np.random.default_rng(17)
    bdy = np.exp(rng.uniform(np.log(0.3), np.log(3.0), b.t.size))
    bX = 5.0 + bdy * rng.normal(size=b.t.size)
    bargs = (d(b.t_off), d(b.t), d(bX), d(b.f0), d(b.df), d(b.nf))
    bmax = torch.empty(b.n, dtype=torch.float32, device=dev)
    barg = torch.empty(b.n, dtype=torch.int32, device=dev)
    bctx = lsp.Context(dev.index or 0, stream=stream)
    dy_b = d(bdy)
    bfn = lambda: bctx.batch_gls(*bargs, dy=dy_b, maxP=bmax, argmax=barg)
    b_ms = _time_calls(torch, stream, bfn, 2, 3, flush)
    batch_line = {"workload": "%d noise_batch patterns as measured curves with errors, N_f = 2 N_t" % b.n,
                  "ms": b_ms, "curves_per_s": b.n / (b_ms * 1e-3), "terms_per_s": b.terms / (b_ms * 1e-3)}
    # Monte Carlo of the floating-mean form: noise realizations X = dy z drawn on the device
    nb = synth.noise_batch(n_curves=256, seed=777001)
    ndy = d(np.exp(np.random.default_rng(18).uniform(np.log(0.3), np.log(3.0), nb.t.size)))
    n_real = 16
    nargs = (d(nb.t_off), d(nb.t), d(nb.f0), d(nb.df), d(nb.nf))
    nmax = torch.empty(n_real * nb.n, dtype=torch.float32, device=dev)
    narg = torch.empty(n_real * nb.n, dtype=torch.int32, device=dev)
    nfn = lambda: bctx.batch_gls_noise(*nargs, dy=ndy, seed=3, n_real=n_real, maxP=nmax, argmax=narg)
    n_ms = _time_calls(torch, stream, nfn, 2, 3, flush)
    bctx.close()
    batch_line["noise_mc"] = {"workload": "%d noise_batch patterns x %d realizations with errors (X = dy z)"
                                          % (nb.n, n_real),
                              "ms": n_ms, "periodograms_per_s": n_real * nb.n / (n_ms * 1e-3),
                              "terms_per_s": n_real * nb.terms / (n_ms * 1e-3)}
    return {"workload": "gapped_100k with per-sample errors (dy log-U[0.15, 1.5], 2%% x10), N_t = %d, N_f = %d"
                        % (c.t.size, c.nf),
            "batch": batch_line,
            "ms_per_call": step_ms, "terms_per_s": terms / (step_ms * 1e-3),
            "roofline": {"bound": "alu", "kernel": kernel,
                         "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gterms/s", "frac": achieved / peak,
                         "traffic": _recorded_traffic(kernel, "gls_main_gapped_100k_errors.md", GLS_SOURCES),
                         "peak_basis": "%s: %.2f terms/clk/SM x %d SMs x %.0f MHz (%s sm_max_mhz)" % (
                             roof[0], roof[1], sms, peaks["sm_max_mhz"], peak_src),
                         "main_ms": float(np.mean(main_ms))},
            "clocks": clk.summary()}


def batch_cpu_sample(n_sample=32, seed=1234):
    """The oracle on a random subset of the Monte-Carlo batch's curves (same
    patterns, same Philox noise), as curves/s and terms/s on the host cores."""
    import oracle
    from paper_1007_1658_gb300 import synth
    b = synth.noise_batch(n_curves=4096)
    picks = np.random.default_rng(5).choice(b.n, n_sample, replace=False)
    terms = 0
    t0 = time.perf_counter()
    for c in picks:
        t = b.curve_t(int(c))
        X = oracle.noise(seed, int(c), 0, t.size)
        oracle.periodogram(t, X, b.f0[c], b.df[c], b.nf[c])
        terms += t.size * int(b.nf[c])
    sec = time.perf_counter() - t0
    return {"value": n_sample / sec, "unit": "curves/s", "terms_per_s": terms / sec, "cores": oracle.num_threads(),
            "kind": "oracle", "sample": "%d random curves of the 4096 (%.3g terms)" % (n_sample, terms)}


def mrhs_ops_per_term(R, n_real):
    """FMA-pipe operations per term and realization of an lsp_batch call with
    groups of R realizations: 6 one at a time; else 2 (XC, XS) + 2 recurrence
    shared by the group, plus CC and CS either in every group (2 / R) or, with
    four groups or more per pattern, once per pattern in the window pass
    (4 / n_real)."""
    if R == 1:
        return 6.0
    if n_real >= 4 * R:
        return 2.0 + 2.0 / R + 4.0 / n_real
    return 2.0 + 4.0 / R


def run_mrhs_bench(torch, dev, stream, n_patterns=256, n_real=64, groups=(1, 2, 4, 8), clk_sm=None):
    """Many realizations per pattern (the surrogate's training shape: 256
    noise_batch patterns x 64 realizations, one lsp_batch call) for each
    multi-RHS group size; every result is bit-identical across group sizes.
    With clk_sm (SMs x clock in Hz) each group also gets its FMA-pipe roof
    (128 lanes/clk/SM over mrhs_ops_per_term) and the fraction reached."""
    from paper_1007_1658_gb300 import lsp, synth
    b = synth.noise_batch(n_curves=n_patterns, seed=777001)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    off, t, f0, df, nf = d(b.t_off), d(b.t), d(b.f0), d(b.df), d(b.nf)
    maxP = torch.empty(n_real * b.n, dtype=torch.float32, device=dev)
    arg = torch.empty(n_real * b.n, dtype=torch.int32, device=dev)
    out = []
    for rhs in groups:
        mctx = lsp.Context(dev.index or 0, stream=stream, batch_rhs=rhs)
        with torch.cuda.stream(stream):
            mctx.batch(off, t, f0, df, nf, seed=1, n_real=n_real, maxP=maxP, argmax=arg)
            mctx.sync(300.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for r in range(3):
                mctx.batch(off, t, f0, df, nf, seed=2 + r, n_real=n_real, maxP=maxP, argmax=arg)
            e1.record(stream)
            mctx.sync(300.0)
        ms = e0.elapsed_time(e1) / 3
        mctx.close()
        row = {"batch_rhs": rhs, "ms": ms, "periodograms_per_s": n_real * b.n / (ms * 1e-3),
               "terms_per_s": n_real * b.terms / (ms * 1e-3)}
        if clk_sm:
            ops = mrhs_ops_per_term(min(rhs, n_real), n_real)
            row["ops_per_term"] = ops
            row["frac_of_roof"] = row["terms_per_s"] / (128.0 / ops * clk_sm)
        out.append(row)
    return {"workload": "%d noise_batch patterns x %d realizations" % (b.n, n_real), "by_group": out}


def run_batch_bench(ctx, torch, dev, stream, args):
    """Monte-Carlo batch (4096 pure-noise curves, N_t log-uniform in
    [200, 20000], gapped patterns, N_f = 2 N_t): one graph-captured persistent
    launch (lsp_batch, noise drawn on the device, per-curve max P) against the
    plain form, one lsp_periodogram call per curve on the same stream (same
    noise values, copied in beforehand; its per-curve maxima are not counted)."""
    from paper_1007_1658_gb300 import lsp, synth
    b = synth.noise_batch(n_curves=args.batch_curves)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    off, t, f0, df, nf = d(b.t_off), d(b.t), d(b.f0), d(b.df), d(b.nf)
    maxP = torch.empty(b.n, dtype=torch.float32, device=dev)
    arg = torch.empty(b.n, dtype=torch.int32, device=dev)
    bctx = lsp.Context(dev.index or 0, stream=stream)
    seed = 1234
    with torch.cuda.stream(stream), ClockSampler(dev.index or 0) as clk:
        for _ in range(2):
            bctx.batch(off, t, f0, df, nf, seed=seed, maxP=maxP, argmax=arg)
        bctx.sync(300.0)
        reps = max(2, args.batch_reps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for r in range(reps):
            bctx.batch(off, t, f0, df, nf, seed=seed + r, maxP=maxP, argmax=arg)
        e1.record(stream)
        bctx.sync(300.0)
    torch.cuda.synchronize(dev)
    batch_ms = e0.elapsed_time(e1) / reps
    # the same batch after lsp_autotune_batch (launch shape chosen by timing on this batch)
    tctx = lsp.Context(dev.index or 0, stream=stream)
    with torch.cuda.stream(stream):
        tctx.autotune_batch(off, t, f0, df, nf, n_real=1)
        tctx.batch(off, t, f0, df, nf, seed=seed, maxP=maxP, argmax=arg)
        tctx.sync(300.0)
        tuned_shape = tctx.test_last_batch_shape()
        e0.record(stream)
        for r in range(reps):
            tctx.batch(off, t, f0, df, nf, seed=seed + r, maxP=maxP, argmax=arg)
        e1.record(stream)
        tctx.sync(300.0)
    tuned_ms = e0.elapsed_time(e1) / reps
    tctx.close()
    # plain form: the same noise (realization 0 of seed 1234), one call per curve
    X = torch.empty(b.t.size, dtype=torch.float64, device=dev)
    tmp = torch.empty(int(np.diff(b.t_off).max()), dtype=torch.float32, device=dev)
    for c in range(b.n):
        n = int(b.t_off[c + 1] - b.t_off[c])
        bctx.noise(seed, c, 0, n, out=tmp[:n])
        X[int(b.t_off[c]):int(b.t_off[c + 1])] = tmp[:n].double()
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    P = torch.empty(int(P_off[-1]), dtype=torch.float32, device=dev)
    pctx = lsp.Context(dev.index or 0, stream=stream)
    views = [(t[int(b.t_off[c]):int(b.t_off[c + 1])], X[int(b.t_off[c]):int(b.t_off[c + 1])],
              float(b.f0[c]), float(b.df[c]), int(b.nf[c]), P[int(P_off[c]):int(P_off[c + 1])]) for c in range(b.n)]
    with torch.cuda.stream(stream):
        for v in views[:64]:
            pctx.periodogram(v[0], v[1], v[2], v[3], v[4], out=v[5])
        pctx.sync(300.0)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        launches = 0
        for v in views:
            pctx.periodogram(v[0], v[1], v[2], v[3], v[4], out=v[5])
            launches += pctx.last_launch_count()
        e3.record(stream)
        pctx.sync(300.0)
    torch.cuda.synchronize(dev)
    plain_ms = e2.elapsed_time(e3)
    # the two forms agree on the maxima (same noise, same arithmetic up to summation order)
    Pn = P.cpu().numpy()
    pmax = np.array([Pn[P_off[c]:P_off[c + 1]].max() for c in range(b.n)])
    bctx.batch(off, t, f0, df, nf, seed=seed, maxP=maxP, argmax=arg)
    bctx.sync(300.0)
    agree = float(np.max(np.abs(pmax - maxP.cpu().numpy()) / pmax))
    bctx.close()
    pctx.close()
    return {"workload": "noise_batch: %d pure-noise curves, N_t log-U[200,20000], N_f = 2 N_t" % b.n,
            "clocks": clk.summary(), "terms": b.terms, "plain_launches": launches, "batch_launches": 1,
            "max_rel_diff_batch_vs_plain": agree, "plain_terms_per_s": b.terms / (plain_ms * 1e-3),
            "terms_per_s": b.terms / (batch_ms * 1e-3), "plain_curves_per_s": b.n / (plain_ms * 1e-3),
            "tuned_shape": dict(zip(("mode", "F", "R", "tailF", "tile"), tuned_shape)), "graph_ms_tuned": tuned_ms,
            "curves_per_s": b.n / (batch_ms * 1e-3), "plain_ms": plain_ms, "graph_ms": batch_ms,
            "speedup_vs_plain": plain_ms / batch_ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--mode", type=int, default=0,
                    help="sin/cos mode: 0 auto (= 4), 1 MUFU, 2 recurrence, 3 three-term recurrence, "
                         "4 three-term recurrence in packed FP32x2")
    ap.add_argument("--F", type=int, default=0, help="frequencies per thread (0 = auto)")
    ap.add_argument("--ref-bins", type=int, default=2048, help="reference arm: oracle frequencies per step")
    ap.add_argument("--cpu-bins", type=int, default=16384, help="cpu_baseline: oracle frequencies (~10-30 s)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-gls", dest="gls", action="store_false", help="skip the floating-mean periodogram leg")
    ap.add_argument("--no-paper", dest="paper", action="store_false", help="skip the paper-shape N_t sweep")
    ap.add_argument("--no-probe", dest="probe", action="store_false", help="skip the pipe-rate probe")
    ap.add_argument("--no-cadence", dest="cadence", action="store_false",
                    help="skip the 65k-cadence precision comparison (naive FP32 vs fixed-point phase)")
    ap.add_argument("--nf", type=int, default=0, help="override N_f (smaller profiling case)")
    ap.add_argument("--batch-curves", type=int, default=4096)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--mrhs-patterns", type=int, default=256, help="multi-realization leg: sampling patterns")
    ap.add_argument("--mrhs-real", type=int, default=64, help="multi-realization leg: realizations per pattern")
    ap.add_argument("--mrhs-groups", default="1,2,4,8", help="multi-realization leg: group sizes to time")
    ap.add_argument("--no-mc", dest="mc", action="store_false",
                    help="skip the 4096-curve graph-vs-plain leg (keeps the multi-realization leg)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    dist = None
    if world > 1:
        import torch
        import torch.distributed as d
        backend = "nccl" if (args.impl == "gb300" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
        d.init_process_group(backend=backend)
        dist = d
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_gpu(args, rank, world, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
