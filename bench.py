#!/usr/bin/env python3
"""Benchmark of the CudaChain hull on GB300.

One step = the hull of each of three 20M-point float64 sets (uniform unit
square, unit disk, isotropic Gaussian sigma = 1), inputs resident in HBM.
`value` is Mpoints/s over all ranks (replicas: every rank runs its own hulls);
the roofline object reports the dominant streaming kernel against the
measured HBM bandwidth; `e2e` is the same metric through the host entry point
(H2D of the points and D2H of the result inside the timed region);
`cpu_baseline` times the CPU oracle on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoints/s (20M-pt hull, % of HBM roofline); batched hulls/s + p99 vs per-call"
KINDS = ("square", "disk", "gauss")
WORKLOAD = ("20M float64 points each of: uniform in unit square (seed 2), uniform in unit disk "
            "(seed 3), isotropic Gaussian sigma=1 (seed 4); one exact hull per distribution per step")

# Per-launch DRAM traffic of the streaming kernels from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, bytes per input point), valid
# only for the kernel source it was taken on.
NCU_TRAFFIC = {
    # kernel: (bytes per point, source file, src_sha1 of that file when captured)
    # mean over the three 20M float64 sets (one-pass dram__bytes_read.sum +
    # dram__bytes_write.sum per launch, cold caches)
    "k_classify": (16.1866, "paper_1508_05488_gb300/csrc/k_round1.cu", "9dc0ac72539fb509225d6a099219b8dbc46c7c3e"),
    "k_extremes": (16.1458, "paper_1508_05488_gb300/csrc/k_round1.cu", "9dc0ac72539fb509225d6a099219b8dbc46c7c3e"),
}


def src_sha1(rel):
    """sha1 of a source file's code: `//` comments, indentation and blank
    lines left out, so that a comment edit keeps a capture valid."""
    import hashlib
    lines = []
    with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
        for line in f:
            k = line.find("//")
            line = (line[:k] if k >= 0 else line).strip()
            if line:
                lines.append(line)
    return hashlib.sha1("\n".join(lines).encode()).hexdigest()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"cch_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["active_mask", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, r in rows:
            for nm, v in zip(names[1:], r[1:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm = [r[0] for r in rows]
        loaded = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def gen_inputs(n, kinds=KINDS):
    from paper_1508_05488_gb300 import inputs
    return {k: inputs.headline_f64(k, n) for k in kinds}


def max_over_ranks(x, dist, device):
    """The largest value of `x` over the ranks (the slowest rank bounds a
    step); `dist` is torch.distributed, or None for one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def hull_alg_bytes(S, n, s1, s2, h, W=None):
    """The method's algorithmic bytes for one hull (the measurement
    contract's accounting): the input read twice (extremes, then
    classification), the round-1 records written, sorted (one read and one
    write), scanned, the SPA survivors written and read by the chain step,
    and the hull written.  S = bytes per input point, W = record bytes."""
    W = W or (20 if S == 16 else 12)
    return 2 * S * n + W * s1 + 2 * W * s1 + (W * s1 + W * s2) + W * s2 + 4 * h


def whole_job_rate(points_all_ranks, ms_step):
    """Mpoints/s of the whole job: every rank's points over the slowest rank's step time."""
    return points_all_ranks / (ms_step * 1e-3) / 1e6


def cpu_baseline(pts, sample_n):
    """The C oracle (single thread, as it stands) on the first `sample_n` points of each set;
    beside it (key `parallel`) the multi-core CPU baseline on the same sample and every core
    OpenMP offers, checked equal to the oracle."""
    import numpy as np
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    tot = 0
    ref = {}
    for k in pts:
        p = pts[k][:sample_n]
        ref[k] = oracle.hull(p)
        tot += len(p)
    dt = time.perf_counter() - t0
    line = {"value": tot / dt / 1e6, "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
            "sample": f"first {sample_n} points of each of the {len(pts)} sets ({tot} points), C Andrew hull "
                      f"with exact predicates, one thread, {dt:.1f} s"}
    line["parallel"] = None
    try:
        if oracle.parallel_available():
            for k in pts:                                  # warm the thread pool
                oracle.parallel_hull(pts[k][:1000])
            same = True
            best = None
            for _ in range(3):
                t0 = time.perf_counter()
                for k in pts:
                    same &= bool(np.array_equal(oracle.parallel_hull(pts[k][:sample_n]), ref[k]))
                t = time.perf_counter() - t0
                best = t if best is None else min(best, t)
            line["parallel"] = {"value": tot / best / 1e6, "unit": "Mpoints/s", "cores": oracle.parallel_threads(),
                                "kind": "openmp: octagon filter, parallel merge sort, Andrew chain, "
                                        "FP64 filter before the exact predicates",
                                "identical_to_oracle": same}
    except Exception as e:  # the baseline is context, never a reason to lose the line
        line["parallel"] = {"unavailable": str(e)[:200]}
    return line


def run_reference(args):
    """Reference arm: the CPU oracle on host cores, one bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1508_05488_gb300 import inputs
    import oracle
    oracle.build()
    n = args.ref_n
    pts = {k: inputs.headline_f64(k, n) for k in KINDS}
    for _ in range(args.warmup):
        for k in KINDS:
            oracle.hull(pts[k])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for k in KINDS:
            oracle.hull(pts[k])
    dt = time.perf_counter() - t0
    v = args.steps * 3 * n / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Mpoints/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_points_per_set": n, "n_per_hull": n,
                   "note": "CPU oracle (C Andrew monotone chain, exact predicates) on the box's host core"},
        "cpu_baseline": {"value": v, "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n} points of each of the 3 sets per step"},
        "e2e": {"value": v, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched_bench(cch, torch, dev, stream, nsets):
    """4096 int32 sets of log-uniform size in [256, 2^20] (square or disk by a
    fair coin, seed 7): one cch_hull_batched launch sequence for all of them
    against one cch_hull call per set, inputs resident; per-set results of the
    two paths compared element-wise on the device."""
    from paper_1508_05488_gb300 import inputs
    pts, off = inputs.batched_i32(nsets, seed=7)
    n_tot = int(off[-1])
    d = torch.from_numpy(pts).to(dev)
    del pts
    idx_b = torch.empty(max(n_tot, 1), dtype=torch.int32, device=dev)
    cnt_b = torch.empty(nsets, dtype=torch.int32, device=dev)
    idx_c = torch.empty(max(n_tot, 1), dtype=torch.int32, device=dev)
    cnt_c = torch.empty(nsets, dtype=torch.int32, device=dev)
    offs = [int(v) for v in off]

    def batched():
        cch.hull_batched_async(d, off, idx_b, cnt_b, stream=stream)

    def per_call(ev=None):
        for s_ in range(nsets):
            a, b = offs[s_], offs[s_ + 1]
            if ev is not None:
                ev[s_][0].record(stream)
            cch.hull_async(d[a:b], idx_c[a:], cnt_c[s_:s_ + 1], stream=stream)
            if ev is not None:
                ev[s_][1].record(stream)

    for _ in range(2):
        batched()
        per_call()
    torch.cuda.synchronize()
    same = bool(torch.equal(cnt_b, cnt_c))
    if same:
        for s_ in range(nsets):
            c = int(cnt_b[s_])
            if c > 0 and not torch.equal(idx_b[offs[s_]:offs[s_] + c], idx_c[offs[s_]:offs[s_] + c]):
                same = False
                break
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_batched():
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            batched()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_default = time_batched()
    # the run-time choices tuned on this batch (outside the timed region),
    # then the same measurement with them
    tuned = cch.autotune_batched(d, off, idx_b, cnt_b, reps=2, stream=stream)
    batched()
    torch.cuda.synchronize()
    same_tuned = bool(torch.equal(cnt_b, cnt_c))
    if same_tuned:
        for s_ in range(nsets):
            c = int(cnt_b[s_])
            if c > 0 and not torch.equal(idx_b[offs[s_]:offs[s_] + c], idx_c[offs[s_]:offs[s_] + c]):
                same_tuned = False
                break
    ms_batch = time_batched()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsets)]
    torch.cuda.synchronize()
    e0.record(stream)
    per_call(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_calls = e0.elapsed_time(e1)
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    q = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
    hbm, _ = peaks()
    return {"config": f"{nsets} int32 sets, sizes log-uniform in [256, 2^20] (seed 7), square or disk",
            "points": n_tot, "hulls_per_s": nsets / (ms_batch * 1e-3), "ms_per_batch": ms_batch,
            "hbm_frac": 2 * 8 * n_tot / (ms_batch * 1e-3) / 1e9 / hbm,
            "hbm_frac_note": "two reads of every 8-byte point over the batch time, against the measured copy bandwidth",
            "default_choices_ms_per_batch": ms_default, "tuned_choices": tuned,
            "identical_with_tuned_choices": same_tuned,
            "per_call_hulls_per_s": nsets / (ms_calls * 1e-3), "per_call_ms_total": ms_calls,
            "per_call_p50_ms": q(0.50), "per_call_p99_ms": q(0.99),
            "speedup_vs_per_call": ms_calls / ms_batch, "identical_to_per_call": same}


def serve_bench(cch, torch, dev, requests_per_load, window=256):
    """Poisson stream of float64 hull requests (sizes log-uniform in [1e3,
    2e7], square / disk / Gaussian / shell, seed 8): `requests_per_load`
    distinct requests, drawn in device memory and submitted from there
    (cch_serve_submit_device: the request state stays device-resident).
    First the saturated rate (closed loop, at most `window` requests
    outstanding, measured twice: the higher is reported with the lower
    beside it), then offered loads of 0.5, 0.8 and 0.95 of the lower.  Every
    result is compared with the hull of the same request computed alone
    (cch_hull).  `hulls_per_s` counts every request over first submit ->
    last result; `drain_ms` is last result - last arrival."""
    import numpy as np
    from paper_1508_05488_gb300 import inputs
    reqs, alone = [], []
    for i in range(requests_per_load):
        d = inputs.serve_request_device(i, dev)
        reqs.append(d)
        alone.append(cch.hull(d).cpu().numpy())
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def run(rate):
        arrivals = inputs.poisson_arrivals(requests_per_load, rate) if rate else None
        res, which = {}, {}
        with cch.Server(np.float64) as srv:
            t0 = time.perf_counter()
            t_arr = t0
            for i in range(requests_per_load):
                if arrivals is not None:
                    wait = t0 + arrivals[i] - time.perf_counter()
                    if wait > 0:
                        time.sleep(wait)
                else:
                    while i - len(res) >= window:           # closed loop: bounded outstanding work
                        for t, st, h, lat in srv.poll():
                            res[t] = (st, h)
                t_arr = time.perf_counter()
                which[srv.submit(reqs[i], stream=stream)] = i
                for t, st, h, lat in srv.poll():
                    res[t] = (st, h)
            while len(res) < requests_per_load:
                for t, st, h, lat in srv.poll():
                    res[t] = (st, h)
                time.sleep(0.0001)
            t_end = time.perf_counter()
            stats = srv.stats()
        ok = all(st == 0 and np.array_equal(h, alone[which[t]]) for t, (st, h) in res.items())
        return {"offered_hulls_per_s": rate, "hulls_per_s": requests_per_load / (t_end - t0),
                "arrival_window_s": t_arr - t0, "drain_ms": (t_end - t_arr) * 1e3,
                "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "samples": len(res),
                "identical_to_alone": bool(ok)}

    # the saturated rate twice (it varies from run to run on a shared box);
    # the offered loads are fractions of the lower one
    sat, sat2 = run(None), run(None)
    if sat2["hulls_per_s"] > sat["hulls_per_s"]:
        sat, sat2 = sat2, sat
    sat["other_run_hulls_per_s"] = sat2["hulls_per_s"]
    loads = [run(f * sat2["hulls_per_s"]) for f in (0.5, 0.8, 0.95)]
    sizes = [int(r.shape[0]) for r in reqs]
    del reqs
    torch.cuda.empty_cache()
    return {"config": f"{requests_per_load} distinct float64 requests per load (sizes log-uniform in [1e3, 2e7], "
                      "square/disk/Gaussian/shell, seed 8), drawn and submitted in device memory; budget 64 GiB; "
                      f"saturated rate in a closed loop of at most {window} outstanding requests",
            "mean_points_per_request": float(np.mean(sizes)), "total_points": int(np.sum(sizes)),
            "saturated": sat, "loads": loads}


# The other single-hull configurations: timed beside the headline step (not
# part of `value`).  name: (generator, n, dtype, description)
EXTRA_CONFIGS = (
    ("degenerate_20M", "degenerate_f64", 20_000_000, "f64",
     "20M float64: 4M points on the unit circle and 16M in the disk of radius 1-2^-10, all on the 2^-20 grid, "
     "1% exact duplicates, shuffled (seed 5)"),
    ("circle_2M", "circle_f64", 2_000_000, "f64",
     "2M float64 points at angles 2 pi k / n on the unit circle, shuffled (seed 6): every point is a hull vertex"),
    ("int32_1M", "square_i32", 1_000_000, "i32", "1M int32 points uniform in [0, 2^29)^2 (seed 1)"),
)


def extra_configs_bench(cch, torch, dev, reps, hbm):
    """Mpoints/s, stage times and survivor counts of the degenerate, all-extreme
    and int32 configurations; for the multi-block sort (k_big) a roofline over
    the record bytes it moves: one read of the records for the histograms, one
    read and one write per radix pass actually run (passes whose digit is the
    same for every record are skipped), the SPA phase's read of every record's
    index and point and write of the survivors' chain slots."""
    from paper_1508_05488_gb300 import inputs
    out = {}
    for name, gen, n, dt, desc in EXTRA_CONFIGS:
        host = getattr(inputs, gen)(n, {"degenerate_f64": 5, "circle_f64": 6, "square_i32": 1}[gen])
        pts = torch.from_numpy(host).to(dev)
        del host
        idx = torch.empty(n, dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        for _ in range(3):
            cch.hull_async(pts, idx, cnt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            cch.hull_async(pts, idx, cnt)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        h = int(cnt.item())
        cch.profile(True)
        cch.profile_read()
        for _ in range(3):
            cch.hull_async(pts, idx, cnt)
        st_ms, calls = cch.profile_read()
        cch.profile(False)
        st_ms = {k: v / max(calls, 1) for k, v in st_ms.items()}
        ours = cch.stages(pts, prefilter=True)
        paper = cch.stages(pts, prefilter=False)
        s1 = int(ours["counts"][0])
        s2 = int(ours["counts"][5:9].sum())
        passes = ours["passes"]
        S = 16 if dt == "f64" else 8
        rec = 12                     # record: 8-byte sort key + 4-byte value
        big_bytes = rec * s1 + passes * 2 * rec * s1 + (4 + S) * s1 + (S + 4) * s2 if passes else 0
        big_ms = st_ms.get("big", 0.0)
        b_alg = hull_alg_bytes(S, n, s1, s2, h)
        entry = {"config": desc, "n": n, "dtype": dt, "ms_per_hull": ms, "mpoints_s": n / ms / 1e3,
                 "hull_roofline": {"algorithmic_bytes": b_alg, "frac": b_alg / (ms * 1e-3) / 1e9 / hbm},
                 "hull_size": h, "stage_ms_per_hull": st_ms,
                 "round1_paper": int(paper["counts"][0]), "round1": s1, "spa": s2,
                 "identical_spa_both_modes": all(bool((a == b).all()) and len(a) == len(b)
                                                 for a, b in zip(ours["spa"], paper["spa"])),
                 "sort_path": "multi-block" if passes else "shared-memory",
                 "radix_passes": passes}
        if passes and big_ms > 0:
            ach = big_bytes / (big_ms * 1e-3) / 1e9
            entry["k_big_roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                       "frac": ach / hbm, "algorithmic_bytes": big_bytes,
                                       "kernel_ms_per_launch": big_ms,
                                       "note": "record buffers of this size are partly L2-resident"
                                               if big_bytes < 120e6 else ""}
        out[name] = entry
        del pts, idx
        torch.cuda.empty_cache()
    return out


# Sizes of the paper's randomly distributed point sets (Table 2).
SURVIVOR_SIZES = (100_000, 200_000, 500_000, 1_000_000, 2_000_000, 5_000_000, 10_000_000, 20_000_000)


def f32soa_bench(cch, torch, host, reps):
    """The paper's input form (Fig. 6: two float32 coordinate vectors): each
    synthetic set rounded to float32, through cch_hull_f32soa (round 1 reads
    the vectors, 8 bytes a point; later stages carry the exactly widened
    float64 values), beside cch_hull on the same points as float64 pairs
    (16 bytes a point).  Inputs resident on the device and larger than L2."""
    import numpy as np

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    sets = {}
    for kind in [k for k in KINDS if k in host]:
        p32 = host[kind].astype(np.float32)
        x = torch.from_numpy(np.ascontiguousarray(p32[:, 0])).cuda()
        y = torch.from_numpy(np.ascontiguousarray(p32[:, 1])).cuda()
        n = x.shape[0]
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        ms = timed(lambda: cch.hull_f32soa_async(x, y, idx, cnt))
        h = int(cnt.item())
        wide = torch.stack([x, y], 1).double()
        idx64 = torch.empty(n, dtype=torch.int32, device="cuda")
        cnt64 = torch.zeros(1, dtype=torch.int32, device="cuda")
        ms64 = timed(lambda: cch.hull_async(wide, idx64, cnt64))
        same = h == int(cnt64.item()) and bool(torch.equal(idx[:h], idx64[:h]))
        sets[kind] = {"mpoints_s": n / ms / 1e3, "ms_per_hull": ms, "float64_pairs_ms_per_hull": ms64,
                      "hull_size": h, "identical_to_float64_path": same}
        del x, y, idx, wide, idx64
        torch.cuda.empty_cache()
    if not sets:
        return None
    first = sets[next(iter(sets))]
    n = next(iter(host.values())).shape[0]
    return {"config": f"{n} float32 points of each synthetic set as two coordinate vectors",
            "value": first["mpoints_s"], "value_set": next(iter(sets)), "unit": "Mpoints/s", "sets": sets}


def survivors(kinds, sizes, reps):
    """Points left after each round of discarding against n (Sec. 3.3, Fig. 11),
    on the synthetic sets, with the time of the whole hull at each size.

    Round 1 of the paper (outside the quadrilateral) is counted with the
    dominance prefilters off; round 1 of this implementation with them on; the
    SPA survivors and the hull are the same either way (checked here).  The
    algorithmic bytes follow the per-step accounting: two reads of the input,
    the round-1 records written, sorted (one read and one write) and scanned,
    the SPA survivors written and read by the chain step, and the hull."""
    import numpy as np
    import torch
    import paper_1508_05488_gb300 as cch
    from paper_1508_05488_gb300 import inputs
    rows = []
    for kind in kinds:
        for n in sizes:
            pts = torch.from_numpy(inputs.headline_f64(kind, n)).cuda()
            paper = cch.stages(pts, prefilter=False)
            ours = cch.stages(pts, prefilter=True)
            same = (np.array_equal(paper["hull"], ours["hull"]) and
                    all(np.array_equal(a, b) for a, b in zip(paper["spa"], ours["spa"])))
            assert same, (kind, n)
            idx = torch.empty(n, dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
            for _ in range(3):
                cch.hull_async(pts, idx, cnt)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                cch.hull_async(pts, idx, cnt)
            e1.record()
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / reps
            s1 = int(sum(len(a) for a in paper["r1"]))
            s1p = int(sum(len(a) for a in ours["r1"]))
            s2 = int(sum(len(a) for a in paper["spa"]))
            h = int(paper["count"])
            balg = hull_alg_bytes(16, n, s1, s2, h)
            rows.append({"kind": kind, "n": n, "round1": s1, "round1_prefiltered": s1p, "spa": s2, "hull": h,
                         "us_per_hull": round(us, 1), "mpoints_s": round(n / us, 1),
                         "alg_bytes": balg, "alg_gbs": round(balg / us / 1e3, 1)})
            del pts, idx
    return rows


def profile_run(args):
    """Warm-up calls, then `--steps` calls of one workload (for ncu launch
    lists and captures): the batched 4096-set call or one extra configuration."""
    import torch
    import paper_1508_05488_gb300 as cch
    from paper_1508_05488_gb300 import inputs
    dev = torch.device("cuda", 0)
    if args.profile == "h2d":
        # pinned host -> device copy bandwidth with 1, 2, 4 and 8 streams
        # (the floor under the end-to-end number: the step's inputs cross it)
        nbytes = 320_000_000
        out = {}
        for ns in (1, 2, 4, 8):
            hs = [torch.empty(nbytes // ns, dtype=torch.uint8).pin_memory() for _ in range(ns)]
            ds = [torch.empty(nbytes // ns, dtype=torch.uint8, device=dev) for _ in range(ns)]
            sts = [torch.cuda.Stream(device=dev) for _ in range(ns)]
            for _ in range(2):
                for h, d_, st in zip(hs, ds, sts):
                    with torch.cuda.stream(st):
                        d_.copy_(h, non_blocking=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                for h, d_, st in zip(hs, ds, sts):
                    with torch.cuda.stream(st):
                        d_.copy_(h, non_blocking=True)
            torch.cuda.synchronize()
            out[ns] = nbytes * args.steps / (time.perf_counter() - t0) / 1e9
        print(json.dumps({"profile": "h2d", "bytes_per_copy_round": nbytes, "rounds": args.steps,
                          "gb_per_s_by_streams": out}))
        return 0
    if args.profile == "modes":
        # the comparison modes on the 20M float64 sets: round 1 with the
        # quadrilateral (the paper's), with the octagon, and with the dominance
        # prefilters (this implementation's default); the paper's chunked SPA
        # against the exact scan, both after the multi-block sort
        rows = {}
        for kind in KINDS:
            d = torch.from_numpy(inputs.headline_f64(kind, args.n)).to(dev)
            row = {}
            for name, kw in (("prefiltered", {}), ("paper", {"prefilter": False}), ("octagon", {"octagon": True}),
                             ("paper_blocked_spa", {"blocked": True})):
                for _ in range(2):
                    st = cch.stages(d, **kw)
                cch.profile(True)
                cch.profile_read()
                for _ in range(args.steps):
                    st = cch.stages(d, **kw)
                ms, calls = cch.profile_read()
                cch.profile(False)
                ms = {k: v / max(calls, 1) for k, v in ms.items()}
                row[name] = {"round1": int(st["counts"][0]), "spa": int(st["counts"][5:9].sum()),
                             "hull": int(st["count"]), "radix_passes": st["passes"],
                             "pipeline_ms": sum(v for k, v in ms.items() if k != "blocked_spa"),
                             "stage_ms": {k: round(v, 4) for k, v in ms.items()}}
            rows[kind] = row
            del d
            torch.cuda.empty_cache()
        print(json.dumps({"profile": "modes", "n": args.n, "calls": args.steps, "sets": rows}))
        return 0
    if args.profile in ("hull", "hull_f32"):
        # `--steps` hulls of each of `--kinds` at `--n` points: float64 pairs
        # (`hull`) or the same points rounded to float32 vectors (`hull_f32`)
        calls = []
        for kind in args.kinds.split(","):
            p = inputs.headline_f64(kind, args.n)
            idx = torch.empty(args.n, dtype=torch.int32, device=dev)
            cnt = torch.zeros(1, dtype=torch.int32, device=dev)
            if args.profile == "hull":
                d = torch.from_numpy(p).to(dev)
                calls.append(lambda d=d, idx=idx, cnt=cnt: cch.hull_async(d, idx, cnt))
            else:
                import numpy as np
                p32 = p.astype(np.float32)
                x = torch.from_numpy(np.ascontiguousarray(p32[:, 0])).to(dev)
                y = torch.from_numpy(np.ascontiguousarray(p32[:, 1])).to(dev)
                calls.append(lambda x=x, y=y, idx=idx, cnt=cnt: cch.hull_f32soa_async(x, y, idx, cnt))
        cnt = None
        call = lambda: [c() for c in calls]
    elif args.profile == "batched":
        pts, off = inputs.batched_i32(args.batched_sets, seed=7)
        d = torch.from_numpy(pts).to(dev)
        n = int(off[-1])
        idx = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        cnt = torch.empty(args.batched_sets, dtype=torch.int32, device=dev)
        call = lambda: cch.hull_batched_async(d, off, idx, cnt)
    else:
        cfg = {c[0]: c for c in EXTRA_CONFIGS}[args.profile]
        seed = {"degenerate_f64": 5, "circle_f64": 6, "square_i32": 1}[cfg[1]]
        d = torch.from_numpy(getattr(inputs, cfg[1])(cfg[2], seed)).to(dev)
        idx = torch.empty(cfg[2], dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        call = lambda: cch.hull_async(d, idx, cnt)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "calls": args.steps, "ms_per_call": e0.elapsed_time(e1) / args.steps,
                      "count0": int(cnt[0]) if cnt is not None else None}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=20_000_000)
    ap.add_argument("--cpu-n", type=int, default=4_000_000)
    ap.add_argument("--ref-n", type=int, default=2_000_000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--survivors", action="store_true",
                    help="print the survivors-after-each-round table against n (Sec. 3.3) instead")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the degenerate, all-extreme circle and int32 configurations")
    ap.add_argument("--batched-sets", type=int, default=4096)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests per offered load (0: skip the serving measurement)")
    ap.add_argument("--profile", default=None,
                    help="profiling run: `hull` / `hull_f32` (`--kinds` at `--n`, float64 pairs or float32 "
                         "vectors), `batched` (the 4096-set call), `h2d` (pinned copy bandwidth), `modes` "
                         "(the round-1 and SPA comparison modes on the 20M sets) or a configuration name "
                         "(degenerate_20M, circle_2M, int32_1M): warm-up calls, then --steps calls, "
                         "one summary line, nothing else")
    ap.add_argument("--kinds", default=",".join(KINDS),
                    help="comma-separated subset of square,disk,gauss (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    kinds = tuple(k for k in args.kinds.split(",") if k)
    assert kinds and all(k in KINDS for k in kinds), kinds
    if args.profile:
        return profile_run(args)
    if args.survivors:
        print(json.dumps({"survivors": survivors(kinds, SURVIVOR_SIZES, max(args.steps, 1)), "unit_time": "us",
                          "dtype": "f64", "data": "synthetic"}))
        return

    import numpy as np
    import torch
    import paper_1508_05488_gb300 as cch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    host = gen_inputs(args.n, kinds)
    dpts = {k: torch.from_numpy(host[k]).to(dev) for k in kinds}
    outs = {k: (torch.empty(args.n, dtype=torch.int32, device=dev),
                torch.empty(1, dtype=torch.int32, device=dev)) for k in kinds}
    stream = torch.cuda.current_stream()

    def step():
        for k in kinds:
            cch.hull_async(dpts[k], outs[k][0], outs[k][1], stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness guard of the timed configuration: counts are hull sizes
    counts = {k: int(outs[k][1].item()) for k in kinds}
    assert all(c > 0 for c in counts.values()), counts

    # stage breakdown from a short profiled pass outside the timed region
    # (events around every stage cost a few microseconds each) ...
    cch.profile(True)
    cch.profile_read()
    for _ in range(3):
        step()
    stage_all, calls_all = cch.profile_read()
    stage_all = {k: v / max(calls_all, 1) for k, v in stage_all.items()}
    # the same per set, for the streaming kernels' fraction on each
    stage_set = {}
    for k in kinds:
        for _ in range(3):
            cch.hull_async(dpts[k], outs[k][0], outs[k][1], stream=stream)
        ms_k, calls_k = cch.profile_read()
        stage_set[k] = {s_: v / max(calls_k, 1) for s_, v in ms_k.items()}
    # ... and, inside the timed region, events around the dominant streaming
    # kernel only
    dom = max(("k_extremes", "k_classify"), key=lambda k: stage_all[k])
    cch.profile_stages([dom])
    cch.profile_read()
    l0 = cch.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = cch.launch_count() - l0
    stage_ms, calls = cch.profile_read()
    cch.profile(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ms_step = ms / args.steps
    pts_step = len(kinds) * args.n * world
    value = whole_job_rate(pts_step, ms_step)

    # roofline of the dominant streaming kernel (one read of the points per launch)
    hbm, hbm_src = peaks()
    dom_ms = stage_ms[dom] / max(calls, 1)
    alg_bytes = 16.0 * args.n
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9
    traffic = None
    if dom in NCU_TRAFFIC:
        bpp, rel, sha = NCU_TRAFFIC[dom]
        if src_sha1(rel) == sha:
            traffic = bpp * args.n
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "peak_source": hbm_src,
                "algorithmic_bytes_per_launch": alg_bytes,
                "kernel_ms_per_launch": dom_ms,
                "stage_ms_per_hull": stage_all,
                "stage_note": "stage times come from events recorded between the launches, which keep "
                              "k_stairs from overlapping a1's tail; a hull without events (per_set.*.hull.ms) "
                              "takes less than the sum of its stages"}
    # the whole step against the method's floor: two reads of every input
    # point (the extremes must be known before the classification)
    step_bytes = 2 * 16.0 * args.n * len(kinds)
    # per set, from the profiled pass (events around every stage): the two
    # streaming kernels' 16 B per point over their stage time
    roofline["per_set"] = {
        k: {kern: {"ms": v[kern], "frac": alg_bytes / (v[kern] * 1e-3) / 1e9 / hbm}
            for kern in ("k_extremes", "k_classify") if v.get(kern)}
        for k, v in stage_set.items()}
    roofline["step"] = {"algorithmic_bytes": step_bytes, "ms": ms_step,
                        "achieved": step_bytes / (ms_step * 1e-3) / 1e9,
                        "frac": step_bytes / (ms_step * 1e-3) / 1e9 / hbm}

    # each set's whole hull against its algorithmic bytes (measured s1, s2, h)
    for k in kinds:
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(10):
            cch.hull_async(dpts[k], outs[k][0], outs[k][1], stream=stream)
        h1.record(stream)
        torch.cuda.synchronize()
        ms_k = h0.elapsed_time(h1) / 10
        st_k = cch.stages(dpts[k])
        s1, s2 = int(st_k["counts"][0]), int(st_k["counts"][5:9].sum())
        b_k = hull_alg_bytes(16, args.n, s1, s2, int(st_k["count"]))
        roofline["per_set"][k]["hull"] = {"ms": ms_k, "round1": s1, "spa": s2, "algorithmic_bytes": b_k,
                                          "frac": b_k / (ms_k * 1e-3) / 1e9 / hbm}

    # the same step with the three independent hulls issued on three streams
    # (each a single-hull call with its own workspace): one hull's
    # latency-bound stages overlap another's streaming ones.  Reported beside
    # `value`, which is the sequential single-stream step.
    side = [torch.cuda.Stream(device=dev) for _ in kinds]

    def step_streams():
        for st, k in zip(side, kinds):
            st.wait_stream(stream)
            cch.hull_async(dpts[k], outs[k][0], outs[k][1], stream=st)
        for st in side:
            stream.wait_stream(st)

    for _ in range(args.warmup):
        step_streams()
    torch.cuda.synchronize()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(args.steps):
        step_streams()
    c1.record(stream)
    torch.cuda.synchronize()
    assert all(int(outs[k][1].item()) == counts[k] for k in kinds)
    ms_conc = max_over_ranks(c0.elapsed_time(c1), dist, dev) / args.steps
    concurrent = {"value": whole_job_rate(pts_step, ms_conc), "unit": "Mpoints/s", "ms_per_step": ms_conc,
                  "how": "the step's hulls as single-hull calls on one CUDA stream each"}

    # end to end through the host entry point (pinned host inputs)
    pinned = {k: torch.from_numpy(host[k]).pin_memory() for k in kinds}
    hidx = {k: torch.empty(args.n, dtype=torch.int32).pin_memory() for k in kinds}
    hcnt = {k: torch.zeros(1, dtype=torch.int32).pin_memory() for k in kinds}

    # the step's sets are independent calls: one host thread and one stream
    # per set, so one set's host-to-device copy overlaps another's hull (the
    # copies themselves share the host link)
    from concurrent.futures import ThreadPoolExecutor
    e2e_streams = {k: torch.cuda.Stream(device=dev) for k in kinds}
    pool = ThreadPoolExecutor(max_workers=len(kinds))

    def one(k):
        rc = cch.hull_host_ptr(pinned[k].data_ptr(), args.n, cch.CCH_F64, hidx[k].data_ptr(),
                               hcnt[k].data_ptr(), stream=e2e_streams[k])
        assert rc == 0, rc
        return 4 + 4 * int(hcnt[k][0])

    def e2e_step():
        return sum(pool.map(one, kinds))

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 4)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        d2h = e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, dev)
    pool.shutdown()
    e2e = {"value": pts_step / e2e_s / 1e6, "unit": "Mpoints/s", "h2d_bytes_per_step": len(kinds) * 16 * args.n,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
           "api": "cch_hull_host from pinned host memory, one host thread and stream per set"}

    if rank != 0:
        return 0
    cpu = None if args.no_cpu else cpu_baseline(host, args.cpu_n)
    del dpts, outs
    torch.cuda.empty_cache()
    f32soa = f32soa_bench(cch, torch, host, max(args.steps, 3))
    torch.cuda.empty_cache()
    extra = None if args.no_extra else extra_configs_bench(cch, torch, dev, max(args.steps // 2, 5), hbm)
    torch.cuda.empty_cache()
    batched = None if args.no_batched else batched_bench(cch, torch, dev, stream, args.batched_sets)
    torch.cuda.empty_cache()
    serving = serve_bench(cch, torch, dev, args.serve_requests) if args.serve_requests > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if kinds == KINDS else f"{args.n} float64 points of {kinds}",
                   "n_per_hull": args.n, "hulls_per_step": len(kinds),
                   "hull_sizes": counts, "l2": "inputs larger than L2 (320 MB per set)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
        "gpu_launches": launches, "concurrent_streams": concurrent, "batched": batched, "serving": serving,
        "f32soa": f32soa,
        "configs": extra,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
